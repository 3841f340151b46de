"""Python face of the FP64 CPU oracle (``sfp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg.  The product path never imports this
module, and this module imports nothing from the product package.

All arithmetic lives in ``sfp_oracle.c``; this file only compiles it (plain
gcc, OpenMP) and marshals numpy arrays.  Units are the paper's scaled units
(lengths in d, time in xi/lambda; Sec. 3, Eqs. b3-b5).  State arrays are
``[chain][axis][index]`` float64 with the p = 0 (centre-of-mass) mode included.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ct.POINTER(ct.c_double)
_U32 = ct.POINTER(ct.c_uint32)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ct.CDLL(build())
            L.orc_philox4x32_10.argtypes = [_U32, _U32, _U32]
            L.orc_u01.argtypes = [ct.c_uint32]
            L.orc_u01.restype = ct.c_double
            L.orc_bead_normals.argtypes = [ct.c_uint32, ct.c_uint32, ct.c_int64,
                                           ct.c_uint32, ct.c_int, _D]
            L.orc_model_new.argtypes = [ct.c_int, ct.c_double, ct.c_double, ct.c_double]
            L.orc_model_new.restype = ct.c_void_p
            L.orc_model_free.argtypes = [ct.c_void_p]
            L.orc_model_tables.argtypes = [ct.c_void_p] + [_D] * 8
            for name in ("orc_modes_to_beads", "orc_beads_to_modes", "orc_delta_H",
                         "orc_full_force"):
                getattr(L, name).argtypes = [ct.c_void_p, _D, _D]
            L.orc_energy.argtypes = [ct.c_void_p, _D]
            L.orc_energy.restype = ct.c_double
            L.orc_mode_step_z.argtypes = [ct.c_void_p, _D, ct.c_double, ct.c_int, _D]
            L.orc_mode_step_Zm.argtypes = [ct.c_void_p, _D, ct.c_double, ct.c_int, _D]
            L.orc_mode_normals.argtypes = [ct.c_uint32, ct.c_uint32, ct.c_int64, ct.c_int, _D]
            L.orc_euler_step_z.argtypes = [ct.c_void_p, _D, ct.c_double, _D]
            L.orc_run_modes.argtypes = [ct.c_void_p, ct.c_int, ct.c_uint32, _U32,
                                        ct.c_int64, ct.c_int64, ct.c_double, ct.c_int,
                                        _D, ct.c_int]
            L.orc_run_modes_mk.argtypes = L.orc_run_modes.argtypes
            L.orc_run_euler.argtypes = [ct.c_void_p, ct.c_int, ct.c_uint32, _U32,
                                        ct.c_int64, ct.c_int64, ct.c_double, _D, ct.c_int]
            L.orc_ground_bonds.argtypes = [ct.c_void_p, _D]
            L.orc_equilibrium_start.argtypes = [ct.c_void_p, ct.c_uint32, ct.c_uint32, _D]
            L.orc_observables.argtypes = [ct.c_void_p, _D, _D]
            L.orc_threads.restype = ct.c_int
            L.orc_run_mc.argtypes = [ct.c_void_p, ct.c_int, ct.c_uint32, _U32, ct.c_int64,
                                     ct.c_int64, _D, _D, ct.POINTER(ct.c_int64), _D, ct.c_int]
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _up(a: np.ndarray):
    assert a.dtype == np.uint32 and a.flags.c_contiguous
    return a.ctypes.data_as(_U32)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_up(c), _up(k), _up(out))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def bead_normals(seed: int, job: int, step: int, tag: int, M: int) -> np.ndarray:
    z = np.zeros((3, M))
    lib().orc_bead_normals(seed, job, step, tag, M, _dp(z))
    return z


def mode_normals(seed: int, job: int, step: int, M: int) -> np.ndarray:
    """Mode-keyed noise Z[alpha][p] of one chain and step (Philox tag 2)."""
    Z = np.zeros((3, M))
    lib().orc_mode_normals(seed, job, step, M, _dp(Z))
    return Z


def threads() -> int:
    return lib().orc_threads()


class Model:
    """Tables and per-chain primitives for one (M, T*, nu, dtau)."""

    def __init__(self, M: int, Tstar: float = 0.034, nu: float = 0.35, dtau: float = 1.0):
        self.M, self.Tstar, self.nu, self.dtau = int(M), float(Tstar), float(nu), float(dtau)
        self._h = lib().orc_model_new(self.M, self.Tstar, self.nu, self.dtau)
        if not self._h:
            raise ValueError("invalid oracle model parameters")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_model_free(h)
            self._h = None

    def tables(self) -> dict:
        M = self.M
        t = {k: np.zeros(M) for k in ("zl", "zeta", "decay", "h", "w", "g")}
        t["phi"] = np.zeros((M, M))
        t["chi"] = np.zeros((M - 1, M))
        lib().orc_model_tables(self._h, _dp(t["phi"]), _dp(t["chi"]), _dp(t["zl"]),
                               _dp(t["zeta"]), _dp(t["decay"]), _dp(t["h"]),
                               _dp(t["w"]), _dp(t["g"]))
        return t

    def _map(self, fn, x):
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(3, self.M)
        y = np.zeros((3, self.M))
        getattr(lib(), fn)(self._h, _dp(x), _dp(y))
        return y

    def modes_to_beads(self, R):
        return self._map("orc_modes_to_beads", R)

    def beads_to_modes(self, r):
        return self._map("orc_beads_to_modes", r)

    def delta_H(self, r):
        return self._map("orc_delta_H", r)

    def full_force(self, r):
        return self._map("orc_full_force", r)

    def energy(self, r) -> float:
        x = np.ascontiguousarray(r, dtype=np.float64).reshape(3, self.M)
        return lib().orc_energy(self._h, _dp(x))

    def mode_step_z(self, R, z, shear: float = 0.0, coupling: bool = True):
        R = np.array(R, dtype=np.float64).reshape(3, self.M)
        z = np.ascontiguousarray(z, dtype=np.float64).reshape(3, self.M)
        lib().orc_mode_step_z(self._h, _dp(z), float(shear), int(bool(coupling)), _dp(R))
        return R

    def mode_step_Zm(self, R, Z, shear: float = 0.0, coupling: bool = True):
        """One mode step with the mode noise Z given directly."""
        R = np.array(R, dtype=np.float64).reshape(3, self.M)
        Z = np.ascontiguousarray(Z, dtype=np.float64).reshape(3, self.M)
        lib().orc_mode_step_Zm(self._h, _dp(Z), float(shear), int(bool(coupling)), _dp(R))
        return R

    def euler_step_z(self, r, z, shear: float = 0.0):
        r = np.array(r, dtype=np.float64).reshape(3, self.M)
        z = np.ascontiguousarray(z, dtype=np.float64).reshape(3, self.M)
        lib().orc_euler_step_z(self._h, _dp(z), float(shear), _dp(r))
        return r

    def run_modes(self, R, seed: int, jobs, step0: int, nsteps: int, shear: float = 0.0,
                  coupling: bool = True, nthreads: int = 0, mode_noise: bool = False):
        """nsteps mode-space steps of C chains; mode_noise: noise drawn per mode
        (orc_run_modes_mk) instead of per bead."""
        R = np.array(R, dtype=np.float64)
        C = R.shape[0]
        R = R.reshape(C, 3, self.M).copy()
        j = np.ascontiguousarray(jobs, dtype=np.uint32)
        assert j.shape == (C,)
        fn = lib().orc_run_modes_mk if mode_noise else lib().orc_run_modes
        fn(self._h, C, seed, _up(j), step0, nsteps, float(shear), int(bool(coupling)), _dp(R), nthreads)
        return R

    def run_euler(self, r, seed: int, jobs, step0: int, nsteps: int, shear: float = 0.0,
                  nthreads: int = 0):
        r = np.array(r, dtype=np.float64)
        C = r.shape[0]
        r = r.reshape(C, 3, self.M).copy()
        j = np.ascontiguousarray(jobs, dtype=np.uint32)
        lib().orc_run_euler(self._h, C, seed, _up(j), step0, nsteps, float(shear),
                            _dp(r), nthreads)
        return r

    def ground_bonds(self) -> np.ndarray:
        l = np.zeros(self.M - 1)
        lib().orc_ground_bonds(self._h, _dp(l))
        return l

    def equilibrium_start(self, seed: int, job: int) -> np.ndarray:
        R = np.zeros((3, self.M))
        lib().orc_equilibrium_start(self._h, seed, job, _dp(R))
        return R

    def equilibrium_starts(self, seed: int, jobs) -> np.ndarray:
        return np.stack([self.equilibrium_start(seed, int(j)) for j in jobs])

    def observables(self, R) -> np.ndarray:
        x = np.ascontiguousarray(R, dtype=np.float64).reshape(3, self.M)
        out = np.zeros(6)
        lib().orc_observables(self._h, _dp(x), _dp(out))
        return out

    def run_mc(self, R, seed: int, jobs, sweep0: int, n_sweeps: int, step, sample: bool = False,
               nthreads: int = 0):
        """Metropolis sweeps in the mode representation (Sec. 5A), see ``orc_mc_sweeps``.

        Returns ``(R, acc, obs)``: the new states ``[C][3][M]``, accepted moves per
        chain and mode ``[C][M]`` and, if ``sample``, per-chain sums of |L|^2,
        |u_m|^2, |r_m - r_cm|^2 and the sample count ``[C][4]`` (else None).
        """
        R = np.array(R, dtype=np.float64)
        C = R.shape[0]
        R = R.reshape(C, 3, self.M).copy()
        j = np.ascontiguousarray(jobs, dtype=np.uint32)
        assert j.shape == (C,)
        s = np.ascontiguousarray(step, dtype=np.float64)
        assert s.shape == (self.M,)
        acc = np.zeros((C, self.M), dtype=np.int64)
        obs = np.zeros((C, 4)) if sample else None
        lib().orc_run_mc(self._h, C, seed, _up(j), sweep0, n_sweeps, _dp(s), _dp(R),
                         acc.ctypes.data_as(ct.POINTER(ct.c_int64)),
                         _dp(obs) if sample else None, nthreads)
        return R, acc, obs

    def mc_tuned_steps(self, R, seed: int, jobs, rounds: int = 8, sweeps: int = 50,
                       target: float = 0.4):
        """Per-mode MC step sizes tuned toward ``target`` acceptance during a burn-in.

        Starts from sqrt(T*/zeta^l_p) and rescales each s_p by its acceptance over
        ``sweeps`` sweeps, ``rounds`` times (sweep counters 2^40 + k, away from the
        sampling sweeps).  Returns ``(step, R)``: the step sizes, to be held fixed
        while sampling, and the burnt-in states.
        """
        zl = self.tables()["zl"]
        step = np.zeros(self.M)
        step[1:] = np.sqrt(self.Tstar / zl[1:])
        C = np.asarray(R).shape[0]
        for k in range(rounds):
            R, acc, _ = self.run_mc(R, seed, jobs, (1 << 40) + k * sweeps, sweeps, step)
            rate = acc.sum(axis=0) / (3.0 * sweeps * C)
            step[1:] *= np.clip(rate[1:] / target, 0.25, 4.0)
        return step, R
