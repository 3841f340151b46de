"""GB300 mode-space Langevin dynamics of the extensible bead-spring model of
semiflexible polymers (Panja, Barkema, van Leeuwen, arXiv:1411.3487).

The simulation runs in the CUDA library ``_build/libsfp.so`` behind the C ABI
of ``include/sfp.h``; this package is its Python binding.  Host arrays are
numpy; the CUDA stream may be a ``torch.cuda.Stream`` or a raw handle.
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import _lib
from ._lib import (SFP_FP32, SFP_FP32_SIMT, SFP_FP64, SFP_MIXED_BF16, SFP_MIXED_BF16_2, SFP_MIXED_TF32,
                   SFP_OBS_ACCUM, SFP_OBS_COM,
                   SFP_OBS_BOND_MSD, SFP_OBS_COM_MSD, SFP_OBS_E2E2_MEAN, SFP_OBS_E2E_MSD, SFP_OBS_MID_MSD,
                   SFP_OBS_MODE_POWER, SFP_OBS_MODE_VAR,
                   SFP_OBS_MODES, SFP_OBS_MODES_F32, SFP_OBS_POSITIONS,
                   SFP_INTEGRATOR_EULER, SFP_INTEGRATOR_MODES, SFP_NOISE_BEADS, SFP_NOISE_MODES, SFP_OBS_SHAPE, SFP_OBS_STEP,
                   SFP_PATH_FUSED, SFP_PATH_STAGED, SFP_PROBE_BONDS, SFP_PROBE_DH,
                   SFP_PROBE_FORCE, SFP_PROBE_NOISE, SFP_PROBE_ZMODE, SfpChainDesc, SfpError,
                   SfpParams)

__all__ = ["Batch", "Server", "params_dsdna", "derive", "philox_words", "SfpError", "SFP_FP32",
           "SFP_MIXED_TF32", "SFP_MIXED_BF16", "SFP_MIXED_BF16_2", "SFP_FP64", "SFP_FP32_SIMT"]


def params_dsdna() -> SfpParams:
    """The paper's dsDNA parameter set (Sec. 2A, Sec. 7B)."""
    p = SfpParams()
    _lib.check(_lib.load().sfp_params_dsdna(ct.byref(p)))
    return p


def derive(p: SfpParams | None = None) -> dict:
    """Derived constants: T*, nu, c (ps per scaled time unit, Eq. g2), d (nm), b, l_p/a,
    lambda, kappa (pN/nm)."""
    p = p or params_dsdna()
    out = (ct.c_double * 8)()
    _lib.check(_lib.load().sfp_derive(ct.byref(p), out))
    keys = ("Tstar", "nu", "c_ps", "d_nm", "b", "lp_over_a", "lambda_pN_per_nm", "kappa_pN_per_nm")
    return dict(zip(keys, list(out)))


def philox_words(seed: int, job: int, step: int, tag: int, count: int) -> np.ndarray:
    """Raw Philox4x32-10 words computed on the GPU, shape [count, 4]."""
    out = np.zeros((count, 4), dtype=np.uint32)
    _lib.check(_lib.load().sfp_philox_words(seed, job, step, tag, count, out.ctypes.data))
    return out


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


class Batch:
    """A batch of independent chains advanced together on one GPU.

    ``chains`` is a sequence of dicts with ``n_beads`` and one of ``dt_ps`` or
    ``dtau``, optional ``shear_rate_per_s`` and ``job_id`` (default: index).
    """

    def __init__(self, chains, seed: int = 1, precision: int = SFP_FP32, params: SfpParams | None = None,
                 stream=None, hbm_budget_bytes: int = 0):
        L = _lib.load()
        self.params = params or params_dsdna()
        n = len(chains)
        arr = (SfpChainDesc * n)()
        self.n_beads = np.zeros(n, dtype=np.int64)
        for i, c in enumerate(chains):
            arr[i].n_beads = int(c["n_beads"])
            arr[i].dt_ps = float(c.get("dt_ps", 0.0))
            arr[i].dtau = float(c.get("dtau", 0.0))
            arr[i].shear_rate_per_s = float(c.get("shear_rate_per_s", 0.0))
            arr[i].job_id = int(c.get("job_id", i))
            self.n_beads[i] = arr[i].n_beads
        self.offsets = np.concatenate([[0], np.cumsum(3 * self.n_beads)])
        self.n_chains = n
        self.precision = precision
        self._n_lags = self._lags_next = 4
        h = ct.c_void_p()
        _lib.check(L.sfp_create(ct.byref(self.params), arr, n, seed, precision, _stream_handle(stream),
                                hbm_budget_bytes, ct.byref(h)))
        self._h = h

    # -- lifecycle -----------------------------------------------------------
    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib.check(_lib.load().sfp_destroy(self._h))
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- state ---------------------------------------------------------------
    def init_equilibrium(self, burn_in_steps: int = 0) -> None:
        _lib.check(_lib.load().sfp_init_equilibrium(self._h, burn_in_steps))

    def _packed(self, a, dtype=np.float64) -> np.ndarray:
        if isinstance(a, (list, tuple)):
            a = np.concatenate([np.asarray(x, dtype=dtype).ravel() for x in a])
        a = np.ascontiguousarray(a, dtype=dtype).ravel()
        if a.size != self.offsets[-1]:
            raise ValueError(f"expected {self.offsets[-1]} values, got {a.size}")
        return a

    def set_modes(self, modes) -> None:
        """Mode amplitudes, packed [3][M_c] per chain; a float32 array (or a list
        of them) goes through sfp_set_modes_f32 (half the host traffic)."""
        f32 = (isinstance(modes, np.ndarray) and modes.dtype == np.float32) or (
            isinstance(modes, (list, tuple)) and len(modes) > 0 and all(
                isinstance(x, np.ndarray) and x.dtype == np.float32 for x in modes))
        if f32:
            a = self._packed(modes, np.float32)
            _lib.check(_lib.load().sfp_set_modes_f32(self._h, a.ctypes.data, a.size))
            return
        a = self._packed(modes)
        _lib.check(_lib.load().sfp_set_modes(self._h, a.ctypes.data, a.size))

    def set_positions(self, pos_nm) -> None:
        a = self._packed(pos_nm)
        _lib.check(_lib.load().sfp_set_positions(self._h, a.ctypes.data, a.size))

    def set_step(self, step: int) -> None:
        _lib.check(_lib.load().sfp_set_step(self._h, step))

    def step(self, n_steps: int = 1) -> None:
        _lib.check(_lib.load().sfp_step(self._h, n_steps))

    # -- outputs ---------------------------------------------------------------
    def _unpack(self, flat: np.ndarray):
        if np.all(self.n_beads == self.n_beads[0]):
            return flat.reshape(self.n_chains, 3, int(self.n_beads[0]))
        return [flat[self.offsets[i]:self.offsets[i + 1]].reshape(3, -1) for i in range(self.n_chains)]

    def set_path(self, path: int) -> None:
        """SFP_PATH_FUSED (one kernel per step) or SFP_PATH_STAGED (one per stage, probes kept)."""
        _lib.check(_lib.load().sfp_set_path(self._h, int(path)))

    def set_graph(self, enable: bool = True) -> None:
        """Replay each chunk of steps from a captured CUDA graph."""
        _lib.check(_lib.load().sfp_set_graph(self._h, int(bool(enable))))

    def set_grouped(self, enable: bool = True) -> None:
        """One launch of clusters of two CTAs for the fused groups of all lengths (default), or one per group."""
        _lib.check(_lib.load().sfp_set_grouped(self._h, int(bool(enable))))

    def set_noise(self, keying: int) -> None:
        """SFP_NOISE_BEADS (default: bead noise projected, Eq. c4) or SFP_NOISE_MODES (Z drawn per mode)."""
        _lib.check(_lib.load().sfp_set_noise(self._h, int(keying)))

    def autotune(self, trial_steps: int = 20) -> list:
        """Choose chains per tile of the fused groups by timing; returns them per group."""
        out = (ct.c_int32 * self.n_chains)()          # at most one group per chain
        _lib.check(_lib.load().sfp_autotune(self._h, int(trial_steps), out))
        return list(out[:len({(int(n), 0) for n in self.n_beads})])

    def set_integrator(self, integrator: int) -> None:
        """SFP_INTEGRATOR_MODES (Sec. 4) or SFP_INTEGRATOR_EULER (bead-position Euler, Sec. 3A)."""
        _lib.check(_lib.load().sfp_set_integrator(self._h, int(integrator)))

    def set_sampling(self, every_steps: int) -> None:
        """Sample observables i-iii, mode power and CoM windows every ``every_steps`` steps."""
        _lib.check(_lib.load().sfp_set_sampling(self._h, int(every_steps)))
        if every_steps > 0:
            self._n_lags = self._lags_next

    def set_msd_lags(self, lags) -> None:
        """Lags (in sampling intervals, 1..8 of them) of the CoM and middle-bead MSD
        windows, used from the next ``set_sampling``."""
        a = (ct.c_int32 * len(lags))(*[int(x) for x in lags])
        _lib.check(_lib.load().sfp_set_msd_lags(self._h, len(lags), a))
        self._lags_next = len(lags)

    def observe(self, what: int):
        L = _lib.load()
        if what in (SFP_OBS_MODES, SFP_OBS_MODES_F32, SFP_OBS_POSITIONS, SFP_OBS_MODE_POWER, SFP_OBS_MODE_VAR):
            out = np.zeros(int(self.offsets[-1]), dtype=np.float32 if what == SFP_OBS_MODES_F32 else np.float64)
            _lib.check(L.sfp_observe(self._h, what, out.ctypes.data, out.nbytes))
            return self._unpack(out)
        if what == SFP_OBS_COM:
            out = np.zeros((self.n_chains, 3))
        elif what == SFP_OBS_STEP:
            out = np.zeros(self.n_chains, dtype=np.int64)
        elif what in (SFP_OBS_SHAPE, SFP_OBS_ACCUM):
            out = np.zeros((self.n_chains, 4))
        elif what in (SFP_OBS_COM_MSD, SFP_OBS_MID_MSD, SFP_OBS_E2E_MSD, SFP_OBS_BOND_MSD):
            out = np.zeros((self.n_chains, self._n_lags, 2))
        elif what == SFP_OBS_E2E2_MEAN:
            out = np.zeros(self.n_chains)
        else:
            raise ValueError(what)
        _lib.check(L.sfp_observe(self._h, what, out.ctypes.data, out.nbytes))
        return out

    def modes(self):
        return self.observe(SFP_OBS_MODES)

    def positions_nm(self):
        return self.observe(SFP_OBS_POSITIONS)

    def probe(self, what: int):
        out = np.zeros(int(self.offsets[-1]))
        _lib.check(_lib.load().sfp_probe(self._h, what, out.ctypes.data, out.nbytes))
        return self._unpack(out)

    def save(self) -> bytes:
        L = _lib.load()
        need = ct.c_size_t()
        _lib.check(L.sfp_save(self._h, None, 0, ct.byref(need)))
        buf = ct.create_string_buffer(need.value)
        _lib.check(L.sfp_save(self._h, buf, need.value, ct.byref(need)))
        return buf.raw

    def load(self, blob: bytes) -> None:
        _lib.check(_lib.load().sfp_load(self._h, blob, len(blob)))

    def stage_timing(self, enable: bool = True) -> None:
        _lib.check(_lib.load().sfp_stage_timing(self._h, int(bool(enable))))

    def stage_times(self) -> dict:
        """Average device time per group-step of each stage, in microseconds."""
        out = (ct.c_double * 6)()
        n = ct.c_int64()
        _lib.check(_lib.load().sfp_stage_times(self._h, out, ct.byref(n)))
        k = max(1, n.value)
        names = ("inverse_us", "force_us", "noise_us", "forward_us", "update_us", "step_us")
        d = {nm: out[i] / k for i, nm in enumerate(names)}
        d["group_steps"] = n.value
        return d

    def info(self) -> dict:
        out = (ct.c_int64 * 4)()
        _lib.check(_lib.load().sfp_info(self._h, out))
        return {"chains": out[0], "beads": out[1], "device_bytes": out[2], "launches": out[3]}


class Server:
    """Continuous-batching request loop (``sfp_server_*``): submit jobs at any
    time, poll finished ones.  A job is a dict with ``n_beads``, ``n_steps``,
    one of ``dt_ps`` / ``dtau``, optional ``shear_rate_per_s`` and ``job_id``."""

    def __init__(self, params: SfpParams | None = None, seed: int = 1, precision: int = SFP_FP32,
                 slots_per_pool: int = 512, quantum_steps: int = 64, keep_results: bool = True,
                 hbm_budget_bytes: int = 0):
        L = _lib.load()
        cfg = _lib.SfpServerConfig()
        _lib.check_server(L.sfp_server_config_default(ct.byref(cfg)))
        cfg.seed, cfg.precision, cfg.slots_per_pool = seed, precision, slots_per_pool
        cfg.quantum_steps, cfg.keep_results, cfg.hbm_budget_bytes = quantum_steps, int(keep_results), hbm_budget_bytes
        self.params = params or params_dsdna()
        h = ct.c_void_p()
        _lib.check_server(L.sfp_server_create(ct.byref(self.params), ct.byref(cfg), ct.byref(h)))
        self._h = h
        self._beads = {}

    def submit(self, job: dict) -> int:
        j = _lib.SfpJob()
        j.n_beads = int(job["n_beads"])
        j.dt_ps = float(job.get("dt_ps", 0.0))
        j.dtau = float(job.get("dtau", 0.0))
        j.shear_rate_per_s = float(job.get("shear_rate_per_s", 0.0))
        j.n_steps = int(job["n_steps"])
        j.job_id = int(job.get("job_id", 0))
        t = ct.c_uint64()
        _lib.check_server(_lib.load().sfp_server_submit(self._h, ct.byref(j), ct.byref(t)))
        self._beads[t.value] = j.n_beads
        return t.value

    def poll(self, max_results: int = 1024) -> list:
        arr = (_lib.SfpJobResult * max_results)()
        n = ct.c_int32()
        _lib.check_server(_lib.load().sfp_server_poll(self._h, arr, max_results, ct.byref(n)))
        out = []
        for r in arr[:n.value]:
            out.append({"ticket": r.ticket, "job_id": r.job_id, "n_beads": r.n_beads, "status": r.status,
                        "n_steps": r.n_steps, "submit_s": r.submit_s, "admit_s": r.admit_s,
                        "finish_s": r.finish_s, "latency_s": r.finish_s - r.submit_s,
                        "com_nm": list(r.com_nm)})
        return out

    def modes(self, ticket: int) -> np.ndarray:
        M = self._beads[ticket]
        out = np.zeros((3, M))
        _lib.check_server(_lib.load().sfp_server_result_modes(self._h, ticket, out.ctypes.data, out.size))
        return out

    def wait_idle(self, timeout_s: float = 600.0) -> None:
        _lib.check_server(_lib.load().sfp_server_wait_idle(self._h, float(timeout_s)))

    def stats(self) -> dict:
        out = (ct.c_double * 10)()
        _lib.check_server(_lib.load().sfp_server_stats(self._h, out))
        keys = ("submitted", "finished", "waiting", "running", "device_bytes", "p50_s", "p99_s", "max_s",
                "clock_s", "bead_steps")
        return dict(zip(keys, list(out)))

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            _lib.load().sfp_server_destroy(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
