"""ctypes binding of ``libsfp.so`` (the C ABI of ``include/sfp.h``).

Argument marshalling only: every step of the simulation runs in the CUDA
library.  There is no fallback: if the library is missing or cannot be
loaded, every entry point raises.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libsfp.so")

SFP_OK, SFP_EINVAL, SFP_ENOMEM, SFP_ECUDA, SFP_ETIMEDOUT, SFP_ENONFINITE, SFP_ENOTSUP = 0, -1, -2, -3, -4, -5, -6
SFP_FP32, SFP_FP64, SFP_MIXED_BF16, SFP_FP32_SIMT = 0, 1, 2, 4
SFP_MIXED_TF32 = SFP_FP32   # FP32 state, TF32x3 transforms
SFP_MIXED_BF16_2 = 3        # FP32 state, two-pass BF16 transforms (tables rounded to BF16)
SFP_OBS_MODES, SFP_OBS_POSITIONS, SFP_OBS_COM, SFP_OBS_STEP, SFP_OBS_SHAPE = 0, 1, 2, 3, 4
SFP_OBS_ACCUM, SFP_OBS_MODE_POWER, SFP_OBS_COM_MSD = 5, 6, 7
SFP_OBS_MID_MSD, SFP_OBS_E2E2_MEAN, SFP_OBS_MODE_VAR, SFP_OBS_E2E_MSD, SFP_OBS_BOND_MSD = 8, 9, 10, 11, 12
SFP_OBS_MODES_F32 = 13
SFP_PATH_FUSED, SFP_PATH_STAGED = 0, 1
SFP_INTEGRATOR_MODES, SFP_INTEGRATOR_EULER = 0, 1
SFP_NOISE_BEADS, SFP_NOISE_MODES = 0, 1
SFP_PROBE_BONDS, SFP_PROBE_FORCE, SFP_PROBE_NOISE, SFP_PROBE_DH, SFP_PROBE_ZMODE = 0, 1, 2, 3, 4

# Every entry point declared in include/sfp.h.
EXPORTS = (
    "sfp_params_dsdna", "sfp_derive", "sfp_create", "sfp_init_equilibrium", "sfp_set_modes", "sfp_set_modes_f32",
    "sfp_set_positions", "sfp_set_step", "sfp_step", "sfp_observe", "sfp_probe", "sfp_save",
    "sfp_load", "sfp_info", "sfp_destroy", "sfp_last_error", "sfp_philox_words",
    "sfp_stage_timing", "sfp_stage_times", "sfp_step_noalloc", "sfp_set_sampling", "sfp_set_msd_lags",
    "sfp_set_path", "sfp_set_integrator", "sfp_set_graph", "sfp_set_grouped", "sfp_set_noise", "sfp_autotune", "sfp_server_config_default", "sfp_server_create", "sfp_server_submit",
    "sfp_server_poll", "sfp_server_result_modes", "sfp_server_wait_idle", "sfp_server_stats",
    "sfp_server_destroy", "sfp_server_last_error",
)


class SfpParams(ct.Structure):
    _fields_ = [("lambda_pN_per_nm", ct.c_double), ("kappa_pN_per_nm", ct.c_double),
                ("a_nm", ct.c_double), ("xi_kg_per_s", ct.c_double), ("kT_pN_nm", ct.c_double),
                ("T_star", ct.c_double), ("nu", ct.c_double), ("a2xi_over_kT_ps", ct.c_double)]


class SfpChainDesc(ct.Structure):
    _fields_ = [("n_beads", ct.c_int32), ("reserved", ct.c_int32), ("dt_ps", ct.c_double),
                ("dtau", ct.c_double), ("shear_rate_per_s", ct.c_double), ("job_id", ct.c_uint64)]


class SfpServerConfig(ct.Structure):
    _fields_ = [("seed", ct.c_uint64), ("precision", ct.c_int32), ("slots_per_pool", ct.c_int32),
                ("quantum_steps", ct.c_int32), ("keep_results", ct.c_int32), ("hbm_budget_bytes", ct.c_size_t)]


class SfpJob(ct.Structure):
    _fields_ = [("n_beads", ct.c_int32), ("reserved", ct.c_int32), ("dt_ps", ct.c_double),
                ("dtau", ct.c_double), ("shear_rate_per_s", ct.c_double), ("n_steps", ct.c_int64),
                ("job_id", ct.c_uint64)]


class SfpJobResult(ct.Structure):
    _fields_ = [("ticket", ct.c_uint64), ("job_id", ct.c_uint64), ("n_beads", ct.c_int32),
                ("status", ct.c_int32), ("n_steps", ct.c_int64), ("submit_s", ct.c_double),
                ("admit_s", ct.c_double), ("finish_s", ct.c_double), ("com_nm", ct.c_double * 3)]


class SfpError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sfp error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load the library (raises if it is absent: there is no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"CUDA library not built: {p} (run paper_1411_3487_gb300.build)")
        L = ct.CDLL(p)
        vp, sz, i32, i64, u32, u64 = ct.c_void_p, ct.c_size_t, ct.c_int32, ct.c_int64, ct.c_uint32, ct.c_uint64
        L.sfp_params_dsdna.argtypes = [ct.POINTER(SfpParams)]
        L.sfp_derive.argtypes = [ct.POINTER(SfpParams), ct.POINTER(ct.c_double)]
        L.sfp_create.argtypes = [ct.POINTER(SfpParams), ct.POINTER(SfpChainDesc), i32, u64, i32, vp, sz,
                                 ct.POINTER(vp)]
        L.sfp_init_equilibrium.argtypes = [vp, i64]
        L.sfp_set_modes.argtypes = [vp, vp, sz]
        L.sfp_set_modes_f32.argtypes = [vp, vp, sz]
        L.sfp_set_positions.argtypes = [vp, vp, sz]
        L.sfp_set_step.argtypes = [vp, i64]
        L.sfp_step.argtypes = [vp, i64]
        L.sfp_observe.argtypes = [vp, i32, vp, sz]
        L.sfp_probe.argtypes = [vp, i32, vp, sz]
        L.sfp_save.argtypes = [vp, vp, sz, ct.POINTER(sz)]
        L.sfp_load.argtypes = [vp, vp, sz]
        L.sfp_info.argtypes = [vp, ct.POINTER(i64)]
        L.sfp_destroy.argtypes = [vp]
        L.sfp_last_error.restype = ct.c_char_p
        L.sfp_philox_words.argtypes = [u32, u32, i64, u32, i32, vp]
        L.sfp_stage_timing.argtypes = [vp, i32]
        L.sfp_stage_times.argtypes = [vp, ct.POINTER(ct.c_double), ct.POINTER(i64)]
        L.sfp_set_sampling.argtypes = [vp, i32]
        L.sfp_set_path.argtypes = [vp, i32]
        L.sfp_set_integrator.argtypes = [vp, i32]
        L.sfp_set_graph.argtypes = [vp, i32]
        L.sfp_set_grouped.argtypes = [vp, i32]
        L.sfp_set_noise.argtypes = [vp, i32]
        L.sfp_autotune.argtypes = [vp, i32, vp]
        L.sfp_server_config_default.argtypes = [ct.POINTER(SfpServerConfig)]
        L.sfp_server_create.argtypes = [ct.POINTER(SfpParams), ct.POINTER(SfpServerConfig), ct.POINTER(vp)]
        L.sfp_server_submit.argtypes = [vp, ct.POINTER(SfpJob), ct.POINTER(u64)]
        L.sfp_server_poll.argtypes = [vp, ct.POINTER(SfpJobResult), i32, ct.POINTER(i32)]
        L.sfp_server_result_modes.argtypes = [vp, u64, vp, sz]
        L.sfp_server_wait_idle.argtypes = [vp, ct.c_double]
        L.sfp_server_stats.argtypes = [vp, ct.POINTER(ct.c_double)]
        L.sfp_server_destroy.argtypes = [vp]
        L.sfp_server_last_error.restype = ct.c_char_p
        L.sfp_step_noalloc.argtypes = [ct.POINTER(SfpParams), ct.POINTER(SfpChainDesc), i32, u64, i64, vp, vp,
                                       i64, vp]
        for name in EXPORTS:
            if name not in ("sfp_last_error", "sfp_server_last_error"):
                getattr(L, name).restype = ct.c_int
        _lib = L
        return _lib


def check(rc: int) -> None:
    if rc != SFP_OK:
        raise SfpError(rc, load().sfp_last_error().decode())


def check_server(rc: int) -> None:
    if rc != SFP_OK:
        raise SfpError(rc, load().sfp_server_last_error().decode())
