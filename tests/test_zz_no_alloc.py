"""The allocation-free step, sfp_step_noalloc, checked against sfp_step.

Some callers cannot allocate device memory: code inside a host framework that
owns every device buffer (its own pool or a budget enforced elsewhere), or a
latency-critical loop in which a cudaMalloc, which may synchronise the whole
device, would stall other streams.  For them the library has one entry point
whose scratch and tables live in a static device array.  This test calls it
through the C ABI on caller-owned device buffers (allocated here with torch)
twice in a row, and compares each result with an SFP_FP32_SIMT batch advanced
by sfp_step from the same start, within the trajectory tolerance used by the
other parity tests (1e-5 relative per chain).  A second case takes the
scalar branches of the kernels (100 beads, not a multiple of 4), a step given
in ps and a shear rate, and is also held against the oracle, whose step and
shear come from the paper's printed constants.  The file name makes pytest
collect it last.
"""
import ctypes as ct
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import C_PS, shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import _lib, build

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


@pytest.mark.parametrize("M,C,dtau,dt_ps,shear", [(256, 40, 100.0, 0.0, 0.0), (100, 8, 0.0, 7.96, 5.0e7)],
                         ids=["256bp", "100bp_ps_shear"])
def test_noalloc_step_matches_sfp_step_on_two_calls(M, C, dtau, dt_ps, shear):
    torch = pytest.importorskip("torch")
    n, seed, job0 = 25, 3, 500
    m = O.Model(M, dtau=dtau if dtau > 0 else dt_ps / C_PS)
    R0 = np.stack([m.equilibrium_start(seed, job0 + c) for c in range(C)])
    R0[:, :, 0] = np.array([0.5, -1.0, 2.0]) * math.sqrt(M)        # off-origin centre of mass

    ref = sfp.Batch([{"n_beads": M, "dtau": dtau, "dt_ps": dt_ps, "shear_rate_per_s": shear, "job_id": job0 + c}
                     for c in range(C)], seed=seed, precision=sfp.SFP_FP32_SIMT)
    ref.set_modes(R0)

    init = R0.copy()
    init[:, :, 0] = 0.0
    modes = torch.tensor(init, dtype=torch.float32, device="cuda")          # caller-owned state
    com = torch.tensor(R0[:, :, 0] / math.sqrt(M), dtype=torch.float64, device="cuda")
    params = sfp.params_dsdna()
    desc = _lib.SfpChainDesc(n_beads=M, reserved=0, dt_ps=dt_ps, dtau=dtau, shear_rate_per_s=shear, job_id=job0)
    L = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        _lib.check(L.sfp_step_noalloc(ct.byref(params), ct.byref(desc), C, seed, call * n,
                                      modes.data_ptr(), com.data_ptr(), n, stream))
        ref.step(n)
        torch.cuda.synchronize()
        G = ref.modes()
        mine = modes.double().cpu().numpy()
        assert np.all(mine[:, :, 0] == 0.0)
        mine[:, :, 0] = com.cpu().numpy() * math.sqrt(M)
        err = (np.linalg.norm((mine - G)[:, :, 1:].reshape(C, -1), axis=1)
               / np.linalg.norm(G[:, :, 1:].reshape(C, -1), axis=1))
        assert err.max() < TOL, (call, err.max())
        assert np.abs(mine[:, :, 0] - G[:, :, 0]).max() < 1e-9 * math.sqrt(M) + 1e-6 * np.abs(G[:, :, 0]).max()
    if shear:
        # the step and shear conversions of the entry point against the oracle
        O_ref = m.run_modes(R0, seed, job0 + np.arange(C), 0, 2 * n, shear=shear_tau(shear))
        err = (np.linalg.norm((mine - O_ref)[:, :, 1:].reshape(C, -1), axis=1)
               / np.linalg.norm(O_ref[:, :, 1:].reshape(C, -1), axis=1))
        assert err.max() < TOL, err.max()
    ref.close()


def test_noalloc_rejects_requests_beyond_the_static_array():
    torch = pytest.importorskip("torch")
    params = sfp.params_dsdna()
    desc = _lib.SfpChainDesc(n_beads=512, reserved=0, dt_ps=0.0, dtau=100.0, shear_rate_per_s=0.0, job_id=0)
    modes = torch.zeros(1, dtype=torch.float32, device="cuda")
    com = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = _lib.load().sfp_step_noalloc(ct.byref(params), ct.byref(desc), 100000, 1, 0, modes.data_ptr(),
                                      com.data_ptr(), 1, None)
    assert rc == _lib.SFP_EINVAL
    assert "static array" in _lib.load().sfp_last_error().decode()
