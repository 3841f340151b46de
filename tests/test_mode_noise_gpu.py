"""Mode-keyed noise (SFP_NOISE_MODES, the reading of Eq. c4 in which Z is drawn
per mode): every path against the oracle's mode-keyed integrator on the same
starts and keys, at the tolerances of the bead-noise parity tests."""
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu

DT = {64: 10.0, 100: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def rel_err(G, R):
    C = G.shape[0]
    d = (G - R)[:, :, 1:].reshape(C, -1)
    return np.linalg.norm(d, axis=1) / np.linalg.norm(R[:, :, 1:].reshape(C, -1), axis=1)


def run_pair(M, C, precision, path, steps, calls=1, rates=None, seed=5):
    dtau = DT[M]
    rates = rates if rates is not None else [0.0] * C
    chains = [{"n_beads": M, "dtau": dtau, "job_id": 40 + c, "shear_rate_per_s": rates[c]} for c in range(C)]
    m = O.Model(M, dtau=dtau)
    R0 = np.stack([m.equilibrium_start(seed, 40 + c) for c in range(C)])
    b = sfp.Batch(chains, seed=seed, precision=precision)
    b.set_path(path)
    b.set_noise(sfp.SFP_NOISE_MODES)
    b.set_modes(R0)
    for _ in range(calls):
        b.step(steps // calls)
    G = b.modes()
    b.close()
    ref = np.stack([m.run_modes(R0[c][None], seed, [40 + c], 0, steps, shear=shear_tau(rates[c]),
                                mode_noise=True)[0] for c in range(C)])
    return G, ref, R0


@pytest.mark.parametrize("precision", [sfp.SFP_MIXED_BF16, sfp.SFP_MIXED_TF32], ids=["bf16x3", "tf32x3"])
@pytest.mark.parametrize("M,C", [(64, 37), (128, 21), (256, 30)])
def test_fused_mode_noise_against_the_oracle(precision, M, C):
    """The fused step without noise blocks: the noise warps draw Z one step
    ahead into a two-step buffer and the epilogue adds w_p Z_p; 500 steps in
    calls of 250 (two launches), a third of the chains sheared."""
    rates = [1.0e8 if c % 3 == 0 else 0.0 for c in range(C)]
    G, ref, _ = run_pair(M, C, precision, sfp.SFP_PATH_FUSED, 500, calls=2, rates=rates)
    err = rel_err(G, ref)
    assert err.max() < 1e-5, err.max()
    assert np.abs(G[:, :, 0] - ref[:, :, 0]).max() < 1e-6 * (1 + np.abs(ref[:, :, 0]).max())


@pytest.mark.parametrize("M", [64, 256])
def test_fused_mode_noise_one_call_equals_many(M):
    """A launch of many steps draws the same Z as launches of one step."""
    C = 24
    a, _, _ = run_pair(M, C, sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED, 40, calls=1)
    b, _, _ = run_pair(M, C, sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED, 40, calls=40)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("precision,path,M,tol",
                         [(sfp.SFP_FP32_SIMT, sfp.SFP_PATH_STAGED, 100, 1e-5),
                          (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_STAGED, 256, 1e-5),
                          (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED, 512, 1e-5),
                          (sfp.SFP_FP64, sfp.SFP_PATH_FUSED, 64, 1e-9),
                          (sfp.SFP_FP64, sfp.SFP_PATH_STAGED, 100, 1e-9)],
                         ids=["simt_100bp", "staged_bf16_256bp", "512bp_on_staged", "fp64_cluster", "fp64_staged"])
def test_other_paths_mode_noise_against_the_oracle(precision, path, M, tol):
    """The staged kernels (Z drawn straight into the mode-space buffer, the
    forward transform's force half alone), 512 beads (staged under mode noise)
    and the FP64 kernels (a cluster per chain for few chains)."""
    C = 6
    G, ref, _ = run_pair(M, C, precision, path, 200, rates=[0.0, 5e7, 0.0, 0.0, 1e8, 0.0])
    err = rel_err(G, ref)
    assert err.max() < tol, err.max()


def test_mode_noise_is_not_the_bead_noise_and_rejects_unknown_keying():
    M, C = 64, 8
    chains = [{"n_beads": M, "dtau": 10.0, "job_id": c} for c in range(C)]
    out = []
    for keying in (sfp.SFP_NOISE_BEADS, sfp.SFP_NOISE_MODES):
        b = sfp.Batch(chains, seed=2, precision=sfp.SFP_MIXED_BF16)
        b.init_equilibrium(0)
        b.set_noise(keying)
        b.step(3)
        out.append(b.modes())
        if keying == sfp.SFP_NOISE_MODES:
            with pytest.raises(sfp.SfpError):
                b.set_noise(7)
        b.close()
    assert not np.allclose(out[0], out[1])
