"""The default bead-position Euler scheme on the GPU (Sec. 3A, Eqs. b3-b5)
against the oracle's Euler integrator, same bead noise, through the C ABI."""
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def rel_err(A, B):
    A, B = np.asarray(A)[:, :, 1:], np.asarray(B)[:, :, 1:]
    return np.linalg.norm((A - B).reshape(len(A), -1), axis=1) / np.linalg.norm(B.reshape(len(B), -1), axis=1)


@pytest.mark.parametrize("precision,tol", [(sfp.SFP_FP32, 1e-5), (sfp.SFP_FP32_SIMT, 1e-5),
                                           (sfp.SFP_FP64, 1e-10)], ids=["fp32_tc", "fp32_simt", "fp64"])
@pytest.mark.parametrize("M,C,shear", [(64, 9, 0.0), (67, 4, 1.0e9), (256, 5, 0.0)])
def test_euler_matches_oracle(precision, tol, M, C, shear):
    dtau, n = 0.1, 300
    m = O.Model(M, dtau=dtau)
    R0 = np.stack([m.equilibrium_start(2, j) for j in range(C)])
    R0[:, :, 0] = np.array([0.5, -1.0, 2.0]) * math.sqrt(M)        # centre of mass off the origin
    b = sfp.Batch([{"n_beads": M, "dtau": dtau, "shear_rate_per_s": shear}] * C, seed=2, precision=precision)
    b.set_modes(R0)
    b.set_integrator(sfp.SFP_INTEGRATOR_EULER)
    b.step(120)
    b.step(n - 120)                                                # two calls: conversions in between
    G = b.modes()
    r0 = np.stack([m.modes_to_beads(x) for x in R0])
    r = m.run_euler(r0, 2, np.arange(C), 0, n, shear=shear_tau(shear))
    ref = np.stack([m.beads_to_modes(x) for x in r])
    assert rel_err(G, ref).max() < tol
    # centre of mass: FP64 on both sides, noise projected in FP32 or FP64
    dcm = np.abs(G[:, :, 0] - ref[:, :, 0]).max() / math.sqrt(M)
    assert dcm < (1e-5 if precision != sfp.SFP_FP64 else 1e-11) * math.sqrt(6 * 0.034 * dtau * n / M) + 1e-12
    assert np.all(b.observe(sfp.SFP_OBS_STEP) == n)


def test_euler_then_modes_continue_one_trajectory():
    """Switching integrators keeps the state and the step counter: Euler steps
    then mode-space steps equal the oracle doing the same."""
    M, C, dtau = 64, 6, 0.1
    m = O.Model(M, dtau=dtau)
    R0 = np.stack([m.equilibrium_start(4, j) for j in range(C)])
    b = sfp.Batch([{"n_beads": M, "dtau": dtau}] * C, seed=4, precision=sfp.SFP_FP64)
    b.set_modes(R0)
    b.set_integrator(sfp.SFP_INTEGRATOR_EULER)
    b.step(50)
    b.set_integrator(sfp.SFP_INTEGRATOR_MODES)
    b.step(50)
    r = m.run_euler(np.stack([m.modes_to_beads(x) for x in R0]), 4, np.arange(C), 0, 50)
    R = np.stack([m.beads_to_modes(x) for x in r])
    R = m.run_modes(R, 4, np.arange(C), 50, 50)
    assert rel_err(b.modes(), R).max() < 1e-10
