"""Paper experiments on the GPU path: the Fig. 1 ratio of the full to the
residual mode force, and the headless tumbling run of Sec. 8."""
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import C_PS, PAPER, shear_tau
from oracle import oracle as O
from paper_1411_3487_gb300 import build
from paper_1411_3487_gb300.tumbling import run_tumbling

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_fig1_full_to_residual_force_ratio():
    """[<H_p^2>/<DeltaH_p^2>]^(1/2) over an equilibrium ensemble at N = 63
    (Fig. 1), with H_p = (1-2nu) 4 sin^2(theta_p/2) R_p + DeltaH_p (Eqs. e8, e10).
    The residual force is small for the slow modes (ratio >> 1 at low p).  The
    GPU's sums over its first chains equal the oracle's on the same trajectory."""
    M, C, dtau, nu, sub = 64, 512, 10.0, 0.35, 8
    m = O.Model(M, dtau=dtau)
    b = sfp.Batch([{"n_beads": M, "dtau": dtau}] * C, seed=6, precision=sfp.SFP_FP32)
    b.set_path(sfp.SFP_PATH_STAGED)            # keeps DeltaH for the probe
    b.init_equilibrium(0)
    b.step(400)
    R = b.modes()[:sub].copy()                  # the oracle follows these chains from here
    coef = (1 - 2 * nu) * 4 * np.sin(0.5 * np.pi * np.arange(M) / M) ** 2
    num, den = np.zeros(M), np.zeros(M)         # whole GPU ensemble
    gnum, gden, onum, oden = np.zeros(M), np.zeros(M), np.zeros(M), np.zeros(M)
    step = 400
    for _ in range(20):
        b.step(25)
        Rg = b.modes()
        b.step(1)                               # its DeltaH is the force of state Rg
        dH = b.probe(sfp.SFP_PROBE_DH)
        H = coef * Rg + dH
        num += np.sum(H ** 2, axis=(0, 1))
        den += np.sum(dH ** 2, axis=(0, 1))
        gnum += np.sum(H[:sub] ** 2, axis=(0, 1))
        gden += np.sum(dH[:sub] ** 2, axis=(0, 1))
        R = m.run_modes(R, 6, np.arange(sub), step, 25)
        for c in range(sub):
            dHo = m.delta_H(m.modes_to_beads(R[c]))
            onum += np.sum((coef * R[c] + dHo) ** 2, axis=0)
            oden += np.sum(dHo ** 2, axis=0)
        R = m.run_modes(R, 6, np.arange(sub), step + 25, 1)
        step += 26
    ratio = np.sqrt(num[1:] / den[1:])
    print("Fig. 1 ratio p = 1..8:", np.round(ratio[:8], 1), "last 8:", np.round(ratio[-8:], 2))
    assert ratio[0] > 10 and ratio[:4].mean() > 3 * ratio[-8:].mean()
    assert np.abs(np.sqrt(gnum[1:] / gden[1:]) / np.sqrt(onum[1:] / oden[1:]) - 1).max() < 1e-2


def test_headless_tumbling_snapshots():
    """Sec. 8 run at its parameters, shortened: 255 bp, 1.54e8 1/s, 16 ps steps,
    snapshots 8 ns apart, written as positions (nm); the first snapshots equal
    the oracle's sheared trajectory from the same start."""
    n = 6
    pos = run_tumbling(n_snapshots=n)
    assert pos.shape == (n + 1, 3, 255) and np.isfinite(pos).all()
    dtau = 16.0 / C_PS                       # 16 ps steps, c from the printed values (Eq. g2)
    d_nm = PAPER["a_nm"] * (1.0 - 2.0 * PAPER["nu"])
    m = O.Model(255, dtau=dtau)
    R = m.equilibrium_start(1, 0)
    steps = int(round(8.0e3 / 16.0))
    R1 = m.run_modes(R[None], 1, [0], 0, steps, shear=shear_tau(1.54e8))[0]
    ref = m.modes_to_beads(R1) * d_nm
    err = np.linalg.norm(pos[1] - ref) / np.linalg.norm(ref - ref.mean(axis=1, keepdims=True))
    assert err < 1e-5
