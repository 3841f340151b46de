"""Largest step from the equilibrium quantities (Sec. 5B, Fig. 2, Table 1
column 2) on the GPU path: for N = 63 the equilibrium <|L|^2>, <|u_m|^2> and
<|r_m - r_cm|^2> of the dynamics lie within 5% of the Monte Carlo benchmark
(Sec. 5A) for every step up to the paper's dtau_max of 50."""
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu

# Table 1, N = 63: dtau_max from equilibrium quantities (column 2)
DTAU_MAX_EQ_63 = 50.0


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_dtau_max_from_equilibrium_quantities_64bp():
    """Scan dtau = 10, 20, 50, 100, 200 at N = 63: 4096 chains relaxed for
    2e5 tau, then sampled over 2e5 tau every 1000 tau (every 5 steps at
    dtau = 200), tensor-core path.  Monte Carlo: the oracle's sampler, 64
    chains x 2e4 sweeps after tuning.  Prints the scan; requires the 5%
    criterion for every dtau <= 50."""
    M = 64
    m = O.Model(M, dtau=10.0)
    Cm = 64
    R = np.stack([m.equilibrium_start(9, j) for j in range(Cm)])
    step, R = m.mc_tuned_steps(R, 9, np.arange(Cm))
    R, _, _ = m.run_mc(R, 9, np.arange(Cm), 0, 4000, step)
    R, _, obs = m.run_mc(R, 9, np.arange(Cm), 4000, 20000, step, sample=True)
    mc_per = obs[:, :3] / obs[:, 3:4]
    mc = mc_per.mean(axis=0)
    mc_se = mc_per.std(axis=0, ddof=1) / math.sqrt(Cm)
    d2 = sfp.derive()["d_nm"] ** 2
    rows = []
    for dtau in (10.0, 20.0, 50.0, 100.0, 200.0):
        n_relax = int(round(2e5 / dtau))
        every = max(1, int(round(1e3 / dtau)))
        b = sfp.Batch([{"n_beads": M, "dtau": dtau}] * 4096, seed=11, precision=sfp.SFP_FP32)
        b.init_equilibrium(0)
        b.step(n_relax)
        b.set_sampling(every)
        b.step(n_relax)
        acc = b.observe(sfp.SFP_OBS_ACCUM)
        per = acc[:, :3] / acc[:, 3:4] / d2
        ratio = per.mean(axis=0) / mc
        se = np.hypot(per.std(axis=0, ddof=1) / math.sqrt(len(per)) / mc, mc_se / mc)
        rows.append((dtau, ratio, se))
        b.close()
    print("MC <|L|^2>, <|u_m|^2>, <|r_m - r_cm|^2> (d^2):", mc, "+-", mc_se)
    for dtau, ratio, se in rows:
        ok = np.all(np.abs(ratio - 1) < 0.05)
        print(f"dtau {dtau:6.1f}: GPU/MC {np.round(ratio, 4)} +- {np.round(se, 4)}  {'within 5%' if ok else 'outside 5%'}")
    for dtau, ratio, _ in rows:
        if dtau <= DTAU_MAX_EQ_63:
            assert np.all(np.abs(ratio - 1) < 0.05), (dtau, ratio)
