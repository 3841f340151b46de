"""The step-size tests of Sec. 5B on the GPU path.

Table 1 lists, per chain length, the largest usable step dtau_max from two
groups of quantities: the equilibrium values Q(0) of (i) the end-to-end
vector L, (ii) the middle bond u_m and (iii) the middle bead relative to the
centre of mass (within 5% of a Monte Carlo benchmark, Fig. 2), and their time
dependence Q(t) (the effective decay constant ln(Q(2t)/Q(t))/t within 10% of
the smallest step's, Fig. 3).  Fig. 4 shows the Q(t) curves of N = 255 for
dtau_min .. dtau_max on top of each other.

Everything here runs through the library's public calls: the equilibrium
sums (SFP_OBS_ACCUM) and the lag windows of L, u_m and r_m - r_cm
(SFP_OBS_E2E_MSD, SFP_OBS_BOND_MSD, SFP_OBS_MID_MSD).  For a stationary chain
the autocorrelation follows from the windows, <X(t).X(0)> = <X^2> - <|X(t) -
X(0)|^2> / 2.  Lengths are returned in nm, times in scaled units tau.
"""
from __future__ import annotations

import numpy as np

from . import (SFP_FP32, SFP_OBS_ACCUM, SFP_OBS_BOND_MSD, SFP_OBS_E2E_MSD, SFP_OBS_MID_MSD, Batch)


def equilibrium_values(M: int, dtau: float, chains: int = 4096, relax_tau: float = 2e5, samples: int = 200,
                       seed: int = 11, precision: int = SFP_FP32) -> np.ndarray:
    """Per-chain equilibrium means of |L|^2, |u_m|^2, |r_m - r_cm|^2 (nm^2), shape
    [chains][3]: equilibrium starts, `relax_tau` of relaxation, then `samples`
    samples spread over another `relax_tau`."""
    n = max(1, int(round(relax_tau / dtau)))
    with Batch([{"n_beads": M, "dtau": dtau}] * chains, seed=seed, precision=precision) as b:
        b.init_equilibrium(0)
        b.step(n)
        b.set_sampling(max(1, n // samples))
        b.step(n)
        acc = b.observe(SFP_OBS_ACCUM)
    return acc[:, :3] / acc[:, 3:4]


def dynamic_q(M: int, dtau: float, lags_tau, sample_tau: float, run_tau: float, chains: int = 2048,
              relax_tau: float = 2e4, seed: int = 21, precision: int = SFP_FP32) -> dict:
    """Q(t) of observables i-iii at the times `lags_tau` (at most 8, multiples of
    `sample_tau`, which must be a multiple of dtau): the normalised time
    autocorrelations of L and u_m and the mean-square displacement of r_m - r_cm
    (nm^2), from non-overlapping windows over `run_tau` after `relax_tau`."""
    every = int(round(sample_tau / dtau))
    if every < 1 or abs(every * dtau - sample_tau) > 1e-9 * sample_tau:
        raise ValueError("sample_tau must be a multiple of dtau")
    lags = [int(round(t / sample_tau)) for t in lags_tau]
    if any(l < 1 or abs(l * sample_tau - t) > 1e-9 * t for l, t in zip(lags, lags_tau)):
        raise ValueError("every lag must be a multiple of sample_tau")
    with Batch([{"n_beads": M, "dtau": dtau}] * chains, seed=seed, precision=precision) as b:
        b.init_equilibrium(0)
        b.step(int(round(relax_tau / dtau)))
        b.set_msd_lags(lags)
        b.set_sampling(every)
        b.step(every * int(round(run_tau / sample_tau)))
        acc = b.observe(SFP_OBS_ACCUM)
        w = {k: b.observe(k) for k in (SFP_OBS_E2E_MSD, SFP_OBS_BOND_MSD, SFP_OBS_MID_MSD)}
    mean = acc[:, :3].sum(axis=0) / acc[:, 3].sum()

    def ratio(k):
        return w[k][:, :, 0].sum(axis=0) / w[k][:, :, 1].sum(axis=0)

    return {"t": np.asarray(lags_tau, dtype=float), "dtau": dtau,
            "Q_L": 1.0 - ratio(SFP_OBS_E2E_MSD) / (2.0 * mean[0]),
            "Q_u": 1.0 - ratio(SFP_OBS_BOND_MSD) / (2.0 * mean[1]),
            "Q_msd": ratio(SFP_OBS_MID_MSD),
            "windows": w[SFP_OBS_MID_MSD][:, :, 1].sum(axis=0)}


def decay_ratio(q: dict, base: dict, taus) -> np.ndarray:
    """Ratio of effective decay constants ln(Q(2 tau)/Q(tau)) / tau of run `q`
    to those of the smallest-step run `base`, rows tau, columns L, u_m, msd (the
    1/tau cancels).  Both runs must hold the times tau and 2 tau."""
    t = list(q["t"])
    out = []
    for tau in taus:
        i, j = t.index(tau), t.index(2 * tau)
        row = []
        for k in ("Q_L", "Q_u", "Q_msd"):
            row.append(np.log(q[k][j] / q[k][i]) / np.log(base[k][j] / base[k][i]))
        out.append(row)
    return np.array(out)


def stack_curves(runs, path: str | None = None) -> dict:
    """Q(t) curves of several dynamic_q runs (the same times) as arrays
    [len(runs)][len(t)] of Q_L, Q_u, Q_msd with their steps; written to `path`
    (numpy .npz) when given: the headless form of Fig. 4."""
    out = {"t": np.asarray(runs[0]["t"], dtype=float), "dtau": np.asarray([r["dtau"] for r in runs], dtype=float)}
    for k in ("Q_L", "Q_u", "Q_msd"):
        out[k] = np.stack([r[k] for r in runs])
    if path:
        np.savez(path, **out)
    return out


def fig4_curves(dtaus=(1.0, 10.0, 50.0, 100.0), M: int = 256,
                lags_tau=(1e3, 3e3, 1e4, 2e4, 3e4, 1e5, 2e5, 3e5), sample_tau: float = 1e3, run_tau: float = 1e6,
                chains: int = 4096, relax_tau: float = 1e5, path: str | None = None, precision: int = SFP_FP32) -> dict:
    """The Q(t) curves of Fig. 4 (N = 255 by default) for each step in `dtaus`."""
    runs = [dynamic_q(M, d, lags_tau, sample_tau, run_tau, chains=chains, relax_tau=relax_tau, precision=precision)
            for d in dtaus]
    return stack_curves(runs, path)
