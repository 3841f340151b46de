"""Headless tumbling run under steady shear (Sec. 8): one chain in the flow
v = gamma-dot y x, snapshots of the absolute bead positions written as an
array instead of a movie.  The paper's run: 255 bp, gamma-dot = 1.54e8 1/s,
dt = 16 ps, 3000 snapshots 8 ns apart."""
from __future__ import annotations

import numpy as np

from . import SFP_FP32, Batch


def run_tumbling(n_beads: int = 255, shear_rate_per_s: float = 1.54e8, dt_ps: float = 16.0,
                 snapshot_ns: float = 8.0, n_snapshots: int = 3000, seed: int = 1, job_id: int = 0,
                 precision: int = SFP_FP32, out_path: str | None = None) -> np.ndarray:
    """Positions [n_snapshots + 1][3][n_beads] in nm (snapshot 0 = the start);
    saved with numpy.save when out_path is given."""
    steps = max(1, int(round(snapshot_ns * 1e3 / dt_ps)))
    b = Batch([{"n_beads": n_beads, "dt_ps": dt_ps, "shear_rate_per_s": shear_rate_per_s, "job_id": job_id}],
              seed=seed, precision=precision)
    b.init_equilibrium(0)
    out = np.zeros((n_snapshots + 1, 3, n_beads))
    out[0] = b.positions_nm()[0]
    for k in range(1, n_snapshots + 1):
        b.step(steps)
        out[k] = b.positions_nm()[0]
    b.close()
    if out_path:
        np.save(out_path, out)
    return out
