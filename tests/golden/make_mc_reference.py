"""Write tests/golden/mc_reference.txt: the oracle's Monte Carlo benchmark of the
equilibrium observables (Sec. 5A) that the step-size scans of Sec. 5B compare
with (Fig. 2, Table 1 column 2).

Calls only the oracle (oracle/oracle.py): for each chain length, 64 chains from
the oracle's equilibrium starts (seed 9), per-mode step sizes tuned toward 40%
acceptance, 4000 sweeps of burn-in, then 2e4 sweeps sampled every sweep;
per-chain means of |L|^2, |u_m|^2, |r_m - r_cm|^2 in scaled units (d^2), and
over chains their mean and standard error.  Run from the repository root:

    python tests/golden/make_mc_reference.py 64 128 256 512
"""
import math
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
from oracle import oracle as O  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "mc_reference.txt")
CHAINS, SEED, BURN, SWEEPS = 64, 9, 4000, 20000


def run(M):
    m = O.Model(M, dtau=10.0)
    R = np.stack([m.equilibrium_start(SEED, j) for j in range(CHAINS)])
    step, R = m.mc_tuned_steps(R, SEED, np.arange(CHAINS))
    R, _, _ = m.run_mc(R, SEED, np.arange(CHAINS), 0, BURN, step)
    R, _, obs = m.run_mc(R, SEED, np.arange(CHAINS), BURN, SWEEPS, step, sample=True)
    per = obs[:, :3] / obs[:, 3:4]
    return per.mean(axis=0), per.std(axis=0, ddof=1) / math.sqrt(CHAINS)


def main(lengths):
    rows = {}
    if os.path.exists(OUT):
        for line in open(OUT):
            if line.strip() and not line.startswith("#"):
                rows[int(line.split()[0])] = line
    for M in lengths:
        mean, se = run(M)
        rows[M] = f"{M:4d} " + " ".join(f"{x:.10e}" for x in (*mean, *se)) + "\n"
        print(rows[M], end="", flush=True)
    with open(OUT, "w") as f:
        f.write("# Monte Carlo benchmark (Sec. 5A) of the equilibrium observables i-iii, written by\n"
                "# tests/golden/make_mc_reference.py from the oracle alone: dsDNA (T* = 0.034, nu = 0.35),\n"
                f"# {CHAINS} chains, seed {SEED}, tuned single-mode moves, {BURN} burn-in + {SWEEPS} sampled sweeps.\n"
                "# beads  <|L|^2>  <|u_m|^2>  <|r_m - r_cm|^2>  (means over chains, d^2)  then their standard errors\n")
        for M in sorted(rows):
            f.write(rows[M])


if __name__ == "__main__":
    main([int(x) for x in sys.argv[1:]] or [64, 128, 256, 512])
