"""Reader for ``tests/golden/paper_constants.txt`` (values printed in the paper)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.txt")


def load() -> dict:
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            kv, _cite = line.split("|", 1)
            k, v = kv.split("=", 1)
            out[k.strip()] = float(v)
    return out


PAPER = load()

# c = T* (1 - 2 nu)^2 a^2 xi / kT (Eq. g2) from the printed values alone: the
# scaled time unit in ps, and a shear rate in 1/s as a rate per unit of scaled
# time (Eq. btum).  Tests convert shear rates with these, never with the
# library's own constant.
C_PS = PAPER["Tstar"] * (1.0 - 2.0 * PAPER["nu"]) ** 2 * PAPER["a2xi_over_kT_ps"]


def shear_tau(rate_per_s: float) -> float:
    return rate_per_s * C_PS * 1e-12
