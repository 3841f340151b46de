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
