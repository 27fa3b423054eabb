"""Reader for tests/golden/paper_values.txt (numbers printed in the paper)."""
import os

_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_values.txt")


def load():
    out = {}
    with open(_PATH) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, vals, _cite = [s.strip() for s in line.split("|")]
            out[name] = [float(v) for v in vals.split()]
    return out
