import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def load_golden(name="cases.txt"):
    """Parse tests/golden/cases.txt into a list of dicts."""
    from fractions import Fraction
    path = os.path.join(ROOT, "tests", "golden", name)
    cases, cur = [], None
    for raw in open(path):
        line = raw.strip()
        if not line or line.startswith("#"):
            continue
        key, _, rest = line.partition(" ")
        vals = rest.split()
        if key == "case":
            cur = {"name": rest.strip(), "frames": None}
            cases.append(cur)
        elif key in ("order", "T", "stride"):
            cur[key] = int(vals[0])
        elif key == "spikes":
            cur["spikes"] = [int(v) for v in vals]
        elif key == "segments":
            cur["segments"] = [tuple(int(u) for u in v.split(":")) for v in vals]
        elif key == "frames":
            cur["frames"] = [Fraction(v) for v in vals]
        else:
            raise ValueError(f"unknown key {key!r} in {path}")
    return cases
