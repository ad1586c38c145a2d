import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: large sizes; still part of the default suite")


def load_grid(name):
    """Reads a golden grid file; returns {(x, y): key} (rows are printed top row first)."""
    path = os.path.join(ROOT, "tests", "golden", name)
    rows = []
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(t) for t in line.split()])
    side = len(rows)
    out = {}
    for r, vals in enumerate(rows):
        y = side - 1 - r
        for x, v in enumerate(vals):
            out[(x, y)] = v
    return out
