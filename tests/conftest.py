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


@pytest.fixture(scope="session")
def cuda():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19891_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


def to_dev(a, dev):
    import torch
    return torch.from_numpy(a).to(dev)


def u32(t):
    """int32 tensor holding uint32 ids -> numpy uint32."""
    return t.cpu().numpy().view("uint32")


def u64(t):
    return t.cpu().numpy().view("uint64")
