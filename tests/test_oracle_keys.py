"""Pins for the oracle's curve keys (Alg. 2; Sec. 2.1; Def. 2.1 / Def. 2.3 / Lemma 1).

Each check is something the paper or the mathematics fixes, not a retyping of the oracle:
hand-enumerated order-1/order-2 tables, the prefix property of Def. 2.3 at w = 30, the
recursive block structure of Def. 2.1, bijectivity and (Hilbert) edge adjacency of
consecutive cells.
"""
import numpy as np
import pytest

import oracle
from conftest import load_grid

CURVES = {"z": oracle.key_z, "h": oracle.key_h}
GOLDEN = {("z", 1): "morton_order1.txt", ("z", 2): "morton_order2.txt",
          ("h", 1): "hilbert_order1.txt", ("h", 2): "hilbert_order2.txt"}


@pytest.mark.parametrize("curve,w", list(GOLDEN))
def test_golden_tables(curve, w):
    grid = load_grid(GOLDEN[(curve, w)])
    for (x, y), k in grid.items():
        assert CURVES[curve](x, y, w) == k, (curve, w, x, y)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("k", [1, 2])
def test_prefix_property_w30(curve, k):
    """Def. 2.3: the label of a level-(30-k) cell is the prefix of its points' labels, and the
    top 2k bits at w = 30 reproduce the order-k table."""
    grid = load_grid(GOLDEN[(curve, k)])
    f = CURVES[curve]
    rng = np.random.default_rng(7)
    sh = 30 - k
    for (x, y), key in grid.items():
        for _ in range(4):
            lx, ly = (int(v) for v in rng.integers(0, 1 << sh, size=2))
            full = f((x << sh) | lx, (y << sh) | ly, 30)
            assert full >> (2 * sh) == key


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("w", [1, 2, 3, 4, 5])
def test_bijection_and_blocks(curve, w):
    """The keys of the 2^w x 2^w grid are a permutation of [0, 4^w), and every aligned
    2^l x 2^l block maps to one aligned interval of length 4^l (Def. 2.1, recursively)."""
    f = CURVES[curve]
    side = 1 << w
    keys = np.array([[f(x, y, w) for x in range(side)] for y in range(side)], dtype=np.int64)
    assert sorted(keys.ravel().tolist()) == list(range(side * side))
    for l in range(w + 1):
        b = 1 << l
        for by in range(0, side, b):
            for bx in range(0, side, b):
                blk = keys[by:by + b, bx:bx + b]
                lo = blk.min()
                assert lo % (b * b) == 0
                assert blk.max() == lo + b * b - 1


@pytest.mark.parametrize("w", [1, 2, 3, 4, 5, 6])
def test_hilbert_adjacency(w):
    """Consecutive Hilbert cells share an edge (Sec. 2.1: consecutive points are close);
    with this orientation the curve starts at (0,0) and ends at (2^w - 1, 0)."""
    side = 1 << w
    pos = {}
    for y in range(side):
        for x in range(side):
            pos[oracle.key_h(x, y, w)] = (x, y)
    for k in range(side * side - 1):
        (x0, y0), (x1, y1) = pos[k], pos[k + 1]
        assert abs(x0 - x1) + abs(y0 - y1) == 1
    assert pos[0] == (0, 0)
    assert pos[side * side - 1] == (side - 1, 0)


def test_hilbert_endpoints_w30():
    assert oracle.key_h(0, 0, 30) == 0
    assert oracle.key_h((1 << 30) - 1, 0, 30) == (1 << 60) - 1
    assert oracle.key_z((1 << 30) - 1, (1 << 30) - 1, 30) == (1 << 60) - 1


@pytest.mark.parametrize("curve", ["z", "h"])
def test_vector_keys_match_scalar(curve):
    rng = np.random.default_rng(3)
    xy = rng.integers(0, 1 << 30, size=(200, 2)).astype(np.int32)
    ks = oracle.keys(xy, 30, curve)
    f = CURVES[curve]
    for (x, y), k in zip(xy.tolist(), ks.tolist()):
        assert f(x, y, 30) == k


def test_morton_single_bits():
    """Alg. 2 read bit by bit: x = 2^i lands on bit 2i, y = 2^i on bit 2i + 1."""
    for i in range(30):
        assert oracle.key_z(1 << i, 0, 30) == 1 << (2 * i)
        assert oracle.key_z(0, 1 << i, 30) == 1 << (2 * i + 1)
