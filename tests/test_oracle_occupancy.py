"""Pins for the early-termination quadtree (Sec. 2.2, "Early termination"): one boolean per
node of the complete quadtree of depth D over the domain, true iff the node's cell holds a
point.  Checked against the cells of the points computed from their coordinates alone (not
from the keys), against the tree structure (a node is the OR of its four children) and, for
the Z order, against de-interleaved node labels."""
import numpy as np
import pytest

import oracle


def _popcount_range(bits, start, count):
    out = 0
    for b in range(start, start + count):
        out += (int(bits[b // 32]) >> (b % 32)) & 1
    return out


def _deinterleave(v, t):
    x = y = 0
    for i in range(t):
        x |= ((v >> (2 * i)) & 1) << i
        y |= ((v >> (2 * i + 1)) & 1) << i
    return x, y


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("w,D,n", [(4, 4, 40), (6, 4, 300), (6, 6, 20), (30, 6, 3000)])
def test_occupied_cells_match_coordinates(curve, w, D, n):
    rng = np.random.default_rng(w * 100 + D)
    pts = rng.integers(0, 1 << w, size=(n, 2)).astype(np.int32)
    if w == 30:   # clustered, so that many nodes are empty
        pts = (rng.normal(1 << 29, 1 << 24, size=(n, 2))).clip(0, (1 << 30) - 1).astype(np.int32)
    bits = oracle.occupancy(oracle.keys(pts, w, curve), D, w)
    kf = oracle.key_z if curve == "z" else oracle.key_h
    for t in range(D + 1):
        l = w - t
        cells = {(int(x) >> l, int(y) >> l) for x, y in pts}
        start = (4 ** t - 1) // 3
        assert _popcount_range(bits, start, 4 ** t) == len(cells)
        for cx, cy in cells:
            v = kf(cx << l, cy << l, w) >> (2 * l)
            assert oracle.occupancy_bit(bits, t, v) == 1
        if curve == "z" and t <= 4:
            for v in range(4 ** t):
                assert oracle.occupancy_bit(bits, t, v) == int(_deinterleave(v, t) in cells)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_node_is_or_of_children(curve):
    rng = np.random.default_rng(3)
    pts = rng.integers(0, 1 << 8, size=(60, 2)).astype(np.int32)
    D = 5
    bits = oracle.occupancy(oracle.keys(pts, 8, curve), D, 8)
    for t in range(D):
        for v in range(4 ** t):
            kids = [oracle.occupancy_bit(bits, t + 1, 4 * v + c) for c in range(4)]
            assert oracle.occupancy_bit(bits, t, v) == int(any(kids))
    assert oracle.occupancy_bit(bits, 0, 0) == 1
    assert not oracle.occupancy(np.zeros(0, np.uint64), 3, 8).any()


@pytest.mark.parametrize("curve", ["z", "h"])
def test_cell_occupied_exhaustive(curve):
    """Every aligned cell of a 32 x 32 grid: at depth <= D the answer is exactly "holds a
    point"; finer cells answer for their depth-D ancestor."""
    w, D = 5, 3
    rng = np.random.default_rng(8)
    pts = rng.integers(0, 1 << w, size=(25, 2)).astype(np.int32)
    bits = oracle.occupancy(oracle.keys(pts, w, curve), D, w)
    kf = oracle.key_z if curve == "z" else oracle.key_h
    for l in range(w + 1):
        for cy in range(1 << (w - l)):
            for cx in range(1 << (w - l)):
                lo = (kf(cx << l, cy << l, w) >> (2 * l)) << (2 * l)
                la = max(l, w - D)
                has = any((int(x) >> la) == (cx << l) >> la and (int(y) >> la) == (cy << l) >> la
                          for x, y in pts)
                assert oracle.cell_occupied(bits, D, l, lo, w) == has
