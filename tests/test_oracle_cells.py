"""Pins for cells(Q) (definition before Alg. 1) and the Observation's key interval.

Exhaustive over every query centre and radius of small grids: at most four cells
(Sec. 1.2, 2^d with d = 2), cell size |Q| <= |C| < 2|Q| with |.| the side, coverage of every
grid point of Q, disjointness, and that each cell meets Q.  Special cases: delta = 0 gives
the point's own unit interval, a radius of at least half the domain gives the whole domain.
"""
import numpy as np
import pytest

import oracle


def _grid_keys(w, curve):
    side = 1 << w
    f = oracle.key_z if curve == "z" else oracle.key_h
    return np.array([[f(x, y, w) for x in range(side)] for y in range(side)], dtype=np.int64)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("w", [3, 4])
def test_cells_exhaustive(curve, w):
    side = 1 << w
    keys = _grid_keys(w, curve)
    for qy in range(side):
        for qx in range(side):
            for delta in range(0, 2 * side + 1):
                rngs, l = oracle.cells(qx, qy, delta, w, curve)
                assert 1 <= len(rngs) <= 4
                # level: 2*delta <= 2^l < 4*delta (capped at w); delta = 0 -> l = 0
                if delta == 0:
                    assert l == 0
                elif l < w:
                    assert 2 * delta <= (1 << l) < 4 * delta
                else:
                    assert (1 << w) < 4 * delta
                for lo, hi in rngs:
                    assert hi - lo + 1 == 4 ** l
                    assert lo % (4 ** l) == 0
                # sorted and disjoint
                for (a, b), (c, d) in zip(rngs, rngs[1:]):
                    assert b < c
                x0, x1 = max(0, qx - delta), min(side - 1, qx + delta)
                y0, y1 = max(0, qy - delta), min(side - 1, qy + delta)
                inq = keys[y0:y1 + 1, x0:x1 + 1].ravel()
                # coverage: every grid point of Q has its key inside some interval
                covered = np.zeros(inq.shape, bool)
                for lo, hi in rngs:
                    covered |= (inq >= lo) & (inq <= hi)
                assert covered.all()
                # every cell meets Q
                for lo, hi in rngs:
                    assert ((inq >= lo) & (inq <= hi)).any()


@pytest.mark.parametrize("curve", ["z", "h"])
def test_cells_same_total_length(curve):
    """Both curves label the same quadtree cells, so the covered key length agrees."""
    rng = np.random.default_rng(11)
    for _ in range(300):
        qx, qy = (int(v) for v in rng.integers(0, 1 << 30, size=2))
        delta = int(rng.integers(0, 1 << 24))
        rz, lz = oracle.cells(qx, qy, delta, 30, "z")
        rh, lh = oracle.cells(qx, qy, delta, 30, "h")
        assert lz == lh and len(rz) == len(rh)
        assert sum(b - a + 1 for a, b in rz) == sum(b - a + 1 for a, b in rh)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_cells_special_cases_w30(curve):
    f = oracle.key_z if curve == "z" else oracle.key_h
    rng = np.random.default_rng(5)
    for _ in range(50):
        qx, qy = (int(v) for v in rng.integers(0, 1 << 30, size=2))
        r, l = oracle.cells(qx, qy, 0, 30, curve)
        k = f(qx, qy, 30)
        assert l == 0 and r == [(k, k)]
        r, l = oracle.cells(qx, qy, 1 << 29, 30, curve)
        assert l == 30 and r == [(0, (1 << 60) - 1)]
        r, l = oracle.cells(qx, qy, 2 ** 31 - 1, 30, curve)
        assert l == 30 and r == [(0, (1 << 60) - 1)]


def test_level_values():
    assert oracle.level(0) == 0
    assert oracle.level(1) == 1        # 2 <= 2 < 4
    assert oracle.level(2) == 2        # 4 <= 4 < 8
    assert oracle.level(3) == 3        # 6 <= 8 < 12
    assert oracle.level(8366) == 15    # 16732 <= 32768 < 33464
    assert oracle.level((1 << 28) + 1) == 30
    assert oracle.level(1 << 28) == 29


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("drop", [0, 1, 2])
def test_refined_cells_exhaustive(curve, drop):
    """Finer covers: every integer point of the closed ball is covered, every kept cell holds a
    point of the ball, cells are disjoint, at most (2^drop + 1)^2 of them, all of side
    2^max(0, l - drop)."""
    w = 4
    side = 1 << w
    keys = _grid_keys(w, curve)
    ys, xs = np.mgrid[0:side, 0:side]
    for qy in range(0, side, 3):
        for qx in range(0, side, 2):
            for delta in range(0, side + 2):
                rngs = oracle.cells_refined(qx, qy, delta, w, curve, drop)
                l = max(0, oracle.level(delta, w) - drop)
                assert len(rngs) <= (2 ** drop + 1) ** 2
                inball = (xs - qx) ** 2 + (ys - qy) ** 2 <= delta * delta
                kb = keys[inball]
                cov = np.zeros(kb.shape, bool)
                for lo, hi in rngs:
                    assert hi - lo + 1 == 4 ** l and lo % (4 ** l) == 0
                    cell = (keys >= lo) & (keys <= hi)
                    assert (cell & inball).any()          # the cell meets the ball
                    cov |= (kb >= lo) & (kb <= hi)
                assert cov.all()                            # the ball is covered
                for (a, b), (c, d) in zip(rngs, rngs[1:]):
                    assert b < c


def test_refined_drop0_is_subset_of_cells():
    rng = np.random.default_rng(4)
    for _ in range(200):
        qx, qy = (int(v) for v in rng.integers(0, 1 << 30, 2))
        delta = int(rng.integers(0, 1 << 22))
        full, _ = oracle.cells(qx, qy, delta)
        sub = oracle.cells_refined(qx, qy, delta, drop=0)
        assert set(sub) <= set(full) and len(sub) >= 1


@pytest.mark.parametrize("intervals,merged", [
    ([], []),                                                     # no interval
    ([(5, 9)], [(5, 9)]),                                         # single
    ([(0, 3), (4, 7)], [(0, 7)]),                                 # abutting: 3 + 1 == 4
    ([(0, 3), (5, 7)], [(0, 3), (5, 7)]),                         # one key apart: kept apart
    ([(0, 3), (4, 7), (8, 8), (10, 12), (13, 15)], [(0, 8), (10, 15)]),   # chains and a gap
    ([(16, 31), (32, 47), (64, 79), (80, 95)], [(16, 47), (64, 95)]),     # aligned cells of 16 keys
    ([(2 ** 60 - 8, 2 ** 60 - 5), (2 ** 60 - 4, 2 ** 60 - 1)], [(2 ** 60 - 8, 2 ** 60 - 1)]),   # top of the key space
    ([(0, 0), (1, 1), (2, 2), (3, 3)], [(0, 3)]),                 # cells of one key (level 0)
])
def test_merge_abutting_table(intervals, merged):
    """Intervals sorted by lo and pairwise disjoint (as the cells of a cover are): those whose
    end is followed by the next one's start are joined, the others kept; the keys covered
    are unchanged."""
    assert oracle.merge_abutting(intervals) == merged
    keys = lambda iv: [k for a, z in iv for k in range(a, z + 1)] if all(z - a < 64 for a, z in iv) else None
    if keys(intervals) is not None and keys(merged) is not None:
        assert keys(merged) == keys(intervals)
