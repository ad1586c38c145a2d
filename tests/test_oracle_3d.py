"""Pins for the 3-D oracle (the Z curve in Z^3; the paper's d-dimensional remark, Sec. 2.1,
with at most 2^d = 8 cells per query, Sec. 1.2): the hand-enumerated order-1 table, the
recursive (prefix-label) construction of order 2 and 3 from it, bijection, cells(Q) invariants
on every query of a small grid, and Alg. 1 against brute force."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "morton3_order1.txt")


def _order1():
    t = np.loadtxt(GOLDEN, dtype=np.int64)
    return {(int(x), int(y), int(z)): int(k) for x, y, z, k in t}


def test_order1_table():
    for (x, y, z), k in _order1().items():
        assert oracle.key_z3(x, y, z, 1) == k


@pytest.mark.parametrize("w", [2, 3])
def test_recursive_labels(w):
    """Def. 2.3 in 3-D: a child's label is its parent's label followed by the 3-bit label of
    its octant in the order-1 curve."""
    t1 = _order1()
    side = 1 << w
    for x in range(side):
        for y in range(side):
            for z in range(side):
                k = 0
                for lvl in range(w - 1, -1, -1):
                    k = 8 * k + t1[((x >> lvl) & 1, (y >> lvl) & 1, (z >> lvl) & 1)]
                assert oracle.key_z3(x, y, z, w) == k


def test_bijection_w3():
    ks = sorted(oracle.key_z3(x, y, z, 3) for x in range(8) for y in range(8) for z in range(8))
    assert ks == list(range(512))


def test_cells3_exhaustive():
    w = 3
    side = 1 << w
    g = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij"), -1).reshape(-1, 3)
    keys = np.array([oracle.key_z3(*p, w) for p in g], dtype=np.int64)
    rng = np.random.default_rng(3)
    for qi in rng.choice(len(g), 60, replace=False):
        q = g[qi]
        for d in range(0, 2 * side + 1):
            rngs, l = oracle.cells3(*q, d, w)
            assert 1 <= len(rngs) <= 8
            if d == 0:
                assert l == 0
            elif l < w:
                assert 2 * d <= (1 << l) < 4 * d
            inq = np.all(np.abs(g - q) <= d, axis=1)
            kq = keys[inq]
            cov = np.zeros(kq.shape, bool)
            for lo, hi in rngs:
                assert hi - lo + 1 == 8 ** l and lo % (8 ** l) == 0
                assert ((kq >= lo) & (kq <= hi)).any()      # every cell meets Q
                cov |= (kq >= lo) & (kq <= hi)
            assert cov.all()
            for (a, b), (c, e) in zip(rngs, rngs[1:]):
                assert b < c


@pytest.mark.parametrize("w,maxd,n", [(4, 6, 600), (10, 200, 4000), (21, 1 << 18, 4000)])
def test_query3_matches_brute_force(w, maxd, n):
    rng = np.random.default_rng(w)
    pts = rng.integers(0, 1 << w, size=(n, 3)).astype(np.int32)
    pts[:30] = pts[30]
    qs = np.concatenate([pts[rng.integers(0, n, 300)], rng.integers(0, 1 << w, size=(100, 3)).astype(np.int32)])
    qs[:3] = [[0, 0, 0], [(1 << w) - 1] * 3, [-1, 0, 0]]
    d = rng.integers(0, maxd, len(qs)).astype(np.int32)
    d[5] = -1
    ix = oracle.build3(pts, w)
    off, ids = oracle.query3(ix, qs, d)
    boff, bids = oracle.brute3(pts, qs, d, w)
    assert np.array_equal(off, boff)
    assert all(np.array_equal(a, b) for a, b in zip(oracle.sorted_lists(off, ids), oracle.sorted_lists(boff, bids)))
    assert off[1] - off[0] >= 0 and off[3] == off[2]    # the invalid centre reports nothing
    # ids come out in ascending (key, id) order
    kmap = oracle.keys3(pts, w)
    for i in range(len(qs)):
        seg = ids[off[i]:off[i + 1]]
        pairs = list(zip(kmap[seg], seg))
        assert pairs == sorted(pairs)


@pytest.mark.parametrize("drop", [1, 2])
def test_cells3_refined(drop):
    """Finer 3-D covers: every integer point of the closed ball is covered, every kept cell
    holds one, disjoint, at most (2^drop + 1)^3 cells of side 2^max(0, l - drop)."""
    w = 3
    side = 1 << w
    g = np.stack(np.meshgrid(np.arange(side), np.arange(side), np.arange(side), indexing="ij"), -1).reshape(-1, 3)
    keys = np.array([oracle.key_z3(*p, w) for p in g], dtype=np.int64)
    rng = np.random.default_rng(drop)
    for qi in rng.choice(len(g), 40, replace=False):
        q = g[qi]
        for d in range(0, side + 2):
            r = oracle.cells3_refined(*q, d, w, drop)
            l = max(0, oracle.level(d, w) - drop)
            assert len(r) <= (2 ** drop + 1) ** 3
            inball = ((g - q) ** 2).sum(axis=1) <= d * d
            kb = keys[inball]
            cov = np.zeros(kb.shape, bool)
            for lo, hi in r:
                assert hi - lo + 1 == 8 ** l and lo % (8 ** l) == 0
                assert (((keys >= lo) & (keys <= hi)) & inball).any()
                cov |= (kb >= lo) & (kb <= hi)
            assert cov.all()
            for (a, b), (c, e) in zip(r, r[1:]):
                assert b < c
