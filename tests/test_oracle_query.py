"""Pins for the oracle's construction and Alg. 1 query against brute force (problem
statement of Sec. 2) and the library sort."""
import numpy as np
import pytest

import oracle
import workloads as W


def _same_sets(a_off, a_ids, b_off, b_ids):
    assert np.array_equal(np.asarray(a_off, np.uint64), np.asarray(b_off, np.uint64))
    for x, y in zip(oracle.sorted_lists(a_off, a_ids), oracle.sorted_lists(b_off, b_ids)):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_build_matches_library_sort(curve):
    pts, _, _ = W.tiny_dense(1, 5000, 1, 6, 0)        # many duplicate keys
    idx = oracle.build(pts, 30, curve)
    k = oracle.keys(pts, 30, curve)
    order = np.lexsort((np.arange(len(k)), k))          # by key, then input index
    assert np.array_equal(idx.keys, k[order])
    assert np.array_equal(idx.ids, order.astype(np.uint32))
    assert np.array_equal(idx.xy, pts[order])


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("seed,side_bits,max_delta", [(1, 4, 6), (2, 6, 20), (3, 10, 300),
                                                       (4, 30, 1 << 28)])
def test_query_vs_brute_small(curve, seed, side_bits, max_delta):
    pts, qs, d = W.tiny_dense(seed, 1500, 400, side_bits, max_delta)
    idx = oracle.build(pts, 30, curve)
    off, ids = oracle.query(idx, qs, d)
    boff, bids = oracle.brute(pts, qs, d)
    _same_sets(off, ids, boff, bids)
    # per-query output is in ascending position of the sorted array, i.e. (key, id) order
    pos = np.empty(idx.n, np.int64)
    pos[idx.ids] = np.arange(idx.n)
    for i in range(len(qs)):
        p = pos[ids[off[i]:off[i + 1]]]
        assert np.all(np.diff(p) > 0)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_closed_ball_boundary(curve):
    """Points exactly at distance delta are reported (closed ball), one unit further are not."""
    c = (1 << 29) + 12345
    for s in [1, 7, 1000]:
        on, out = W.pythagorean_ring(c, c + 3, s)
        pts = np.concatenate([on, out])
        idx = oracle.build(pts, 30, curve)
        off, ids = oracle.query(idx, np.array([[c, c + 3]], np.int32), np.array([5 * s], np.int32))
        assert sorted(ids.tolist()) == list(range(len(on)))


def test_empty_and_degenerate():
    idx = oracle.build(np.zeros((0, 2), np.int32))
    off, ids = oracle.query(idx, np.array([[5, 5]], np.int32), np.array([100], np.int32))
    assert off.tolist() == [0, 0] and ids.size == 0
    pts = np.array([[5, 5], [5, 5], [6, 5]], np.int32)
    idx = oracle.build(pts)
    off, ids = oracle.query(idx, np.array([[5, 5], [5, 5], [-1, 3], [5, 5]], np.int32),
                            np.array([0, 1, 10, -1], np.int32))
    assert off.tolist() == [0, 2, 5, 5, 5]
    assert ids.tolist() == [0, 1, 0, 1, 2]          # invalid queries report nothing


@pytest.mark.parametrize("curve", ["z", "h"])
def test_uniform_1e5_vs_brute(curve):
    """The whole uniform-1e5 workload (10^9 pair tests) against brute force."""
    wl = W.uniform_1e5()
    idx = oracle.build(wl.points, 30, curve)
    off, ids, scanned = oracle.query(idx, wl.queries, wl.delta, threads=8, want_scanned=True)
    boff, bids = oracle.brute(wl.points, wl.queries, wl.delta, threads=8)
    _same_sets(off, ids, boff, bids)
    mean_k = off[-1] / wl.m
    # expected ~20 hits per query, minus an edge loss of a couple of percent
    assert 18.5 < mean_k < 20.5
    ratio = scanned.sum() / off[-1]
    assert 4.0 < ratio < 12.0   # scan amplification (c+1)^2 4/pi, c in [1, 2)


def test_threads_do_not_change_results():
    wl = W.mixed_1e7(scale=0.002)
    idx = oracle.build(wl.points)
    a = oracle.query(idx, wl.queries, wl.delta, threads=1)
    b = oracle.query(idx, wl.queries, wl.delta, threads=7)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
