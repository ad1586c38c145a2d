"""Pins for the dynamic oracle (Sec. 2.1 "Dynamic implementation", Sec. 3.3): after every
batch, its answers equal brute force over the live set, and rejected batches change nothing."""
import numpy as np
import pytest

import oracle
from oracle.dynamic import DynamicOracle, NotFound
import workloads as W


def test_dynamic_vs_brute():
    rng = np.random.default_rng(9)
    pts, qs, d = W.tiny_dense(4, 800, 100, 8, 40)
    dyn = DynamicOracle(pts)
    for r in range(5):
        live = np.nonzero(dyn.alive)[0]
        dels = rng.choice(live, size=60, replace=False)
        ins = rng.integers(0, 256, size=(90, 2)).astype(np.int32)
        first = dyn.apply(ins, dels)
        assert first == 800 + 90 * r
        live = np.nonzero(dyn.alive)[0]
        off, ids = dyn.query(qs, d)
        boff, bids = oracle.brute(dyn.xy_by_id[live], qs, d)
        bids = live[bids].astype(np.uint32)
        assert np.array_equal(off, boff)
        for a, b in zip(oracle.sorted_lists(off, ids), oracle.sorted_lists(boff, bids)):
            assert np.array_equal(a, b)
        # the index is sorted by (key, id)
        k = dyn.index.keys.astype(object)
        assert all((k[i], dyn.index.ids[i]) < (k[i + 1], dyn.index.ids[i + 1])
                   for i in range(dyn.n - 1))


def test_rejected_batch_changes_nothing():
    pts, _, _ = W.tiny_dense(5, 50, 1, 8, 0)
    dyn = DynamicOracle(pts)
    dyn.apply(np.zeros((0, 2), np.int32), np.array([3, 4]))
    keys_before = dyn.index.keys.copy()
    for bad in ([3], [7, 7], [50], [-1]):
        with pytest.raises(NotFound):
            dyn.apply(np.array([[1, 1]], np.int32), np.array(bad))
        assert np.array_equal(dyn.index.keys, keys_before) and dyn.next_id == 50
