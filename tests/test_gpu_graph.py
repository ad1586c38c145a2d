"""Whole-pipeline CUDA graphs (rebuild + model fit + query batch captured once, replayed):
replays equal eager calls and the oracle, also after new inputs are written into the same
buffers (the sort's look-back epochs advance on the device, so replays never see stale words)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _ref(pts, qs, d, curve):
    return oracle.query(oracle.build(pts, 30, curve), qs, d)


@pytest.mark.parametrize("curve,bounds", [("h", "binary"), ("h", "learned"), ("z", "learned")])
def test_graph_replays_match_oracle(cuda, curve, bounds):
    wl = W.roads_3e7(scale=0.01)
    wl2 = W.roads_3e7(scale=0.01, seed=33)
    roff, rids = _ref(wl.points, wl.queries, wl.delta, curve)
    roff2, rids2 = _ref(wl2.points, wl2.queries, wl2.delta, curve)
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    idx = sfc.sfc_build(pts, curve, bounds=bounds)
    total = max(int(roff[-1]), int(roff2[-1]))
    off = torch.zeros(wl.m + 1, dtype=torch.int64, device=cuda)
    ids = torch.zeros(total, dtype=torch.int32, device=cuda)
    g = sfc.sfc_graph_capture(idx, pts, q, d, off, ids)
    for _ in range(3):
        off.zero_()
        ids.zero_()
        g.launch()
        torch.cuda.synchronize()
        assert np.array_equal(u64(off), roff)
        assert np.array_equal(u32(ids[: int(roff[-1])]), rids)
    # new points and queries in the same buffers (same sizes): the next replay answers them
    assert wl2.n == wl.n and wl2.m == wl.m
    pts.copy_(to_dev(wl2.points, cuda))
    q.copy_(to_dev(wl2.queries, cuda))
    d.copy_(to_dev(wl2.delta, cuda))
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u64(off), roff2)
    assert np.array_equal(u32(ids[: int(roff2[-1])]), rids2)
    assert sfc.sfc_device_status(idx) == (0, 0)
    g.close()


def test_query_only_graph(cuda):
    wl = W.mixed_1e7(scale=0.01)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned")
    ref = oracle.build(wl.points)
    q, d = to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    roff, rids = oracle.query(ref, wl.queries, wl.delta)
    off = torch.zeros(wl.m + 1, dtype=torch.int64, device=cuda)
    ids = torch.zeros(int(roff[-1]) * 2, dtype=torch.int32, device=cuda)
    g = sfc.sfc_graph_capture(idx, None, q, d, off, ids)
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids[: int(roff[-1])]), rids)
    rng = np.random.default_rng(8)
    sel = rng.integers(0, wl.n, wl.m)
    qs2 = wl.points[sel].copy()
    d2 = (wl.delta // 2).astype(np.int32)
    q.copy_(to_dev(qs2, cuda))
    d.copy_(to_dev(d2, cuda))
    g.launch()
    torch.cuda.synchronize()
    roff2, rids2 = oracle.query(ref, qs2, d2)
    assert np.array_equal(u64(off), roff2) and np.array_equal(u32(ids[: int(roff2[-1])]), rids2)


def test_rebuild_in_place(cuda):
    a = W.mixed_1e7(scale=0.005, seed=40)
    b = W.mixed_1e7(scale=0.004, seed=41)
    idx = sfc.sfc_build(to_dev(a.points, cuda), "h", bounds="learned")
    sfc.sfc_rebuild(idx, to_dev(b.points, cuda))
    keys, ids, xy = sfc.sfc_get_sorted(idx)
    ref = oracle.build(b.points, 30, "h")
    assert np.array_equal(u64(keys), ref.keys) and np.array_equal(u32(ids), ref.ids)
    off, out = sfc.query(idx, to_dev(b.queries, cuda), to_dev(b.delta, cuda))
    roff, rids = oracle.query(ref, b.queries, b.delta)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(out), rids)
