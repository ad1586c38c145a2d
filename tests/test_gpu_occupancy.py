"""Early termination (Sec. 2.2) on the GPU: the bitmap built with the index equals the
oracle's bit for bit (every depth, both curves, after updates and in graph replays), queries
with it report exactly the oracle's answer, and the cells it drops are the oracle's empty
cells."""
import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _gpu_bits(idx, D):
    return sfc.sfc_get_occupancy(idx, D).cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("D", [1, 6, 12, 13])
def test_bitmap_matches_oracle(cuda, curve, D):
    wl = W.mixed_1e7(scale=0.01)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), curve, occupancy_depth=D)
    ref = oracle.build(wl.points, 30, curve)
    assert np.array_equal(_gpu_bits(idx, D), oracle.occupancy(ref.keys, D))


@pytest.mark.parametrize("n", [0, 1, 2])
def test_bitmap_tiny(cuda, n):
    pts = np.array([[5, 9], [5, 9]], np.int32)[:n]
    idx = sfc.sfc_build(to_dev(pts.reshape(-1, 2), cuda), "z", occupancy_depth=4)
    assert np.array_equal(_gpu_bits(idx, 4), oracle.occupancy(oracle.keys(pts.reshape(-1, 2)), 4))


def test_bitmap_absent_is_an_error(cuda):
    idx = sfc.sfc_build(to_dev(W.uniform_1e5(scale=0.01).points, cuda), "z")
    with pytest.raises(sfc.SfcError) as e:
        sfc.sfc_get_occupancy(idx, 4)
    assert e.value.status == sfc.SFC_ERR_STATE
    with pytest.raises(sfc.SfcError):
        sfc.sfc_build(to_dev(W.uniform_1e5(scale=0.01).points, cuda), "z", occupancy_depth=14)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 1, 2])
@pytest.mark.parametrize("bounds", ["binary", "learned"])
def test_queries_with_early_termination(cuda, curve, cover, bounds):
    """The paper's setting for early termination: Normal points, uniformly placed queries (many
    windows empty), plus queries at data points."""
    wl = W.normal_uniform_queries(200_000, 4000, 1e-3)
    pts = wl.points
    qs = np.concatenate([wl.queries, pts[:2000]])
    d = np.concatenate([wl.delta, np.random.default_rng(1).integers(0, 1 << 20, 2000).astype(np.int32)])
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, occupancy_depth=12, cover_refine=cover, bounds=bounds)
    off, ids = sfc.query(idx, to_dev(qs, cuda), to_dev(d, cuda))
    roff, rids = oracle.query(oracle.build(pts, 30, curve), qs, d)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)
    cs = sfc.sfc_query_cell_stats(idx)
    assert 0 < cs["empty"] < cs["cells"]
    assert sfc.sfc_device_status(idx) == (0, 0)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 1])
def test_dropped_cells_are_the_empty_ones(cuda, curve, cover):
    """Ranges export with the bitmap: exactly the cover's cells the oracle's bitmap shows
    occupied, merged where they abut; the dropped count is the oracle's."""
    D = 10
    rng = np.random.default_rng(21)
    pts = W.normal_points(rng, 50_000)
    qs = W.uniform_points(rng, 3000)
    d = rng.integers(0, 1 << 22, 3000).astype(np.int32)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, occupancy_depth=D, cover_refine=cover)
    K = sfc.sfc_query_max_intervals(idx)
    lo, hi, b, e, c = sfc.sfc_query_ranges(idx, to_dev(qs, cuda), to_dev(d, cuda))
    lo, hi, c = u64(lo), u64(hi), c.cpu().numpy()
    ref = oracle.build(pts, 30, curve)
    bits = oracle.occupancy(ref.keys, D)
    empty = cells = 0
    for i in range(len(qs)):
        x, y, r = int(qs[i, 0]), int(qs[i, 1]), int(d[i])
        if cover == 0:
            cl, l = oracle.cells(x, y, r, 30, curve)
        else:
            cl = oracle.cells_refined(x, y, r, 30, curve, cover)
            l = max(0, oracle.level(r) - cover)
        keep = [(a, z) for a, z in cl if oracle.cell_occupied(bits, D, l, a)]
        cells += len(cl)
        empty += len(cl) - len(keep)
        merged = oracle.merge_abutting(keep)
        assert c[i] == len(merged)
        for j, (a, z) in enumerate(merged):
            assert (int(lo[K * i + j]), int(hi[K * i + j])) == (a, z)
    # a query batch counts the same cells
    sfc.query(idx, to_dev(qs, cuda), to_dev(d, cuda))
    assert sfc.sfc_query_cell_stats(idx) == {"cells": cells, "empty": empty}
    assert empty > 0


def test_bitmap_follows_updates_and_graph_replays(cuda):
    wl = W.mixed_1e7(scale=0.005)
    D = 12
    pts = to_dev(wl.points, cuda)
    idx = sfc.sfc_build(pts, "h", occupancy_depth=D)
    rng = np.random.default_rng(5)
    ins = W.uniform_points(rng, 3000)
    dels = rng.choice(wl.n, 2000, replace=False).astype(np.int32)
    sfc.sfc_update(idx, to_dev(ins, cuda), to_dev(dels, cuda))
    live = np.delete(np.concatenate([wl.points, ins]), dels, axis=0)
    assert np.array_equal(_gpu_bits(idx, D), oracle.occupancy(oracle.keys(live, 30, "h"), D))
    # rebuild graph: a replay over new points in the same buffer rebuilds the bitmap
    idx2 = sfc.sfc_build(pts, "z", occupancy_depth=D)
    q, d = to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta)
    p2 = W.uniform_points(rng, wl.n)
    roff2, rids2 = oracle.query(oracle.build(p2), wl.queries, wl.delta)
    off = torch.zeros(wl.m + 1, dtype=torch.int64, device=cuda)
    ids = torch.zeros(max(int(roff[-1]), int(roff2[-1]), 1), dtype=torch.int32, device=cuda)
    g = sfc.sfc_graph_capture(idx2, pts, q, d, off, ids)
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids[: int(roff[-1])]), rids)
    pts.copy_(to_dev(p2, cuda))
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(_gpu_bits(idx2, D), oracle.occupancy(oracle.keys(p2), D))
    assert np.array_equal(u64(off), roff2) and np.array_equal(u32(ids[: int(roff2[-1])]), rids2)
    g.close()
