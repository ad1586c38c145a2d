"""3-D points on the GPU (the Z curve in Z^3, the paper's d-dimensional remark): keys, the
sorted array, cells(Q) with at most 8 cells and their bounds, and the query results,
bit-exact against the 3-D oracle; host buffers, rebuilds, graphs and the documented
rejections."""
import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu

S3 = 1 << 21


def _pts(rng, n, side=S3):
    return rng.integers(0, side, size=(n, 3)).astype(np.int32)


def test_keys3(cuda):
    rng = np.random.default_rng(1)
    p = _pts(rng, 5000)
    p[:4] = [[0, 0, 0], [S3 - 1, S3 - 1, S3 - 1], [S3 - 1, 0, 0], [0, 0, S3 - 1]]
    k = sfc.sfc_keys3(to_dev(p, cuda)).cpu().numpy().view(np.uint64)
    assert np.array_equal(k, oracle.keys3(p))


@pytest.mark.parametrize("n", [0, 1, 1000, 70_001])
def test_build3_sorted_arrays(cuda, n):
    rng = np.random.default_rng(n)
    p = _pts(rng, n) if n else np.zeros((0, 3), np.int32)
    if n > 10:
        p[: n // 10] = p[n // 10]                     # duplicates: ties broken by id
    idx = sfc.sfc_build3(to_dev(p, cuda))
    assert sfc.lib().sfc_index_dim(idx.handle) == 3
    k, i, x = sfc.sfc_get_sorted(idx)
    ref = oracle.build3(p)
    assert np.array_equal(u64(k), ref.keys) and np.array_equal(u32(i), ref.ids)
    xs = x.cpu().numpy()
    assert np.array_equal(xs[:, :3], ref.xy) and not xs[:, 3].any()


@pytest.mark.parametrize("cover", [0, 1])
def test_ranges3(cuda, cover):
    rng = np.random.default_rng(5)
    p = _pts(rng, 20_000)
    qs = np.concatenate([p[:1500], _pts(rng, 500)])
    d = rng.integers(0, 1 << 18, 2000).astype(np.int32)
    d[:20] = 0
    d[20:30] = S3
    qs[30:34] = [[0, 0, 0], [S3 - 1, S3 - 1, S3 - 1], [0, S3 - 1, 5], [7, 7, S3 - 1]]
    idx = sfc.sfc_build3(to_dev(p, cuda), cover_refine=cover)
    K = sfc.sfc_query_max_intervals(idx)
    assert K == (8 if cover == 0 else 27)
    lo, hi, b, e, c = sfc.sfc_query_ranges(idx, to_dev(qs, cuda), to_dev(d, cuda))
    lo, hi, b, e, c = u64(lo), u64(hi), b.cpu().numpy(), e.cpu().numpy(), c.cpu().numpy()
    ref = oracle.build3(p)
    for j in range(len(qs)):
        if cover == 0:
            cells, _ = oracle.cells3(*qs[j], int(d[j]))
        else:
            cells = oracle.cells3_refined(*qs[j], int(d[j]), drop=1)
        merged = oracle.merge_abutting(cells)
        assert c[j] == len(merged) <= K
        for r, (a, z) in enumerate(merged):
            assert (int(lo[K * j + r]), int(hi[K * j + r])) == (a, z)
            assert b[K * j + r] == oracle.lower_bound(ref.keys, a)
            assert e[K * j + r] == oracle.lower_bound(ref.keys, z + 1)


def _same(idx, p, qs, d, cuda):
    off, ids = sfc.query(idx, to_dev(qs, cuda), to_dev(d, cuda))
    roff, rids = oracle.query3(oracle.build3(p), qs, d)
    assert np.array_equal(u64(off), roff)
    assert np.array_equal(u32(ids), rids)
    return off, ids


@pytest.mark.parametrize("chunk", [32, 1024, 4096])
@pytest.mark.parametrize("cover", [0, 1])
def test_mixed3d_vs_oracle(cuda, chunk, cover):
    wl = W.mixed3d(scale=0.005)
    idx = sfc.sfc_build3(to_dev(wl.points, cuda), chunk=chunk, cover_refine=cover)
    _same(idx, wl.points, wl.queries, wl.delta, cuda)
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_dense_small_grid_edge_cases(cuda):
    """Duplicates, whole-domain balls, radius 0, invalid centres and radii, a mask budget
    small enough that the write pass re-filters."""
    rng = np.random.default_rng(9)
    p = _pts(rng, 30_000, side=64)
    p[:300] = [3, 4, 5]
    qs = np.concatenate([p[rng.integers(0, len(p), 3000)], np.array([[3, 4, 5], [0, 0, 0], [-1, 0, 0], [0, S3, 0]], np.int32)])
    d = np.concatenate([rng.integers(0, 12, 3000), np.array([0, 2 ** 31 - 1, 5, 5])]).astype(np.int32)
    d[7] = -2
    idx = sfc.sfc_build3(to_dev(p, cuda), mask_budget_mb=1, cover_refine=1)
    off, _ = _same(idx, p, qs, d, cuda)
    o = u64(off)
    assert o[3001] - o[3000] >= 300 and o[3002] - o[3001] == len(p)
    st, bits = sfc.sfc_device_status(idx)
    assert st == sfc.SFC_ERR_INVALID and bits & sfc.SFC_DEV_BAD_QUERY


def test_host_rebuild_graph_autotune(cuda):
    wl = W.mixed3d(scale=0.003)
    wl2 = W.mixed3d(scale=0.003, seed=81)
    idx = sfc.sfc_build3_host(wl.points)
    roff, rids = oracle.query3(oracle.build3(wl.points), wl.queries, wl.delta)
    off, ids = sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, capacity=int(roff[-1]))
    assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    tuned = sfc.sfc_autotune(idx, q, d, force=True)
    assert tuned["cover"] == 0   # built with the default cover_refine = 0: not tuned
    idx_t = sfc.sfc_build3(pts, cover_refine=-1)
    assert sfc.sfc_autotune(idx_t, q, d, force=True)["cover"] in (0, 1)
    _same(idx_t, wl.points, wl.queries, wl.delta, cuda)
    roff2, rids2 = oracle.query3(oracle.build3(wl2.points), wl.queries, wl.delta)
    total = max(int(roff[-1]), int(roff2[-1]))
    o = torch.zeros(wl.m + 1, dtype=torch.int64, device=cuda)
    i = torch.zeros(total, dtype=torch.int32, device=cuda)
    g = sfc.sfc_graph_capture(idx, pts, q, d, o, i)
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u64(o), roff) and np.array_equal(u32(i[: int(roff[-1])]), rids)
    pts.copy_(to_dev(wl2.points, cuda))
    g.launch()
    torch.cuda.synchronize()
    assert np.array_equal(u64(o), roff2) and np.array_equal(u32(i[: int(roff2[-1])]), rids2)
    g.close()
    sfc.sfc_rebuild(idx, to_dev(wl.points, cuda))
    _same(idx, wl.points, wl.queries, wl.delta, cuda)


def test_rejections(cuda):
    p = to_dev(_pts(np.random.default_rng(2), 1000), cuda)
    for bad in ({"bounds": "learned"}, {"cover_refine": 2}, {"occupancy_depth": 4}, {"query_norm": "square"}):
        with pytest.raises(sfc.SfcError):
            sfc.sfc_build3(p, **bad)
    idx = sfc.sfc_build3(p)
    with pytest.raises(sfc.SfcError):
        sfc.sfc_update(idx, None, torch.zeros(1, dtype=torch.int32, device=cuda))
    with pytest.raises(sfc.SfcError):
        sfc.sfc_train_model(idx)
    with pytest.raises(sfc.SfcError):
        sfc.sfc_set_cover(idx, 2)
    sfc.sfc_set_cover(idx, 1)
    with pytest.raises(sfc.SfcError):
        sfc.sfc_set_query_norm(idx, "square")
    bad = to_dev(np.array([[0, 0, S3]], np.int32), cuda)
    idx2 = sfc.sfc_build3(bad)
    assert sfc.sfc_device_status(idx2)[1] & sfc.SFC_DEV_BAD_POINT


def test_big_balls_split_over_warps(cuda):
    """3-D queries of many chunks are written chunk by chunk by many warps: a dense Gaussian
    cloud with 20 balls covering most of it among small ones equals the oracle, with chunks of
    32 points (the chunk hit counts then come from one mask word per chunk) and of 4096."""
    rng = np.random.default_rng(43)
    c = rng.normal(1 << 20, 1 << 14, size=(150_000, 3))
    u = rng.integers(0, 1 << 21, size=(50_000, 3))
    p = np.clip(np.concatenate([c, u]), 0, (1 << 21) - 1).astype(np.int32)
    qs = p[rng.choice(len(p), 5_000, replace=False)].copy()
    d = rng.integers(0, 1 << 9, 5_000).astype(np.int32)
    qs[:20] = (1 << 20) + rng.integers(-(1 << 12), 1 << 12, size=(20, 3))
    d[:20] = 1 << 15
    for chunk in (32, 4096):
        idx = sfc.sfc_build3(to_dev(p, cuda), chunk=chunk, cover_refine=1)
        off, _ = _same(idx, p, qs, d, cuda)
        assert int(np.diff(u64(off)).max()) > 50_000
        assert sfc.sfc_device_status(idx) == (0, 0)
