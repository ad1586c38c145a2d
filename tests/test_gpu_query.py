"""GPU parity of the query path (Alg. 1 for a batch): ranges of cells(Q), bounds, counts,
offsets and the id lists, element by element against the oracle.  Integer work: bit-exact,
including the per-query order (ascending (key, id))."""
import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def run_gpu(pts, qs, d, curve, dev, **opts):
    idx = sfc.sfc_build(to_dev(pts, dev), curve, **opts)
    off, ids = sfc.query(idx, to_dev(qs, dev), to_dev(d, dev))
    st = sfc.sfc_device_status(idx)
    return idx, u64(off), u32(ids), st


def assert_same(pts, qs, d, curve, dev, **opts):
    idx, off, ids, st = run_gpu(pts, qs, d, curve, dev, **opts)
    ref = oracle.build(pts, 30, curve)
    roff, rids = oracle.query(ref, qs, d)
    assert np.array_equal(off, roff)
    assert np.array_equal(ids, rids)
    return idx, st


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 1, 2])
def test_ranges_and_bounds(cuda, curve, cover):
    pts, qs, d = W.tiny_dense(11, 3000, 2000, 30, 1 << 26)
    d[:50] = 0
    d[50:60] = 1 << 29
    d[60:70] = 2 ** 31 - 1
    d[70:90] = np.arange(1, 21)
    qs[90:100] = [[0, 0], [(1 << 30) - 1, (1 << 30) - 1]] * 5
    qs[100:110] = [[1 << 29, 5], [7, (1 << 30) - 2]] * 5
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, cover_refine=cover)
    K = sfc.sfc_query_max_intervals(idx)
    assert K == (2 ** cover + 1) ** 2 if cover else K == 4
    lo, hi, b, e, c = sfc.sfc_query_ranges(idx, to_dev(qs, cuda), to_dev(d, cuda))
    lo, hi, b, e, c = u64(lo), u64(hi), b.cpu().numpy(), e.cpu().numpy(), c.cpu().numpy()
    ref = oracle.build(pts, 30, curve)
    for i in range(len(qs)):
        if cover == 0:
            cells, _ = oracle.cells(int(qs[i, 0]), int(qs[i, 1]), int(d[i]), 30, curve)
        else:
            cells = oracle.cells_refined(int(qs[i, 0]), int(qs[i, 1]), int(d[i]), 30, curve, cover)
        # the GPU merges intervals that abut in key order; the covered key set is the same
        merged = oracle.merge_abutting(cells)
        assert c[i] == len(merged) <= K
        for r, (a, z) in enumerate(merged):
            assert (int(lo[K * i + r]), int(hi[K * i + r])) == (a, z)
            assert b[K * i + r] == oracle.lower_bound(ref.keys, a)
            assert e[K * i + r] == oracle.lower_bound(ref.keys, z + 1)
        for r in range(len(merged), K):
            assert (int(lo[K * i + r]), int(hi[K * i + r])) == (1, 0)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 1, 2])
@pytest.mark.parametrize("seed,side_bits,max_delta", [(1, 4, 6), (2, 6, 20), (3, 10, 300),
                                                       (4, 30, 1 << 27), (5, 16, 70000)])
def test_tiny_vs_oracle(cuda, curve, cover, seed, side_bits, max_delta):
    """Every cover reports the oracle's answer (Alg. 1 over cells(Q)) in the same order."""
    pts, qs, d = W.tiny_dense(seed, 5000, 3000, side_bits, max_delta)
    assert_same(pts, qs, d, curve, cuda, cover_refine=cover)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [1, 2])
def test_finer_cover_scans_less(cuda, curve, cover):
    """A finer cover scans at most what cells(Q) scans (its cells lie inside cells(Q)'s), the
    scanned total equals the oracle's per-query scan over its own intervals, and the answer,
    with learned bounds too, is unchanged."""
    wl = W.mixed_1e7(scale=0.01)
    q, d = to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    scanned = {}
    for cv in (0, cover):
        idx, st = assert_same(wl.points, wl.queries, wl.delta, curve, cuda, cover_refine=cv,
                              bounds="learned")
        assert st == (0, 0)
        scanned[cv] = sfc.sfc_query_stats(idx)["scanned"]
    assert scanned[cover] <= scanned[0]
    ref = oracle.build(wl.points, 30, curve)
    want = 0
    for i in range(wl.m):
        for a, z in oracle.merge_abutting(oracle.cells_refined(int(wl.queries[i, 0]), int(wl.queries[i, 1]),
                                                               int(wl.delta[i]), 30, curve, cover)):
            want += oracle.lower_bound(ref.keys, z + 1) - oracle.lower_bound(ref.keys, a)
    assert scanned[cover] == want


@pytest.mark.parametrize("cover", [1, 2])
def test_finer_cover_chunks_and_rescan(cuda, cover):
    """Finer covers across chunk sizes and with the bitmask budget exhausted (the write pass
    re-filters), where a chunk spans many short intervals."""
    wl = W.mixed_1e7(scale=0.005)
    for chunk in (32, 1024, 4096):
        assert_same(wl.points, wl.queries, wl.delta, "h", cuda, cover_refine=cover, chunk=chunk)
    assert_same(wl.points, wl.queries, wl.delta, "z", cuda, cover_refine=cover, mask_budget_mb=1)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("chunk", [32, 96, 256, 1024, 2048, 4096])
def test_chunk_sizes(cuda, curve, chunk):
    """Every chunk size gives the same answer (chunks split one query's scan across warps)."""
    wl = W.mixed_1e7(scale=0.003)
    assert_same(wl.points, wl.queries, wl.delta, curve, cuda, chunk=chunk)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_rescan_past_mask_budget(cuda, curve):
    """With a 1 MB bitmask budget most chunks take the re-scan path of the write pass."""
    wl = W.mixed_1e7(scale=0.01)
    assert_same(wl.points, wl.queries, wl.delta, curve, cuda, mask_budget_mb=1)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_boundary_and_invalid(cuda, curve):
    c = (1 << 29) + 77
    on, out = W.pythagorean_ring(c, c - 5, 1000)
    pts = np.concatenate([on, out, np.array([[c, c - 5]], np.int32)])
    qs = np.array([[c, c - 5], [c, c - 5], [-1, 0], [0, 1 << 30], [c, c - 5], [c, c - 5]], np.int32)
    d = np.array([5000, 0, 10, 10, -3, 4999], np.int32)
    idx, st = assert_same(pts, qs, d, curve, cuda)
    assert st[0] == sfc.SFC_ERR_INVALID and st[1] & sfc.SFC_DEV_BAD_QUERY


def test_empty_batch_and_capacity(cuda):
    wl = W.uniform_1e5(scale=0.02)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z")
    q = to_dev(wl.queries, cuda)
    d = to_dev(wl.delta, cuda)
    off = torch.empty(1, dtype=torch.int64, device=cuda)
    sfc.sfc_query_batch(idx, q[:0], d[:0], off, torch.empty(0, dtype=torch.int32, device=cuda))
    assert off.tolist() == [0]
    # capacity too small: offsets complete, ids written only below capacity, flag raised
    full_off, full_ids = sfc.query(idx, q, d)
    total = int(full_off[-1])
    cap = total // 2
    off = torch.empty(wl.m + 1, dtype=torch.int64, device=cuda)
    ids = torch.full((total,), -1, dtype=torch.int32, device=cuda)
    sfc.sfc_query_batch(idx, q, d, off, ids, capacity=cap)
    st, bits = sfc.sfc_device_status(idx)
    assert st == sfc.SFC_ERR_CAPACITY and bits & sfc.SFC_DEV_CAPACITY
    assert torch.equal(off, full_off)
    assert torch.equal(ids[:cap], full_ids[:cap])
    assert bool((ids[cap:] == -1).all())


def test_write_requires_matching_count(cuda):
    wl = W.uniform_1e5(scale=0.01)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z")
    q = to_dev(wl.queries, cuda)
    d = to_dev(wl.delta, cuda)
    ids = torch.empty(10, dtype=torch.int32, device=cuda)
    off = torch.empty(wl.m + 1, dtype=torch.int64, device=cuda)
    with pytest.raises(sfc.SfcError) as e:
        sfc.sfc_query_write(idx, q, d, off, ids)
    assert e.value.status == sfc.SFC_ERR_STATE


@pytest.mark.parametrize("curve", ["z", "h"])
def test_uniform_1e5_full(cuda, curve):
    """The whole uniform-1e5 workload, bit-exact against the oracle and by set against brute
    force."""
    wl = W.uniform_1e5()
    idx, st = assert_same(wl.points, wl.queries, wl.delta, curve, cuda)
    assert st == (0, 0)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_host_buffer_api(cuda, curve):
    wl = W.mixed_1e7(scale=0.002)
    idx = sfc.sfc_build_host(wl.points, curve)
    ref = oracle.build(wl.points, 30, curve)
    roff, rids = oracle.query(ref, wl.queries, wl.delta)
    off, ids = sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, capacity=int(roff[-1]))
    assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    with pytest.raises(sfc.SfcError) as e:
        sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, capacity=int(roff[-1]) - 1)
    assert e.value.status == sfc.SFC_ERR_CAPACITY


def test_host_buffer_api_pinned_output(cuda):
    """Pinned and pageable host output buffers both receive the oracle's answer."""
    wl = W.mixed_1e7(scale=0.003)
    idx = sfc.sfc_build_host(wl.points, "z")
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta)
    total = int(roff[-1])
    pinned = torch.full((total,), -1, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    off, ids = sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, total, out_ids=pinned)
    assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    pageable = np.full(total, 7, np.uint32)
    off, ids = sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, total, out_ids=pageable)
    assert np.array_equal(ids, rids)


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("reorder", [0, 1])
def test_host_buffer_api_sliced_copy(cuda, pinned, reorder):
    """A batch with more than 32 MB of ids: the write pass runs in query slices and each
    slice's ids are copied out on a second stream while the next are written; with curve-order
    processing the order is first regrouped by slice."""
    wl = W.mixed_1e7(scale=0.05)
    idx = sfc.sfc_build_host(wl.points, "z", bounds="learned", cover_refine=1, reorder_queries=reorder)
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta, threads=8)
    total = int(roff[-1])
    assert total * 4 >= 32 << 20
    if pinned:
        out = torch.full((total,), -1, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    else:
        out = np.full(total, 7, np.uint32)
    for _ in range(2):
        off, ids = sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, total, out_ids=out)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)
    assert sfc.sfc_device_status(idx) == (0, 0)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("reorder", [0, 1])
def test_small_query_boundary(cuda, curve, reorder):
    """Queries that scan at most 64 points are counted and written one thread each: a stack
    of 64 equal points and one of 65, both queried with delta 0 (every scanned point a hit),
    plus scans of a few points among a background, equal the oracle on both sides of 64."""
    rng = np.random.default_rng(21)
    bg = rng.integers(0, 1 << 30, size=(5000, 2), dtype=np.int64)
    a, b = (1 << 20, 3 << 22), (5 << 25, 7 << 21)
    pts = np.concatenate([bg, np.tile(a, (64, 1)), np.tile(b, (65, 1))]).astype(np.int32)
    pts = pts[rng.permutation(len(pts))]
    qs = np.concatenate([[a, b, a, b], bg[:300]]).astype(np.int32)
    d = np.concatenate([[0, 0, 1, 1], rng.integers(0, 1 << 16, 300)]).astype(np.int32)
    for bounds in ("binary", "learned"):
        idx, st = assert_same(pts, qs, d, curve, cuda, bounds=bounds, reorder_queries=reorder)
        assert st == (0, 0)
    ref = oracle.build(pts, 30, curve)
    roff, _ = oracle.query(ref, qs, d)
    assert roff[1] - roff[0] == 64 and roff[2] - roff[1] == 65


def test_roads_scaled(cuda):
    wl = W.roads_3e7(scale=0.005)
    assert_same(wl.points, wl.queries, wl.delta, "h", cuda)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("reorder", [0, 1, 2])
def test_processing_order_does_not_change_results(cuda, curve, reorder):
    """Queries handed out in curve order of their centres (option 1) or input order (0) give
    identical offsets and id lists; invalid centres sort last."""
    wl = W.mixed_1e7(scale=0.01)
    qs = wl.queries.copy()
    d = wl.delta.copy()
    qs[::97] = [-5, 3]          # a few invalid centres
    for bounds in ("binary", "learned"):
        idx, st = assert_same(wl.points, qs, d, curve, cuda, reorder_queries=reorder, bounds=bounds)
        assert st[1] & ~sfc.SFC_DEV_BAD_QUERY == 0


def test_autotune(cuda):
    """The autotuner picks among the documented candidates, caches its choice per shape, and
    the answers after tuning still equal the oracle's."""
    wl = W.mixed_1e7(scale=0.02)
    q, d = to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned")
    choice = sfc.sfc_autotune(idx, q, d, force=True)
    assert choice["chunk"] in (256, 512, 1024, 2048, 4096) and choice["cover"] == 0
    assert choice["batch"] in (1, 2, 4, 8, 16) and choice["qbatch"] in (1, 2, 4, 8, 16)
    idx2 = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned")
    assert sfc.sfc_autotune(idx2, q, d) == choice          # served from the cache
    off, ids = sfc.query(idx2, q, d)
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)
    # cover chosen by the tuner (cover_refine = -1), then set by hand
    idx3 = sfc.sfc_build(to_dev(wl.points, cuda), "z", cover_refine=-1)
    assert sfc.sfc_cover_refine(idx3) == 1
    c3 = sfc.sfc_autotune(idx3, q, d, force=True)
    assert c3["cover"] in (0, 1, 2) and sfc.sfc_cover_refine(idx3) == c3["cover"]
    off, ids = sfc.query(idx3, q, d)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)
    sfc.sfc_set_cover(idx3, 2)
    assert sfc.sfc_query_max_intervals(idx3) == 25
    off, ids = sfc.query(idx3, q, d)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)
    with pytest.raises(sfc.SfcError):
        sfc.sfc_set_cover(idx3, 3)


def test_set_tuning(cuda):
    """Scan settings set by hand (chunk, count-pass and write-pass grabs), the extremes among
    them: the answers equal the oracle's under each; values out of range are refused and leave
    the last valid settings in place."""
    wl = W.mixed_1e7(scale=0.02)
    q, d = to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned", cover_refine=1)
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta)
    for chunk, batch, qbatch in [(32, 1, 1), (96, 3, 5), (4096, 16, 2), (4096, 1024, 1024)]:
        sfc.sfc_set_tuning(idx, chunk, batch, qbatch)
        off, ids = sfc.query(idx, q, d)
        assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids), (chunk, batch, qbatch)
    for bad in [(16, 1, 1), (4128, 1, 1), (100, 1, 1), (1024, 0, 1), (1024, 1, 0), (1024, 1025, 1),
                (1024, 1, 1025)]:
        with pytest.raises(sfc.SfcError):
            sfc.sfc_set_tuning(idx, *bad)
    off, ids = sfc.query(idx, q, d)   # the last valid settings are still in place
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 2])
def test_extreme_radii(cuda, curve, cover):
    """Queries whose disc covers the whole domain (every point reported, the scan is the whole
    array and spans hundreds of chunks), radius 0 on stacked duplicates, and tiny queries in the
    same batch."""
    rng = np.random.default_rng(12)
    pts = rng.integers(0, 1 << 30, size=(200_000, 2)).astype(np.int32)
    pts[:500] = [777, 999]                         # 500 duplicates of one point
    qs = np.concatenate([np.array([[0, 0], [(1 << 30) - 1, 5], [777, 999], [777, 999]], np.int32),
                         pts[rng.integers(0, 200_000, 300)]])
    d = np.concatenate([np.array([2 ** 31 - 1, 1 << 30, 0, 3], np.int32),
                        rng.integers(0, 1 << 16, 300).astype(np.int32)])
    idx, st = assert_same(pts, qs, d, curve, cuda, cover_refine=cover)
    off = oracle.query(oracle.build(pts, 30, curve), qs[:3], d[:3])[0]
    assert off[1] - off[0] == 200_000 and off[3] - off[2] == 500
    assert st == (0, 0)


@pytest.mark.parametrize("dim", [2, 3])
def test_rebuild_host_equals_rebuild(cuda, dim):
    """sfc_rebuild_host (points in host memory, staged by the index) leaves the index exactly as
    sfc_rebuild over the same points in device memory: sorted arrays and query results."""
    rng = np.random.default_rng(31)
    hi = 1 << (30 if dim == 2 else 21)
    p0 = rng.integers(0, hi, size=(20_000, dim), dtype=np.int64).astype(np.int32)
    p1 = rng.integers(0, hi, size=(30_000, dim), dtype=np.int64).astype(np.int32)
    q = p1[:500].copy()
    d = rng.integers(0, hi >> 8, 500).astype(np.int32)
    if dim == 2:
        a = sfc.sfc_build(torch.from_numpy(p0).to(cuda), "z", bounds="learned")
        b = sfc.sfc_build(torch.from_numpy(p0).to(cuda), "z", bounds="learned")
    else:
        a = sfc.sfc_build3(torch.from_numpy(p0).to(cuda))
        b = sfc.sfc_build3(torch.from_numpy(p0).to(cuda))
    for _ in range(2):
        sfc.sfc_rebuild(a, torch.from_numpy(p1).to(cuda))
        sfc.sfc_rebuild_host(b, p1)
        torch.cuda.synchronize()
        for x, y in zip(sfc.sfc_get_sorted(a), sfc.sfc_get_sorted(b)):
            assert torch.equal(x, y)
        qa, da = torch.from_numpy(q).to(cuda), torch.from_numpy(d).to(cuda)
        oa, ia = sfc.query(a, qa, da)
        ob, ib = sfc.query(b, qa, da)
        assert torch.equal(oa, ob) and torch.equal(ia, ib)
    assert sfc.sfc_device_status(a) == (0, 0) and sfc.sfc_device_status(b) == (0, 0)


@pytest.mark.parametrize("reorder", [0, 1])
@pytest.mark.parametrize("chunk", [256, 4096])
def test_big_queries_split_over_warps(cuda, reorder, chunk):
    """Queries that scan at least 8 chunks are written chunk by chunk by many warps, each chunk
    at its query's offset plus the hits of the query's earlier chunks.  A Gaussian cluster with
    40 discs covering most of it (about 2.6·10^5 hits each) among 20,000 small queries equals the
    oracle in both processing orders, through the device call and through the host call (whose
    write pass runs in slices: more than 32 MB of ids)."""
    rng = np.random.default_rng(41)
    c = rng.normal(1 << 29, 1 << 22, size=(300_000, 2))
    u = rng.integers(0, 1 << 30, size=(100_000, 2))
    pts = np.clip(np.concatenate([c, u]), 0, (1 << 30) - 1).astype(np.int32)
    qs = pts[rng.choice(len(pts), 20_000, replace=False)].copy()
    d = rng.integers(0, 1 << 16, 20_000).astype(np.int32)
    qs[:40] = (1 << 29) + rng.integers(-(1 << 20), 1 << 20, size=(40, 2))
    d[:40] = 1 << 23
    ref = oracle.build(pts, 30, "z")
    roff, rids = oracle.query(ref, qs, d, threads=8)
    assert int(roff[-1]) * 4 >= 32 << 20 and int(np.diff(roff).max()) > 200_000
    for bounds in ("binary", "learned"):
        idx, off, ids, st = run_gpu(pts, qs, d, "z", cuda, bounds=bounds, chunk=chunk, reorder_queries=reorder,
                                    cover_refine=1)
        assert st == (0, 0)
        assert np.array_equal(off, roff) and np.array_equal(ids, rids)
        hoff, hids = sfc.sfc_query_batch_host(idx, qs, d, int(roff[-1]))
        assert np.array_equal(hoff, roff) and np.array_equal(hids, rids)


def test_big_queries_with_small_mask_budget(cuda):
    """With a 1 MB hit-mask budget only the big queries whose chunks all have mask slots are
    split over warps; the others, and the chunks past the budget, are re-filtered by the query
    walk.  Results equal the oracle for chunk sizes that do and do not keep 16-byte mask rows."""
    rng = np.random.default_rng(47)
    c = rng.normal(1 << 29, 1 << 22, size=(200_000, 2))
    pts = np.clip(c, 0, (1 << 30) - 1).astype(np.int32)
    qs = pts[rng.choice(len(pts), 5_000, replace=False)].copy()
    d = rng.integers(0, 1 << 15, 5_000).astype(np.int32)
    qs[:30] = (1 << 29) + rng.integers(-(1 << 21), 1 << 21, size=(30, 2))
    d[:30] = 1 << 23
    for chunk in (96, 256):
        idx, st = assert_same(pts, qs, d, "z", cuda, chunk=chunk, mask_budget_mb=1, cover_refine=1,
                              reorder_queries=1)
        assert st == (0, 0)
