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
def test_ranges_and_bounds(cuda, curve):
    pts, qs, d = W.tiny_dense(11, 3000, 2000, 30, 1 << 26)
    d[:50] = 0
    d[50:60] = 1 << 29
    d[60:70] = 2 ** 31 - 1
    qs[70:80] = [[0, 0], [(1 << 30) - 1, (1 << 30) - 1]] * 5
    idx = sfc.sfc_build(to_dev(pts, cuda), curve)
    lo, hi, b, e, c = sfc.sfc_query_ranges(idx, to_dev(qs, cuda), to_dev(d, cuda))
    lo, hi, b, e, c = u64(lo), u64(hi), b.cpu().numpy(), e.cpu().numpy(), c.cpu().numpy()
    ref = oracle.build(pts, 30, curve)
    for i in range(len(qs)):
        cells, _ = oracle.cells(int(qs[i, 0]), int(qs[i, 1]), int(d[i]), 30, curve)
        # the GPU merges intervals that abut in key order; the covered key set is the same
        merged = []
        for a, z in cells:
            if merged and merged[-1][1] + 1 == a:
                merged[-1] = (merged[-1][0], z)
            else:
                merged.append((a, z))
        assert c[i] == len(merged) <= 4
        for r, (a, z) in enumerate(merged):
            assert (int(lo[4 * i + r]), int(hi[4 * i + r])) == (a, z)
            assert b[4 * i + r] == oracle.lower_bound(ref.keys, a)
            assert e[4 * i + r] == oracle.lower_bound(ref.keys, z + 1)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("seed,side_bits,max_delta", [(1, 4, 6), (2, 6, 20), (3, 10, 300),
                                                       (4, 30, 1 << 27), (5, 16, 70000)])
def test_tiny_vs_oracle(cuda, curve, seed, side_bits, max_delta):
    pts, qs, d = W.tiny_dense(seed, 5000, 3000, side_bits, max_delta)
    assert_same(pts, qs, d, curve, cuda)


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
    assert choice["chunk"] in (256, 512, 1024, 2048, 4096)
    assert choice["batch"] in (1, 2, 4, 8, 16) and choice["qbatch"] in (1, 2, 4, 8, 16)
    idx2 = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned")
    assert sfc.sfc_autotune(idx2, q, d) == choice          # served from the cache
    off, ids = sfc.query(idx2, q, d)
    roff, rids = oracle.query(oracle.build(wl.points), wl.queries, wl.delta)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_extreme_radii(cuda, curve):
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
    idx, st = assert_same(pts, qs, d, curve, cuda)
    off = oracle.query(oracle.build(pts, 30, curve), qs[:3], d[:3])[0]
    assert off[1] - off[0] == 200_000 and off[3] - off[2] == 500
    assert st == (0, 0)
