"""Parity at the workloads' full sizes, in the launch configuration bench.py uses.

The whole batch runs on the GPU; the oracle checks sampled queries one by one (exact id lists
in order, or by set against brute force), and the sorted arrays are checked completely by
properties that determine them uniquely: (key, id) strictly increasing, every key equal to the
oracle key of its id's point, and the ids exactly the live set."""
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
THREADS = os.cpu_count() or 1


def check_sorted_arrays(idx, xy_by_id, live_ids, curve, key_sample=None):
    keys, ids, xy = sfc.sfc_get_sorted(idx)
    k, i, p = u64(keys), u32(ids), xy.cpu().numpy()
    assert k.shape[0] == live_ids.shape[0]
    # (key, id) strictly increasing
    dk = np.diff(k.astype(np.int64))
    assert np.all(dk >= 0)
    same = dk == 0
    assert np.all(np.diff(i.astype(np.int64))[same] > 0)
    # ids are exactly the live set
    mark = np.zeros(xy_by_id.shape[0], bool)
    mark[i] = True
    assert mark.sum() == live_ids.shape[0] and mark[live_ids].all()
    # every key is the oracle key of its id's point, and xy is that point (all positions, or
    # a sample of positions when key_sample is given)
    sel = slice(None) if key_sample is None else np.random.default_rng(key_sample[0]).choice(
        k.shape[0], min(key_sample[1], k.shape[0]), replace=False)
    assert np.array_equal(p[sel], xy_by_id[i[sel]])
    assert np.array_equal(oracle.keys(p[sel], 30, curve), k[sel])


def check_sampled_queries(off, ids, pts, qs, d, sample, sorted_pos=None):
    off = u64(off)
    out = u32(ids)
    boff, bids = oracle.brute(pts, qs[sample], d[sample], threads=THREADS)
    for j, qi in enumerate(sample):
        got = out[off[qi]:off[qi + 1]]
        want = bids[boff[j]:boff[j + 1]]
        assert np.array_equal(np.sort(got), want), qi
        if sorted_pos is not None and got.size > 1:
            assert np.all(np.diff(sorted_pos[got]) > 0)   # ascending (key, id) order


@pytest.mark.parametrize("curve", ["z", "h"])
def test_mixed_1e7_full(cuda, curve):
    wl = W.mixed_1e7()
    pts = to_dev(wl.points, cuda)
    idx = sfc.sfc_build(pts, curve, bounds="learned")
    check_sorted_arrays(idx, wl.points, np.arange(wl.n), curve)
    off, ids = sfc.query(idx, to_dev(wl.queries, cuda), to_dev(wl.delta, cuda))
    # exact lists (in order) for a sample, against the oracle's Alg. 1
    ref = oracle.build(wl.points, 30, curve)
    sample = np.random.default_rng(0).choice(wl.m, 5000, replace=False)
    roff, rids = oracle.query(ref, wl.queries[sample], wl.delta[sample], threads=THREADS)
    o, out = u64(off), u32(ids)
    for j, qi in enumerate(sample):
        assert np.array_equal(out[o[qi]:o[qi + 1]], rids[roff[j]:roff[j + 1]]), qi
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_roads_3e7_graph_full(cuda):
    """The road-like workload at full size, Hilbert order, whole pipeline as one CUDA graph."""
    wl = W.roads_3e7()
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    idx = sfc.sfc_build(pts, "h")
    off, ids = sfc.query(idx, q, d)          # eager result, also sizes the output
    total = int(off[-1].item())
    goff = torch.zeros_like(off)
    gids = torch.zeros(total, dtype=torch.int32, device=cuda)
    g = sfc.sfc_graph_capture(idx, pts, q, d, goff, gids)
    g.launch()
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(goff, off) and torch.equal(gids, ids)
    check_sorted_arrays(idx, wl.points, np.arange(wl.n), "h")
    keys, sid, _ = sfc.sfc_get_sorted(idx)
    pos = np.empty(wl.n, np.int64)
    pos[u32(sid)] = np.arange(wl.n)
    sample = np.random.default_rng(1).choice(wl.m, 300, replace=False)
    check_sampled_queries(goff, gids, wl.points, wl.queries, wl.delta, sample, pos)
    mean_k = total / wl.m
    assert 25 < mean_k < 100, mean_k   # about 50 points per query by construction
    g.close()


def test_mixed_1e8_learned_vs_binary_full(cuda):
    """10^8 points, 10^7 queries, Z order, 4096-leaf learned model: the learned-bounds output is
    bit-identical to the binary-search output, 10^5 sampled queries equal the oracle's id lists
    (in order) and 100 of them match brute force."""
    wl = W.mixed_1e8()
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    idx = sfc.sfc_build(pts, "z", bounds="learned", leaves=4096)
    off_l, ids_l = sfc.query(idx, q, d)
    stats = sfc.sfc_model_stats(idx)
    sfc.sfc_set_bounds_mode(idx, "binary")
    off_b = sfc.sfc_query_count(idx, q, d)
    assert torch.equal(off_b, off_l)
    ids_b = torch.empty_like(ids_l)
    sfc.sfc_query_write(idx, q, d, off_b, ids_b)
    assert torch.equal(ids_b, ids_l)
    del ids_b
    assert stats["misses"] <= 0.001 * stats["endpoints"], stats
    # exact id lists, in order, of 10^5 sampled queries against the oracle's Alg. 1 over the
    # whole point set, and 100 of them by set against brute force
    ref = oracle.build(wl.points, 30, "z")
    sample = np.sort(np.random.default_rng(2).choice(wl.m, 100_000, replace=False))
    roff, rids = oracle.query(ref, wl.queries[sample], wl.delta[sample], threads=THREADS)
    o, out = u64(off_l), u32(ids_l)
    got_len = (o[sample + 1] - o[sample]).astype(np.int64)
    assert np.array_equal(got_len, np.diff(roff.astype(np.int64)))
    got = np.concatenate([out[o[qi]:o[qi + 1]] for qi in sample])
    assert np.array_equal(got, rids)
    check_sampled_queries(off_l, ids_l, wl.points, wl.queries, wl.delta, sample[:100])
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_dynamic_5e7_rounds_full(cuda):
    """Base 5*10^7 clustered points, 20 rounds of 5*10^5 deletes + 10^6 inserts + 10^6 queries;
    after every round the arrays equal a rebuild from scratch over the live set (by the
    properties above: order and id set on every round, keys of all positions on the first,
    middle and last round and of 10^6 sampled positions on the others) and sampled queries
    match brute force over the live points."""
    dwl = W.dynamic_5e7(rounds=20)
    idx = sfc.sfc_build(to_dev(dwl.base, cuda), "z", bounds="learned")
    xy_by_id = dwl.base.copy()
    alive = np.ones(dwl.base.shape[0], bool)
    cluster = dwl.meta["base_cluster"]
    rng = np.random.default_rng(3)
    for r, rd in enumerate(dwl.rounds):
        live = np.nonzero(alive)[0]
        dels = live[rd["delete_rank"]].astype(np.uint32)
        first = sfc.sfc_update(idx, to_dev(rd["inserts"], cuda), to_dev(dels.view(np.int32), cuda))
        assert first == xy_by_id.shape[0]
        alive[dels] = False
        xy_by_id = np.concatenate([xy_by_id, rd["inserts"]])
        alive = np.concatenate([alive, np.ones(rd["inserts"].shape[0], bool)])
        cluster = np.concatenate([cluster, rd["insert_cluster"]])
        live = np.nonzero(alive)[0]
        full = r in (0, len(dwl.rounds) // 2, len(dwl.rounds) - 1)
        check_sorted_arrays(idx, xy_by_id, live, "z", None if full else (r, 1_000_000))
        qs, d = W.dynamic_round_queries(dwl, r, xy_by_id[live], cluster[live])
        off, ids = sfc.query(idx, to_dev(qs, cuda), to_dev(d, cuda))
        sample = rng.choice(qs.shape[0], 40, replace=False)
        off_h, ids_h = u64(off), u32(ids)
        boff, bids = oracle.brute(xy_by_id[live], qs[sample], d[sample], threads=THREADS)
        for j, qi in enumerate(sample):
            got = np.sort(ids_h[off_h[qi]:off_h[qi + 1]])
            want = live[bids[boff[j]:boff[j + 1]]].astype(np.uint32)
            assert np.array_equal(got, want), (r, qi)
    assert sfc.sfc_device_status(idx) == (0, 0)
