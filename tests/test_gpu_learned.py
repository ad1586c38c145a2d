"""GPU learned bounds: the training kernels against the fp64 oracle (gradient, Adam step),
and the learned bound search against binary search (bit-exact positions and outputs)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import learned as OL
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu

H = 16


def _sample(keys_sorted, s):
    n = keys_sorted.shape[0]
    i = (np.arange(s, dtype=np.float64) * n / s).astype(np.int64)
    return keys_sorted[i], (i / n)


K = 256


@pytest.mark.parametrize("root", ["mlp", "pwl"])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_fp64_oracle(cuda, root, seed):
    """The training kernels' loss and gradient against the fp64 analytic reference (itself
    pinned by finite differences), relative tolerance 1e-3 (fp32 accumulation)."""
    assert sfc.sfc_model_hidden() == H
    assert sfc.sfc_model_params("mlp") == 3 * H + 1 and sfc.sfc_model_params("pwl") == K + 1
    wl = (W.mixed_1e7(scale=0.01, seed=seed + 10) if seed != 2
          else W.normal_uniform_queries(100_000, 1, 0.001))
    ref = oracle.build(wl.points)
    k, y = _sample(ref.keys, 4096)
    rng = np.random.default_rng(seed)
    x = k.astype(np.float64) / 2.0 ** 60
    y32 = y.astype(np.float32).astype(np.float64)
    if root == "mlp":
        theta = (OL.init_params(H) + rng.normal(0, 0.3, 3 * H + 1)).astype(np.float32)
        rloss, rg = OL.root_loss_grad(theta.astype(np.float64), x, y32, H)
    else:
        theta = OL.pwl_project(OL.pwl_init(K) + rng.normal(0, 0.01, K + 1)).astype(np.float32)
        rloss, rg = OL.pwl_loss_grad(theta.astype(np.float64), x, y32, K)
    loss, g = sfc.sfc_model_loss_grad(theta, to_dev(k.view(np.int64), cuda),
                                      to_dev(y.astype(np.float32), cuda), root=root)
    assert loss == pytest.approx(rloss, rel=1e-3)
    scale = np.abs(rg).max()
    np.testing.assert_allclose(g, rg, rtol=1e-3, atol=1e-3 * scale)


@pytest.mark.parametrize("npar", [3 * H + 1, K + 1])
def test_adam_step_matches_oracle(cuda, npar):
    rng = np.random.default_rng(4)
    th = rng.normal(0, 1, npar)
    m = rng.normal(0, 0.1, npar)
    v = np.abs(rng.normal(0, 0.1, npar))
    g = rng.normal(0, 1, npar)
    for t in (1, 2, 50):
        p, mm, vv = sfc.sfc_model_adam_step(th, m, v, g, t, 0.02)
        rp, rm, rv = OL.adam_step(th, g, m, v, t, 0.02)
        np.testing.assert_allclose(mm, rm, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(vv, rv, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(p, rp, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("root", ["mlp", "pwl"])
def test_training_lowers_the_loss(cuda, root):
    wl = W.normal_uniform_queries(200_000, 1, 0.001)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned", root=root, train_steps=25)
    model = sfc.sfc_model_get(idx)
    assert model["root"] == root
    ref = oracle.build(wl.points)
    k, y = _sample(ref.keys, 65536)
    x = k.astype(np.float64) / 2.0 ** 60
    p = model["params"].astype(np.float64)
    if root == "mlp":
        trained, initial = OL.root_loss(p, x, y, H), OL.root_loss(OL.init_params(H), x, y, H)
    else:
        trained, initial = OL.pwl_loss(p, x, y, K), OL.pwl_loss(OL.pwl_init(K), x, y, K)
    assert trained < 0.5 * initial, (trained, initial)
    # leaves tile the array: first/end are monotone and cover [0, n)
    first, end = model["first"].astype(np.int64), model["end"].astype(np.int64)
    assert first[0] == 0 and end[-1] == wl.n
    assert np.all(end >= first) and np.all(first[1:] == end[:-1])


@pytest.mark.parametrize("root", ["pwl", "mlp"])
@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("make", ["uniform", "mixed", "dups", "tiny", "normal"])
def test_learned_equals_binary(cuda, curve, make, root):
    if make == "uniform":
        wl = W.uniform_1e5()
        pts, qs, d = wl.points, wl.queries, wl.delta
    elif make == "mixed":
        wl = W.mixed_1e7(scale=0.02)
        pts, qs, d = wl.points, wl.queries, wl.delta
    elif make == "dups":
        pts, qs, d = W.tiny_dense(3, 20000, 3000, 6, 10)
    elif make == "normal":
        wl = W.normal_uniform_queries(100_000, 5000, 0.003)
        pts, qs, d = wl.points, wl.queries, wl.delta
    else:
        pts, qs, d = W.tiny_dense(4, 3, 500, 30, 1 << 20)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, bounds="learned", leaves=512, root=root)
    qt, dt = to_dev(qs, cuda), to_dev(d, cuda)
    lo, hi, bl, el, cl = sfc.sfc_query_ranges(idx, qt, dt)
    offl, idsl = sfc.query(idx, qt, dt)
    stats = sfc.sfc_model_stats(idx)
    sfc.sfc_set_bounds_mode(idx, "binary")
    lo2, hi2, bb, eb, cb = sfc.sfc_query_ranges(idx, qt, dt)
    offb, idsb = sfc.query(idx, qt, dt)
    assert torch.equal(cl, cb) and torch.equal(lo, lo2) and torch.equal(hi, hi2)
    assert torch.equal(bl, bb) and torch.equal(el, eb)
    assert torch.equal(offl, offb) and torch.equal(idsl, idsb)
    ref = oracle.build(pts, 30, curve)
    roff, rids = oracle.query(ref, qs, d)
    assert np.array_equal(u64(offl), roff) and np.array_equal(u32(idsl), rids)
    # the window misses at most a sliver of endpoints (they fall back to binary search)
    assert stats["endpoints"] > 0
    assert stats["misses"] <= 0.01 * stats["endpoints"] + 2, stats
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_learned_on_empty_and_single(cuda):
    for n in (0, 1, 2):
        pts = np.array([[5, 9], [5, 9]][:n], np.int32).reshape(-1, 2)
        idx = sfc.sfc_build(to_dev(pts, cuda), "z", bounds="learned")
        q = to_dev(np.array([[5, 9], [0, 0]], np.int32), cuda)
        d = to_dev(np.array([0, 3], np.int32), cuda)
        off, ids = sfc.query(idx, q, d)
        assert off.tolist() == [0, n, n]


def test_learned_vs_binary_timed(cuda):
    """What the learned model changes, timed: the plan phase (range derivation + bound search)
    of one query batch over 3 * 10^7 points (keys beyond L2) with learned bounds (trained root),
    learned bounds with the root left at its start (0 Adam steps) and binary search over the
    same index, each best of 3 by CUDA events; all three times are printed and the outputs are
    bit-identical.  The mean searched window of the learned bounds (fence bracket within the
    error window) is a few hundred keys against the whole array for binary search; whether that
    makes the phase faster is what the times show (bench.py's bounds_comparison reports the same
    at 10^8 with medians and spread)."""
    wl = W.mixed_1e8(scale=0.3)
    pts, qt, dt = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    trained = sfc.sfc_build(pts, "z", bounds="learned", cover_refine=1, profile=1)
    untrained = sfc.sfc_build(pts, "z", bounds="learned", cover_refine=1, profile=1, train_steps=0)
    runs = {}
    outs = {}
    for name, idx, mode in (("learned", trained, "learned"), ("binary", trained, "binary"),
                            ("learned_0_steps", untrained, "learned")):
        sfc.sfc_set_bounds_mode(idx, mode)
        best = float("inf")
        for _ in range(3):
            sfc.sfc_profile_read(idx, reset=True)
            off = sfc.sfc_query_count(idx, qt, dt)
            best = min(best, sfc.sfc_profile_read(idx, reset=True)["plan"][1])
        runs[name] = best
        off, ids = sfc.query(idx, qt, dt)
        outs[name] = (off, ids)
        if mode == "learned":
            st = sfc.sfc_model_stats(idx)
            runs[name + "_window"] = st["window_sum"] / st["endpoints"]
            assert st["misses"] <= 0.001 * st["endpoints"], st
    print("plan phase ms (best of 3), n = 3e7, m = 3e6:", runs)
    for name in ("learned", "learned_0_steps"):
        assert torch.equal(outs[name][0], outs["binary"][0]) and torch.equal(outs[name][1], outs["binary"][1])
        assert runs[name + "_window"] < 1000, runs
    for v in runs.values():
        assert v > 0
    trained.close()
    untrained.close()


def test_trained_vs_untrained_root(cuda):
    """Training the root against the key CDF spreads the keys more evenly over the leaves
    (the largest leaf shrinks against the untrained identity root); the mean windows of both
    are recorded.  Both stay far below n."""
    wl = W.normal_uniform_queries(1_000_000, 50_000, 0.001)
    pts, qt, dt = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    res = {}
    for root in ("pwl", "mlp"):
        for steps in (0, 300):
            idx = sfc.sfc_build(pts, "z", bounds="learned", train_steps=steps, root=root)
            sfc.query(idx, qt, dt)
            st = sfc.sfc_model_stats(idx)
            m = sfc.sfc_model_get(idx)
            sizes = (m["end"].astype(np.int64) - m["first"].astype(np.int64))
            res[(root, steps)] = (st["window_sum"] / st["endpoints"], int(sizes.max()))
    print("normal points: (mean window, largest leaf) by (root, steps):", res)
    assert res[("pwl", 300)][1] < res[("pwl", 0)][1], res
    for v in res.values():
        assert v[0] < wl.n / 100


@pytest.mark.parametrize("curve", ["z", "h"])
def test_fence_matches_oracle(cuda, curve):
    """The leaves' coarse (16) and fine (256) fences are the keys at the positions the
    definition gives (oracle learned.leaf_fence over the oracle's sorted keys and the GPU's leaf
    ranges), and a learned query batch still equals binary search."""
    from oracle import learned as L
    wl = W.mixed_1e7(scale=0.02)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), curve, bounds="learned")
    m = sfc.sfc_model_get(idx)
    fence = sfc.sfc_model_fence(idx)
    fine = sfc.sfc_model_fence_fine(idx)
    ref = oracle.build(wl.points, 30, curve)
    for j in range(len(m["first"])):
        f, e = int(m["first"][j]), int(m["end"][j])
        assert np.array_equal(fence[j], L.leaf_fence(ref.keys, f, e)), j
        assert np.array_equal(fine[j], L.leaf_fence(ref.keys, f, e, k=256)), j
        assert np.array_equal(fine[j][::16], fence[j]), j   # coarse key s is fine key 16 s
    off, ids = sfc.query(idx, to_dev(wl.queries, cuda), to_dev(wl.delta, cuda))
    roff, rids = oracle.query(ref, wl.queries, wl.delta)
    assert np.array_equal(u64(off), roff) and np.array_equal(u32(ids), rids)
    st = sfc.sfc_model_stats(idx)
    assert st["misses"] == 0 and st["window_sum"] / st["endpoints"] < 0.5 * wl.n / 4096 + 2


def _leaf_stage_points(kind):
    if kind == "clustered":   # all clustered (the dynamic workload's base shape), n = 10^6
        return W.dynamic_5e7(scale=0.02, rounds=1).base
    return W.mixed_1e7(scale=0.1 if kind == "mixed-1e6" else 1.0).points


@pytest.mark.parametrize("curve,root,kind", [("z", "pwl", "mixed-1e6"), ("h", "pwl", "mixed-1e6"),
                                             ("z", "mlp", "mixed-1e6"), ("z", "pwl", "clustered"),
                                             ("z", "pwl", "mixed-1e7")])
def test_leaf_stage_matches_oracle(cuda, curve, root, kind):
    """The leaf stage of the fit against the oracle, leaf by leaf over the oracle's sorted keys.

    Line: the GPU's least-squares line of position against key offset (fitted in fp32) equals
    oracle.learned.leaf_fit (fp64 normal equations): slope within a relative 1e-3, and the two
    lines within 1e-3 * (keys in the leaf) + 1e-3 positions of each other at both ends of the
    leaf's key range (fp32 sums over up to a few 10^4 keys lose about 1e-5 relative; a wrong
    term or sign is off by whole positions).
    Error window: err_lo and err_hi are exactly the min and max of position - prediction over
    the leaf's keys, with the prediction taken by the query-time fp32 function
    (oracle.learned.predict_positions) from the leaf's own slope and intercept -- so every key
    of every leaf lies in its window and both ends are attained; empty leaves get (0, 0).  (On
    all-clustered points most of the 4,096 leaves stay empty: the 256-knot root cannot resolve
    1,000 narrow clusters, so a few hundred leaves hold all keys.)"""
    pts = _leaf_stage_points(kind)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, bounds="learned", root=root)
    m = sfc.sfc_model_get(idx)
    keys = oracle.build(pts, 30, curve).keys
    n = keys.shape[0]
    first, end = m["first"].astype(np.int64), m["end"].astype(np.int64)
    assert first[0] == 0 and end[-1] == n and np.all(end >= first)
    L = first.shape[0]
    checked = 0
    for j in range(L):
        f, e = int(first[j]), int(end[j])
        c = e - f
        if c == 0:
            assert m["err_lo"][j] == 0 and m["err_hi"][j] == 0, j
            continue
        kk = keys[f:e]
        base = int(kk[0])
        u = (kk - np.uint64(base)).astype(np.float64)
        s_ref, c_ref = OL.leaf_fit(u, np.arange(c, dtype=np.float64))
        s_gpu, c_gpu = float(m["slope"][j]), float(m["icpt"][j])
        if c >= 2:
            assert abs(s_gpu - s_ref) <= 1e-3 * abs(s_ref) + 1e-30, (j, s_gpu, s_ref)
            for uu in (0.0, float(u[-1])):
                assert abs((s_gpu * uu + c_gpu) - (s_ref * uu + c_ref)) <= 1e-3 * c + 1e-3, (j, uu)
        pred = OL.predict_positions(m["slope"][j], m["icpt"][j], f, base, kk)
        res = np.clip(np.arange(f, e, dtype=np.int64) - pred, -0x7fffffff, 0x7fffffff)
        assert int(m["err_lo"][j]) == int(res.min()) and int(m["err_hi"][j]) == int(res.max()), \
            (j, int(m["err_lo"][j]), int(m["err_hi"][j]), int(res.min()), int(res.max()))
        checked += c
    assert checked == n   # every key of every leaf was checked
    idx.close()
