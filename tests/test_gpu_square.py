"""Square-window queries on the GPU (the windows of the paper's experiments, Sec. 3): bit-exact
against the oracle's Alg. 1 with the square window, on tiny adversarial inputs and on the
paper's three synthetic distributions, under every cover, both bound searches, early
termination, and when one index switches between disc and square windows."""
import numpy as np
import pytest

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _same(idx, qs, d, ref, cuda, norm="square"):
    off, ids = sfc.query(idx, to_dev(qs, cuda), to_dev(d, cuda))
    roff, rids = oracle.query(ref, qs, d, norm=norm)
    assert np.array_equal(u64(off), roff)
    assert np.array_equal(u32(ids), rids)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [0, 1, 2])
@pytest.mark.parametrize("seed,side_bits,max_delta", [(1, 4, 6), (3, 10, 300), (4, 30, 1 << 27)])
def test_tiny_square(cuda, curve, cover, seed, side_bits, max_delta):
    pts, qs, d = W.tiny_dense(seed, 5000, 3000, side_bits, max_delta)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, query_norm="square", cover_refine=cover)
    _same(idx, qs, d, oracle.build(pts, 30, curve), cuda)


@pytest.mark.parametrize("dist", ["uniform", "normal", "skewed"])
@pytest.mark.parametrize("rel", [1e-4, 1e-3, 1e-2])
def test_paper_distributions_square(cuda, dist, rel):
    wl = W.paper_static(dist, 200_000, 5000, rel)
    for curve, bounds in (("z", "learned"), ("h", "binary")):
        idx = sfc.sfc_build(to_dev(wl.points, cuda), curve, query_norm="square", bounds=bounds,
                            cover_refine=1, occupancy_depth=12)
        _same(idx, wl.queries, wl.delta, oracle.build(wl.points, 30, curve), cuda)
        assert sfc.sfc_device_status(idx) == (0, 0)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("cover", [1, 2])
def test_square_ranges(cuda, curve, cover):
    pts, qs, d = W.tiny_dense(11, 3000, 1500, 30, 1 << 26)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve, query_norm="square", cover_refine=cover)
    K = sfc.sfc_query_max_intervals(idx)
    lo, hi, b, e, c = sfc.sfc_query_ranges(idx, to_dev(qs, cuda), to_dev(d, cuda))
    lo, hi, c = u64(lo), u64(hi), c.cpu().numpy()
    for i in range(len(qs)):
        merged = oracle.merge_abutting(oracle.cells_refined(int(qs[i, 0]), int(qs[i, 1]), int(d[i]), 30, curve,
                                                            cover, norm="square"))
        assert c[i] == len(merged)
        for r, (a, z) in enumerate(merged):
            assert (int(lo[K * i + r]), int(hi[K * i + r])) == (a, z)


def test_switch_norm_on_one_index(cuda):
    wl = W.mixed_1e7(scale=0.01)
    idx = sfc.sfc_build(to_dev(wl.points, cuda), "z", bounds="learned", cover_refine=1)
    ref = oracle.build(wl.points)
    _same(idx, wl.queries, wl.delta, ref, cuda, norm="disc")
    sfc.sfc_set_query_norm(idx, "square")
    _same(idx, wl.queries, wl.delta, ref, cuda, norm="square")
    sfc.sfc_set_query_norm(idx, "disc")
    _same(idx, wl.queries, wl.delta, ref, cuda, norm="disc")
    assert sfc.lib().sfc_set_query_norm(idx.handle, 2) == sfc.SFC_ERR_INVALID
