"""GPU parity of key generation (Alg. 2, Sec. 2.1), the construction sort (Sec. 3.1.1) and
the exclusive scan, against the oracle / library routines.  Integer work: bit-exact."""
import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _points(kind, n, seed=0):
    rng = np.random.default_rng(seed)
    if kind == "uniform":
        return rng.integers(0, 1 << 30, size=(n, 2)).astype(np.int32)
    if kind == "dups":
        return rng.integers(0, 8, size=(n, 2)).astype(np.int32)
    if kind == "equal":
        return np.full((n, 2), 12345, np.int32)
    if kind == "top":   # only the top bits vary: only the highest digits are live
        return (rng.integers(0, 4, size=(n, 2)) << 28).astype(np.int32)
    if kind == "corner":
        return np.array([[0, 0], [(1 << 30) - 1, 0], [0, (1 << 30) - 1], [(1 << 30) - 1] * 2] * (n // 4 + 1),
                        np.int32)[:n]
    if kind == "small":
        return rng.integers(0, 1 << 20, size=(n, 2)).astype(np.int32)
    raise ValueError(kind)


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("n", [1, 2, 3, 1000, 65537])
def test_keys_and_decode(cuda, curve, n):
    pts = _points("uniform", n, n)
    pts[:4 if n >= 4 else n] = _points("corner", min(n, 4))
    k = sfc.sfc_keys(to_dev(pts, cuda), curve)
    ref = oracle.keys(pts, 30, curve)
    assert np.array_equal(u64(k), ref)
    back = sfc.sfc_decode(k, curve)
    assert np.array_equal(back.cpu().numpy(), pts)


@pytest.mark.parametrize("curve", ["z", "h"])
def test_keys_unaligned_pointer(cuda, curve):
    pts = _points("uniform", 1001, 5)
    t = to_dev(pts, cuda)
    out = torch.empty(1001, dtype=torch.int64, device=cuda)
    sfc.sfc_keys(t[1:], curve, out=out[1:])
    assert np.array_equal(u64(out[1:]), oracle.keys(pts[1:], 30, curve))


@pytest.mark.parametrize("curve", ["z", "h"])
@pytest.mark.parametrize("kind,n", [("uniform", 100_003), ("dups", 50_000), ("equal", 9000),
                                    ("top", 20_000), ("small", 4096), ("small", 4097),
                                    ("uniform", 1), ("uniform", 5), ("corner", 33)])
def test_build_sort_matches_oracle(cuda, curve, kind, n):
    pts = _points(kind, n, 3)
    idx = sfc.sfc_build(to_dev(pts, cuda), curve)
    keys, ids, xy = sfc.sfc_get_sorted(idx)
    ref = oracle.build(pts, 30, curve)
    assert np.array_equal(u64(keys), ref.keys)
    assert np.array_equal(u32(ids), ref.ids)
    assert np.array_equal(xy.cpu().numpy(), ref.xy)
    assert sfc.sfc_device_status(idx) == (0, 0)


def test_build_empty(cuda):
    idx = sfc.sfc_build(torch.empty((0, 2), dtype=torch.int32, device=cuda), "z")
    keys, ids, xy = sfc.sfc_get_sorted(idx)
    assert keys.numel() == 0
    off, out = sfc.query(idx, torch.tensor([[5, 5]], dtype=torch.int32, device=cuda),
                         torch.tensor([100], dtype=torch.int32, device=cuda))
    assert off.tolist() == [0, 0] and out.numel() == 0


def test_build_flags_bad_points(cuda):
    pts = np.array([[1, 2], [-1, 3], [5, 1 << 30]], np.int32)
    idx = sfc.sfc_build(to_dev(pts, cuda), "z")
    st, bits = sfc.sfc_device_status(idx)
    assert st == sfc.SFC_ERR_INVALID and bits & sfc.SFC_DEV_BAD_POINT
    assert sfc.sfc_device_status(idx) == (0, 0)     # reading clears the word


@pytest.mark.parametrize("kind", ["random", "sorted", "reversed", "equal", "topdigit", "twovals"])
@pytest.mark.parametrize("n", [1, 4095, 4096, 70_001])
def test_sort_pairs(cuda, kind, n):
    rng = np.random.default_rng(n)
    if kind == "random":
        k = rng.integers(0, 1 << 60, size=n, dtype=np.int64)
    elif kind == "sorted":
        k = np.sort(rng.integers(0, 1 << 60, size=n, dtype=np.int64))
    elif kind == "reversed":
        k = np.sort(rng.integers(0, 1 << 60, size=n, dtype=np.int64))[::-1].copy()
    elif kind == "equal":
        k = np.full(n, 77, np.int64)
    elif kind == "topdigit":
        k = rng.integers(0, 16, size=n, dtype=np.int64) << 56
    else:
        k = rng.integers(0, 2, size=n, dtype=np.int64) * ((1 << 60) - 1)
    vals = rng.permutation(n).astype(np.int32)
    ko, io = sfc.sfc_sort_pairs(to_dev(k, cuda), to_dev(vals, cuda))
    order = np.lexsort((np.arange(n), k))    # stable by key
    assert np.array_equal(ko.cpu().numpy(), k[order])
    assert np.array_equal(io.cpu().numpy(), vals[order])


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 4095, 4096, 4097, 1_000_003])
def test_exclusive_scan(cuda, n):
    rng = np.random.default_rng(n)
    x = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        x[:10] = 0xFFFFFFFF      # sums past 2^32 need the 64-bit accumulator
    out = sfc.sfc_exclusive_scan(to_dev(x.view(np.int32), cuda))
    ref = np.zeros(n + 1, np.uint64)
    np.cumsum(x.astype(np.uint64), out=ref[1:])
    assert np.array_equal(u64(out), ref)


def test_scan_unaligned(cuda):
    x = np.arange(10_001, dtype=np.int32)
    t = to_dev(x, cuda)
    out = sfc.sfc_exclusive_scan(t[1:])
    ref = np.zeros(10_001, np.uint64)
    np.cumsum(x[1:].astype(np.uint64), out=ref[1:])
    assert np.array_equal(u64(out), ref)
