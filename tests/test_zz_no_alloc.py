"""The scan entry point that allocates no device memory (sfc_exclusive_scan_noalloc) gives
the same result as the allocating one (sfc_exclusive_scan), on two calls in a row.

It exists for callers that must not allocate device memory (a host framework's caching pool
owns the memory, or a loop cannot take cudaMalloc's implicit synchronisation); its scratch is
a fixed array in device memory shared by all calls, with a status word that
sfc_exclusive_scan_noalloc_status reads.  This file is collected last so that a
stop-at-first-failure run has already run every other test; it also passes on its own.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2508_19891_gb300 as sfc

pytestmark = pytest.mark.gpu

MAX_ITEMS = 16384 * 4096


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_19891_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    return torch.device("cuda", 0)


@pytest.mark.parametrize("n", [1, 4096, 4097, 1_000_003])
def test_noalloc_scan_matches_allocating_scan_twice(dev, n):
    rng = np.random.default_rng(n)
    for call in range(2):
        x = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
        x[: min(n, 8)] = 0xFFFFFFFF
        t = torch.from_numpy(x.view(np.int32)).to(dev)
        ref = sfc.sfc_exclusive_scan(t)
        out = sfc.sfc_exclusive_scan_noalloc(t)
        assert sfc.sfc_exclusive_scan_noalloc_status() == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, call)


@pytest.mark.parametrize("n", [MAX_ITEMS - 1, MAX_ITEMS])
def test_noalloc_scan_at_the_array_limit(dev, n):
    """The largest sizes use every word of the fixed array (16,384 tiles); checked against the
    allocating scan and, at the sampled positions, against int64 partial sums."""
    rng = np.random.default_rng(n % 1000)
    x = rng.integers(0, 2 ** 32, size=n, dtype=np.uint64).astype(np.uint32)
    t = torch.from_numpy(x.view(np.int32)).to(dev)
    for call in range(2):
        out = sfc.sfc_exclusive_scan_noalloc(t)
        assert sfc.sfc_exclusive_scan_noalloc_status() == 0
        ref = sfc.sfc_exclusive_scan(t)
        assert torch.equal(out, ref), call
    cs = np.concatenate([[0], np.cumsum(x.astype(np.uint64))])
    pos = np.array([0, 1, 4095, 4096, n // 2, n - 4097, n - 1, n])
    assert np.array_equal(out[torch.from_numpy(pos).to(dev)].cpu().numpy().view(np.uint64), cs[pos])
    del t, out, ref


def test_noalloc_scan_limits(dev):
    out = torch.empty(1, dtype=torch.int64, device=dev)
    sfc.sfc_exclusive_scan_noalloc(torch.empty(0, dtype=torch.int32, device=dev), out=out)
    assert out.tolist() == [0]
    assert sfc.sfc_exclusive_scan_noalloc_status() == 0
    # one past the maximum is rejected before anything is enqueued (no buffer is read)
    L = sfc.lib()
    st = L.sfc_exclusive_scan_noalloc(ctypes.c_void_p(out.data_ptr()), MAX_ITEMS + 1,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == sfc.SFC_ERR_CAPACITY
    assert L.sfc_exclusive_scan_noalloc(None, 5, ctypes.c_void_p(out.data_ptr()), None) == sfc.SFC_ERR_INVALID
    assert L.sfc_exclusive_scan_noalloc(ctypes.c_void_p(out.data_ptr()), 5, None, None) == sfc.SFC_ERR_INVALID


def test_noalloc_binding_rejects_bad_buffers(dev):
    x = torch.arange(10, dtype=torch.int32, device=dev)
    with pytest.raises(ValueError):
        sfc.sfc_exclusive_scan_noalloc(x, out=torch.empty(10, dtype=torch.int64, device=dev))      # n, not n + 1
    with pytest.raises(ValueError):
        sfc.sfc_exclusive_scan_noalloc(x, out=torch.empty(11, dtype=torch.int32, device=dev))      # dtype
    with pytest.raises(ValueError):
        sfc.sfc_exclusive_scan_noalloc(x, out=torch.empty(22, dtype=torch.int64, device=dev)[::2])  # strided
    with pytest.raises(ValueError):
        sfc.sfc_exclusive_scan_noalloc(x, out=torch.empty(11, dtype=torch.int64))                  # host
    with pytest.raises(ValueError):
        sfc.sfc_exclusive_scan_noalloc(x.to(torch.int64))                                          # 64-bit input
    out = sfc.sfc_exclusive_scan_noalloc(x, out=torch.empty(12, dtype=torch.int64, device=dev))
    assert out[:11].tolist() == [0, 0, 1, 3, 6, 10, 15, 21, 28, 36, 45]
