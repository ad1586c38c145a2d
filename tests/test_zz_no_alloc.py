"""The scan entry point that allocates no device memory (sfc_exclusive_scan_noalloc) gives
the same result as the allocating one (sfc_exclusive_scan), on two calls in a row.

It exists for callers that must not allocate device memory (a host framework's caching pool
owns the memory, or a loop cannot take cudaMalloc's implicit synchronisation); its scratch is
a fixed array in device memory shared by all calls.  This file is collected last so that a
stop-at-first-failure run has already run every other test; it also passes on its own.
"""
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
        torch.cuda.synchronize()
        assert torch.equal(out, ref), (n, call)


def test_noalloc_scan_limits(dev):
    out = torch.empty(1, dtype=torch.int64, device=dev)
    sfc.sfc_exclusive_scan_noalloc(torch.empty(0, dtype=torch.int32, device=dev), out=out)
    assert out.tolist() == [0]
    # one past the maximum is rejected before anything is enqueued (no buffer is read)
    L = sfc.lib()
    import ctypes
    st = L.sfc_exclusive_scan_noalloc(ctypes.c_void_p(out.data_ptr()), MAX_ITEMS + 1,
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
    assert st == sfc.SFC_ERR_CAPACITY
