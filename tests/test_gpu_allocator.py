"""The caller's allocator (sfc_allocator) owns all of an index's device memory: with
PyTorch's caching allocator routed through the callbacks, every buffer of the index comes from
them (the library's own pool does not grow), torch counts the memory, results equal those of
an index on the library's pool and the oracle, and destroying the index hands every block back."""
import gc

import numpy as np
import pytest
import torch

import oracle
import paper_2508_19891_gb300 as sfc
import workloads as W
from conftest import to_dev, u32, u64

pytestmark = pytest.mark.gpu


def _pool_settled():
    """The library's own pool bytes once earlier tests' unreferenced indexes are gone."""
    gc.collect()
    torch.cuda.synchronize()
    return sfc.sfc_pool_bytes_in_use()


@pytest.mark.parametrize("bounds,curve", [("learned", "z"), ("binary", "h")])
def test_torch_allocator_owns_every_index_buffer(cuda, bounds, curve):
    wl = W.mixed_1e7(scale=0.02)
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    A = sfc.TorchAllocator(cuda)
    pool0 = _pool_settled()
    torch0 = torch.cuda.memory_allocated(cuda)
    idx = sfc.sfc_build(pts, curve, bounds=bounds, cover_refine=-1, allocator=A)
    sfc.sfc_autotune(idx, q, d)
    off, ids = sfc.query(idx, q, d)
    # a dynamic round (update workspaces) and the host-buffer batch (staging buffers)
    rng = np.random.default_rng(5)
    dels = torch.from_numpy(rng.choice(wl.n, 1000, replace=False).astype(np.int32)).to(cuda)
    ins = pts[:2000].clone()
    sfc.sfc_update(idx, ins, dels)
    sfc.sfc_query_batch_host(idx, wl.queries, wl.delta, int(off[-1].item()) * 2)
    assert _pool_settled() <= pool0              # nothing from the library's own pool
    assert A.allocs > 0 and A.live
    keys, iids, xy = sfc.sfc_get_sorted(idx, copy=False)
    n = keys.numel()
    assert A.owns(keys.data_ptr(), 8 * n) and A.owns(iids.data_ptr(), 4 * n) and A.owns(xy.data_ptr(), 8 * n)
    held = sum(A.live.values())
    assert torch.cuda.memory_allocated(cuda) - torch0 >= held   # torch accounts for the index
    # same answers as an index on the library's pool, and as the oracle
    ref = sfc.sfc_build(pts, curve, bounds=bounds, cover_refine=-1)
    sfc.sfc_autotune(ref, q, d)
    sfc.sfc_update(ref, ins, dels)
    off_a, ids_a = sfc.query(idx, q, d)
    off_r, ids_r = sfc.query(ref, q, d)
    assert torch.equal(off_a, off_r) and torch.equal(ids_a, ids_r)
    ref.close()
    first = wl.n
    alive = np.ones(wl.n + ins.shape[0], bool)
    alive[dels.cpu().numpy()] = False
    allpts = np.concatenate([wl.points, ins.cpu().numpy()])
    live = np.nonzero(alive)[0]
    boff, bids = oracle.brute(allpts[live], wl.queries[:200], wl.delta[:200])
    o, out = u64(off_a), u32(ids_a)
    for j in range(200):
        assert np.array_equal(np.sort(out[o[j]:o[j + 1]]), live[bids[boff[j]:boff[j + 1]]].astype(np.uint32)), j
    assert first == wl.n
    assert sfc.sfc_device_status(idx) == (0, 0)
    idx.close()
    torch.cuda.synchronize()
    assert not A.live and A.frees == A.allocs    # every block handed back
    assert _pool_settled() <= pool0


def test_torch_allocator_graph_and_3d(cuda):
    """A CUDA graph over an allocator-backed index (its buffers are reserved through the
    callbacks before capture) and a 3-D index built from host points."""
    wl = W.roads_3e7(scale=0.003)
    pts, q, d = to_dev(wl.points, cuda), to_dev(wl.queries, cuda), to_dev(wl.delta, cuda)
    A = sfc.TorchAllocator(cuda)
    pool0 = _pool_settled()
    idx = sfc.sfc_build(pts, "h", bounds="learned", allocator=A)
    off, ids = sfc.query(idx, q, d)
    goff = torch.zeros_like(off)
    gids = torch.zeros_like(ids)
    g = sfc.sfc_graph_capture(idx, pts, q, d, goff, gids)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(goff, off) and torch.equal(gids, ids)
    g.close()
    idx.close()
    w3 = W.mixed3d(scale=0.002)
    i3 = sfc.sfc_build3_host(w3.points, allocator=A)
    o3, d3 = sfc.query(i3, to_dev(w3.queries, cuda), to_dev(w3.delta, cuda))
    roff, rids = oracle.query3(oracle.build3(w3.points), w3.queries, w3.delta)
    assert np.array_equal(u64(o3), roff) and np.array_equal(u32(d3), rids)
    i3.close()
    torch.cuda.synchronize()
    assert _pool_settled() <= pool0 and not A.live and A.frees == A.allocs


def test_allocator_out_of_memory_is_reported(cuda):
    """An allocator that has no memory makes the build fail with SFC_ERR_OOM, cleanly."""
    A = sfc.TorchAllocator(cuda)
    budget = {"left": 4}

    def stingy(nbytes, stream, ctx):
        if budget["left"] == 0:
            return None
        budget["left"] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), cuda.index, int(stream or 0))
        A.live[int(p)] = int(nbytes)
        A.allocs += 1
        return int(p)

    A._alloc = sfc.SFC_ALLOC_FN(stingy)
    A.struct = sfc.sfc_allocator(A._alloc, A._free, None)
    pts = to_dev(W.uniform_1e5(scale=0.1).points, cuda)
    with pytest.raises(sfc.SfcError) as e:
        sfc.sfc_build(pts, "z", allocator=A)
    assert e.value.status == sfc.SFC_ERR_OOM
    torch.cuda.synchronize()
    assert not A.live and A.frees == A.allocs
