// Dynamic setting (Sec. 2.1 "Dynamic implementation"; Sec. 3.3) and index bookkeeping.
#include "sfc_internal.cuh"
#include "index.cuh"

namespace sfc {

sfc_status ensure_alive_bits(sfc_index* idx, uint64_t ids, cudaStream_t st)
{
    const uint64_t words = (ids + 31) / 32 + 1;
    const size_t old = idx->alive.bytes;
    if (words * 4 <= old) return SFC_OK;
    DevBuf nb;
    SFC_TRY(nb.ensure(words * 4, st));
    SFC_CUDA_TRY(cudaMemsetAsync(nb.ptr, 0xff, nb.bytes, st));
    idx->alive.release(st);
    idx->alive = nb;
    return SFC_OK;
}

void release_index(sfc_index* idx, cudaStream_t st)
{
    idx->keys.release(st);
    idx->ids.release(st);
    idx->xy.release(st);
    idx->xy_by_id.release(st);
    idx->alive.release(st);
    idx->status.release(st);
    release_sort_ws(idx->sort_ws, st);
    idx->scan_ws.flags.release(st);
    QueryWs& q = idx->qws;
    q.ranges.release(st); q.nchunks.release(st); q.chunk_base.release(st);
    q.counts.release(st); q.masks.release(st); q.ctr.release(st);
    HostStage& h = idx->stage;
    h.q.release(st); h.delta.release(st); h.offsets.release(st); h.ids.release(st);
    idx->model.leaves.release(st);
    idx->model.scratch.release(st);
    UpdateWs& u = idx->uws;
    u.a.release(st); u.b.release(st); u.c.release(st); u.d.release(st);
    u.e.release(st); u.f.release(st); u.g.release(st); u.h.release(st);
}

}  // namespace sfc

extern "C" sfc_status sfc_update(sfc_index* idx, const int32_t* d_inserts, uint64_t k_ins,
                                 const uint32_t* d_delete_ids, uint64_t k_del, uint32_t* h_first_new_id,
                                 void* stream)
{
    (void)idx; (void)d_inserts; (void)k_ins; (void)d_delete_ids; (void)k_del; (void)h_first_new_id;
    (void)stream;
    return SFC_ERR_STATE;
}
