// Dynamic setting (Sec. 2.1 "Dynamic implementation"; Sec. 3.3), batched.
//
// The paper keeps (pi(p), p) in a B-tree multimap and applies one element at a time.  Here a
// whole batch is applied to the sorted arrays at once; the result is exactly the array a
// rebuild from scratch over the live points would produce, because the order is (key, id)
// and every inserted id is larger than every existing one:
//
//   del_keys_kernel    key of each deleted id from the id -> coordinates table
//   radix sort         deletes by (key, id)
//   del_check_kernel   each delete must be an issued, live id, and not repeated
//   (host)             one synchronisation: a bad batch is rejected before anything changes
//   del_locate_kernel  array position of each delete: lexicographic lower_bound of (key, id)
//   radix sort         inserts by key with ids next_id + i (keys computed from the points)
//   ins_rank_kernel    rank of each insert among the old entries: upper_bound of its key
//   shift counts       v[p] = 1 - deleted(p) + (inserts ranked at p); one exclusive scan T
//                      gives every surviving entry p its new slot T[p] + inserts_at(p)
//   move_kernel        surviving entries to their new slots
//   ins_place_kernel   insert j to slot r_j - (deletes before r_j) + j
//   then: liveness bits, the id -> coordinates table, and a refit of a trained model.
#include <algorithm>

#include "sfc_internal.cuh"
#include "index.cuh"

namespace sfc {

namespace {

constexpr int kT = 256;

int grid_of(uint64_t n)
{
    uint64_t g = (n + kT - 1) / kT;
    const uint64_t cap = (uint64_t)num_sms() * 16;
    return (int)std::max<uint64_t>(1, std::min(g, cap));
}

__global__ void del_keys_kernel(const uint32_t* __restrict__ del, uint64_t k, const int2* __restrict__ xy_by_id,
                                uint32_t next_id, int curve, uint64_t* keys_out)
{
    __shared__ HilbertTables tb;
    if (curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < k; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t id = del[t];
        uint64_t key = 0;
        if (id < next_id) {
            const int2 p = xy_by_id[id];
            key = curve_key(curve, &tb, (uint32_t)p.x & (kSide - 1), (uint32_t)p.y & (kSide - 1));
        }
        keys_out[t] = key;
    }
}

__global__ void del_check_kernel(const uint64_t* __restrict__ skeys, const uint32_t* __restrict__ sids, uint64_t k,
                                 const uint32_t* __restrict__ alive, uint32_t next_id, uint32_t* bad)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < k; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t id = sids[t];
        bool ok = id < next_id && ((alive[id >> 5] >> (id & 31)) & 1u);
        if (t > 0 && sids[t - 1] == id && skeys[t - 1] == skeys[t]) ok = false;   // repeated id
        if (!ok) atomicOr(bad, 1u);
    }
}

// Position of (key, id) in the array sorted by (key, id); flags a delete that is not found.
__global__ void del_locate_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids, uint32_t n,
                                  const uint64_t* __restrict__ dkeys, const uint32_t* __restrict__ dids, uint64_t k,
                                  uint32_t* dpos, uint8_t* deleted, uint32_t* bad)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < k; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t kk = dkeys[t];
        const uint32_t id = dids[t];
        uint32_t lo = 0, len = n;
        while (len > 0) {
            const uint32_t half = len >> 1;
            const uint32_t mid = lo + half;
            const uint64_t km = keys[mid];
            const bool less = km < kk || (km == kk && ids[mid] < id);
            lo = less ? mid + 1 : lo;
            len = less ? len - half - 1 : half;
        }
        if (lo < n && keys[lo] == kk && ids[lo] == id) {
            dpos[t] = lo;
            deleted[lo] = 1;
        } else {
            dpos[t] = n;
            atomicOr(bad, 2u);
        }
    }
}

// Rank of each (sorted) insert among the old entries: all old ids are smaller, so it is the
// number of old keys <= the insert's key.
__global__ void ins_rank_kernel(const uint64_t* __restrict__ keys, uint32_t n, const uint64_t* __restrict__ ikeys,
                                uint64_t k, uint32_t* rank, uint32_t* v)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t kk = ikeys[j];
        uint32_t lo = 0, len = n;
        while (len > 0) {
            const uint32_t half = len >> 1;
            const bool le = keys[lo + half] <= kk;
            lo = le ? lo + half + 1 : lo;
            len = le ? len - half - 1 : half;
        }
        rank[j] = lo;
        atomicAdd(v + lo, 1u);
    }
}

// v[p] = 1 - deleted[p] for p < n, v[n] = 0 (the insert counts are added afterwards).
__global__ void shift_init_kernel(const uint8_t* __restrict__ deleted, uint32_t n, uint32_t* v)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p <= n; p += (uint64_t)gridDim.x * blockDim.x)
        v[p] = p < n ? 1u - deleted[p] : 0u;
}

__global__ void move_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ ids,
                            const int2* __restrict__ xy, uint32_t n, const uint8_t* __restrict__ deleted,
                            const uint32_t* __restrict__ v, const uint64_t* __restrict__ T, uint64_t* nkeys,
                            uint32_t* nids, int2* nxy)
{
    for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
        if (deleted[p]) continue;
        const uint64_t dst = T[p] + (v[p] - 1u);   // v[p] - 1 = inserts placed before p
        nkeys[dst] = keys[p];
        nids[dst] = ids[p];
        nxy[dst] = xy[p];
    }
}

__global__ void ins_place_kernel(const uint64_t* __restrict__ ikeys, const uint32_t* __restrict__ iids,
                                 const int2* __restrict__ ixy, uint64_t k, const uint32_t* __restrict__ rank,
                                 const uint32_t* __restrict__ dpos, uint64_t kdel, uint64_t* nkeys, uint32_t* nids,
                                 int2* nxy)
{
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < k; j += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rank[j];
        // deletes at positions < r (dpos is ascending)
        uint64_t lo = 0, len = kdel;
        while (len > 0) {
            const uint64_t half = len >> 1;
            const bool lt = dpos[lo + half] < r;
            lo = lt ? lo + half + 1 : lo;
            len = lt ? len - half - 1 : half;
        }
        const uint64_t dst = (uint64_t)r - lo + j;
        nkeys[dst] = ikeys[j];
        nids[dst] = iids[j];
        nxy[dst] = ixy[j];
    }
}

__global__ void alive_clear_kernel(const uint32_t* __restrict__ del, uint64_t k, uint32_t* alive)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < k; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t id = del[t];
        atomicAnd(alive + (id >> 5), ~(1u << (id & 31)));
    }
}

}  // namespace

sfc_status ensure_alive_bits(sfc_index* idx, uint64_t ids, cudaStream_t st)
{
    // ids >= next_id are never treated as live (checks compare against next_id first), so
    // new words can start all-ones: an inserted id is live as soon as next_id passes it.
    const uint64_t words = (ids + 31) / 32 + 1;
    if (words * 4 <= idx->alive.bytes) return SFC_OK;
    DevBuf nb;
    SFC_TRY(nb.ensure(words * 4, st));
    SFC_CUDA_TRY(cudaMemsetAsync(nb.ptr, 0xff, nb.bytes, st));
    if (idx->alive.ptr)
        SFC_CUDA_TRY(cudaMemcpyAsync(nb.ptr, idx->alive.ptr, idx->alive.bytes, cudaMemcpyDeviceToDevice, st));
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
    idx->occ.release(st);
    idx->xyz.release(st);
    idx->keys_in.release(st);
    release_sort_ws(idx->sort_ws, st);
    idx->scan_ws.flags.release(st);
    QueryWs& q = idx->qws;
    q.ranges.release(st); q.nchunks.release(st); q.chunk_base.release(st);
    q.counts.release(st); q.masks.release(st); q.ctr.release(st);
    q.qkeys.release(st); q.qkeys_sorted.release(st); q.perm.release(st);
    q.nch_sorted.release(st); q.wbase.release(st); q.small_list.release(st); q.small_mask.release(st);
    q.chunk_hits.release(st); q.big_items.release(st); q.big_list.release(st);
    HostStage& h = idx->stage;
    h.q.release(st); h.delta.release(st); h.offsets.release(st); h.ids.release(st);
    h.points.release(st); h.slice_keys.release(st); h.slice_keys_sorted.release(st); h.slice_perm.release(st);
    if (h.copy) {
        cudaStreamSynchronize(h.copy);
        cudaStreamDestroy(h.copy);
        h.copy = nullptr;
        for (auto& e : h.done) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    }
    ModelState& M = idx->model;
    M.state.release(st); M.samples.release(st); M.partial.release(st);
    M.tmp.release(st); M.leaves.release(st); M.fence.release(st);
    M.fence_fine.release(st);
    UpdateWs& u = idx->uws;
    u.a.release(st); u.b.release(st); u.c.release(st); u.d.release(st);
    u.e.release(st); u.f.release(st); u.g.release(st); u.h.release(st);
    u.keys.release(st); u.ids.release(st); u.xy.release(st);
    u.mark.release(st); u.v.release(st); u.t.release(st);
}

sfc_status apply_update(sfc_index* idx, const int32_t* d_inserts, uint64_t k_ins, const uint32_t* d_del,
                        uint64_t k_del, uint32_t* h_first, cudaStream_t st)
{
    UpdateWs& U = idx->uws;
    const uint32_t n = (uint32_t)idx->n;
    const uint32_t next_id = idx->next_id;
    const int curve = idx->curve;
    if ((uint64_t)next_id + k_ins >= 0xffffffffull || (uint64_t)n + k_ins >= 0xffffffffull) return SFC_ERR_INVALID;
    uint32_t* status = idx->status.as<uint32_t>();
    // scratch: a = flags, b = delete keys in / sorted, c = delete ids sorted, d = delete positions
    SFC_TRY(U.a.ensure(16, st));
    uint32_t* bad = U.a.as<uint32_t>();
    SFC_CUDA_TRY(cudaMemsetAsync(bad, 0, 16, st));
    uint64_t* dkeys_in = nullptr;
    uint64_t* dkeys = nullptr;
    uint32_t* dids = nullptr;
    uint32_t* dpos = nullptr;
    if (k_del) {
        SFC_TRY(U.b.ensure(k_del * 16, st));
        SFC_TRY(U.c.ensure(k_del * 4, st));
        SFC_TRY(U.d.ensure(k_del * 4, st));
        dkeys_in = U.b.as<uint64_t>();
        dkeys = dkeys_in + k_del;
        dids = U.c.as<uint32_t>();
        dpos = U.d.as<uint32_t>();
        del_keys_kernel<<<grid_of(k_del), kT, 0, st>>>(d_del, k_del, idx->xy_by_id.as<int2>(), next_id, curve, dkeys_in);
        count_launch();
        SortSource src;
        src.keys = dkeys_in;
        src.vals = d_del;
        SortDest dst;
        dst.keys = dkeys;
        dst.vals = dids;
        dst.curve = curve;
        SFC_TRY(radix_sort(src, k_del, dst, idx->sort_ws, status, st));
        del_check_kernel<<<grid_of(k_del), kT, 0, st>>>(dkeys, dids, k_del, idx->alive.as<uint32_t>(), next_id, bad);
        count_launch();
        SFC_TRY(launch_status());
        uint32_t hbad = 0;
        SFC_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, st));
        SFC_CUDA_TRY(cudaStreamSynchronize(st));
        if (hbad) return SFC_ERR_NOT_FOUND;   // nothing has been changed yet
    }
    // ---- inserts: keys, sort, decoded coordinates ----
    uint64_t* ikeys = nullptr;
    uint32_t* iids = nullptr;
    int2* ixy = nullptr;
    uint32_t* irank = nullptr;
    if (k_ins) {
        SFC_TRY(U.e.ensure(k_ins * 8, st));
        SFC_TRY(U.f.ensure(k_ins * 4, st));
        SFC_TRY(U.g.ensure(k_ins * 8, st));
        SFC_TRY(U.h.ensure(k_ins * 4, st));
        ikeys = U.e.as<uint64_t>();
        iids = U.f.as<uint32_t>();
        ixy = U.g.as<int2>();
        irank = U.h.as<uint32_t>();
        SortSource src;
        src.points = reinterpret_cast<const int2*>(d_inserts);
        src.curve = curve;
        src.val_base = next_id;
        SortDest dst;
        dst.keys = ikeys;
        dst.vals = iids;
        dst.xy = ixy;
        dst.curve = curve;
        SFC_TRY(radix_sort(src, k_ins, dst, idx->sort_ws, status, st));
    }
    // ---- shift counts and the new arrays ----
    const uint64_t new_n = (uint64_t)n - k_del + k_ins;
    SFC_TRY(U.keys.ensure(std::max<uint64_t>(new_n, 1) * 8, st));
    SFC_TRY(U.ids.ensure(std::max<uint64_t>(new_n, 1) * 4, st));
    SFC_TRY(U.xy.ensure(std::max<uint64_t>(new_n, 1) * 8, st));
    DevBuf& delmark = U.mark;
    DevBuf& vbuf = U.v;
    DevBuf& tbuf = U.t;
    SFC_TRY(delmark.ensure((size_t)n + 16, st));
    SFC_TRY(vbuf.ensure(((size_t)n + 1) * 4, st));
    SFC_TRY(tbuf.ensure(((size_t)n + 2) * 8, st));
    uint8_t* deleted = delmark.as<uint8_t>();
    uint32_t* v = vbuf.as<uint32_t>();
    uint64_t* T = tbuf.as<uint64_t>();
    SFC_CUDA_TRY(cudaMemsetAsync(deleted, 0, (size_t)n + 1, st));
    const uint64_t* keys = idx->keys.as<uint64_t>();
    const uint32_t* ids = idx->ids.as<uint32_t>();
    if (k_del) {
        del_locate_kernel<<<grid_of(k_del), kT, 0, st>>>(keys, ids, n, dkeys, dids, k_del, dpos, deleted, bad);
        count_launch();
    }
    shift_init_kernel<<<grid_of((uint64_t)n + 1), kT, 0, st>>>(deleted, n, v);
    count_launch();
    if (k_ins) {
        ins_rank_kernel<<<grid_of(k_ins), kT, 0, st>>>(keys, n, ikeys, k_ins, irank, v);
        count_launch();
    }
    SFC_TRY(launch_status());
    SFC_TRY(exclusive_scan_u32(v, (uint64_t)n + 1, T, idx->scan_ws, status, st));
    uint64_t* nkeys = U.keys.as<uint64_t>();
    uint32_t* nids = U.ids.as<uint32_t>();
    int2* nxy = U.xy.as<int2>();
    if (n) {
        move_kernel<<<grid_of(n), kT, 0, st>>>(keys, ids, idx->xy.as<int2>(), n, deleted, v, T, nkeys, nids, nxy);
        count_launch();
    }
    if (k_ins) {
        ins_place_kernel<<<grid_of(k_ins), kT, 0, st>>>(ikeys, iids, ixy, k_ins, irank, dpos, k_del, nkeys, nids, nxy);
        count_launch();
    }
    // ---- liveness and the id -> coordinates table ----
    if (k_del) {
        alive_clear_kernel<<<grid_of(k_del), kT, 0, st>>>(d_del, k_del, idx->alive.as<uint32_t>());
        count_launch();
    }
    SFC_TRY(launch_status());
    if (k_ins) {
        const uint64_t ids_after = (uint64_t)next_id + k_ins;
        if (ids_after * sizeof(int2) > idx->xy_by_id.bytes) {
            DevBuf nb;
            SFC_TRY(nb.ensure(ids_after * sizeof(int2) + ids_after * sizeof(int2) / 2, st));
            if (next_id)
                SFC_CUDA_TRY(cudaMemcpyAsync(nb.ptr, idx->xy_by_id.ptr, (size_t)next_id * sizeof(int2),
                                             cudaMemcpyDeviceToDevice, st));
            idx->xy_by_id.release(st);
            idx->xy_by_id = nb;
        }
        SFC_CUDA_TRY(cudaMemcpyAsync(idx->xy_by_id.as<int2>() + next_id, d_inserts, k_ins * sizeof(int2),
                                     cudaMemcpyDeviceToDevice, st));
        SFC_TRY(ensure_alive_bits(idx, ids_after, st));
    }
    // ---- swap in the new arrays ----
    std::swap(idx->keys, U.keys);
    std::swap(idx->ids, U.ids);
    std::swap(idx->xy, U.xy);
    idx->n = new_n;
    idx->next_id = next_id + (uint32_t)k_ins;
    if (h_first) *h_first = next_id;
    idx->qws.pending.valid = false;
    SFC_TRY(build_occupancy(idx, st));
    if (idx->model.trained) {
        const int steps = std::max(20, idx->opt.train_steps / 5);
        SFC_TRY(refit_model(idx, steps, st));
    }
    return SFC_OK;
}

}  // namespace sfc

extern "C" sfc_status sfc_update(sfc_index* idx, const int32_t* d_inserts, uint64_t k_ins,
                                 const uint32_t* d_delete_ids, uint64_t k_del, uint32_t* h_first_new_id,
                                 void* stream)
{
    if (!idx || (k_ins && !d_inserts) || (k_del && !d_delete_ids) || idx->dim != 2) return SFC_ERR_INVALID;
    if (k_del > idx->n || k_ins >= 0xffffffffull) return k_del > idx->n ? SFC_ERR_NOT_FOUND : SFC_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    idx->last_stream = st;
    sfc::AllocScope alloc_scope(idx->allocator());
    sfc::ProfScope ps(idx, "update", st);
    return sfc::apply_update(idx, d_inserts, k_ins, d_delete_ids, k_del, h_first_new_id, st);
}
