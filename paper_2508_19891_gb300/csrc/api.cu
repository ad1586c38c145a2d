// C ABI of the library (include/sfc.h): argument checks, the index object and its
// workspaces, and the order of kernel launches for each call.  No computation of the method
// happens here; every step runs in the kernels of keygen.cu, radix.cu, scan.cu, query.cu,
// learned.cu and update.cu.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "sfc_internal.cuh"
#include "query.cuh"
#include "index.cuh"

namespace sfc {

std::atomic<uint64_t> g_launches{0};

int num_sms()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        cached[dev] = v;
    }
    return cached[dev];
}

// The library allocates through the device's default stream-ordered pool.  By default that
// pool returns freed memory to the system at every synchronisation, so an index built after
// another was destroyed would map its memory again; keep freed memory cached in the pool
// instead (once per device), as a caching allocator does.
static void keep_pool_memory()
{
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done[dev] = true;
}

thread_local const sfc_allocator* t_alloc = nullptr;
static std::atomic<uint64_t> g_pool_bytes{0};   // held from the library's own pool

sfc_status dev_alloc(void** p, size_t bytes, cudaStream_t st, const sfc_allocator** owner)
{
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    const sfc_allocator* a = t_alloc;
    if (owner) *owner = a;
    if (a) {   // the caller's allocator: stream-ordered on st, NULL when it has no memory
        *p = a->alloc(bytes, reinterpret_cast<void*>(st), a->ctx);
        return *p ? SFC_OK : SFC_ERR_OOM;
    }
    keep_pool_memory();
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SFC_ERR_OOM : SFC_ERR_CUDA;
    }
    g_pool_bytes.fetch_add(bytes, std::memory_order_relaxed);
    return SFC_OK;
}

void dev_free(void* p, size_t bytes, cudaStream_t st, const sfc_allocator* owner)
{
    if (!p) return;
    if (owner) {
        owner->free(p, reinterpret_cast<void*>(st), owner->ctx);
    } else {
        cudaFreeAsync(p, st);
        g_pool_bytes.fetch_sub(bytes == 0 ? 16 : bytes, std::memory_order_relaxed);
    }
}

}  // namespace sfc

using namespace sfc;

namespace {

cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

sfc_status ensure_status_buf(sfc_index* idx, cudaStream_t st)
{
    if (idx->status.ptr) return SFC_OK;
    SFC_TRY(idx->status.ensure(16 + sizeof(unsigned long long) * 8, st));
    SFC_CUDA_TRY(cudaMemsetAsync(idx->status.ptr, 0, idx->status.bytes, st));
    return SFC_OK;
}

uint32_t* status_word(sfc_index* idx) { return idx->status.as<uint32_t>(); }
// status buffer: u32 status word, padding, then u64 counters [0..2] learned-bounds
// statistics, [3] points scanned by the last batch, [4] cover cells, [5] of them found empty
// by the early-termination bitmap
unsigned long long* model_stats(sfc_index* idx)
{
    return reinterpret_cast<unsigned long long*>(idx->status.as<unsigned char>() + 16);
}
unsigned long long* scan_stats(sfc_index* idx) { return model_stats(idx) + 3; }

sfc_status build_from_device(sfc_index* idx, const int32_t* d_points, cudaStream_t st)
{
    const uint64_t n = idx->n;
    SFC_TRY(idx->keys.ensure(n * sizeof(uint64_t), st));
    SFC_TRY(idx->ids.ensure(n * sizeof(uint32_t), st));
    SFC_TRY(idx->xy.ensure(n * sizeof(int2), st));
    SortSource src;
    src.points = reinterpret_cast<const int2*>(d_points);
    src.curve = idx->curve;
    SortDest dst;
    dst.keys = idx->keys.as<uint64_t>();
    dst.vals = idx->ids.as<uint32_t>();
    dst.xy = idx->xy.as<int2>();
    dst.curve = idx->curve;
    {
        ProfScope ps(idx, "sort", st);
        SFC_TRY(radix_sort(src, n, dst, idx->sort_ws, status_word(idx), st));
    }
    if (idx->opt.occupancy_depth > 0) {
        ProfScope ps(idx, "occupancy", st);
        SFC_TRY(build_occupancy(idx, st));
    }
    // the id -> coordinates table of the dynamic setting starts as a copy of the input
    SFC_TRY(idx->xy_by_id.ensure(n * sizeof(int2), st));
    if (n) SFC_CUDA_TRY(cudaMemcpyAsync(idx->xy_by_id.ptr, d_points, n * sizeof(int2),
                                        cudaMemcpyDeviceToDevice, st));
    idx->next_id = (uint32_t)n;
    SFC_TRY(ensure_alive_bits(idx, n, st));
    return SFC_OK;
}

// 3-D: keys of the input points, the (key, id) sort, and the coordinates decoded from the sorted
// keys into 16-byte records.
sfc_status build3_from_device(sfc_index* idx, const int32_t* d_points, cudaStream_t st)
{
    const uint64_t n = idx->n;
    SFC_TRY(idx->keys.ensure(n * sizeof(uint64_t), st));
    SFC_TRY(idx->ids.ensure(n * sizeof(uint32_t), st));
    SFC_TRY(idx->xyz.ensure(n * sizeof(int4), st));
    SFC_TRY(idx->keys_in.ensure(n * sizeof(uint64_t), st));
    ProfScope ps(idx, "sort", st);
    SFC_TRY(launch_keys3(d_points, n, idx->keys_in.as<uint64_t>(), status_word(idx), st));
    SortSource src;
    src.keys = idx->keys_in.as<uint64_t>();
    SortDest dst;
    dst.keys = idx->keys.as<uint64_t>();
    dst.vals = idx->ids.as<uint32_t>();
    SFC_TRY(radix_sort(src, n, dst, idx->sort_ws, status_word(idx), st));
    SFC_TRY(launch_decode3(idx->keys.as<uint64_t>(), n, idx->xyz.as<int4>(), st));
    idx->next_id = (uint32_t)n;
    return SFC_OK;
}

QueryArgs base_args(sfc_index* idx, const int32_t* q, const int32_t* delta, uint64_t m)
{
    QueryArgs a{};
    a.curve = idx->curve;
    a.keys = idx->keys.as<uint64_t>();
    a.ids = idx->ids.as<uint32_t>();
    a.xy = idx->xy.as<int2>();
    a.n = (uint32_t)idx->n;
    a.q = q;
    a.delta = delta;
    a.m = m;
    a.status = status_word(idx);
    a.drop = idx->drop;
    a.kint = (uint32_t)query_intervals(idx->dim, idx->drop);
    a.norm = idx->norm;
    a.dim = idx->dim;
    a.xyz = idx->xyz.as<int4>();
    if (idx->opt.occupancy_depth > 0 && idx->occ.ptr) {
        a.occ = idx->occ.as<uint32_t>();
        a.occ_depth = idx->opt.occupancy_depth;
    }
    a.cells = model_stats(idx) + 4;
    return a;
}

sfc_status ensure_query_ws(sfc_index* idx, uint64_t m, cudaStream_t st)
{
    QueryWs& w = idx->qws;
    SFC_TRY(w.ranges.ensure(m * 2 * query_intervals(idx->dim, idx->drop) * sizeof(uint32_t), st));
    SFC_TRY(w.nchunks.ensure(m * sizeof(uint32_t), st));
    SFC_TRY(w.chunk_base.ensure((m + 1) * sizeof(uint64_t), st));
    SFC_TRY(w.counts.ensure(m * sizeof(uint32_t), st));
    SFC_TRY(w.ctr.ensure(kCtrWords * sizeof(unsigned long long), st));
    SFC_TRY(w.small_list.ensure(m * sizeof(uint32_t), st));
    SFC_TRY(w.small_mask.ensure(m * kSmallWords * sizeof(unsigned long long), st));
    SFC_TRY(w.chunk_hits.ensure((kChunkHitsPerQuery * m + 1024) * sizeof(uint32_t), st));
    SFC_TRY(w.big_items.ensure((kChunkHitsPerQuery * m + 1024) * sizeof(uint32_t), st));
    SFC_TRY(w.big_list.ensure(m * sizeof(uint32_t), st));
    if (idx->opt.reorder_queries != 0 && idx->dim == 2) {
        SFC_TRY(w.qkeys.ensure(m * sizeof(uint64_t), st));
        SFC_TRY(w.qkeys_sorted.ensure(m * sizeof(uint64_t), st));
        SFC_TRY(w.perm.ensure(m * sizeof(uint32_t), st));
        SFC_TRY(w.nch_sorted.ensure(m * sizeof(uint32_t), st));
        SFC_TRY(w.wbase.ensure((m + 1) * sizeof(uint64_t), st));
        SFC_TRY(reserve_sort(idx->sort_ws, std::max<uint64_t>(m, 1), st));
    }
    const uint64_t budget = (uint64_t)idx->opt.mask_budget_mb << 20;
    // one bit per scanned point: 1 KB per query covers batches whose mean scan is up to 8,192
    // points; chunks past the buffer are re-filtered by the write pass
    uint64_t want = m * 1024ull + (1ull << 20);
    if (want > budget) want = budget;
    if (w.masks.bytes < want) SFC_TRY(w.masks.ensure(want, st));
    return SFC_OK;
}

const LearnedModelView* model_view(sfc_index* idx, LearnedModelView& v)
{
    if (idx->bounds != SFC_BOUNDS_LEARNED || !idx->model.trained) return nullptr;
    v.root = model_root_device(idx);
    v.leaf = idx->model.leaves.as<LeafParams>();
    v.fence = idx->model.fence.as<uint64_t>();
    v.fence_fine = idx->model.fence_fine.as<uint64_t>();
    v.stats = model_stats(idx);
    return &v;
}

// Curve-order processing pays off once the coordinates no longer fit in L2 (n >= 2^24, i.e.
// 128 MB of coordinates); option 1 forces it, 0 disables it.
bool use_curve_order(const sfc_index* idx, uint64_t m)
{
    if (m < 2 || idx->opt.reorder_queries == 0 || idx->dim != 2) return false;
    if (idx->opt.reorder_queries == 1) return true;
    return idx->n >= (1ull << 24);
}

// The chunk hit counts of big queries (count pass) and their in-query offsets (write pass).
void set_big_queries(QueryWs& w, QueryArgs& a)
{
    a.chunk_hits = w.chunk_hits.as<uint32_t>();
    a.big_items = w.big_items.as<uint32_t>();
    a.big_list = w.big_list.as<uint32_t>();
    a.big_cap = std::min<uint64_t>(std::min(w.chunk_hits.bytes, w.big_items.bytes) / sizeof(uint32_t), a.mask_chunks);
    a.big_warps = (uint32_t)num_sms() * 64u * kBigShare;
}

sfc_status do_count(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                    uint64_t* d_out_offsets, cudaStream_t st)
{
    SFC_TRY(ensure_status_buf(idx, st));
    if (m == 0) {
        SFC_CUDA_TRY(cudaMemsetAsync(d_out_offsets, 0, sizeof(uint64_t), st));
        idx->qws.pending = {true, d_q, d_delta, 0, d_out_offsets, 0, false, idx->drop, idx->norm};
        return SFC_OK;
    }
    SFC_TRY(ensure_query_ws(idx, m, st));
    QueryWs& w = idx->qws;
    QueryArgs a = base_args(idx, d_q, d_delta, m);
    a.ranges = w.ranges.as<uint32_t>();
    a.nchunks = w.nchunks.as<uint32_t>();
    a.chunk_base = w.chunk_base.as<uint64_t>();
    a.counts = w.counts.as<uint32_t>();
    a.masks = w.masks.as<uint32_t>();
    a.chunk = idx->chunk;
    a.mask_chunks = w.masks.bytes / (a.chunk / 8);
    set_big_queries(w, a);
    a.batch = idx->batch;
    a.qbatch = idx->qbatch;
    a.work_ctr = w.ctr.as<unsigned long long>();
    a.small_list = w.small_list.as<uint32_t>();
    a.small_mask = w.small_mask.as<unsigned long long>();
    a.out_offsets = d_out_offsets;
    a.scanned = scan_stats(idx);
    // per-batch statistics: learned-bounds counters and the scanned total
    SFC_CUDA_TRY(cudaMemsetAsync(model_stats(idx), 0, 6 * sizeof(unsigned long long), st));
    SFC_CUDA_TRY(cudaMemsetAsync(a.counts, 0, m * sizeof(uint32_t), st));
    SFC_CUDA_TRY(cudaMemsetAsync(a.work_ctr, 0, kCtrWords * sizeof(unsigned long long), st));
    LearnedModelView lv;
    const bool ordered = use_curve_order(idx, m);
    if (ordered) {
        // processing order: queries sorted by the curve key of their centre, so that queries
        // scanning overlapping ranges run close together and share the cache
        ProfScope ps(idx, "order", st);
        SFC_TRY(launch_query_keys(d_q, m, idx->curve, w.qkeys.as<uint64_t>(), st));
        SortSource src;
        src.keys = w.qkeys.as<uint64_t>();
        SortDest dst;
        dst.keys = w.qkeys_sorted.as<uint64_t>();
        dst.vals = w.perm.as<uint32_t>();
        dst.curve = idx->curve;
        SFC_TRY(radix_sort(src, m, dst, idx->sort_ws, a.status, st));
        a.perm = w.perm.as<uint32_t>();   // the plan already runs in processing order
    }
    {
        ProfScope ps(idx, "plan", st);
        SFC_TRY(launch_plan(a, model_view(idx, lv), st));
    }
    {
        ProfScope ps(idx, "scan", st);
        SFC_TRY(exclusive_scan_u32(a.nchunks, m, a.chunk_base, idx->scan_ws, a.status, st));
        if (ordered) {
            SFC_TRY(launch_gather_u32(a.nchunks, w.perm.as<uint32_t>(), m, w.nch_sorted.as<uint32_t>(), st));
            SFC_TRY(exclusive_scan_u32(w.nch_sorted.as<uint32_t>(), m, w.wbase.as<uint64_t>(), idx->scan_ws,
                                       a.status, st));
            a.wbase = w.wbase.as<uint64_t>();
        }
    }
    {
        ProfScope ps(idx, "count", st);
        SFC_TRY(launch_count(a, st));
    }
    {
        ProfScope ps(idx, "scan", st);
        SFC_TRY(exclusive_scan_u32(a.counts, m, d_out_offsets, idx->scan_ws, a.status, st));
        SFC_TRY(launch_chunk_prefix(a, st));
    }
    w.pending = {true, d_q, d_delta, m, d_out_offsets, a.chunk, ordered, a.drop, a.norm};
    return SFC_OK;
}

// The write pass for the queries [q_begin, q_end) of the pending count (no state checks).
sfc_status do_write_range(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                          const uint64_t* d_out_offsets, uint32_t* d_out_ids, uint64_t cap, cudaStream_t st,
                          uint64_t q_begin, uint64_t q_end, const uint32_t* perm = nullptr)
{
    QueryWs& w = idx->qws;
    QueryArgs a = base_args(idx, d_q, d_delta, m);
    a.drop = w.pending.drop;
    a.kint = (uint32_t)query_intervals(idx->dim, a.drop);
    a.norm = w.pending.norm;
    a.ranges = w.ranges.as<uint32_t>();
    a.nchunks = w.nchunks.as<uint32_t>();
    a.chunk_base = w.chunk_base.as<uint64_t>();
    a.counts = w.counts.as<uint32_t>();
    a.masks = w.masks.as<uint32_t>();
    a.chunk = w.pending.chunk;
    a.mask_chunks = w.masks.bytes / (a.chunk / 8);
    set_big_queries(w, a);
    a.batch = idx->batch;
    a.qbatch = idx->qbatch;
    a.work_ctr = w.ctr.as<unsigned long long>();
    a.small_list = w.small_list.as<uint32_t>();
    a.small_mask = w.small_mask.as<unsigned long long>();
    a.out_offsets = const_cast<uint64_t*>(d_out_offsets);
    a.out_ids = d_out_ids;
    if (w.pending.ordered) {
        a.perm = perm ? perm : w.perm.as<uint32_t>();
        a.wbase = w.wbase.as<uint64_t>();
    }
    a.ids_capacity = d_out_ids ? cap : 0;
    a.q_begin = q_begin;
    a.q_end = q_end;
    // the write pass's own work counters start at zero (a repeated write stays correct)
    SFC_CUDA_TRY(cudaMemsetAsync(a.work_ctr + kCtrWrite, 0, 2 * sizeof(unsigned long long), st));
    SFC_CUDA_TRY(cudaMemsetAsync(a.work_ctr + kCtrWriteBig, 0, sizeof(unsigned long long), st));
    ProfScope ps(idx, "write", st);
    return launch_write(a, st);
}

sfc_status do_write(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                    const uint64_t* d_out_offsets, uint32_t* d_out_ids, uint64_t cap, cudaStream_t st)
{
    QueryWs& w = idx->qws;
    if (!w.pending.valid || w.pending.q != d_q || w.pending.delta != d_delta || w.pending.m != m ||
        w.pending.offsets != d_out_offsets)
        return SFC_ERR_STATE;
    w.pending.valid = false;
    if (m == 0) return SFC_OK;
    return do_write_range(idx, d_q, d_delta, m, d_out_offsets, d_out_ids, cap, st, 0, m);
}

}  // namespace

extern "C" {

void sfc_default_options(sfc_options* opt)
{
    if (!opt) return;
    opt->bounds = SFC_BOUNDS_BINARY;
    opt->leaves = 4096;
    opt->train_steps = 8;
    opt->train_samples = 16384;
    opt->learning_rate = 0.02f;
    opt->chunk = 0;
    opt->mask_budget_mb = 4096;
    opt->reorder_queries = 2;
    opt->profile = 0;
    opt->root = SFC_ROOT_PWL;
    opt->cover_refine = 0;
    opt->occupancy_depth = 0;
    opt->query_norm = SFC_NORM_DISC;
}

sfc_status sfc_build(sfc_index** out, const int32_t* d_points, uint64_t n, sfc_curve curve,
                     const sfc_options* opt, const sfc_allocator* alloc, void* stream)
{
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n >= 0xffffffffull || (n && !d_points)) return SFC_ERR_INVALID;
    if (curve != SFC_CURVE_Z && curve != SFC_CURVE_HILBERT) return SFC_ERR_INVALID;
    if (alloc && (!alloc->alloc || !alloc->free)) return SFC_ERR_INVALID;
    sfc_options o;
    sfc_default_options(&o);
    if (opt) o = *opt;
    if (o.leaves < 1 || o.leaves > (1 << 20) || o.mask_budget_mb < 1 || o.train_samples < 2 ||
        o.train_steps < 0 || o.reorder_queries < 0 || o.reorder_queries > 2 || (o.chunk != 0 && (o.chunk < 32 || o.chunk > 4096 || (o.chunk & 31))) ||
        (o.bounds != SFC_BOUNDS_BINARY && o.bounds != SFC_BOUNDS_LEARNED) ||
        (o.root != SFC_ROOT_PWL && o.root != SFC_ROOT_MLP) || o.cover_refine < -1 || o.cover_refine > 2 ||
        o.occupancy_depth < 0 || o.occupancy_depth > 13 ||
        (o.query_norm != SFC_NORM_DISC && o.query_norm != SFC_NORM_SQUARE))
        return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    sfc_index* idx = new (std::nothrow) sfc_index();
    if (!idx) return SFC_ERR_OOM;
    cudaGetDevice(&idx->device);
    if (alloc) {
        idx->alloc = *alloc;
        idx->has_alloc = true;
    }
    AllocScope scope(idx->allocator());
    idx->curve = curve;
    idx->n = n;
    idx->opt = o;
    idx->bounds = SFC_BOUNDS_BINARY;
    idx->chunk = o.chunk ? (uint32_t)o.chunk : 1024u;
    idx->drop = o.cover_refine < 0 ? 1 : o.cover_refine;
    idx->norm = o.query_norm;
    idx->last_stream = st;
    idx->prof.on = o.profile != 0;
    sfc_status s = ensure_status_buf(idx, st);
    if (s == SFC_OK) s = build_from_device(idx, d_points, st);
    if (s == SFC_OK && o.bounds == SFC_BOUNDS_LEARNED) {
        ProfScope ps(idx, "train", st);
        s = train_model(idx, st);
        if (s == SFC_OK) idx->bounds = SFC_BOUNDS_LEARNED;
    }
    if (s != SFC_OK) {
        sfc_destroy(idx);
        return s;
    }
    *out = idx;
    return SFC_OK;
}

sfc_status sfc_build_host(sfc_index** out, const int32_t* h_points, uint64_t n, sfc_curve curve,
                          const sfc_options* opt, const sfc_allocator* alloc, void* stream)
{
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n >= 0xffffffffull || (n && !h_points)) return SFC_ERR_INVALID;
    if (alloc && (!alloc->alloc || !alloc->free)) return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    AllocScope scope(alloc);   // the staging copy of the points comes from the same allocator
    void* d = nullptr;
    const sfc_allocator* owner = nullptr;
    SFC_TRY(dev_alloc(&d, n * sizeof(int2), st, &owner));
    cudaError_t e = n ? cudaMemcpyAsync(d, h_points, n * sizeof(int2), cudaMemcpyHostToDevice, st) : cudaSuccess;
    sfc_status s = e == cudaSuccess ? sfc_build(out, static_cast<int32_t*>(d), n, curve, opt, alloc, stream)
                                    : SFC_ERR_CUDA;
    dev_free(d, n * sizeof(int2), st, owner);
    return s;
}

void sfc_destroy(sfc_index* idx)
{
    if (!idx) return;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = idx->last_stream;
    for (const ProfRec& r : idx->prof.recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    idx->prof.recs.clear();
    release_index(idx, st);
    delete idx;
}

sfc_status sfc_rebuild(sfc_index* idx, const int32_t* d_points, uint64_t n, void* stream)
{
    if (!idx || n >= 0xffffffffull || (n && !d_points)) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    idx->last_stream = st;
    idx->n = n;
    idx->qws.pending.valid = false;
    SFC_TRY(ensure_status_buf(idx, st));
    // every issued id is live again
    if (idx->dim == 3) return build3_from_device(idx, d_points, st);
    if (idx->alive.ptr) SFC_CUDA_TRY(cudaMemsetAsync(idx->alive.ptr, 0xff, idx->alive.bytes, st));
    SFC_TRY(build_from_device(idx, d_points, st));
    if (idx->opt.bounds == SFC_BOUNDS_LEARNED) {
        ProfScope ps(idx, "train", st);
        SFC_TRY(train_model(idx, st));
    }
    return SFC_OK;
}

sfc_status sfc_rebuild_host(sfc_index* idx, const int32_t* h_points, uint64_t n, void* stream)
{
    if (!idx || n >= 0xffffffffull || (n && !h_points)) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    const size_t bytes = n * (size_t)idx->dim * sizeof(int32_t);
    SFC_TRY(idx->stage.points.ensure(bytes ? bytes : 1, st));
    if (n) SFC_CUDA_TRY(cudaMemcpyAsync(idx->stage.points.ptr, h_points, bytes, cudaMemcpyHostToDevice, st));
    return sfc_rebuild(idx, idx->stage.points.as<int32_t>(), n, stream);
}

sfc_status sfc_reserve(sfc_index* idx, uint64_t n_max, uint64_t m_max, void* stream)
{
    if (!idx || n_max >= 0xffffffffull) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    SFC_TRY(ensure_status_buf(idx, st));
    const uint64_t n1 = n_max ? n_max : 1;
    SFC_TRY(idx->keys.ensure(n1 * sizeof(uint64_t), st));
    SFC_TRY(idx->ids.ensure(n1 * sizeof(uint32_t), st));
    if (idx->dim == 3) {
        SFC_TRY(idx->xyz.ensure(n1 * sizeof(int4), st));
        SFC_TRY(idx->keys_in.ensure(n1 * sizeof(uint64_t), st));
    } else {
        SFC_TRY(idx->xy.ensure(n1 * sizeof(int2), st));
        SFC_TRY(idx->xy_by_id.ensure(n1 * sizeof(int2), st));
        SFC_TRY(ensure_alive_bits(idx, n1, st));
    }
    if (idx->opt.occupancy_depth > 0)
        SFC_TRY(idx->occ.ensure(occupancy_words(idx->opt.occupancy_depth) * sizeof(uint32_t), st));
    SFC_TRY(reserve_sort(idx->sort_ws, n1, st));
    SFC_TRY(ensure_query_ws(idx, m_max, st));
    SFC_TRY(reserve_scan(idx->scan_ws, std::max<uint64_t>(m_max, n1) + 1, st));
    if (idx->opt.bounds == SFC_BOUNDS_LEARNED) SFC_TRY(reserve_model(idx, n1, st));
    return SFC_OK;
}

}  // extern "C"

struct sfc_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

sfc_status sfc_graph_capture(sfc_index* idx, unsigned flags, const int32_t* d_points, uint64_t n,
                             const int32_t* d_q, const int32_t* d_delta, uint64_t m, uint64_t* d_out_offsets,
                             uint32_t* d_out_ids, uint64_t ids_capacity, sfc_graph** out, void* stream)
{
    if (!idx || !out || !flags || (flags & ~(SFC_GRAPH_REBUILD | SFC_GRAPH_QUERY))) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    *out = nullptr;
    const bool rb = flags & SFC_GRAPH_REBUILD, qb = flags & SFC_GRAPH_QUERY;
    if (rb && (n >= 0xffffffffull || (n && !d_points))) return SFC_ERR_INVALID;
    if (qb && (!d_out_offsets || (m && (!d_q || !d_delta)) || (ids_capacity && !d_out_ids))) return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    SFC_TRY(sfc_reserve(idx, rb ? n : idx->n, qb ? m : 0, stream));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));   // set-up done before capture starts
    cudaStream_t cs = nullptr;
    SFC_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    sfc_graph* g = new (std::nothrow) sfc_graph();
    if (!g) { cudaStreamDestroy(cs); return SFC_ERR_OOM; }
    sfc_status s = SFC_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) s = SFC_ERR_CUDA;
    if (s == SFC_OK && rb) s = sfc_rebuild(idx, d_points, n, cs);
    if (s == SFC_OK && qb) s = sfc_query_batch(idx, d_q, d_delta, m, d_out_offsets, d_out_ids, ids_capacity, cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (s == SFC_OK && ce != cudaSuccess) s = SFC_ERR_CUDA;
    if (s == SFC_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) s = SFC_ERR_CUDA;
    g->graph = graph;
    cudaStreamDestroy(cs);
    idx->last_stream = st;
    if (s != SFC_OK) {
        cudaGetLastError();
        sfc_graph_destroy(g);
        return s;
    }
    *out = g;
    return SFC_OK;
}

sfc_status sfc_graph_launch(sfc_graph* g, void* stream)
{
    if (!g || !g->exec) return SFC_ERR_INVALID;
    SFC_CUDA_TRY(cudaGraphLaunch(g->exec, as_stream(stream)));
    count_launch();
    return SFC_OK;
}

void sfc_graph_destroy(sfc_graph* g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

sfc_status sfc_query_count(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                           uint64_t* d_out_offsets, void* stream)
{
    if (!idx || !d_out_offsets || (m && (!d_q || !d_delta)) || m >= 0xffffffffull) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    idx->last_stream = as_stream(stream);
    return do_count(idx, d_q, d_delta, m, d_out_offsets, as_stream(stream));
}

sfc_status sfc_query_write(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                           const uint64_t* d_out_offsets, uint32_t* d_out_ids, uint64_t ids_capacity,
                           void* stream)
{
    if (!idx || !d_out_offsets || (ids_capacity && !d_out_ids)) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    idx->last_stream = as_stream(stream);
    return do_write(idx, d_q, d_delta, m, d_out_offsets, d_out_ids, ids_capacity, as_stream(stream));
}

sfc_status sfc_query_batch(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                           uint64_t* d_out_offsets, uint32_t* d_out_ids, uint64_t ids_capacity,
                           void* stream)
{
    SFC_TRY(sfc_query_count(idx, d_q, d_delta, m, d_out_offsets, stream));
    return sfc_query_write(idx, d_q, d_delta, m, d_out_offsets, d_out_ids, ids_capacity, stream);
}

}  // extern "C"

namespace {

struct TuneKey {
    int device, curve, lgn, lgm, bounds, cover, norm;   // cover: the option (-1 = tuned)
    bool operator==(const TuneKey& o) const
    {
        return device == o.device && curve == o.curve && lgn == o.lgn && lgm == o.lgm && bounds == o.bounds &&
               cover == o.cover && norm == o.norm;
    }
};

struct TuneVal {
    uint32_t chunk, batch, qbatch;
    int drop;
};

std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TuneVal>> g_tune_cache;

int lg2(uint64_t v)
{
    int l = 0;
    while (v > 1) { v >>= 1; ++l; }
    return l;
}

// Device time of fn() on st with CUDA events (best of reps).
template <class F>
sfc_status time_on(cudaStream_t st, int reps, float* best, F fn)
{
    cudaEvent_t a, b;
    SFC_CUDA_TRY(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return SFC_ERR_CUDA; }
    *best = 1e30f;
    sfc_status s = SFC_OK;
    for (int r = 0; r < reps && s == SFC_OK; ++r) {
        cudaEventRecord(a, st);
        s = fn();
        cudaEventRecord(b, st);
        if (s == SFC_OK && cudaEventSynchronize(b) == cudaSuccess) {
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < *best) *best = ms;
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return s;
}

}  // namespace

extern "C" {

sfc_status sfc_autotune(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m, int force,
                        int* h_chunk, int* h_batch, int* h_qbatch, void* stream)
{
    if (!idx || (m && (!d_q || !d_delta)) || m >= 0xffffffffull) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    const TuneKey key{idx->device, (int)idx->curve, lg2(idx->n + 1), lg2(m + 1), (int)idx->bounds,
                      idx->opt.cover_refine, idx->norm};
    bool cached = false;
    if (!force) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        for (const auto& kv : g_tune_cache)
            if (kv.first == key) {
                idx->chunk = kv.second.chunk;
                idx->batch = kv.second.batch;
                idx->qbatch = kv.second.qbatch;
                idx->drop = kv.second.drop;
                cached = true;
            }
    }
    if (!cached && m > 0) {
        const bool prof = idx->prof.on;
        idx->prof.on = false;
        DevBuf off, ids;
        sfc_status s = off.ensure((m + 1) * sizeof(uint64_t), st);
        auto count = [&]() { return do_count(idx, d_q, d_delta, m, off.as<uint64_t>(), st); };
        auto write = [&](uint64_t total) {
            return do_write(idx, d_q, d_delta, m, off.as<uint64_t>(), ids.as<uint32_t>(), total, st);
        };
        // the result (and so its size) is the same under every setting
        uint64_t total = 0;
        if (s == SFC_OK) s = count();
        if (s == SFC_OK && cudaMemcpyAsync(&total, off.as<uint64_t>() + m, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess) s = SFC_ERR_CUDA;
        if (s == SFC_OK && cudaStreamSynchronize(st) != cudaSuccess) s = SFC_ERR_CUDA;
        if (s == SFC_OK) s = ids.ensure(std::max<uint64_t>(total, 1) * sizeof(uint32_t), st);
        idx->qws.pending.valid = false;
        float best = 1e30f, t = 0.0f;
        int bd = idx->drop;
        if (idx->opt.cover_refine < 0) {   // the cover: whole batches (both passes) per candidate
            for (int d : {0, 1, 2}) {
                if (s != SFC_OK) break;
                if (idx->dim == 3 && d > 1) break;   // 3-D covers: cells(Q) or one level finer
                idx->drop = d;
                s = time_on(st, 2, &t, [&]() {
                    sfc_status c = count();
                    return c == SFC_OK ? write(total) : c;
                });
                if (t < best) { best = t; bd = d; }
            }
            idx->drop = bd;
        }
        uint32_t bc = idx->chunk, bb = idx->batch, bq = idx->qbatch;
        best = 1e30f;
        for (uint32_t c : {256u, 512u, 1024u, 2048u, 4096u}) {
            if (s != SFC_OK) break;
            idx->chunk = c;
            idx->batch = 4;
            s = time_on(st, 2, &t, count);
            if (t < best) { best = t; bc = c; }
        }
        idx->chunk = bc;
        best = 1e30f;
        for (uint32_t b : {1u, 2u, 4u, 8u, 16u}) {
            if (s != SFC_OK) break;
            idx->batch = b;
            s = time_on(st, 2, &t, count);
            if (t < best) { best = t; bb = b; }
        }
        idx->batch = bb;
        // write pass: one count with the chosen settings, then time the writes
        if (s == SFC_OK) s = count();
        best = 1e30f;
        for (uint32_t qb : {1u, 2u, 4u, 8u, 16u}) {
            if (s != SFC_OK) break;
            idx->qbatch = qb;
            s = time_on(st, 2, &t, [&]() {
                idx->qws.pending.valid = true;   // the plan of the last count is still in place
                return write(total);
            });
            if (t < best) { best = t; bq = qb; }
        }
        idx->qbatch = bq;
        idx->qws.pending.valid = false;
        ids.release(st);
        off.release(st);
        idx->prof.on = prof;
        cudaStreamSynchronize(st);
        if (s != SFC_OK) return s;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        bool found = false;
        for (auto& kv : g_tune_cache)
            if (kv.first == key) { kv.second = TuneVal{bc, bb, bq, bd}; found = true; }
        if (!found) g_tune_cache.push_back({key, TuneVal{bc, bb, bq, bd}});
    }
    if (h_chunk) *h_chunk = (int)idx->chunk;
    if (h_batch) *h_batch = (int)idx->batch;
    if (h_qbatch) *h_qbatch = (int)idx->qbatch;
    return SFC_OK;
}

sfc_status sfc_set_tuning(sfc_index* idx, int chunk, int batch, int qbatch)
{
    if (!idx || chunk < 32 || chunk > 4096 || (chunk & 31) || batch < 1 || batch > 1024 || qbatch < 1 ||
        qbatch > 1024)
        return SFC_ERR_INVALID;
    idx->chunk = (uint32_t)chunk;
    idx->batch = (uint32_t)batch;
    idx->qbatch = (uint32_t)qbatch;
    return SFC_OK;
}

sfc_status sfc_set_query_norm(sfc_index* idx, sfc_norm norm)
{
    if (!idx || (norm != SFC_NORM_DISC && norm != SFC_NORM_SQUARE)) return SFC_ERR_INVALID;
    if (idx->dim == 3 && norm != SFC_NORM_DISC) return SFC_ERR_INVALID;
    idx->norm = norm;
    return SFC_OK;
}

sfc_status sfc_set_cover(sfc_index* idx, int refine)
{
    if (!idx || refine < 0 || refine > 2 || (idx->dim == 3 && refine > 1)) return SFC_ERR_INVALID;
    idx->drop = refine;
    return SFC_OK;
}

sfc_status sfc_get_occupancy(const sfc_index* cidx, uint32_t* d_out, uint64_t words, int* h_depth, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx || !d_out) return SFC_ERR_INVALID;
    const int D = idx->opt.occupancy_depth;
    if (D <= 0 || !idx->occ.ptr) return SFC_ERR_STATE;
    const uint64_t need = occupancy_words(D);
    if (words < need) return SFC_ERR_CAPACITY;
    if (h_depth) *h_depth = D;
    SFC_CUDA_TRY(cudaMemcpyAsync(d_out, idx->occ.ptr, need * sizeof(uint32_t), cudaMemcpyDeviceToDevice,
                                 as_stream(stream)));
    return SFC_OK;
}

sfc_status sfc_query_cell_stats(const sfc_index* cidx, uint64_t* h_cells, uint64_t* h_empty, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx || !idx->status.ptr) return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    unsigned long long v[2] = {0, 0};
    SFC_CUDA_TRY(cudaMemcpyAsync(v, model_stats(idx) + 4, sizeof(v), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_cells) *h_cells = v[0];
    if (h_empty) *h_empty = v[1];
    return SFC_OK;
}

int sfc_query_max_intervals(const sfc_index* idx) { return idx ? query_intervals(idx->dim, idx->drop) : 0; }

int sfc_cover_refine(const sfc_index* idx) { return idx ? idx->drop : -1; }

sfc_status sfc_query_batch_host(sfc_index* idx, const int32_t* h_q, const int32_t* h_delta, uint64_t m,
                                uint64_t* h_out_offsets, uint32_t* h_out_ids, uint64_t ids_capacity,
                                void* stream)
{
    if (!idx || !h_out_offsets || (m && (!h_q || !h_delta)) || (ids_capacity && !h_out_ids) ||
        m >= 0xffffffffull)
        return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    idx->last_stream = st;
    HostStage& hs = idx->stage;
    const uint64_t qbytes = m * (uint64_t)idx->dim * sizeof(int32_t);
    SFC_TRY(hs.q.ensure(qbytes, st));
    SFC_TRY(hs.delta.ensure(m * sizeof(int32_t), st));
    SFC_TRY(hs.offsets.ensure((m + 1) * sizeof(uint64_t), st));
    int32_t* dq = hs.q.as<int32_t>();
    int32_t* dd = hs.delta.as<int32_t>();
    uint64_t* doff = hs.offsets.as<uint64_t>();
    if (m) {
        SFC_CUDA_TRY(cudaMemcpyAsync(dq, h_q, qbytes, cudaMemcpyHostToDevice, st));
        SFC_CUDA_TRY(cudaMemcpyAsync(dd, h_delta, m * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    }
    SFC_TRY(do_count(idx, dq, dd, m, doff, st));
    SFC_CUDA_TRY(cudaMemcpyAsync(h_out_offsets, doff, (m + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    const uint64_t total = h_out_offsets[m];
    if (total > ids_capacity) {
        idx->qws.pending.valid = false;
        return SFC_ERR_CAPACITY;
    }
    SFC_TRY(hs.ids.ensure(total * sizeof(uint32_t), st));
    uint32_t* d_ids = hs.ids.as<uint32_t>();
    const int S = HostStage::kSlices;
    if (m >= (uint64_t)S && total * sizeof(uint32_t) >= (32ull << 20)) {
        // the write pass in query slices; the ids of each finished slice go out on a second
        // stream while the next slices are written (output offsets are in query order)
        const uint32_t* sperm = nullptr;
        if (idx->qws.pending.ordered) {
            // curve order: regroup the processing order by input slice (a stable one-digit sort
            // of the slice numbers), so slice s is positions [floor(m s / S), floor(m (s + 1) / S))
            // and keeps curve order inside
            SFC_TRY(hs.slice_keys.ensure(m * sizeof(uint64_t), st));
            SFC_TRY(hs.slice_keys_sorted.ensure(m * sizeof(uint64_t), st));
            SFC_TRY(hs.slice_perm.ensure(m * sizeof(uint32_t), st));
            const uint32_t* perm = idx->qws.perm.as<uint32_t>();
            SFC_TRY(launch_slice_keys(perm, m, S, hs.slice_keys.as<uint64_t>(), st));
            SortSource src;
            src.keys = hs.slice_keys.as<uint64_t>();
            src.vals = perm;
            SortDest dst;
            dst.keys = hs.slice_keys_sorted.as<uint64_t>();
            dst.vals = hs.slice_perm.as<uint32_t>();
            SFC_TRY(radix_sort(src, m, dst, idx->sort_ws, status_word(idx), st));
            sperm = hs.slice_perm.as<uint32_t>();
        }
        if (!hs.copy) {
            SFC_CUDA_TRY(cudaStreamCreateWithFlags(&hs.copy, cudaStreamNonBlocking));
            for (auto& e : hs.done) SFC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        }
        idx->qws.pending.valid = false;
        for (int sl = 0; sl < S; ++sl) {
            const uint64_t qa = m * (uint64_t)sl / S, qb = m * (uint64_t)(sl + 1) / S;
            SFC_TRY(do_write_range(idx, dq, dd, m, doff, d_ids, total, st, qa, qb, sperm));
            SFC_CUDA_TRY(cudaEventRecord(hs.done[sl], st));
            SFC_CUDA_TRY(cudaStreamWaitEvent(hs.copy, hs.done[sl], 0));
            const uint64_t a = h_out_offsets[qa], b = h_out_offsets[qb];
            if (b > a)
                SFC_CUDA_TRY(cudaMemcpyAsync(h_out_ids + a, d_ids + a, (b - a) * sizeof(uint32_t),
                                             cudaMemcpyDeviceToHost, hs.copy));
        }
        SFC_CUDA_TRY(cudaStreamSynchronize(hs.copy));
        SFC_CUDA_TRY(cudaStreamSynchronize(st));
        return SFC_OK;
    }
    SFC_TRY(do_write(idx, dq, dd, m, doff, d_ids, total, st));
    if (total)
        SFC_CUDA_TRY(cudaMemcpyAsync(h_out_ids, d_ids, total * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    return SFC_OK;
}

sfc_status sfc_reserve_queries(sfc_index* idx, uint64_t m, void* stream)
{
    if (!idx) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    SFC_TRY(ensure_status_buf(idx, as_stream(stream)));
    return ensure_query_ws(idx, m, as_stream(stream));
}

sfc_status sfc_set_bounds_mode(sfc_index* idx, sfc_bounds mode)
{
    if (!idx || (mode != SFC_BOUNDS_BINARY && mode != SFC_BOUNDS_LEARNED)) return SFC_ERR_INVALID;
    if (idx->dim == 3 && mode != SFC_BOUNDS_BINARY) return SFC_ERR_INVALID;
    if (mode == SFC_BOUNDS_LEARNED && !idx->model.trained) return SFC_ERR_STATE;
    idx->bounds = mode;
    return SFC_OK;
}

sfc_status sfc_train_model(sfc_index* idx, void* stream)
{
    if (!idx || idx->dim != 2) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    idx->last_stream = as_stream(stream);
    ProfScope ps(idx, "train", as_stream(stream));
    return train_model(idx, as_stream(stream));
}

sfc_status sfc_profile_enable(sfc_index* idx, int on)
{
    if (!idx) return SFC_ERR_INVALID;
    idx->prof.on = on != 0;
    return SFC_OK;
}

sfc_status sfc_profile_read(sfc_index* idx, sfc_profile_entry* out, int max, int* count, int reset,
                            void* stream)
{
    if (!idx || (max > 0 && !out)) return SFC_ERR_INVALID;
    SFC_CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
    std::vector<sfc_profile_entry> agg;
    for (const ProfRec& r : idx->prof.recs) {
        float ms = 0.0f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
            cudaGetLastError();
            ms = 0.0f;
        }
        size_t k = 0;
        while (k < agg.size() && std::strncmp(agg[k].name, r.name, sizeof(agg[k].name)) != 0) ++k;
        if (k == agg.size()) {
            sfc_profile_entry e{};
            std::strncpy(e.name, r.name, sizeof(e.name) - 1);
            agg.push_back(e);
        }
        agg[k].launches += 1;
        agg[k].ms += ms;
    }
    if (reset) {
        for (const ProfRec& r : idx->prof.recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        idx->prof.recs.clear();
    }
    const int n = (int)agg.size();
    for (int i = 0; i < n && i < max; ++i) out[i] = agg[i];
    if (count) *count = n;
    return SFC_OK;
}

sfc_status sfc_model_stats(const sfc_index* cidx, uint64_t* h_endpoints, uint64_t* h_misses,
                           uint64_t* h_window_sum, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx) return SFC_ERR_INVALID;
    unsigned long long v[3];
    cudaStream_t st = as_stream(stream);
    SFC_CUDA_TRY(cudaMemcpyAsync(v, model_stats(idx), sizeof(v), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_endpoints) *h_endpoints = v[0];
    if (h_misses) *h_misses = v[1];
    if (h_window_sum) *h_window_sum = v[2];
    return SFC_OK;
}

sfc_status sfc_query_stats(const sfc_index* cidx, uint64_t* h_scanned, uint64_t* h_chunks,
                           uint64_t* h_hits, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx || !idx->status.ptr) return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    unsigned long long s = 0;
    uint64_t g = 0, h = 0;
    SFC_CUDA_TRY(cudaMemcpyAsync(&s, scan_stats(idx), sizeof(s), cudaMemcpyDeviceToHost, st));
    const PendingCount& p = idx->qws.pending;
    if (p.m && idx->qws.chunk_base.ptr)
        SFC_CUDA_TRY(cudaMemcpyAsync(&g, idx->qws.chunk_base.as<uint64_t>() + p.m, sizeof(g),
                                     cudaMemcpyDeviceToHost, st));
    if (p.m && p.offsets)
        SFC_CUDA_TRY(cudaMemcpyAsync(&h, p.offsets + p.m, sizeof(h), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_scanned) *h_scanned = s;
    if (h_chunks) *h_chunks = g;
    if (h_hits) *h_hits = h;
    return SFC_OK;
}

sfc_status sfc_get_sorted(const sfc_index* idx, const uint64_t** d_keys, const uint32_t** d_ids,
                          const int32_t** d_xy, uint64_t* n)
{
    if (!idx) return SFC_ERR_INVALID;
    if (d_keys) *d_keys = idx->keys.as<uint64_t>();
    if (d_ids) *d_ids = idx->ids.as<uint32_t>();
    if (d_xy) *d_xy = idx->dim == 3 ? idx->xyz.as<int32_t>() : idx->xy.as<int32_t>();
    if (n) *n = idx->n;
    return SFC_OK;
}

int sfc_index_dim(const sfc_index* idx) { return idx ? idx->dim : 0; }

sfc_status sfc_keys3(const int32_t* d_points, uint64_t n, uint64_t* d_keys, void* stream)
{
    if (n && (!d_points || !d_keys)) return SFC_ERR_INVALID;
    return launch_keys3(d_points, n, d_keys, nullptr, as_stream(stream));
}

sfc_status sfc_build3(sfc_index** out, const int32_t* d_points, uint64_t n, const sfc_options* opt,
                      const sfc_allocator* alloc, void* stream)
{
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n >= 0xffffffffull || (n && !d_points)) return SFC_ERR_INVALID;
    if (alloc && (!alloc->alloc || !alloc->free)) return SFC_ERR_INVALID;
    sfc_options o;
    sfc_default_options(&o);
    if (opt) o = *opt;
    if (o.bounds != SFC_BOUNDS_BINARY || o.cover_refine > 1 || o.cover_refine < -1 || o.occupancy_depth != 0 ||
        o.query_norm != SFC_NORM_DISC || o.mask_budget_mb < 1 ||
        (o.chunk != 0 && (o.chunk < 32 || o.chunk > 4096 || (o.chunk & 31))))
        return SFC_ERR_INVALID;
    o.reorder_queries = 0;
    cudaStream_t st = as_stream(stream);
    sfc_index* idx = new (std::nothrow) sfc_index();
    if (!idx) return SFC_ERR_OOM;
    cudaGetDevice(&idx->device);
    if (alloc) {
        idx->alloc = *alloc;
        idx->has_alloc = true;
    }
    AllocScope scope(idx->allocator());
    idx->curve = SFC_CURVE_Z;
    idx->dim = 3;
    idx->drop = o.cover_refine < 0 ? 1 : o.cover_refine;
    idx->n = n;
    idx->opt = o;
    idx->chunk = o.chunk ? (uint32_t)o.chunk : 1024u;
    idx->last_stream = st;
    idx->prof.on = o.profile != 0;
    sfc_status s = ensure_status_buf(idx, st);
    if (s == SFC_OK) s = build3_from_device(idx, d_points, st);
    if (s != SFC_OK) {
        sfc_destroy(idx);
        return s;
    }
    *out = idx;
    return SFC_OK;
}

sfc_status sfc_build3_host(sfc_index** out, const int32_t* h_points, uint64_t n, const sfc_options* opt,
                           const sfc_allocator* alloc, void* stream)
{
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n >= 0xffffffffull || (n && !h_points)) return SFC_ERR_INVALID;
    if (alloc && (!alloc->alloc || !alloc->free)) return SFC_ERR_INVALID;
    cudaStream_t st = as_stream(stream);
    AllocScope scope(alloc);
    void* d = nullptr;
    const sfc_allocator* owner = nullptr;
    SFC_TRY(dev_alloc(&d, n * 3 * sizeof(int32_t), st, &owner));
    cudaError_t e = n ? cudaMemcpyAsync(d, h_points, n * 3 * sizeof(int32_t), cudaMemcpyHostToDevice, st) : cudaSuccess;
    sfc_status s = e == cudaSuccess ? sfc_build3(out, static_cast<int32_t*>(d), n, opt, alloc, stream) : SFC_ERR_CUDA;
    dev_free(d, n * 3 * sizeof(int32_t), st, owner);
    return s;
}

sfc_status sfc_device_status(sfc_index* idx, uint32_t* h_bits, void* stream)
{
    if (!idx) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    SFC_TRY(ensure_status_buf(idx, st));
    uint32_t bits = 0;
    SFC_CUDA_TRY(cudaMemcpyAsync(&bits, idx->status.ptr, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaMemsetAsync(idx->status.ptr, 0, sizeof(uint32_t), st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_bits) *h_bits = bits;
    if (bits & SFC_DEV_TIMEOUT) return SFC_ERR_TIMEOUT;
    if (bits & (SFC_DEV_BAD_POINT | SFC_DEV_BAD_QUERY)) return SFC_ERR_INVALID;
    if (bits & SFC_DEV_NOT_FOUND) return SFC_ERR_NOT_FOUND;
    if (bits & SFC_DEV_CAPACITY) return SFC_ERR_CAPACITY;
    return SFC_OK;
}

sfc_status sfc_keys(const int32_t* d_points, uint64_t n, sfc_curve curve, uint64_t* d_keys, void* stream)
{
    if ((n && (!d_points || !d_keys)) || (curve != SFC_CURVE_Z && curve != SFC_CURVE_HILBERT))
        return SFC_ERR_INVALID;
    return launch_keys(reinterpret_cast<const int2*>(d_points), n, curve, d_keys, nullptr, as_stream(stream));
}

sfc_status sfc_decode(const uint64_t* d_keys, uint64_t n, sfc_curve curve, int32_t* d_points, void* stream)
{
    if ((n && (!d_points || !d_keys)) || (curve != SFC_CURVE_Z && curve != SFC_CURVE_HILBERT))
        return SFC_ERR_INVALID;
    return launch_decode(d_keys, n, curve, reinterpret_cast<int2*>(d_points), as_stream(stream));
}

sfc_status sfc_sort_pairs(const uint64_t* d_keys_in, const uint32_t* d_ids_in, uint64_t n,
                          uint64_t* d_keys_out, uint32_t* d_ids_out, void* stream)
{
    if (n >= 0xffffffffull || (n && (!d_keys_in || !d_keys_out || !d_ids_out))) return SFC_ERR_INVALID;
    if (n == 0) return SFC_OK;
    cudaStream_t st = as_stream(stream);
    SortWorkspace ws;
    SortSource src;
    src.keys = d_keys_in;
    src.vals = d_ids_in;
    SortDest dst;
    dst.keys = d_keys_out;
    dst.vals = d_ids_out;
    sfc_status s = radix_sort(src, n, dst, ws, nullptr, st);
    release_sort_ws(ws, st);
    return s;
}

sfc_status sfc_exclusive_scan(const uint32_t* d_in, uint64_t n, uint64_t* d_out, void* stream)
{
    if (!d_out || (n && !d_in)) return SFC_ERR_INVALID;
    return exclusive_scan_standalone(d_in, n, d_out, as_stream(stream));
}

sfc_status sfc_query_ranges(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                            uint64_t* d_lo, uint64_t* d_hi, uint32_t* d_begin, uint32_t* d_end,
                            uint32_t* d_count, void* stream)
{
    if (!idx || (m && (!d_q || !d_delta))) return SFC_ERR_INVALID;
    AllocScope alloc_scope(idx->allocator());
    cudaStream_t st = as_stream(stream);
    SFC_TRY(ensure_status_buf(idx, st));
    QueryArgs a = base_args(idx, d_q, d_delta, m);
    LearnedModelView lv;
    return launch_ranges(a, model_view(idx, lv), d_lo, d_hi, d_begin, d_end, d_count, st);
}

uint64_t sfc_launch_count(void) { return g_launches.load(); }

uint64_t sfc_pool_bytes_in_use(void) { return g_pool_bytes.load(); }

const char* sfc_status_string(sfc_status s)
{
    switch (s) {
        case SFC_OK: return "SFC_OK";
        case SFC_ERR_INVALID: return "SFC_ERR_INVALID";
        case SFC_ERR_OOM: return "SFC_ERR_OOM";
        case SFC_ERR_CAPACITY: return "SFC_ERR_CAPACITY";
        case SFC_ERR_NOT_FOUND: return "SFC_ERR_NOT_FOUND";
        case SFC_ERR_TIMEOUT: return "SFC_ERR_TIMEOUT";
        case SFC_ERR_CUDA: return "SFC_ERR_CUDA";
        case SFC_ERR_STATE: return "SFC_ERR_STATE";
    }
    return "SFC_ERR_UNKNOWN";
}

}  // extern "C"
