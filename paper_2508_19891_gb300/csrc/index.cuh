// The opaque index object behind the C ABI and the host functions that operate on it.
#pragma once

#include <vector>

#include "sfc_internal.cuh"

namespace sfc {

struct PendingCount {       // plan kept between sfc_query_count and sfc_query_write
    bool valid;
    const int32_t* q;
    const int32_t* delta;
    uint64_t m;
    const uint64_t* offsets;
    uint32_t chunk;
    bool ordered;           // queries processed in curve order (perm / wbase valid)
    int drop;               // cover refinement of the plan
    int norm;               // query window of the plan
};

struct QueryWs {
    DevBuf ranges, nchunks, chunk_base, counts, masks, ctr;
    DevBuf small_list, small_mask;   // queries of the small-query path and their hit masks
    DevBuf chunk_hits;               // per-chunk hit counts, then in-query offsets, of big queries
    DevBuf big_items;                // the chunk slots of big queries, listed query by query
    DevBuf big_list;                 // the big queries
    DevBuf qkeys, qkeys_sorted, perm, nch_sorted, wbase;   // curve-order processing
    PendingCount pending{false, nullptr, nullptr, 0, nullptr, 0, false, 0, 0};
};

struct HostStage {          // device staging of sfc_query_batch_host and sfc_rebuild_host
    static constexpr int kSlices = 8;   // write-pass slices whose ids are copied out as they finish
    DevBuf q, delta, offsets, ids;
    DevBuf points;                      // sfc_rebuild_host's copy of the points
    // curve-ordered batches: the processing order regrouped by input slice (stable), so each
    // slice's queries are written together and their ids form one contiguous range
    DevBuf slice_keys, slice_keys_sorted, slice_perm;
    cudaStream_t copy = nullptr;        // stream of the device-to-host copies of the ids
    cudaEvent_t done[kSlices] = {};     // slice s written
};

struct ModelState {
    bool trained = false;
    int nleaves = 0;
    int kind = 0;      // root kind of the trained model
    DevBuf state;      // optimiser state and derived root parameters (layout in learned.cu)
    DevBuf samples;    // training sample x[N], y[N]
    DevBuf partial;    // per-block partial gradients and the completion counter
    DevBuf tmp;        // leaf boundaries (uint32[nleaves + 1]) during a fit
    DevBuf leaves;     // LeafParams[nleaves], read by the query path
    DevBuf fence;      // uint64[nleaves][kFence]: fence keys of each leaf, read by the query path
    DevBuf fence_fine; // uint64[nleaves][kFenceFine]: the fine fence keys of each leaf
};

struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};

struct Profiler {
    bool on = false;
    std::vector<ProfRec> recs;
};

struct UpdateWs {
    DevBuf a, b, c, d, e, f, g, h;   // flags, delete keys/ids/positions, insert keys/ids/xy/ranks
    DevBuf keys, ids, xy;            // the next sorted arrays (swapped with the index's)
    DevBuf mark, v, t;               // deleted marks, shift counts, their exclusive scan
};

}  // namespace sfc

struct sfc_index {
    int device = 0;
    sfc_curve curve = SFC_CURVE_Z;
    uint64_t n = 0;                     // live points
    uint32_t next_id = 0;               // first id not yet issued
    sfc_options opt{};
    sfc_bounds bounds = SFC_BOUNDS_BINARY;
    uint32_t chunk = 1024;              // points per scan chunk
    uint32_t batch = 4;                 // chunks per work-queue grab
    uint32_t qbatch = 8;                // queries per write-queue grab
    int drop = 0;                       // cover refinement: levels below cells(Q) (0..2)
    int norm = 0;                       // query window (sfc_norm)
    int dim = 2;                        // 2, or 3 for indexes made by sfc_build3
    cudaStream_t last_stream = nullptr;
    sfc_allocator alloc{};              // the caller's allocator (used when has_alloc)
    bool has_alloc = false;
    const sfc_allocator* allocator() const { return has_alloc ? &alloc : nullptr; }

    sfc::DevBuf keys, ids, xy;          // the sorted array A_P and its keys
    sfc::DevBuf xy_by_id;               // coordinates by id (dynamic setting)
    sfc::DevBuf alive;                  // liveness bitmap by id
    sfc::DevBuf status;                 // device status word + model statistics
    sfc::DevBuf occ;                    // early-termination bitmap (occupancy_depth > 0)
    sfc::DevBuf xyz;                    // 3-D: coordinates in sorted order (int4 x, y, z, 0)
    sfc::DevBuf keys_in;                // 3-D: keys in input order (the sort's source)

    sfc::SortWorkspace sort_ws;
    sfc::ScanWorkspace scan_ws;
    sfc::QueryWs qws;
    sfc::HostStage stage;
    sfc::ModelState model;
    sfc::UpdateWs uws;
    sfc::Profiler prof;
};

namespace sfc {

sfc_status ensure_alive_bits(sfc_index* idx, uint64_t ids, cudaStream_t st);
void release_index(sfc_index* idx, cudaStream_t st);
sfc_status train_model(sfc_index* idx, cudaStream_t st);
sfc_status fit_leaves(sfc_index* idx, cudaStream_t st);
sfc_status reserve_model(sfc_index* idx, uint64_t n, cudaStream_t st);
sfc_status refit_model(sfc_index* idx, int steps, cudaStream_t st);
sfc_status apply_update(sfc_index* idx, const int32_t* d_inserts, uint64_t k_ins, const uint32_t* d_del,
                        uint64_t k_del, uint32_t* h_first, cudaStream_t st);
const RootParams* model_root_device(sfc_index* idx);
// early-termination bitmap of the sorted keys (no-op when opt.occupancy_depth == 0)
sfc_status build_occupancy(sfc_index* idx, cudaStream_t st);
uint64_t occupancy_words(int depth);

// Records CUDA events around a step when profiling is on.
class ProfScope {
public:
    ProfScope(sfc_index* idx, const char* name, cudaStream_t st) : idx_(idx), st_(st)
    {
        if (!idx || !idx->prof.on) return;
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
        rec_.name = name;
        if (cudaEventCreate(&rec_.a) != cudaSuccess) return;
        if (cudaEventCreate(&rec_.b) != cudaSuccess) { cudaEventDestroy(rec_.a); return; }
        cudaEventRecord(rec_.a, st);
        live_ = true;
    }
    ~ProfScope()
    {
        if (!live_) return;
        cudaEventRecord(rec_.b, st_);
        idx_->prof.recs.push_back(rec_);
    }
private:
    sfc_index* idx_;
    cudaStream_t st_;
    ProfRec rec_{};
    bool live_ = false;
};

}  // namespace sfc
