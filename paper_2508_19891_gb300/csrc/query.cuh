// Arguments and launchers of the query pipeline (query.cu), shared with the C-ABI layer.
#pragma once

#include "sfc_internal.cuh"

namespace sfc {

struct QueryArgs {
    int curve;
    const uint64_t* keys;        // sorted keys [n]
    const uint32_t* ids;         // ids in sorted order [n]
    const int2* xy;              // coordinates in sorted order [n] (2-D)
    const int4* xyz;             // coordinates in sorted order [n] (3-D: x, y, z, 0)
    int dim;                     // 2 or 3; queries are int32[m][dim]
    uint32_t n;
    const int32_t* q;            // [m][dim]
    const int32_t* delta;        // [m]
    uint64_t m;
    uint32_t* ranges;            // [m][2 * kint]: (begin, end) of up to kint intervals
    uint32_t kint;               // intervals stored per query (2-D: 4, 9 or 25 by the cover; 3-D: 8 or 27)
    int drop;                    // cover refinement: 0 cells(Q), 1 or 2 levels finer
    int norm;                    // SFC_NORM_DISC or SFC_NORM_SQUARE
    uint32_t* nchunks;           // [m]
    uint64_t* chunk_base;        // [m + 1]
    uint32_t* counts;            // [m] hits per query
    uint32_t* masks;             // hit bitmask, chunk g at masks + g * (chunk / 32)
    uint64_t mask_chunks;        // chunks that fit in the bitmask buffer
    uint32_t chunk;              // points per chunk (multiple of 32, <= 4096)
    uint32_t batch;              // chunks taken per work-queue grab (count pass)
    uint32_t qbatch;             // queries taken per grab (write pass)
    unsigned long long* work_ctr;  // kCtrWords counters, see kCtrCount ... kCtrSmallCount
    // queries that scan at most kSmallScan points skip the chunked passes: the plan lists them
    // (small_list[0 .. work_ctr[kCtrSmallSize])) and the count and write kernels, once their
    // chunked work is claimed, take them one thread per query, keeping each one's hits as
    // kSmallWords mask words (NULL: no small-query path)
    uint32_t* small_list;
    unsigned long long* small_mask;
    uint64_t* out_offsets;       // [m + 1]
    uint32_t* out_ids;
    uint64_t ids_capacity;
    // write pass: the processing positions [q_begin, q_end) (q_end 0: all m); the caller
    // arranges that they hold exactly the queries with ids in [q_begin, q_end) (input order,
    // or a curve order regrouped by slice), which is also the small queries' filter
    uint64_t q_begin, q_end;
    uint32_t* status;
    unsigned long long* scanned;   // sum of S_q over the batch (statistics)
    // optional processing order: queries handed out in curve order of their centres
    const uint32_t* perm;        // [m] query index at each processing rank (NULL: identity)
    const uint64_t* wbase;       // [m + 1] chunk bases in processing order (NULL: chunk_base)
    // big queries (more chunks than one warp's share, all below big_cap): the plan lists the
    // candidates; after the count pass, each chunk's hit count (from its mask words) is scanned
    // inside each big query into chunk_hits[g] (g = chunk_base[q] + j), the chunk's first output
    // position within the query, and its chunks are listed in big_items
    // (work_ctr[kCtrBigItems] of them); the write pass spreads the listed chunks over many warps
    uint32_t* chunk_hits;
    uint32_t* big_list;          // [m] the queries of at least kBigChunks chunks (work_ctr[kCtrBigList])
    uint32_t* big_items;
    uint64_t big_cap;
    uint32_t big_warps;          // warps the write pass runs (a query is big past G / big_warps chunks)
    // early-termination bitmap (NULL: off) and the cover statistics
    const uint32_t* occ;
    int occ_depth;
    unsigned long long* cells;   // [0] cells of the covers, [1] of them found empty
};

struct LearnedModelView {
    const RootParams* root;      // device memory (written by training, no host copy needed)
    const LeafParams* leaf;
    const uint64_t* fence;       // [leaves][kFence] fence keys
    const uint64_t* fence_fine;  // [leaves][kFenceFine] fine fence keys
    unsigned long long* stats;   // [3]: endpoints, misses, window sum
};

sfc_status launch_plan(const QueryArgs& a, const LearnedModelView* lm, cudaStream_t st);
int cover_intervals(int drop);   // intervals stored per query for a cover refinement
int query_intervals(int dim, int drop);   // ... for an index of dimension dim
sfc_status launch_count(const QueryArgs& a, cudaStream_t st);
// scan length up to which a query takes the small-query path, and its mask words (one per 64
// scanned points)
constexpr uint32_t kSmallScan = 64;
constexpr uint32_t kSmallWords = (kSmallScan + 63) / 64;
// work counters of a query batch: the count pass's chunk queue, the write pass's query queue and
// its small-query queue (adjacent: the write pass clears both), the small-list length, the
// count pass's small-query queue, the write pass's queue of big-query chunks
constexpr int kCtrCount = 0, kCtrWrite = 1, kCtrSmallWrite = 2, kCtrSmallSize = 3, kCtrSmallCount = 4;
constexpr int kCtrWriteBig = 5, kCtrBigItems = 6, kCtrBigList = 7;
constexpr int kCtrWords = 8;
// a query of at least max(kBigChunks, G / big_warps) chunks is written chunk by chunk by many
// warps (one warp would set the write pass's tail: single queries reach 10^6 hits)
#ifndef SFC_BIG_CHUNKS
#define SFC_BIG_CHUNKS 8
#endif
constexpr uint64_t kBigChunks = SFC_BIG_CHUNKS;
// ... where big_warps is this many times the warps the write pass runs: a query is split once
// it has more than a quarter of one warp's share of the chunks.  Measured: splitting from 8
// chunks keeps dynamic-5e7's write pass at 1.6-2.1 ms (2.7-16 ms unsplit), while splitting
// mixed-1e7's queries of 8-20 chunks costs 0.17 ms there (1.14 -> 1.31 ms).
#ifndef SFC_BIG_SHARE
#define SFC_BIG_SHARE 4
#endif
constexpr uint32_t kBigShare = SFC_BIG_SHARE;
// chunk_hits entries per query of a batch (big_cap = min(this * m + 1024, mask chunks))
constexpr uint64_t kChunkHitsPerQuery = 4;
// per big query, chunk_hits[g] <- exclusive scan of the query's chunk hit counts (in place),
// and its chunk slots appended to big_items
sfc_status launch_chunk_prefix(const QueryArgs& a, cudaStream_t st);
// curve key of each query centre (invalid centres sort last) with the query index as value
sfc_status launch_query_keys(const int32_t* q, uint64_t m, int curve, uint64_t* keys, cudaStream_t st);
// out[r] = nchunks[perm[r]]
sfc_status launch_gather_u32(const uint32_t* src, const uint32_t* perm, uint64_t m, uint32_t* out, cudaStream_t st);
sfc_status launch_write(const QueryArgs& a, cudaStream_t st);
// keys[r] = the slice of query perm[r] when queries 0 .. m - 1 are cut into S slices
// [floor(m s / S), floor(m (s + 1) / S))
sfc_status launch_slice_keys(const uint32_t* perm, uint64_t m, int S, uint64_t* keys, cudaStream_t st);
sfc_status launch_ranges(const QueryArgs& a, const LearnedModelView* lm, uint64_t* lo, uint64_t* hi,
                         uint32_t* b, uint32_t* e, uint32_t* cnt, cudaStream_t st);

}  // namespace sfc
