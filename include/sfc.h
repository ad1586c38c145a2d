/*
 * sfc.h — C ABI of the GB300 (sm_103a) library for batched 2-D distance reporting over a
 * point set sorted along a space-filling curve (method of "Simpler is Faster: Practical
 * Distance Reporting by Sorting Along a Space-Filling Curve", arXiv 2508.19891).
 *
 * Problem (Sec. 2, problem statement): store a set P of integer points so that a query
 * (q, delta) returns every point of P within distance delta of q.  Method (Sec. 2, Alg. 1):
 * sort P by its curve key pi(p); a query becomes at most four contiguous key intervals
 * (cells(Q), Observation), each located by lower_bound and scanned with an exact filter.
 *
 * Conventions for every call:
 *   - Coordinates are int32 in [0, 2^30) (w = 30 bits per axis); keys are the 60-bit curve
 *     labels of Def. 2.3 in a uint64.  Points and queries are interleaved (x, y) pairs.
 *   - Radii are int32 >= 0.  A point i is reported for (q, delta) iff
 *     (x_i - q_x)^2 + (y_i - q_y)^2 <= delta^2, evaluated exactly in 64-bit integers
 *     (the closed ball B_delta(q) of the problem statement).
 *   - Ids are input indices (0-based); points added by sfc_update get fresh ids.
 *   - "d_" arguments are DEVICE pointers on the index's device, "h_" arguments HOST
 *     pointers.  The caller owns every buffer it passes; nothing is retained after the call
 *     except inside the opaque index.  All device work is enqueued on `stream` (a
 *     cudaStream_t; NULL = the legacy default stream) and is asynchronous unless a call says
 *     it synchronises.
 *   - Host-detectable argument errors are returned at once and enqueue nothing.  Errors
 *     found on the device (a coordinate outside the domain, a negative radius, output
 *     capacity exceeded, a look-back wait that gave up) are recorded in the index's device
 *     status word and reported by sfc_device_status() or by the next call that synchronises.
 *     No call traps or aborts.
 *   - Nothing falls back to the CPU: every step of every call runs in this library's CUDA
 *     kernels.
 */
#ifndef SFC_H
#define SFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SFC_OK = 0,
    SFC_ERR_INVALID = -1,    /* bad argument, or (device) bad coordinate / radius */
    SFC_ERR_OOM = -2,        /* device allocation failed */
    SFC_ERR_CAPACITY = -3,   /* output capacity smaller than the result; offsets are complete */
    SFC_ERR_NOT_FOUND = -4,  /* update deletes an id that is not live (batch not applied) */
    SFC_ERR_TIMEOUT = -5,    /* a bounded device wait gave up; results of that call are void */
    SFC_ERR_CUDA = -6,       /* a CUDA runtime call failed */
    SFC_ERR_STATE = -7       /* call out of order (e.g. sfc_query_write without a count) */
} sfc_status;

typedef enum { SFC_CURVE_Z = 0, SFC_CURVE_HILBERT = 1 } sfc_curve;
typedef enum { SFC_BOUNDS_BINARY = 0, SFC_BOUNDS_LEARNED = 1 } sfc_bounds;
/* Root of the learned CDF model: monotone piecewise linear over 256 equal key intervals
 * (the key ranges of the level-4 quadtree cells), or a 1-16-1 monotone sigmoid MLP. */
typedef enum { SFC_ROOT_PWL = 0, SFC_ROOT_MLP = 1 } sfc_root;
/* Query window.  SFC_NORM_DISC: the closed disc (x - q_x)^2 + (y - q_y)^2 <= delta^2 of the
 * problem statement (Sec. 2).  SFC_NORM_SQUARE: the closed axis-parallel square
 * max(|x - q_x|, |y - q_y|) <= delta (side 2 delta + 1 grid points), the square windows of the
 * paper's experiments (Sec. 3, "Queries"). */
typedef enum { SFC_NORM_DISC = 0, SFC_NORM_SQUARE = 1 } sfc_norm;

/* Device status bits (sfc_device_status_bits). */
#define SFC_DEV_BAD_POINT   0x1u   /* a point coordinate outside [0, 2^30) */
#define SFC_DEV_BAD_QUERY   0x2u   /* a query centre outside the domain or a radius < 0 */
#define SFC_DEV_CAPACITY    0x4u   /* sfc_query_* output capacity exceeded */
#define SFC_DEV_TIMEOUT     0x8u   /* a look-back or work-queue wait hit its iteration limit */
#define SFC_DEV_NOT_FOUND   0x10u  /* sfc_update: delete of a non-live or duplicate id */

typedef struct sfc_index sfc_index;   /* opaque; owned by the library */

/* Device memory of an index from the caller's allocator instead of the library's.  With an
 * allocator given at build, every device buffer of that index -- the sorted arrays, the
 * learned model, the query and update workspaces, the staging buffers of the host-buffer
 * calls -- is requested from alloc(bytes, stream, ctx) and returned with free(ptr, stream,
 * ctx), both on the stream of the call that needs or drops the buffer (a cudaStream_t;
 * stream-ordered like cudaMallocAsync / cudaFreeAsync: the memory may be used by work
 * enqueued on that stream after alloc returns, and free may hand it to later work on that
 * stream).  alloc returns a device pointer on the index's device, aligned to at least 256
 * bytes, or NULL when it has no memory (the call then returns SFC_ERR_OOM).  The callbacks
 * run on the thread of the library call, never concurrently for one index, and not while a
 * stream is being captured once sfc_reserve has sized the index.  The struct is copied at
 * build; ctx must stay valid until sfc_destroy returns.  This lets a framework's caching
 * allocator (e.g. PyTorch's) own all of the index's memory.  A NULL allocator keeps the
 * library's own stream-ordered pool (cudaMallocAsync on the device's default pool).  Calls
 * that take no index (sfc_sort_pairs, sfc_exclusive_scan, the model-step calls) use the
 * pool. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* ctx);
    void (*free)(void* ptr, void* stream, void* ctx);
    void* ctx;
} sfc_allocator;

typedef struct {
    sfc_bounds bounds;      /* bound search used by queries (default SFC_BOUNDS_BINARY) */
    int leaves;             /* learned model: number of leaf segments (default 4096) */
    int train_steps;        /* learned model: Adam steps of the root (default 8) */
    int train_samples;      /* learned model: keys sampled for root training (default 16384) */
    float learning_rate;    /* learned model: Adam step size (default 0.02) */
    int chunk;              /* scan chunk in points (0 = autotuned/default 1024) */
    int mask_budget_mb;     /* cap on the hit-mask buffer of the two-pass scan, which is sized
                               1 KB per query (default cap 4096 MB) */
    int reorder_queries;    /* order in which queries are processed (outputs are unaffected):
                               0 input order, 1 curve order of the centres (queries that scan
                               overlapping ranges run together and share L2), 2 curve order once
                               the coordinates outgrow L2, n >= 2^24 (default 2) */
    int profile;            /* 1 = record per-step CUDA events from the start (sfc_profile_read) */
    sfc_root root;          /* learned model: root kind (default SFC_ROOT_PWL) */
    int cover_refine;       /* cover of each query's ball (outputs are unaffected): 0 the cells
                               of cells(Q) (Alg. 1, at most 4 cells of level l with
                               2 delta <= 2^l < 4 delta); 1 or 2 the cells of level l - 1 or
                               l - 2 (at most 9 or 25) that hold an integer point of the closed
                               ball, so fewer points are scanned for more key intervals; -1 the
                               choice of sfc_autotune (1 until it runs) (default 0) */
    int occupancy_depth;    /* early termination (Sec. 2.2): depth D of a quadtree over the
                               domain with one bit per node (the cell holds a point), built
                               with the index and after every sfc_update; queries drop the
                               cells of their cover that it shows empty (a cell deeper than D
                               answers for its depth-D ancestor).  0 = off, 1..13; D = 12 (the
                               paper's) takes 2.8 MB (default 0) */
    sfc_norm query_norm;    /* window of the queries (default SFC_NORM_DISC); sfc_set_query_norm */
} sfc_options;

/* Fills *opt with the defaults listed above. */
void sfc_default_options(sfc_options* opt);

/* ---------------------------------------------------------------------------------- */
/* Index construction (Sec. 2: "store P in an array sorted by pi(p)"; Sec. 3.1.1:      */
/* compute the keys and sort once).                                                     */
/* ---------------------------------------------------------------------------------- */

/* Builds an index over n points d_points (int32[n][2], device).  Keys of `curve`, then a
 * stable LSD radix sort of (key, id); the sorted coordinates are written alongside.
 * If opt->bounds is SFC_BOUNDS_LEARNED the learned model is trained as well.
 * n may be 0; n must be < 2^32 - 1.  opt NULL = the defaults.  alloc: the allocator of all
 * the index's device memory (see sfc_allocator), NULL = the library's pool.  *out receives
 * the new index (NULL on error).  Errors: SFC_ERR_INVALID (NULL out, n too large, unknown
 * curve, an allocator without both callbacks), SFC_ERR_OOM, SFC_ERR_CUDA.  Bad coordinates
 * set SFC_DEV_BAD_POINT (keys of such points are unspecified). */
sfc_status sfc_build(sfc_index** out, const int32_t* d_points, uint64_t n, sfc_curve curve,
                     const sfc_options* opt, const sfc_allocator* alloc, void* stream);

/* As sfc_build with the points in host memory (copied inside the call, into device memory
 * from the same allocator). */
sfc_status sfc_build_host(sfc_index** out, const int32_t* h_points, uint64_t n, sfc_curve curve,
                          const sfc_options* opt, const sfc_allocator* alloc, void* stream);

/* 3-D index (the paper's d-dimensional Z curve, Sec. 2.1, for d = 3): d_points int32[n][3]
 * with every coordinate in [0, 2^21); 63-bit keys (bit 3i = x_i, 3i + 1 = y_i, 3i + 2 = z_i);
 * cells(Q) has at most 2^3 = 8 cells.  The query calls (sfc_query_count / _write / _batch /
 * _batch_host, sfc_query_ranges, sfc_autotune, graphs, sfc_rebuild with int32[n][3] points)
 * take int32[m][3] centres on such an index and report the closed ball
 * dx^2 + dy^2 + dz^2 <= delta^2.  Covers: cover_refine 0 (cells(Q)) or 1 (the cells one level
 * finer that hold an integer point of the ball, at most 27), -1 tuned by sfc_autotune.
 * Static and with binary-search bounds only: opt->bounds must be SFC_BOUNDS_BINARY,
 * occupancy_depth 0, query_norm SFC_NORM_DISC, cover_refine -1..1 (else SFC_ERR_INVALID);
 * sfc_update, sfc_train_model, a learned bound search, cover 2 and square windows return
 * SFC_ERR_INVALID on it; queries run in input order. */
sfc_status sfc_build3(sfc_index** out, const int32_t* d_points, uint64_t n, const sfc_options* opt,
                      const sfc_allocator* alloc, void* stream);

/* As sfc_build3 with the points in host memory (copied inside the call). */
sfc_status sfc_build3_host(sfc_index** out, const int32_t* h_points, uint64_t n, const sfc_options* opt,
                           const sfc_allocator* alloc, void* stream);

/* 2 for indexes made by sfc_build / sfc_build_host, 3 for sfc_build3 / sfc_build3_host; 0 for
 * NULL. */
int sfc_index_dim(const sfc_index* idx);

/* Frees the index and everything it owns (stream-ordered on the stream of the last call;
 * memory from a caller's allocator goes back through its free callback). */
void sfc_destroy(sfc_index* idx);

/* Rebuilds the index in place over n new points (device), with the index's curve and
 * options: keys, sort, coordinates, the id table (ids restart at 0..n-1) and, if the index
 * uses learned bounds, a fresh model fit.  Reuses the index's buffers (they only grow), so
 * after sfc_reserve it allocates nothing.  Errors as sfc_build. */
sfc_status sfc_rebuild(sfc_index* idx, const int32_t* d_points, uint64_t n, void* stream);

/* As sfc_rebuild with the points in host memory (int32[n][2], or [n][3] for a 3-D index):
 * they are copied on the stream into a staging buffer that the index keeps (it only grows,
 * and it comes from the index's allocator), then the index is rebuilt from it.  Page-locked
 * h_points must stay unchanged until the stream has run the copy; pageable memory is copied
 * before the call returns.  Errors as sfc_rebuild. */
sfc_status sfc_rebuild_host(sfc_index* idx, const int32_t* h_points, uint64_t n, void* stream);

/* Sizes every buffer of the index for rebuilds of up to n_max points and query batches of up
 * to m_max queries, so that later sfc_rebuild / sfc_query_* calls allocate nothing (needed
 * before capturing them in a CUDA graph). */
sfc_status sfc_reserve(sfc_index* idx, uint64_t n_max, uint64_t m_max, void* stream);

/* ---------------------------------------------------------------------------------- */
/* CUDA graphs: the whole pipeline captured once, replayed with one launch.            */
/* ---------------------------------------------------------------------------------- */

typedef struct sfc_graph sfc_graph;   /* opaque; owned by the library */

#define SFC_GRAPH_REBUILD 0x1u   /* sfc_rebuild(d_points, n) (+ model fit if learned) */
#define SFC_GRAPH_QUERY   0x2u   /* sfc_query_batch(d_q, d_delta, m, offsets, ids, capacity) */

/* Captures the selected steps, with these exact pointers and sizes, into a CUDA graph (on a
 * private stream; `stream` orders the set-up work) and instantiates it.  Replays read the
 * buffers' contents at replay time, so new points or queries written into the same buffers
 * are answered by the next sfc_graph_launch.  Calls sfc_reserve(n, m) first.  The index must
 * outlive the graph and must not be used by other calls while a replay runs. */
sfc_status sfc_graph_capture(sfc_index* idx, unsigned flags, const int32_t* d_points, uint64_t n,
                             const int32_t* d_q, const int32_t* d_delta, uint64_t m,
                             uint64_t* d_out_offsets, uint32_t* d_out_ids, uint64_t ids_capacity,
                             sfc_graph** out, void* stream);

/* Replays a captured pipeline on `stream` (one graph launch). */
sfc_status sfc_graph_launch(sfc_graph* g, void* stream);

/* Frees the graph (not the index). */
void sfc_graph_destroy(sfc_graph* g);

/* ---------------------------------------------------------------------------------- */
/* Queries (Alg. 1 for a batch).                                                        */
/* ---------------------------------------------------------------------------------- */

/* Counting half of a query batch.  d_q: int32[m][2] centres, d_delta: int32[m] radii.
 * Writes d_out_offsets (uint64[m+1], device): out_offsets[i] is where query i's ids start,
 * out_offsets[m] the total.  Keeps the batch's plan in the index so that sfc_query_write
 * can emit the ids without redoing the search or the count.  Invalid queries (centre outside
 * the domain, radius < 0) report nothing and set SFC_DEV_BAD_QUERY. */
sfc_status sfc_query_count(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta,
                           uint64_t m, uint64_t* d_out_offsets, void* stream);

/* Writing half: must follow sfc_query_count on the same index with the same d_q, d_delta,
 * m and d_out_offsets (else SFC_ERR_STATE).  Writes the ids of query i to
 * d_out_ids[out_offsets[i] .. out_offsets[i+1]) in ascending (key, id) order.  Ids whose
 * slot is >= ids_capacity are not written and SFC_DEV_CAPACITY is set. */
sfc_status sfc_query_write(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta,
                           uint64_t m, const uint64_t* d_out_offsets, uint32_t* d_out_ids,
                           uint64_t ids_capacity, void* stream);

/* Both halves in one asynchronous call (capacity mode; capturable in a CUDA graph once
 * sfc_reserve_queries has sized the workspace for m). */
sfc_status sfc_query_batch(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta,
                           uint64_t m, uint64_t* d_out_offsets, uint32_t* d_out_ids,
                           uint64_t ids_capacity, void* stream);

/* Whole query batch with host buffers: copies h_q/h_delta in, runs the batch, copies
 * h_out_offsets (uint64[m+1]) and the ids back (staged in device memory; page-locked host
 * buffers copy fastest).  Past 32 MB of ids the write pass runs in 8 slices of the queries (by
 * input index) and each slice's ids go out on a second stream while the next slices are written.
 * Synchronises `stream`.  If the total exceeds ids_capacity, only h_out_offsets is written and
 * SFC_ERR_CAPACITY is returned. */
sfc_status sfc_query_batch_host(sfc_index* idx, const int32_t* h_q, const int32_t* h_delta,
                                uint64_t m, uint64_t* h_out_offsets, uint32_t* h_out_ids,
                                uint64_t ids_capacity, void* stream);

/* Pre-sizes the query workspace for batches of up to m queries, so that later query calls
 * allocate nothing (needed before capturing them in a CUDA graph). */
sfc_status sfc_reserve_queries(sfc_index* idx, uint64_t m, void* stream);

/* Autotuner: when the index was built with cover_refine = -1, first times whole batches
 * (count + write) under the covers 0, 1 and 2; then times the count pass (plan + scan + count)
 * of this query batch for chunk sizes {256, 512, 1024, 2048, 4096} points (threads-per-query
 * granularity of the scan), then the number of chunks taken per work-queue grab
 * {1, 2, 4, 8, 16}, then the queries per write-pass grab {1, 2, 4, 8, 16}, and keeps the
 * fastest in the index (results do not depend on them).  The choice is cached per (device,
 * curve, log2 n, log2 m, bound search, cover option) for later indexes; force != 0
 * re-measures.  Writes the choice to *h_chunk, *h_batch, *h_qbatch (any may be NULL); the
 * cover is read back with sfc_cover_refine.  Synchronises `stream`; allocates temporary
 * output buffers. */
sfc_status sfc_autotune(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta, uint64_t m, int force,
                        int* h_chunk, int* h_batch, int* h_qbatch, void* stream);

/* Sets the three scan settings that sfc_autotune chooses, without timing anything: the chunk
 * in points (32 ... 4096, a multiple of 32), the chunks per work-queue grab of the count pass
 * (batch) and the queries per grab of the write pass (qbatch), each 1 ... 1024; otherwise
 * SFC_ERR_INVALID and nothing changes.  Results do not depend on them, and a count already
 * made keeps its own chunk for its write.  For replaying a measured choice where timing it
 * again would give another (under a profiler, whose overhead changes the timings). */
sfc_status sfc_set_tuning(sfc_index* idx, int chunk, int batch, int qbatch);

/* Chooses the bound search of later queries.  SFC_BOUNDS_LEARNED requires a trained model
 * (sfc_train_model or opt->bounds at build), else SFC_ERR_STATE. */
sfc_status sfc_set_bounds_mode(sfc_index* idx, sfc_bounds mode);

/* Sets the cover of later queries (0, 1 or 2 as opt->cover_refine; else SFC_ERR_INVALID).
 * A count already made keeps its own cover for its write.  A captured query graph keeps the
 * cover it was captured with; reserve (sfc_reserve_queries) after a change to a finer cover,
 * since the per-query interval table grows with it. */
sfc_status sfc_set_cover(sfc_index* idx, int refine);

/* Copies the early-termination bitmap (opt->occupancy_depth > 0): node v of depth t (the cell
 * of level 30 - t whose key prefix, Def. 2.3, is v) is bit (4^t - 1) / 3 + v, bit b in word
 * b / 32 at position b % 32; ((4^(D+1) - 1) / 3 + 31) / 32 words in all.  d_out uint32[words]
 * in device memory; *h_depth receives D.  SFC_ERR_STATE when the index has no bitmap,
 * SFC_ERR_CAPACITY when words is too small (nothing copied). */
sfc_status sfc_get_occupancy(const sfc_index* idx, uint32_t* d_out, uint64_t words, int* h_depth,
                             void* stream);

/* Cover statistics of the last query batch: *h_cells the cells of all covers, *h_empty those
 * dropped as empty by the early-termination bitmap.  Synchronises `stream`. */
sfc_status sfc_query_cell_stats(const sfc_index* idx, uint64_t* h_cells, uint64_t* h_empty, void* stream);

/* Sets the window of later queries (SFC_NORM_DISC or SFC_NORM_SQUARE, else SFC_ERR_INVALID).
 * A count already made keeps its window for its write; a captured query graph keeps the window
 * it was captured with. */
sfc_status sfc_set_query_norm(sfc_index* idx, sfc_norm norm);

/* The cover currently used by queries (0, 1 or 2), or -1 for idx == NULL. */
int sfc_cover_refine(const sfc_index* idx);

/* Interval slots per query of the current cover: 4, 9 or 25 (3-D: 8 or 27; 0 for idx == NULL); the stride
 * of sfc_query_ranges' outputs. */
int sfc_query_max_intervals(const sfc_index* idx);

/* ---------------------------------------------------------------------------------- */
/* Learned bounds: two-stage CDF model replacing the search tree over the keys          */
/* (Sec. 2.1 "Storing P twice" uses a static B-tree; this library learns the CDF).      */
/* ---------------------------------------------------------------------------------- */

/* (Re)trains the model on the index's sorted keys: the root MLP by Adam on the GPU, then
 * the leaf least-squares lines and the exact per-leaf error windows. */
sfc_status sfc_train_model(sfc_index* idx, void* stream);

/* Number of MLP root hidden units H (the MLP root has 3H + 1 parameters: alpha[H], beta[H],
 * b[H], c; f(x) = c + sum_k exp(alpha_k) sigmoid(exp(beta_k) x + b_k)). */
int sfc_model_hidden(void);

/* Number of parameters of a root kind: MLP 3H + 1; piecewise linear K + 1 = 257, the knot
 * heights h_0 .. h_K of f(x) at x = k / K (kept non-decreasing: after every Adam step each
 * height is raised to the running maximum of those before it); -1 if unknown. */
int sfc_model_params(sfc_root root);

/* Mean-squared error of the root on samples (x = key / 2^60, target y) and its gradient, from
 * the training kernels run once with no update: h_params float[sfc_model_params(root)]
 * (host), d_keys uint64[s] (device), d_y float[s] (device).  Writes *h_loss and
 * h_grad float[sfc_model_params(root)] (host).  Synchronises `stream`. */
sfc_status sfc_model_loss_grad(sfc_root root, const float* h_params, const uint64_t* d_keys,
                               const float* d_y, uint64_t s, float* h_loss, float* h_grad,
                               void* stream);

/* One step of the device Adam optimiser (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected)
 * on host-given state of np parameters: updates h_params, h_m, h_v in place with gradient
 * h_grad at step t >= 1.  Synchronises. */
sfc_status sfc_model_adam_step(float* h_params, float* h_m, float* h_v, const float* h_grad, int np,
                               int t, float lr, void* stream);

/* Copies the trained model out (host): the root kind, its parameters
 * (float[sfc_model_params(kind)]); per leaf j < *h_leaves: first position, end position,
 * slope, intercept, err_lo, err_hi.  Any pointer may be NULL.  SFC_ERR_STATE if no model.
 * Synchronises. */
sfc_status sfc_model_get(const sfc_index* idx, int* h_root, float* h_params, int* h_leaves,
                         uint32_t* h_first, uint32_t* h_end, float* h_slope, float* h_icpt,
                         int32_t* h_err_lo, int32_t* h_err_hi, void* stream);

/* Copies the leaves' coarse fences out (host): uint64[*h_leaves][16], fence s of leaf j = the
 * key at position first_j + floor(s * (end_j - first_j) / 16) of the sorted array (all bits
 * set for a leaf without keys).  h_fence must hold leaves * 16 entries.  SFC_ERR_STATE if no
 * model.  Synchronises. */
sfc_status sfc_model_fence(const sfc_index* idx, uint64_t* h_fence, int* h_leaves, void* stream);

/* Copies the leaves' fine fences out (host): uint64[*h_leaves][256], fine fence key r of leaf j
 * = the key at position first_j + floor(r * (end_j - first_j) / 256) (all bits set for a leaf
 * without keys); coarse fence key s is fine fence key 16 s.  A learned search counts the fine
 * keys inside its error window that lie below the target, which brackets it between two fine
 * keys before the last-mile search.  h_fence must hold leaves * 256 entries.  SFC_ERR_STATE if
 * no model.  Synchronises. */
sfc_status sfc_model_fence_fine(const sfc_index* idx, uint64_t* h_fence, int* h_leaves, void* stream);

/* Work of the last query batch: points scanned (sum over queries of the interval lengths,
 * the S_q of Alg. 1's scan loop), scan chunks (queries that scan at most 64 points have none:
 * one thread scans each of them), and points reported.  Synchronises. */
sfc_status sfc_query_stats(const sfc_index* idx, uint64_t* h_scanned, uint64_t* h_chunks,
                           uint64_t* h_hits, void* stream);

/* Statistics of the last learned-bounds query batch: endpoints searched, endpoints whose
 * window missed (fell back to full binary search), and the sum of window lengths.
 * Synchronises. */
sfc_status sfc_model_stats(const sfc_index* idx, uint64_t* h_endpoints, uint64_t* h_misses,
                           uint64_t* h_window_sum, void* stream);

/* ---------------------------------------------------------------------------------- */
/* Dynamic setting (Sec. 2.1 "Dynamic implementation"; Sec. 3.3), batched.              */
/* ---------------------------------------------------------------------------------- */

/* Applies one batch: deletes d_delete_ids (uint32[k_del], device) first, then inserts
 * d_inserts (int32[k_ins][2], device) with ids first_new_id, first_new_id + 1, ...
 * (written to *h_first_new_id; ids are never reused).  The sorted arrays become those of a
 * rebuild from scratch over the live set; a trained model is refitted.  Synchronises
 * `stream` to validate the deletes: a delete of a non-live or repeated id returns
 * SFC_ERR_NOT_FOUND and changes nothing. */
sfc_status sfc_update(sfc_index* idx, const int32_t* d_inserts, uint64_t k_ins,
                      const uint32_t* d_delete_ids, uint64_t k_del, uint32_t* h_first_new_id,
                      void* stream);

/* ---------------------------------------------------------------------------------- */
/* Introspection and individual steps (used by the parity tests).                       */
/* ---------------------------------------------------------------------------------- */

/* Device views of the sorted arrays (owned by the index; valid until the next
 * sfc_update/sfc_destroy): keys uint64[n], ids uint32[n], coordinates int32[n][2] (a 3-D
 * index: int32[n][4] records x, y, z, 0). */
sfc_status sfc_get_sorted(const sfc_index* idx, const uint64_t** d_keys, const uint32_t** d_ids,
                          const int32_t** d_xy, uint64_t* n);

/* Synchronises `stream`, returns the device status word accumulated since the last call
 * in *h_bits (SFC_DEV_* bits) and clears it.  Returns the sfc_status of the most severe
 * bit (SFC_OK if none). */
sfc_status sfc_device_status(sfc_index* idx, uint32_t* h_bits, void* stream);

/* Curve keys of n points (Alg. 2 for Z; the Hilbert labelling of Sec. 2.1), device in/out. */
sfc_status sfc_keys(const int32_t* d_points, uint64_t n, sfc_curve curve, uint64_t* d_keys,
                    void* stream);

/* 3-D Z keys (uint64[n], device) of int32[n][3] device points. */
sfc_status sfc_keys3(const int32_t* d_points, uint64_t n, uint64_t* d_keys, void* stream);

/* Inverse of sfc_keys: coordinates of n keys (device in/out). */
sfc_status sfc_decode(const uint64_t* d_keys, uint64_t n, sfc_curve curve, int32_t* d_points,
                      void* stream);

/* Stable sort of (key, id) pairs by key with the library's onesweep radix sort: d_keys_in
 * uint64[n], d_ids_in uint32[n] (NULL = ids 0..n-1), outputs d_keys_out / d_ids_out
 * (must not alias the inputs).  Allocates and frees its own workspace on `stream`. */
sfc_status sfc_sort_pairs(const uint64_t* d_keys_in, const uint32_t* d_ids_in, uint64_t n,
                          uint64_t* d_keys_out, uint32_t* d_ids_out, void* stream);

/* Exclusive prefix sum of n uint32 into uint64[n+1] (the last entry is the total), with the
 * library's single-pass decoupled look-back scan.  Allocates and frees its own workspace on
 * `stream` and synchronises `stream`: returns SFC_ERR_TIMEOUT (output void) if a look-back
 * wait gave up. */
sfc_status sfc_exclusive_scan(const uint32_t* d_in, uint64_t n, uint64_t* d_out, void* stream);

/* sfc_exclusive_scan without any device allocation.  No counterpart in the paper: this is
 * for callers that must not allocate device memory, such as code whose device memory is all
 * owned by a caching pool of a host framework (an allocation from inside this library would
 * go around the pool and can fail once the pool holds the memory), or a latency-bound loop
 * that cannot take the implicit device synchronisation of cudaMalloc/cudaFree.  The call
 * only enqueues a memset and one kernel on `stream` and does not synchronise.
 * Scratch: a fixed 131 KB array in device memory of every device that loads the library,
 * held until the process exits; n may be at most 67,108,864 (16,384 tiles of 4,096),
 * larger n returns SFC_ERR_CAPACITY and enqueues nothing.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current, so make
 * that first call before capturing a stream into a CUDA graph; the address is looked up
 * again when the device's CUDA context was destroyed and created again (cudaDeviceReset).
 * All calls share the one array (it keeps the last call's words; each call clears what it
 * uses first), so calls that can overlap on the GPU -- on different streams, or different
 * host threads -- race and must be serialised by the caller.  Output: d_out uint64[n+1] as
 * sfc_exclusive_scan.  A look-back wait that gave up is recorded in the array's status word,
 * read by sfc_exclusive_scan_noalloc_status. */
sfc_status sfc_exclusive_scan_noalloc(const uint32_t* d_in, uint64_t n, uint64_t* d_out, void* stream);

/* Status of the most recent sfc_exclusive_scan_noalloc on the current device: synchronises
 * `stream` (the stream of that call, or one ordered after it), writes the status bits
 * (SFC_DEV_TIMEOUT if a look-back wait gave up and the output is void) to *h_bits (may be
 * NULL) and returns SFC_ERR_TIMEOUT in that case, else SFC_OK.  Allocates nothing; it reads
 * the shared array, so the same serialisation applies as to the scan itself. */
sfc_status sfc_exclusive_scan_noalloc_status(uint32_t* h_bits, void* stream);

/* Ranges and bounds of a query batch (Alg. 1, range derivation and bound search): for each
 * query i, the merged key intervals of its cover -- cells(Q), or the finer cover set by
 * cover_refine -- in K = sfc_query_max_intervals(idx) slots (d_lo/d_hi uint64[K m], slot
 * K i + r, unused slots lo = 1, hi = 0) and their array bounds by the index's current bound
 * search (d_begin/d_end uint32[K m]); d_count uint32[m] receives the number of intervals.
 * Any output may be NULL. */
sfc_status sfc_query_ranges(sfc_index* idx, const int32_t* d_q, const int32_t* d_delta,
                            uint64_t m, uint64_t* d_lo, uint64_t* d_hi, uint32_t* d_begin,
                            uint32_t* d_end, uint32_t* d_count, void* stream);

/* Opt-in timing of the library's steps with CUDA events recorded on the launching stream
 * around each step ("sort", "plan", "scan", "count", "write", "train", "update", ...).
 * Enabling costs two event records per step; leave it off inside CUDA-graph capture. */
typedef struct {
    char name[24];
    uint64_t launches;   /* times the step ran since the last reset */
    double ms;           /* summed device time of those runs */
} sfc_profile_entry;

sfc_status sfc_profile_enable(sfc_index* idx, int on);

/* Synchronises `stream`, aggregates the recorded steps by name into out[0..max) and
 * writes how many entries there are to *count; reset != 0 clears the records. */
sfc_status sfc_profile_read(sfc_index* idx, sfc_profile_entry* out, int max, int* count, int reset,
                            void* stream);

/* Number of this library's kernels launched by this process so far (host counter). */
uint64_t sfc_launch_count(void);

/* Device bytes this process's calls currently hold from the library's own stream-ordered
 * pool (host counter; memory from a caller's sfc_allocator is not counted). */
uint64_t sfc_pool_bytes_in_use(void);

/* Human-readable name of a status code. */
const char* sfc_status_string(sfc_status s);

#ifdef __cplusplus
}
#endif

#endif /* SFC_H */
