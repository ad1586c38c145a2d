// Batched distance query (Alg. 1 for m queries at once).
//
//   plan_kernel    one thread per query (in curve order of the centres when the queries are
//                  reordered): bounding square Q of B_delta(q), the level l with
//                  2 delta <= 2^l < 4 delta, the <= 4 cells of cells(Q) and their key
//                  intervals [pi(C)o0, pi(C)o1] (Observation) -- or, with a refined cover,
//                  the cells one or two levels finer (<= 9 / <= 25) that meet the window;
//                  cells the early-termination bitmap shows empty are dropped -- sorted and
//                  with abutting intervals merged, then lower_bound of both ends of every
//                  interval, by binary search or by the learned model (fence bracket and
//                  error window, verified, with fallback).  The query's scan length S_q is cut
//                  into chunks of C points; a query with S_q <= kSmallScan gets no chunks and
//                  goes onto the small-query list instead.  plan3_kernel does the same for 3-D
//                  points.
//   scan           exclusive scan of the chunk counts -> chunk bases.
//   count_kernel   persistent warps take batches of chunks from a counter (work stealing);
//                  a warp streams the chunk's coordinates, applies the exact window test
//                  (disc dx^2 + dy^2 <= delta^2 in int64, square, or 3-D ball), keeps the warp
//                  ballots as a hit bitmask (one bit per scanned point) and adds the chunk's
//                  popcount to the query's count.  Once the chunks are all claimed, the warps
//                  take the listed small queries, one thread per query, with the same test.
//   scan           exclusive scan of the per-query counts -> the caller's out_offsets.
//   write_kernel   persistent warps take batches of queries; a warp walks its query's
//                  chunks in order, reads the bitmask (or, past the bitmask budget, re-runs
//                  the filter) and writes the ids of the hits with ballot/popc compaction at
//                  out_offsets[q] + rank, so each query's ids come out in array order; then
//                  the small queries, one thread each, from their own masks.
//
// The bitmask makes the second pass read 1 bit instead of 8 bytes per scanned point.  In the
// two scan passes a warp keeps its query's intervals (array shift and end of each, in the
// concatenated order of the scan) in shared memory; a lane moves to the next interval only
// when its index crosses the current one's end.
#include "sfc_internal.cuh"
#include "query.cuh"

namespace sfc {

namespace {

constexpr int kThreads = 256;

// Binary searches in lock step per thread, and the plan kernel's resident blocks per SM (its
// register budget) for each bound search.
#ifndef SFC_BINARY_BATCH
#define SFC_BINARY_BATCH 8
#endif
#ifndef SFC_PLAN_BLOCKS_BINARY
#define SFC_PLAN_BLOCKS_BINARY 4
#endif
#ifndef SFC_PLAN_BLOCKS_LEARNED
#define SFC_PLAN_BLOCKS_LEARNED 4
#endif
#ifndef SFC_LEARNED_BATCH
#define SFC_LEARNED_BATCH 2
#endif
// Targets a warp searches per round: the flat list of its 32 queries' interval endpoints is
// searched in rounds of at most this many (one round for nearly every warp: cover 1 averages
// about 6.5 endpoints per query).  A multiple of 32.
#ifndef SFC_PLAN_CAP
#define SFC_PLAN_CAP 256
#endif
constexpr uint32_t kPlanCap = SFC_PLAN_CAP;

__device__ __forceinline__ bool query_valid(int32_t qx, int32_t qy, int32_t delta)
{
    return point_in_domain(qx, qy) && delta >= 0;
}

// ------------------------------------------------------------------------------------
// Bound search: K lower_bounds in lock step (independent loads in flight together)
// ------------------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void lower_bounds_window(const uint64_t* __restrict__ keys,
                                                    const uint64_t* t, uint32_t* lo,
                                                    uint32_t* len)
{
    // answer of search e lies in [lo[e], lo[e] + len[e]]
    while (true) {
        bool any = false;
#pragma unroll
        for (int e = 0; e < K; ++e) any |= len[e] > 0;
        if (!any) break;
#pragma unroll
        for (int e = 0; e < K; ++e) {
            if (len[e] > 0) {
                uint32_t half = len[e] >> 1;
                uint64_t k = __ldg(keys + lo[e] + half);
                bool right = k < t[e];
                lo[e] = right ? lo[e] + half + 1 : lo[e];
                len[e] = right ? len[e] - half - 1 : half;
            }
        }
    }
}

// E lower_bounds in lock step with one step count for all: the answer of search x lies in
// [base[x], base[x] + len] (the same len for every x, keys[base[x] .. base[x] + len) inside the
// array).  Each step halves len and moves a base past the probed key when that key is below
// the target (Khuong & Morin's branch-free search); the final probe decides between base and
// base + 1.  With one length there is no per-search bookkeeping: a step is an add, the load,
// the 64-bit compare and a select.
template <int E>
__device__ __forceinline__ void lower_bounds_uniform(const uint64_t* __restrict__ keys, const uint64_t* t,
                                                     uint32_t* base, uint32_t len)
{
    if (len == 0) return;
#pragma unroll 1
    while (len > 1) {
        const uint32_t half = len >> 1;
#pragma unroll
        for (int x = 0; x < E; ++x) base[x] = __ldg(keys + base[x] + half) < t[x] ? base[x] + half : base[x];
        len -= half;
    }
#pragma unroll
    for (int x = 0; x < E; ++x) base[x] += __ldg(keys + base[x]) < t[x] ? 1u : 0u;
}

// Per-thread counters of the learned search, summed once per block at the end of the plan.
struct BoundStats {
    unsigned long long endpoints = 0, misses = 0, window = 0;
};

// Bound search functors: lower_bound of t[0..ne) (ne <= E) into r[].
struct BinaryBounds {
    static constexpr bool kStats = false;
    static constexpr int kBatch = SFC_BINARY_BATCH;
    static constexpr bool kFenceSmem = false;
    static constexpr int kMinBlocks = SFC_PLAN_BLOCKS_BINARY;   // endpoints searched in lock step per thread
    __device__ __forceinline__ void prepare(RootParams*) {}
    template <int E>
    __device__ __forceinline__ void search(const uint64_t* keys, uint32_t n, const uint64_t* t, uint32_t* r,
                                           int ne, BoundStats&) const
    {
        uint32_t lo[E], len[E];
#pragma unroll
        for (int e = 0; e < E; ++e) { lo[e] = 0; len[e] = e < ne ? n : 0; }
        lower_bounds_window<E>(keys, t, lo, len);
#pragma unroll
        for (int e = 0; e < E; ++e) r[e] = lo[e];
    }
    // lower_bound over the whole array of the warp's flat list of T targets (each lane takes
    // targets lane, lane + 32, ...; kBatch of them in lock step); results in res
    __device__ __forceinline__ void search_flat(const uint64_t* keys, uint32_t n, const uint64_t* tg, uint32_t* res,
                                                uint32_t T, BoundStats&, uint64_t*) const
    {
        constexpr int E = kBatch;
#pragma unroll 1
        for (uint32_t e0 = lane_id(); e0 < T; e0 += 32 * E) {
            uint64_t t[E];
            uint32_t base[E];
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t e = e0 + 32 * x;
                t[x] = e < T ? tg[e] : 0;
                base[x] = 0;
            }
            lower_bounds_uniform<E>(keys, t, base, n);
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t e = e0 + 32 * x;
                if (e < T) res[e] = base[x];
            }
        }
    }
};

struct LearnedBounds {
    static constexpr bool kStats = true;
    static constexpr bool kFenceSmem = false;
    static constexpr int kBatch = SFC_LEARNED_BATCH;
    static constexpr int kMinBlocks = SFC_PLAN_BLOCKS_LEARNED;
    const RootParams* root;      // device; after prepare() the block's shared-memory copy
    const LeafParams* leaf;
    const uint64_t* fence;       // [leaves][kFence] coarse fence keys
    const uint64_t* fence_fine;  // [leaves][kFenceFine] fine fence keys
    unsigned long long* stats;   // [0] endpoints, [1] misses, [2] window sum
    // every thread of the block calls this, then the block synchronises
    __device__ __forceinline__ void prepare(RootParams* s)
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(root);
        uint32_t* dst = reinterpret_cast<uint32_t*>(s);
        for (unsigned i = threadIdx.x; i < sizeof(RootParams) / 4; i += blockDim.x) dst[i] = src[i];
        root = s;
    }
    // lower_bound over the whole array of the warp's flat list of T targets (each lane takes
    // targets lane, lane + 32, ...; kBatch of them in lock step); results in res.  Per target:
    //   1. the root routes it to leaf j (the keys below it lie in leaves before j, the keys
    //      above it in leaves after j, as the root is monotone);
    //   2. the leaf's line predicts its position p and the stored error window bounds it:
    //      lower_bound(t) lies in [a, b] = [p + err_lo, p + err_hi + 1] within the leaf;
    //   3. the window picks the slice of the leaf's fine fence (the keys at kFenceFine equally
    //      spaced positions of the leaf) that falls inside it, and counting the slice's keys
    //      below t brackets the target between two fence keys;
    //   4. the last-mile search runs over the bracket within the window (every search of a
    //      batch padded to the longest); an answer on the edge of its range is checked against
    //      the key beyond the edge, and a target whose window missed is searched over the whole
    //      array.
    __device__ __forceinline__ void search_flat(const uint64_t* keys, uint32_t n, const uint64_t* tg, uint32_t* res,
                                                uint32_t T, BoundStats& bs, uint64_t*) const
    {
        constexpr int E = kBatch;
#pragma unroll 1
        for (uint32_t e0 = lane_id(); e0 < T; e0 += 32 * E) {
            uint64_t t[E];
            uint32_t lo[E], len[E], fo[E];
            int ne = 0;
            uint32_t F = 0;   // longest fence slice of the batch
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t e = e0 + 32 * x;
                ne += e < T;
                t[x] = e < T ? tg[e] : 0;
                const uint32_t j = (uint32_t)route_leaf(*root, t[x]);
                const LeafParams lp = leaf[j];
                const int64_t p = leaf_predict(lp, t[x]);
                int64_t a = p + lp.err_lo, b = p + (int64_t)lp.err_hi + 1;
                a = min(max(a, (int64_t)lp.first), (int64_t)lp.end);
                b = min(max(b, a), (int64_t)lp.end);
                lo[x] = (uint32_t)a;
                len[x] = (uint32_t)(b - a);
                // fine fence entry r sits at position first + floor(r cnt / kFenceFine): the
                // entries at positions below a are below t, those above b are not, so only
                // entries [ra, rb) need counting; ra and rb from a float estimate widened by one
                // entry on each side (its error is far below one entry)
                const uint32_t cnt = lp.end - lp.first;
                uint32_t ra = 0, rb = 0;
                if (cnt) {
                    const float scale = __fdividef((float)kFenceFine, (float)cnt);
                    const float fa = (float)(uint32_t)(a - lp.first) * scale;
                    const float fbk = (float)(uint32_t)(b - lp.first + 1) * scale;
                    ra = (uint32_t)max((int)fa - 1, 0);
                    rb = (uint32_t)min((int)fbk + 2, kFenceFine);
                }
                fo[x] = j * kFenceFine + ra;
                F = max(F, rb - ra);
            }
            // count the slice's fence keys below t: branch-free, every slice padded to the
            // batch's longest, moved left where it would run past the leaf's fence (the entries
            // it takes in on the left are below t and are counted like the others)
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t r0 = fo[x] % kFenceFine;
                fo[x] -= r0 + F > kFenceFine ? r0 + F - kFenceFine : 0;
            }
            uint32_t c[E];
#pragma unroll
            for (int x = 0; x < E; ++x) c[x] = 0;
            if (F > 0) {
                uint32_t flen = F;
#pragma unroll 1
                while (flen > 1) {
                    const uint32_t half = flen >> 1;
#pragma unroll
                    for (int x = 0; x < E; ++x) c[x] = __ldg(fence_fine + fo[x] + c[x] + half) < t[x] ? c[x] + half : c[x];
                    flen -= half;
                }
#pragma unroll
                for (int x = 0; x < E; ++x) c[x] += __ldg(fence_fine + fo[x] + c[x]) < t[x] ? 1u : 0u;
            }
            uint32_t N = 0;
            unsigned long long wsum = 0;
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t j = fo[x] / kFenceFine;
                const uint64_t first = __ldg(&leaf[j].first), cnt = __ldg(&leaf[j].end) - first;
                // r fine keys below t: lower_bound(t) lies in [P(r - 1) + 1, P(r)], P(r) the
                // position of fine key r, P(kFenceFine) = end
                const uint32_t r = cnt ? fo[x] % kFenceFine + c[x] : 0u;
                const uint64_t bl = r == 0 ? first : first + ((uint64_t)(r - 1) * cnt) / kFenceFine + 1;
                const uint64_t bh = r == 0 ? first : (r == kFenceFine ? first + cnt : first + ((uint64_t)r * cnt) / kFenceFine);
                const uint64_t nl = max((uint64_t)lo[x], bl), nh = min((uint64_t)lo[x] + len[x], bh);
                if (nl <= nh) {
                    lo[x] = (uint32_t)nl;
                    len[x] = (uint32_t)(nh - nl);
                } else {   // both hold lower_bound(t) unless the window is off: keep the bracket
                    lo[x] = (uint32_t)bl;
                    len[x] = (uint32_t)(bh - bl);
                }
                if (e0 + 32 * x < T) wsum += len[x];
                N = max(N, len[x]);
            }
            // pad every range to the longest: [lo, lo + N) still holds the answer, moved left
            // where it would run past the end of the array
            uint32_t lo0[E];
#pragma unroll
            for (int x = 0; x < E; ++x) {
                lo[x] = (uint64_t)lo[x] + N > n ? n - N : lo[x];
                lo0[x] = lo[x];
            }
            lower_bounds_uniform<E>(keys, t, lo, N);
            // an answer strictly inside its range has both neighbours in it, compared by the
            // search; on an edge, the key beyond the edge decides
            uint32_t miss = 0;
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t r = lo[x];
                bool ok = true;
                if (r == lo0[x] && r > 0) ok = __ldg(keys + r - 1) < t[x];
                if (r == lo0[x] + N && r < n) ok = ok && __ldg(keys + r) >= t[x];
                if (!ok && e0 + 32 * x < T) miss |= 1u << x;
            }
            if (miss) {
                uint32_t r2[E];
#pragma unroll
                for (int x = 0; x < E; ++x) r2[x] = 0;
                lower_bounds_uniform<E>(keys, t, r2, n);
#pragma unroll
                for (int x = 0; x < E; ++x) lo[x] = (miss >> x) & 1u ? r2[x] : lo[x];
            }
#pragma unroll
            for (int x = 0; x < E; ++x) {
                const uint32_t e = e0 + 32 * x;
                if (e < T) res[e] = lo[x];
            }
            bs.endpoints += ne;
            bs.misses += __popc(miss);
            bs.window += wsum;
        }
    }
};

// Inclusive prefix sum over the warp (every lane calls).
__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t v)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane >= o) v += t;
    }
    return v;
}

// Sum of v over the warp (every lane calls), returned to every lane.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ------------------------------------------------------------------------------------
// plan_kernel: range derivation and bound search, one thread per query
// ------------------------------------------------------------------------------------
template <int DROP>
struct Cover {
    // cells per axis at most: 2 for cells(Q) (2 delta <= 2^l), 2^DROP + 1 one or two levels finer
    static constexpr int NX = DROP == 0 ? 2 : (1 << DROP) + 1;
    static constexpr int K = NX * NX;   // 4, 9, 25 interval slots per query
};

// Early termination (Sec. 2.2): whether the cell of level l whose key interval starts at c may
// hold a point -- the bit of its own node when the node is within depth D, else of its
// ancestor at depth D.
__device__ __forceinline__ bool cell_occupied(const uint32_t* __restrict__ occ, int D, int l, uint64_t c)
{
    const int t = min(kOmega - l, D);
    const uint64_t b = occupancy_level_start(t) + (c >> (2 * (kOmega - t)));
    return (__ldg(occ + (b >> 5)) >> (b & 31)) & 1u;
}

// The cells of the cover, each as the key of its first point (its key interval is [c, c | span],
// Observation; every cell of a cover has the same level), sorted ascending into the thread's
// column col[0], col[stride], ... of shared memory; returns how many; *span_out = 4^l - 1.
// DROP 0: cells(Q), the cells of level l (2 delta <= 2^l < 4 delta, capped at omega) that meet
// the clipped square Q.  DROP > 0: the cells of level max(0, l - DROP) that hold an integer
// point of the closed ball (the distance from q to the cell's nearest integer point is at most
// delta; for the square window every cell meeting Q qualifies).  With the early-termination
// bitmap (occ != NULL), cells it shows empty are dropped; ncell / nempty count the cover's
// cells and the dropped ones.
template <int DROP>
__device__ __forceinline__ int derive_cells(int curve, int norm, const HilbertTables* tb, int32_t qx, int32_t qy,
                                            int32_t delta, const uint32_t* occ, int D, uint64_t* col, int stride,
                                            uint64_t* span_out, uint32_t& ncell, uint32_t& nempty)
{
    constexpr int K = Cover<DROP>::K;
    const int64_t d = delta;
    const int64_t x0 = max((int64_t)0, (int64_t)qx - d), x1 = min((int64_t)kSide - 1, (int64_t)qx + d);
    const int64_t y0 = max((int64_t)0, (int64_t)qy - d), y1 = min((int64_t)kSide - 1, (int64_t)qy + d);
    int l = 0;
    if (d > 0) {
        l = 64 - __clzll((unsigned long long)(2 * d - 1));   // bit length of 2 delta - 1
        if (l > kOmega) l = kOmega;
    }
    l = max(0, l - DROP);
    const uint64_t span = (l >= kOmega) ? kKeyMax : ((1ull << (2 * l)) - 1);
    *span_out = span;
    constexpr int NX = Cover<DROP>::NX;   // cells per axis at most
    const int64_t cx0 = x0 >> l, cy0 = y0 >> l;
    const int nx = (int)min((int64_t)NX, (x1 >> l) - cx0 + 1), ny = (int)min((int64_t)NX, (y1 >> l) - cy0 + 1);
    // per column: the squared distance from q to the column's nearest x and, for the Z curve,
    // the spread bits of its first x (the key of cell (cx, cy) is spread(cx 2^l) | spread(cy 2^l) << 1)
    int64_t dx2[NX];
    uint64_t sx[NX];
#pragma unroll
    for (int ix = 0; ix < NX; ++ix) {
        const int64_t cx = cx0 + ix;
        const int64_t ax0 = cx << l, ax1 = ((cx + 1) << l) - 1;
        const int64_t dx = qx < ax0 ? ax0 - qx : (qx > ax1 ? qx - ax1 : 0);
        dx2[ix] = dx * dx;
        sx[ix] = curve == SFC_CURVE_Z ? spread_bits((uint32_t)(cx << l)) : 0;
    }
    const int64_t d2 = d * d;
    int cnt = 0;
#pragma unroll
    for (int iy = 0; iy < NX; ++iy) {
        if (iy >= ny) break;
        const int64_t cy = cy0 + iy;
        const int64_t ay0 = cy << l, ay1 = ((cy + 1) << l) - 1;
        const int64_t dy = qy < ay0 ? ay0 - qy : (qy > ay1 ? qy - ay1 : 0);
        const int64_t dy2 = dy * dy;
        const uint64_t sy = curve == SFC_CURVE_Z ? spread_bits((uint32_t)(cy << l)) << 1 : 0;
#pragma unroll
        for (int ix = 0; ix < NX; ++ix) {
            if (ix >= nx) break;
            // every cell meeting Q meets a square window; a disc needs an integer point of the
            // ball in the cell
            if (DROP > 0 && norm == SFC_NORM_DISC && dx2[ix] + dy2 > d2) continue;
            const uint64_t c = (curve == SFC_CURVE_Z ? (sx[ix] | sy)
                                                     : hilbert_key(tb, (uint32_t)((cx0 + ix) << l), (uint32_t)(cy << l))) &
                               ~span;
            ++ncell;
            if (occ && !cell_occupied(occ, D, l, c)) {
                ++nempty;
                continue;
            }
            int j = cnt;
            while (j > 0 && col[(j - 1) * stride] > c) {
                col[j * stride] = col[(j - 1) * stride];
                --j;
            }
            col[j * stride] = c;
            ++cnt;
        }
    }
    return cnt;
}

// Visits the endpoints of the merged key intervals of nc sorted cells (cells whose intervals
// abut in key order form one interval: the scan over them is identical): endpoint 2k is the
// first key of interval k, endpoint 2k + 1 one past its last key (the interval's array range is
// [lower_bound(first key), lower_bound(last key + 1))).  fn(ep, key) in order.
template <class F>
__device__ __forceinline__ void for_each_endpoint(const uint64_t* col, int stride, int nc, uint64_t span, F&& fn)
{
    uint32_t ep = 0;
    uint64_t prev_end = 0;
    for (int k = 0; k < nc; ++k) {
        const uint64_t c = col[k * stride];
        if (k == 0 || c != prev_end) fn(ep++, c);                           // an interval starts
        prev_end = c + span + 1;
        if (k + 1 == nc || col[(k + 1) * stride] != prev_end) fn(ep++, prev_end);   // ... and ends
    }
}

// Appends query i to a list (counter work_ctr[ctr]) where flag is set; one atomic per warp.
// Every lane of the warp calls.
__device__ __forceinline__ void list_append(const QueryArgs& a, bool flag, uint64_t i, int ctr, uint32_t* list)
{
    const uint32_t mask = __ballot_sync(0xffffffffu, flag);
    if (!mask) return;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(a.work_ctr + ctr, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (flag) list[base + __popc(mask & lanemask_lt())] = (uint32_t)i;
}

// Lists query i as small (it scans at most kSmallScan points) for the thread-per-query kernels,
// or as a candidate big query (at least kBigChunks chunks) for the write pass.
__device__ __forceinline__ void plan_lists(const QueryArgs& a, bool active, uint32_t S, uint64_t i)
{
    if (a.small_list) list_append(a, active && S > 0 && S <= kSmallScan, i, kCtrSmallSize, a.small_list);
    if (a.big_list)
        list_append(a, active && S > kSmallScan && (uint64_t)S > (kBigChunks - 1) * a.chunk, i, kCtrBigList,
                    a.big_list);
}

// Optional outputs of the plan (the ranges export); null in the query path.
struct PlanExport {
    uint64_t* lo;
    uint64_t* hi;
    uint32_t* b;
    uint32_t* e;
    uint32_t* cnt;
};


// Dynamic shared memory of plan_kernel<Bounds, DROP, ..>: each thread's column of K cell keys
// (column-major, so that the lanes of a warp touch consecutive words), then per warp the flat
// target list (kPlanCap keys) and its results (kPlanCap positions), and for the learned search
// per warp one leaf's fine fence (kFenceFine keys).
template <class Bounds, int DROP>
constexpr size_t plan_smem_bytes()
{
    return (size_t)Cover<DROP>::K * kThreads * sizeof(uint64_t) +
           (size_t)(kThreads / 32) * kPlanCap * (sizeof(uint64_t) + sizeof(uint32_t)) +
           (Bounds::kFenceSmem ? (size_t)(kThreads / 32) * kFenceFine * sizeof(uint64_t) : 0);
}

// One thread per query for the range derivation: the cells of its cover, sorted, in shared
// memory.  The bound search runs on the warp's endpoints as one flat list in shared memory:
// lane L's query owns list positions [off_L, off_L + 2 cnt_L), the lanes take the list
// round-robin, so every lane searches about the same number of endpoints whatever the spread
// of interval counts over the warp's queries.  Then each thread writes its query's intervals'
// (begin, end) to slots 0.. of its K slots (unused slots (0, 0)), the number of chunks of its
// scan, and adds to the scanned total.  Nothing per query lives in local memory.
template <class Bounds, int DROP, bool EXPORT>
__global__ void __launch_bounds__(kThreads, Bounds::kMinBlocks) plan_kernel(QueryArgs a, Bounds bounds_in, PlanExport ex)
{
    constexpr int K = Cover<DROP>::K;
    __shared__ HilbertTables tb;
    __shared__ RootParams s_root;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    uint64_t* col = reinterpret_cast<uint64_t*>(s_dyn) + threadIdx.x;
    const unsigned warp = threadIdx.x >> 5;
    uint64_t* tg = reinterpret_cast<uint64_t*>(s_dyn) + (size_t)K * kThreads + (size_t)warp * kPlanCap;
    uint32_t* res = reinterpret_cast<uint32_t*>(reinterpret_cast<uint64_t*>(s_dyn) + (size_t)K * kThreads +
                                                (size_t)(kThreads / 32) * kPlanCap) + (size_t)warp * kPlanCap;
    uint64_t* sf = reinterpret_cast<uint64_t*>(s_dyn + (size_t)K * kThreads * sizeof(uint64_t) +
                                               (size_t)(kThreads / 32) * kPlanCap * (sizeof(uint64_t) + sizeof(uint32_t))) +
                   (size_t)warp * kFenceFine;
    Bounds bounds = bounds_in;
    bounds.prepare(&s_root);
    __syncthreads();
    if (a.curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);   // ends with a block barrier
    // thread r takes the query of processing rank r (curve order of the centres when a
    // processing order is given: neighbouring threads then search neighbouring keys)
    const uint64_t r = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = r < a.m;
    const uint64_t i = active && a.perm ? (uint64_t)__ldg(a.perm + r) : r;
    int2 q = make_int2(0, 0);
    int32_t delta = -1;
    if (active) {
        q = __ldg(reinterpret_cast<const int2*>(a.q) + i);
        delta = __ldg(a.delta + i);
    }
    const bool ok = active && query_valid(q.x, q.y, delta);
    if (active && !ok) set_status(a.status, SFC_DEV_BAD_QUERY);
    BoundStats bs;
    uint32_t ncell = 0, nempty = 0;
    uint64_t span = 0;
    const int nc = ok ? derive_cells<DROP>(a.curve, a.norm, &tb, q.x, q.y, delta, a.occ, a.occ_depth, col, kThreads,
                                           &span, ncell, nempty)
                      : 0;
    uint32_t cnt = 0;   // merged intervals
    for_each_endpoint(col, kThreads, nc, span, [&](uint32_t ep, uint64_t) { cnt += ep & 1u; });
    const uint32_t ne = 2u * cnt;
    const uint32_t incl = warp_incl_scan_u32(ne);
    const uint32_t off = incl - ne;
    const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    uint2* rp = (!EXPORT && active) ? reinterpret_cast<uint2*>(a.ranges + (uint64_t)2 * K * i) : nullptr;
    uint64_t S = 0;   // sum of e_k - b_k, gathered endpoint by endpoint
#pragma unroll 1
    for (uint32_t r0 = 0; r0 < T; r0 += kPlanCap) {   // warp-uniform
        const uint32_t r1 = min(T, r0 + kPlanCap);
        for_each_endpoint(col, kThreads, nc, span, [&](uint32_t ep, uint64_t key) {
            const uint32_t f = off + ep;
            if (f >= r0 && f < r1) tg[f - r0] = key;
        });
        __syncwarp();
        bounds.search_flat(a.keys, a.n, tg, res, r1 - r0, bs, sf);
        __syncwarp();
        const uint32_t f0 = max(off, r0), f1 = min(off + ne, r1);
        for (uint32_t f = f0; f < f1; ++f) {
            const uint32_t ep = f - off, k = ep >> 1;
            const uint32_t pos = res[f - r0];
            S += (ep & 1u) ? (uint64_t)pos : (uint64_t)0 - pos;
            if (!EXPORT) {
                if (rp) reinterpret_cast<uint32_t*>(rp + k)[ep & 1u] = pos;
            } else {
                const uint64_t o = (uint64_t)K * i + k;
                const uint64_t key = tg[f - r0];
                if (ep & 1u) {
                    if (ex.hi) ex.hi[o] = key - 1;
                    if (ex.e) ex.e[o] = pos;
                } else {
                    if (ex.lo) ex.lo[o] = key;
                    if (ex.b) ex.b[o] = pos;
                }
            }
        }
        __syncwarp();   // read before the next round's targets overwrite the list
    }
    // warp totals of the statistics: one atomic per warp and counter, no block barrier (a warp
    // that is done leaves without waiting for the rest of its block)
    if (a.scanned) {
        const unsigned long long t = warp_sum_u64(S);
        if (lane_id() == 0 && t) atomicAdd(a.scanned, t);
    }
    if (a.cells) {
        const unsigned long long tc = warp_sum_u64(ncell), te = warp_sum_u64(nempty);
        if (lane_id() == 0 && tc) {
            atomicAdd(a.cells, tc);
            if (te) atomicAdd(a.cells + 1, te);
        }
    }
    if constexpr (Bounds::kStats) {
        if (bounds.stats) {
            const unsigned long long te = warp_sum_u64(bs.endpoints);
            const unsigned long long tm = warp_sum_u64(bs.misses);
            const unsigned long long tw = warp_sum_u64(bs.window);
            if (lane_id() == 0 && te) {
                atomicAdd(bounds.stats + 0, te);
                if (tm) atomicAdd(bounds.stats + 1, tm);
                atomicAdd(bounds.stats + 2, tw);
            }
        }
    }
    const bool small = !EXPORT && a.small_list && active && S > 0 && S <= kSmallScan;
    if (!EXPORT) plan_lists(a, active, S, i);
    if (!active) return;
    if (!EXPORT) {
        for (uint32_t k = cnt; k < (uint32_t)K; ++k) rp[k] = make_uint2(0u, 0u);
        a.nchunks[i] = small ? 0u : (uint32_t)((S + a.chunk - 1) / a.chunk);
    } else {
        for (uint32_t k = cnt; k < (uint32_t)K; ++k) {
            const uint64_t o = (uint64_t)K * i + k;
            if (ex.lo) ex.lo[o] = 1;
            if (ex.hi) ex.hi[o] = 0;
            if (ex.b) ex.b[o] = 0;
            if (ex.e) ex.e[o] = 0;
        }
        if (ex.cnt) ex.cnt[i] = cnt;
    }
}

// ------------------------------------------------------------------------------------
// plan3_kernel: the same for 3-D points (Z curve in Z^3, binary bound search)
// ------------------------------------------------------------------------------------
// cells(Q) in 3-D: at most two cells per axis, 8 in all; one level finer, at most 3 per axis
template <int DROP>
struct Cover3 {
    static constexpr int NX = DROP == 0 ? 2 : 3;
    static constexpr int K = NX * NX * NX;
};

// DROP 0: cells(Q) in 3-D, the cells of level l (2 delta <= 2^l < 4 delta, capped at 21)
// meeting the clipped cube Q.  DROP 1: the cells of level max(0, l - 1) holding an integer
// point of the closed ball.  Key intervals of length 8^l, sorted, abutting ones merged.
template <int DROP>
__device__ __forceinline__ int derive_ranges3(int32_t qx, int32_t qy, int32_t qz, int32_t delta, uint64_t* lo,
                                              uint64_t* hi)
{
    constexpr int K = Cover3<DROP>::K;
    const int64_t d = delta;
    const int64_t c[3] = {qx, qy, qz};
    int64_t a0[3], a1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a0[k] = max((int64_t)0, c[k] - d);
        a1[k] = min((int64_t)kSide3 - 1, c[k] + d);
    }
    int l = 0;
    if (d > 0) {
        l = 64 - __clzll((unsigned long long)(2 * d - 1));
        if (l > kOmega3) l = kOmega3;
    }
    l = max(0, l - DROP);
    const uint64_t span = (1ull << (3 * l)) - 1;   // 3 l <= 63
    int cnt = 0;
    for (int64_t cz = a0[2] >> l; cz <= (a1[2] >> l); ++cz)
        for (int64_t cy = a0[1] >> l; cy <= (a1[1] >> l); ++cy)
            for (int64_t cx = a0[0] >> l; cx <= (a1[0] >> l); ++cx) {
                if (DROP > 0) {
                    const int64_t cc[3] = {cx, cy, cz};
                    int64_t dist2 = 0;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int64_t b0 = cc[k] << l, b1 = ((cc[k] + 1) << l) - 1;
                        const int64_t e = c[k] < b0 ? b0 - c[k] : (c[k] > b1 ? c[k] - b1 : 0);
                        dist2 += e * e;
                    }
                    if (dist2 > d * d) continue;
                }
                if (cnt == K) break;   // unreachable: at most Cover3<DROP>::NX cells per axis
                const uint64_t k0 = morton3_key((uint32_t)(cx << l), (uint32_t)(cy << l), (uint32_t)(cz << l)) & ~span;
                int j = cnt;
                while (j > 0 && lo[j - 1] > k0) { lo[j] = lo[j - 1]; hi[j] = hi[j - 1]; --j; }
                lo[j] = k0;
                hi[j] = k0 | span;
                ++cnt;
            }
    int m = 0;
    for (int i = 0; i < cnt; ++i) {
        if (m > 0 && hi[m - 1] + 1 == lo[i]) {
            hi[m - 1] = hi[i];
        } else {
            lo[m] = lo[i];
            hi[m] = hi[i];
            ++m;
        }
    }
    return m;
}

template <int DROP, bool EXPORT>
__global__ void __launch_bounds__(kThreads, 4) plan3_kernel(QueryArgs a, PlanExport ex)
{
    constexpr int kCells3 = Cover3<DROP>::K;
    constexpr int NB = (2 * kCells3 + 7) / 8;
    const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = i < a.m;
    int32_t qx = 0, qy = 0, qz = 0, delta = -1;
    if (active) {
        qx = __ldg(a.q + 3 * i);
        qy = __ldg(a.q + 3 * i + 1);
        qz = __ldg(a.q + 3 * i + 2);
        delta = __ldg(a.delta + i);
    }
    const bool ok = active && point3_in_domain(qx, qy, qz) && delta >= 0;
    if (active && !ok) set_status(a.status, SFC_DEV_BAD_QUERY);
    uint64_t lo[kCells3], hi[kCells3];
    uint32_t b[kCells3], e[kCells3];
    const int cnt = ok ? derive_ranges3<DROP>(qx, qy, qz, delta, lo, hi) : 0;
    BoundStats bs;
    const BinaryBounds bounds{};
#pragma unroll 1
    for (int bi = 0; bi < NB && 8 * bi < 2 * cnt; ++bi) {
        uint64_t t[8];
        uint32_t r[8];
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int ep = 8 * bi + x;
            t[x] = ep < 2 * cnt ? ((ep & 1) ? hi[ep >> 1] + 1 : lo[ep >> 1]) : 0;
        }
        bounds.search<8>(a.keys, a.n, t, r, min(2 * cnt - 8 * bi, 8), bs);
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int ep = 8 * bi + x;
            if (ep < 2 * cnt) {
                if (ep & 1) e[ep >> 1] = r[x];
                else b[ep >> 1] = r[x];
            }
        }
    }
    uint64_t S = 0;
    for (int k = 0; k < cnt; ++k) S += e[k] - b[k];
    if (!EXPORT) {   // statistics: one atomic per warp and counter
        const unsigned long long ts = warp_sum_u64(S), tc = warp_sum_u64((unsigned long long)cnt);
        if (lane_id() == 0) {
            if (a.scanned && ts) atomicAdd(a.scanned, ts);
            if (a.cells && tc) atomicAdd(a.cells, tc);
        }
    }
    const bool small = !EXPORT && a.small_list && active && S > 0 && S <= kSmallScan;
    if (!EXPORT) plan_lists(a, active, S, i);
    if (!active) return;
    if (!EXPORT) {
        uint2* rp = reinterpret_cast<uint2*>(a.ranges + (uint64_t)2 * kCells3 * i);
#pragma unroll
        for (int k = 0; k < kCells3; ++k) rp[k] = k < cnt ? make_uint2(b[k], e[k]) : make_uint2(0u, 0u);
        a.nchunks[i] = small ? 0u : (uint32_t)((S + a.chunk - 1) / a.chunk);
    } else {
        for (int k = 0; k < kCells3; ++k) {
            const bool u = k < cnt;
            const uint64_t o = (uint64_t)kCells3 * i + k;
            if (ex.lo) ex.lo[o] = u ? lo[k] : 1;
            if (ex.hi) ex.hi[o] = u ? hi[k] : 0;
            if (ex.b) ex.b[o] = u ? b[k] : 0;
            if (ex.e) ex.e[o] = u ? e[k] : 0;
        }
        if (ex.cnt) ex.cnt[i] = (uint32_t)cnt;
    }
}

// ------------------------------------------------------------------------------------
// Shared helpers of the two scan passes
// ------------------------------------------------------------------------------------
constexpr int kMaxInt = 27;   // intervals per query at the finest cover (3-D, one level finer)

// One query's intervals in the concatenated order of its scan (per-warp shared memory):
// array position = concatenated index + shift[r] for indices below end[r].
struct WarpTab {
    uint32_t shift[kMaxInt];
    uint32_t end[kMaxInt];
};

struct QView {
    uint32_t S;      // concatenated length (sum of the interval lengths)
    uint32_t nint;   // intervals stored per query
    int2 q;
    int32_t qz;      // third coordinate of 3-D queries
    int32_t d;       // delta
    int64_t d2;      // -(delta^2 + 1): a point is inside iff dx^2 + dy^2 + d2 < 0
};

// Loads query qi's intervals into the warp's table (lane r takes interval r); every lane calls.
__device__ __forceinline__ QView load_query(const QueryArgs& a, uint64_t qi, WarpTab* tab)
{
    QView v;
    const unsigned lane = lane_id();
    uint32_t b = 0, len = 0;
    if (lane < a.kint) {
        const uint2 r = __ldg(reinterpret_cast<const uint2*>(a.ranges) + qi * a.kint + lane);
        b = r.x;
        len = r.y - r.x;
    }
    const uint32_t incl = warp_incl_scan_u32(len);
    __syncwarp();   // the previous query's table is no longer read
    if (lane < a.kint) {
        tab->shift[lane] = b - (incl - len);
        tab->end[lane] = incl;
    }
    __syncwarp();
    v.S = __shfl_sync(0xffffffffu, incl, 31);
    v.nint = a.kint;
    if (a.dim == 3) {
        v.q = make_int2(__ldg(a.q + 3 * qi), __ldg(a.q + 3 * qi + 1));
        v.qz = __ldg(a.q + 3 * qi + 2);
    } else {
        v.q = __ldg(reinterpret_cast<const int2*>(a.q) + qi);
        v.qz = 0;
    }
    v.d = __ldg(a.delta + qi);
    v.d2 = -((int64_t)v.d * v.d + 1);
    return v;
}

// Moves a lane's interval cursor r forward to the interval holding concatenated index f.
__device__ __forceinline__ void seek(const WarpTab* tab, uint32_t nint, uint32_t f, uint32_t& r, uint32_t& shift,
                                     uint32_t& end)
{
    while (r + 1 < nint && f >= tab->end[r]) ++r;
    shift = tab->shift[r];
    end = tab->end[r];
}

// The scans are specialised by geometry: the 2-D disc, the 2-D square window, and the 3-D
// ball (points stored as 16-byte int4 records).
constexpr int kGeomDisc = SFC_NORM_DISC;
constexpr int kGeomSquare = SFC_NORM_SQUARE;
constexpr int kGeomBall3 = 2;

template <int GEOM>
struct Geom {
    using P = int2;
    static __device__ __forceinline__ const P* points(const QueryArgs& a) { return a.xy; }
    static __device__ __forceinline__ P zero() { return make_int2(0, 0); }
};
template <>
struct Geom<kGeomBall3> {
    using P = int4;
    static __device__ __forceinline__ const P* points(const QueryArgs& a) { return a.xyz; }
    static __device__ __forceinline__ P zero() { return make_int4(0, 0, 0, 0); }
};

// Exact window tests.  Disc (the problem statement's closed ball): |dx|, |dy| < 2^30, so each
// square is one signed 32x32 -> 64-bit multiply-add and the sum stays below 2^61; the test
// dx^2 + dy^2 <= delta^2 is taken as the sign of dx^2 + dy^2 - (delta^2 + 1), read from the
// high word alone (delta^2 + 1 <= 2^62, so nothing overflows).  Square (the experiments'
// windows): max(|dx|, |dy|) <= delta in 32-bit integers.  3-D ball: |dx|, |dy|, |dz| < 2^21,
// the sum of squares stays below 2^44, the same sign test.
template <int GEOM>
__device__ __forceinline__ bool is_hit(const QView& v, int2 p)
{
    const int dx = p.x - v.q.x, dy = p.y - v.q.y;
    if (GEOM == kGeomSquare) return max(abs(dx), abs(dy)) <= v.d;
    const long long s = (long long)dx * dx + ((long long)dy * dy + v.d2);
    return (int)(s >> 32) < 0;
}

template <int GEOM>
__device__ __forceinline__ bool is_hit(const QView& v, int4 p)
{
    const int dx = p.x - v.q.x, dy = p.y - v.q.y, dz = p.z - v.qz;
    const long long s = (long long)dx * dx + ((long long)dy * dy + ((long long)dz * dz + v.d2));
    return (int)(s >> 32) < 0;
}

// Filters points [s0, s1) of the query's concatenated intervals; returns the hit count and
// leaves word w (the ballot of points s0 + 32w ...) in lane w % 32, slot w / 32.  Lane 0 keeps
// each step's four ballots in the warp's word buffer sw (WPL x 32 words, one 16-byte store),
// and every lane reads its own words back at the end.  Points go in groups of 4 x 32: when the
// whole group lies inside the chunk and no lane crosses the end of its interval (one vote), the
// group runs without per-point guards; otherwise each point is checked and the lane looks its
// interval up again when it crosses into the next one.
template <int WPL, int GEOM>
__device__ __forceinline__ uint32_t filter_chunk(const QueryArgs& a, const QView& v, const WarpTab* tab,
                                                 uint32_t s0, uint32_t s1, uint32_t (&words)[WPL],
                                                 uint32_t* __restrict__ sw)
{
    const uint32_t nit = (s1 - s0 + 31) >> 5;
    __syncwarp();   // the previous chunk's words have been read
    using P = typename Geom<GEOM>::P;
    const P* __restrict__ xy = Geom<GEOM>::points(a);
    uint32_t f = s0 + lane_id();
    uint32_t r = 0, shift, end;
    seek(tab, v.nint, f, r, shift, end);
    for (uint32_t it = 0; it < nit; it += 4, f += 128) {
        // sixteen, eight or four steps that lie inside the chunk and inside every lane's interval
        // run without per-point guards (sixteen only for the 8-byte 2-D records)
        if (GEOM != kGeomBall3 && s0 + (it + 16) * 32 <= s1 && __all_sync(0xffffffffu, f + 480 < end)) {
            const P* p = xy + (f + shift);
            P pp[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) pp[u] = __ldg(p + 32 * u);
            uint32_t w[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) w[u] = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, pp[u]));
            if (lane_id() == 0) {
#pragma unroll
                for (int u = 0; u < 16; u += 4)
                    *reinterpret_cast<uint4*>(sw + it + u) = make_uint4(w[u], w[u + 1], w[u + 2], w[u + 3]);
            }
            it += 12;
            f += 384;
            continue;
        }
        if (s0 + (it + 8) * 32 <= s1 && __all_sync(0xffffffffu, f + 224 < end)) {
            const P* p = xy + (f + shift);
            const P p0 = __ldg(p), p1 = __ldg(p + 32), p2 = __ldg(p + 64), p3 = __ldg(p + 96);
            const P p4 = __ldg(p + 128), p5 = __ldg(p + 160), p6 = __ldg(p + 192), p7 = __ldg(p + 224);
            const uint32_t w0 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p0));
            const uint32_t w1 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p1));
            const uint32_t w2 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p2));
            const uint32_t w3 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p3));
            const uint32_t w4 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p4));
            const uint32_t w5 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p5));
            const uint32_t w6 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p6));
            const uint32_t w7 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p7));
            if (lane_id() == 0) {
                *reinterpret_cast<uint4*>(sw + it) = make_uint4(w0, w1, w2, w3);
                *reinterpret_cast<uint4*>(sw + it + 4) = make_uint4(w4, w5, w6, w7);
            }
            it += 4;
            f += 128;
            continue;
        }
        const bool full = s0 + (it + 4) * 32 <= s1;     // warp-uniform
        if (full && __all_sync(0xffffffffu, f + 96 < end)) {
            const P* p = xy + (f + shift);
            const P p0 = __ldg(p), p1 = __ldg(p + 32), p2 = __ldg(p + 64), p3 = __ldg(p + 96);
            const uint32_t w0 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p0));
            const uint32_t w1 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p1));
            const uint32_t w2 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p2));
            const uint32_t w3 = __ballot_sync(0xffffffffu, is_hit<GEOM>(v, p3));
            if (lane_id() == 0) *reinterpret_cast<uint4*>(sw + it) = make_uint4(w0, w1, w2, w3);
        } else {
            P p[4];
            bool val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t fu = f + 32u * u;
                val[u] = fu < s1;
                if (fu >= end) seek(tab, v.nint, fu, r, shift, end);
                p[u] = val[u] ? __ldg(xy + (fu + shift)) : Geom<GEOM>::zero();
            }
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = __ballot_sync(0xffffffffu, val[u] && is_hit<GEOM>(v, p[u]));
            if (lane_id() == 0) *reinterpret_cast<uint4*>(sw + it) = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
        const uint32_t wi = s * 32 + lane_id();
        words[s] = wi < nit ? sw[wi] : 0u;
    }
    uint32_t c = 0;
#pragma unroll
    for (int s = 0; s < WPL; ++s) c += __popc(words[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

// Warp-cooperative search: the query owning chunk g (largest q with base[q] <= g).
__device__ __forceinline__ uint64_t owner_query(const uint64_t* __restrict__ base, uint64_t m, uint64_t g)
{
    uint64_t lo = 0, hi = m;   // base[lo] <= g < base[hi]
    const unsigned lane = lane_id();
    while (hi - lo > 1) {
        const uint64_t step = (hi - lo + 31) >> 5;
        const uint64_t pos = lo + lane * step;
        const bool le = pos < hi && __ldg(base + pos) <= g;
        const uint32_t bal = __ballot_sync(0xffffffffu, le);
        const int last = 31 - __clz(bal);
        const uint64_t nlo = lo + (uint64_t)last * step;
        const uint64_t nhi = min(hi, nlo + step);
        lo = nlo;
        hi = nhi;
    }
    return lo;
}

// ------------------------------------------------------------------------------------
// small queries: one thread per query
// ------------------------------------------------------------------------------------
// A query that scans at most kSmallScan points would spend most of a warp's time in the
// chunked passes on its per-query setup; one thread walks its intervals instead, keeping hit
// f (the f-th scanned point, in scan order) as bit f mod 64 of mask word f / 64.
__device__ __forceinline__ QView small_view(const QueryArgs& a, uint64_t qi)
{
    QView v;
    v.S = 0;
    v.nint = a.kint;
    if (a.dim == 3) {
        v.q = make_int2(__ldg(a.q + 3 * qi), __ldg(a.q + 3 * qi + 1));
        v.qz = __ldg(a.q + 3 * qi + 2);
    } else {
        v.q = __ldg(reinterpret_cast<const int2*>(a.q) + qi);
        v.qz = 0;
    }
    v.d = __ldg(a.delta + qi);
    v.d2 = -((int64_t)v.d * v.d + 1);
    return v;
}

// Each warp claims 32 listed queries at a time from a shared counter, one per lane; the chunked
// kernels run these loops once their own queue is empty, so the small queries fill the tail.
template <int GEOM>
__device__ __forceinline__ void small_count_tail(const QueryArgs& a)
{
    using P = typename Geom<GEOM>::P;
    constexpr uint32_t NW = kSmallWords;
    const P* __restrict__ xy = Geom<GEOM>::points(a);
    const uint64_t ns = a.work_ctr[kCtrSmallSize];
    while (true) {
        unsigned long long t0 = 0;
        if (lane_id() == 0) t0 = atomicAdd(a.work_ctr + kCtrSmallCount, 32ull);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= ns) break;
        const uint64_t t = t0 + lane_id();
        if (t >= ns) continue;
        const uint32_t q = a.small_list[t];
        const QView v = small_view(a, q);
        const uint2* rp = reinterpret_cast<const uint2*>(a.ranges) + (uint64_t)q * a.kint;
        unsigned long long* mw = a.small_mask + t * NW;
        unsigned long long word = 0;
        uint32_t f = 0, hits = 0;
        for (uint32_t r = 0; r < a.kint; ++r) {
            const uint2 be = __ldg(rp + r);
            for (uint32_t pos = be.x; pos < be.y; ++pos) {
                if (is_hit<GEOM>(v, __ldg(xy + pos))) word |= 1ull << (f & 63);
                if ((++f & 63) == 0) {   // a full word of 64 scanned points
                    mw[(f >> 6) - 1] = word;
                    hits += __popcll(word);
                    word = 0;
                }
            }
        }
        if (f & 63) {
            mw[f >> 6] = word;
            hits += __popcll(word);
        }
        a.counts[q] = hits;
    }
}

__device__ __forceinline__ void small_write_tail(const QueryArgs& a)
{
    constexpr uint32_t NW = kSmallWords;
    const uint64_t ns = a.work_ctr[kCtrSmallSize];
    const uint64_t qe = a.q_end ? a.q_end : a.m;
    while (true) {
        unsigned long long t0 = 0;
        if (lane_id() == 0) t0 = atomicAdd(a.work_ctr + kCtrSmallWrite, 32ull);
        t0 = __shfl_sync(0xffffffffu, t0, 0);
        if (t0 >= ns) break;
        const uint64_t t = t0 + lane_id();
        if (t >= ns) continue;
        const uint32_t q = a.small_list[t];
        if (q < a.q_begin || q >= qe) continue;   // a slice of the queries (by query id)
        uint32_t left = __ldg(a.counts + q);
        if (left == 0) continue;
        const unsigned long long* mw = a.small_mask + t * NW;
        const uint2* rp = reinterpret_cast<const uint2*>(a.ranges) + (uint64_t)q * a.kint;
        uint64_t dst = a.out_offsets[q];
        unsigned long long word = mw[0];
        uint32_t f = 0;
        for (uint32_t r = 0; r < a.kint && left; ++r) {
            const uint2 be = __ldg(rp + r);
            for (uint32_t pos = be.x; pos < be.y && left; ++pos) {
                if ((word >> (f & 63)) & 1ull) {
                    if (dst < a.ids_capacity) a.out_ids[dst] = __ldg(a.ids + pos);
                    ++dst;
                    --left;
                }
                if ((++f & 63) == 0 && left) word = mw[f >> 6];
            }
        }
    }
}

// A query whose chunks are split over warps (see QueryArgs::chunk_hits): one whose chunks
// outnumber a warp's share of the batch's G chunks (and at least kBigChunks), so that one warp
// alone would set the write pass's tail.
__device__ __forceinline__ bool is_big(const QueryArgs& a, uint64_t G, uint64_t cb, uint64_t nch)
{
    return a.chunk_hits != nullptr && nch >= max(kBigChunks, G / a.big_warps) && cb + nch <= a.big_cap;
}

// ------------------------------------------------------------------------------------
// count_kernel
// ------------------------------------------------------------------------------------
template <int WPL, int GEOM>
__global__ void __launch_bounds__(kThreads) count_kernel(QueryArgs a)
{
    __shared__ WarpTab s_tab[kThreads / 32];
    __shared__ __align__(16) uint32_t s_words[kThreads / 32][WPL * 32];
    WarpTab* tab = &s_tab[threadIdx.x >> 5];
    uint32_t* sw = s_words[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    // work items are chunks in processing order: wbase (curve order) or chunk_base (input order)
    const uint64_t* wb = a.wbase ? a.wbase : a.chunk_base;
    const uint64_t G = wb[a.m];
    const uint32_t W = a.chunk >> 5;   // mask words per chunk
    while (true) {
        uint64_t g0 = 0;
        if (lane == 0) g0 = atomicAdd(a.work_ctr + kCtrCount, (unsigned long long)a.batch);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if (g0 >= G) break;
        const uint64_t g1 = min(G, g0 + a.batch);
        uint64_t r = owner_query(wb, a.m, g0);
        uint64_t loaded = ~0ull;
        QView v;
        for (uint64_t w = g0; w < g1; ++w) {
            while (__ldg(wb + r + 1) <= w) ++r;
            const uint64_t q = a.perm ? __ldg(a.perm + r) : r;
            if (q != loaded) {   // consecutive chunks of one query share its table
                v = load_query(a, q, tab);
                loaded = q;
            }
            const uint32_t j = (uint32_t)(w - __ldg(wb + r));
            const uint64_t g = a.perm ? __ldg(a.chunk_base + q) + j : w;   // mask slot
            const uint32_t s0 = j * a.chunk;
            const uint32_t s1 = min(v.S, s0 + a.chunk);
            uint32_t words[WPL];
            const uint32_t cnt = filter_chunk<WPL, GEOM>(a, v, tab, s0, s1, words, sw);
            if (g < a.mask_chunks) {
                const uint32_t nw = (s1 - s0 + 31) >> 5;
                uint32_t* mp = a.masks + g * W;
#pragma unroll
                for (int s = 0; s < WPL; ++s) {
                    const uint32_t wi = s * 32 + lane;
                    if (wi < nw) mp[wi] = words[s];
                }
            }
            if (lane == 0 && cnt) atomicAdd(a.counts + q, cnt);
        }
    }
    if (a.small_list) small_count_tail<GEOM>(a);
}

// ------------------------------------------------------------------------------------
// write_kernel
// ------------------------------------------------------------------------------------
// Writes the ids of one chunk (points [s0, s1) of the query's concatenated intervals, mask slot
// g) to out_ids[dst ...]; returns the number written.  cr / shift / end: the lane's interval
// cursor, which only moves forward while the chunks of one query are taken in order.
template <int WPL, int GEOM>
__device__ __forceinline__ uint32_t write_chunk(const QueryArgs& a, const QView& v, const WarpTab* tab, uint16_t* buf,
                                                uint64_t g, uint32_t s0, uint32_t s1, uint64_t dst,
                                                uint32_t& cr, uint32_t& shift, uint32_t& end)
{
    const unsigned lane = lane_id();
    const uint32_t nw = (s1 - s0 + 31) >> 5;
    uint32_t words[WPL];
    if (g < a.mask_chunks) {
        const uint32_t* mp = a.masks + g * (a.chunk >> 5);
#pragma unroll
        for (int s = 0; s < WPL; ++s) {
            const uint32_t wi = s * 32 + lane;
            words[s] = wi < nw ? __ldcs(mp + wi) : 0u;
        }
    } else {
        filter_chunk<WPL, GEOM>(a, v, tab, s0, s1, words, reinterpret_cast<uint32_t*>(buf));
        __syncwarp();   // the words are read before buf takes the staged indices
    }
    // the WPL groups' popcounts in 16-bit fields of one word, scanned together
    unsigned long long pk = 0;
#pragma unroll
    for (int s = 0; s < WPL; ++s) pk |= (unsigned long long)__popc(words[s]) << (16 * s);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, pk, o);
        if (lane >= (unsigned)o) pk += t;
    }
    const unsigned long long ktot = __shfl_sync(0xffffffffu, pk, 31);
    uint32_t rank = 0;
#pragma unroll
    for (int s = 0; s < WPL; ++s) {
        const uint32_t wl = words[s];
        const uint32_t pc = __popc(wl);
        const uint32_t incl = (uint32_t)(pk >> (16 * s)) & 0xffffu;
        const uint32_t K = (uint32_t)(ktot >> (16 * s)) & 0xffffu;
        if (K == 0) continue;
        // each lane lists the group-relative indices of its own word's hits
        uint32_t slot = incl - pc;
        uint32_t bits = wl;
        const uint32_t rbase = lane * 32u;
        while (bits) {
            buf[slot++] = (uint16_t)(rbase + (uint32_t)(__ffs(bits) - 1));
            bits &= bits - 1;
        }
        __syncwarp();
        // coalesced gather of the ids and write of the output; a lane's indices grow with t,
        // so its interval cursor only moves forward
        const uint32_t gbase = s0 + (uint32_t)s * 1024u;
        const uint64_t dst0 = dst + rank;
        if (dst0 + K <= a.ids_capacity) {   // the whole group fits: no per-id check
            uint32_t* __restrict__ out = a.out_ids + dst0;
#pragma unroll 4
            for (uint32_t t = lane; t < K; t += 32) {
                const uint32_t f = gbase + buf[t];
                if (f >= end) seek(tab, v.nint, f, cr, shift, end);
                __stcs(out + t, __ldg(a.ids + (f + shift)));   // written once, not re-read
            }
        } else {
            for (uint32_t t = lane; t < K; t += 32) {
                const uint32_t f = gbase + buf[t];
                if (f >= end) seek(tab, v.nint, f, cr, shift, end);
                const uint64_t d = dst0 + t;
                if (d < a.ids_capacity) a.out_ids[d] = __ldg(a.ids + (f + shift));
            }
        }
        __syncwarp();
        rank += K;
    }
    return rank;
}


// The chunks of big queries, in batches from the list of their chunk slots (a query's chunks
// are listed together); a chunk's output position is its query's offset plus the hits of the
// query's earlier chunks.  Launched before write_kernel, which skips these queries.
template <int WPL, int GEOM>
__global__ void __launch_bounds__(kThreads, 8) write_big_kernel(QueryArgs a)
{
    // per-warp staging of one group of 32 mask words (<= 1024 hits): each hit's index within
    // the group's 1024 points, 16 bits; its array position is resolved in the copy loop
    __shared__ __align__(16) uint16_t s_rel[kThreads / 32][1024];
    __shared__ WarpTab s_tab[kThreads / 32];
    uint16_t* buf = s_rel[threadIdx.x >> 5];
    WarpTab* tab = &s_tab[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    const uint64_t qe = a.q_end ? a.q_end : a.m;
    {
        const uint64_t total = a.work_ctr[kCtrBigItems];
        uint64_t q = 0, cb = 0, ce = 0, off = 0;
        uint32_t k = 0, cr = 0, shift = 0, end = 0;
        QView v;
        while (true) {
            uint64_t b0 = 0;
            if (lane == 0) b0 = atomicAdd(a.work_ctr + kCtrWriteBig, (unsigned long long)a.batch);
            b0 = __shfl_sync(0xffffffffu, b0, 0);
            if (b0 >= total) break;
            const uint64_t b1 = min(total, b0 + a.batch);
            for (uint64_t b = b0; b < b1; ++b) {
                const uint64_t g = __ldg(a.big_items + b);
                if (g < cb || g >= ce) {   // a new query: its table, offset and cursor
                    q = owner_query(a.chunk_base, a.m, g);
                    cb = __ldg(a.chunk_base + q);
                    ce = __ldg(a.chunk_base + q + 1);
                    v = load_query(a, q, tab);
                    off = a.out_offsets[q];
                    k = __ldg(a.counts + q);
                    cr = 0;
                    shift = 0;
                    end = 0;
                }
                if (q < a.q_begin || q >= qe) continue;
                const uint64_t j = g - cb;
                const uint32_t before = __ldg(a.chunk_hits + g);
                const uint32_t after = g + 1 < ce ? __ldg(a.chunk_hits + g + 1) : k;
                if (after == before) continue;   // no hits in this chunk
                const uint32_t s0 = (uint32_t)j * a.chunk;
                write_chunk<WPL, GEOM>(a, v, tab, buf, g, s0, min(v.S, s0 + a.chunk), off + before, cr, shift, end);
            }
        }
    }
}

// A hint that starts moving the line holding p into L2; nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <int WPL, int GEOM>
__global__ void __launch_bounds__(kThreads, 8) write_kernel(QueryArgs a)
{
    // per-warp staging of one group of 32 mask words (<= 1024 hits): each hit's index within
    // the group's 1024 points, 16 bits; its array position is resolved in the copy loop
    __shared__ __align__(16) uint16_t s_rel[kThreads / 32][1024];
    __shared__ WarpTab s_tab[kThreads / 32];
    uint16_t* buf = s_rel[threadIdx.x >> 5];
    WarpTab* tab = &s_tab[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.out_offsets[a.m] > a.ids_capacity)
        set_status(a.status, SFC_DEV_CAPACITY);
    const uint64_t qe = a.q_end ? a.q_end : a.m;
    const uint64_t G = a.chunk_hits ? a.chunk_base[a.m] : 0;
    const uint32_t W = a.chunk >> 5;   // mask words per chunk
    // the queries that are not big (write_big_kernel takes those), one warp each, from a
    // query queue
    while (true) {
        uint64_t q0 = 0;
        if (lane == 0) q0 = atomicAdd(a.work_ctr + kCtrWrite, (unsigned long long)a.qbatch);
        q0 = a.q_begin + __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= qe) break;
        const uint64_t q1 = min(qe, q0 + a.qbatch);
        for (uint64_t qs = q0; qs < q1; qs += 32) {
            const uint32_t nb = (uint32_t)min((uint64_t)32, q1 - qs);
            // lane i loads query qs + i's bookkeeping and starts its intervals and its first
            // chunk's mask words towards L2, so that these loads are in flight for the whole
            // grab together instead of one query after another
            uint64_t mq = 0, mcb = 0;
            uint32_t mk = 0, mnch = 0;
            if (lane < nb) {
                mq = a.perm ? __ldg(a.perm + qs + lane) : qs + lane;
                prefetch_l2(reinterpret_cast<const uint2*>(a.ranges) + mq * a.kint);
                mk = __ldg(a.counts + mq);
                mcb = __ldg(a.chunk_base + mq);
                mnch = (uint32_t)(__ldg(a.chunk_base + mq + 1) - mcb);
                if (mk != 0 && mnch != 0 && mcb < a.mask_chunks) {
                    // the lines of the first chunk's mask that the query surely uses: all when
                    // further chunks follow, else the first (its points may end within it, and
                    // the count pass writes no words past them)
                    const uint32_t pw = mnch > 1 ? W : min(W, 32u);
                    for (uint32_t w = 0; w < pw; w += 32) prefetch_l2(a.masks + mcb * W + w);
                }
            }
            for (uint32_t i = 0; i < nb; ++i) {
                const uint64_t q = __shfl_sync(0xffffffffu, mq, i);
                const uint32_t k = __shfl_sync(0xffffffffu, mk, i);
                const uint64_t cb = __shfl_sync(0xffffffffu, mcb, i);
                const uint32_t nch = __shfl_sync(0xffffffffu, mnch, i);
                if (k == 0 || nch == 0) continue;   // no hits, or a query of the small-query path
                if (is_big(a, G, cb, nch)) continue;  // written by write_big_kernel
                const uint64_t off = a.out_offsets[q];
                const QView v = load_query(a, q, tab);
                uint32_t cr = 0;   // this lane's interval cursor (indices only grow within a query)
                uint32_t shift = 0, end = 0;
                uint32_t rank = 0;
                for (uint32_t j = 0; j < nch && rank < k; ++j) {
                    const uint32_t s0 = j * a.chunk;
                    rank += write_chunk<WPL, GEOM>(a, v, tab, buf, cb + j, s0, min(v.S, s0 + a.chunk), off + rank,
                                                   cr, shift, end);
                }
            }
        }
    }
    // then the small queries
    if (a.small_list) small_write_tail(a);
}

// Per listed query that is big (one warp each): each chunk's hit count from its mask words
// (the count pass's ballots), then chunk_hits[cb .. cb + nch) <- their exclusive scan, and the
// slots cb .. cb + nch - 1 appended to big_items.  The plan listed the queries of at least
// kBigChunks chunks in its processing order, so the big chunks come out close to curve order
// and the write pass's gathers of neighbouring big queries share the cache.
__global__ void chunk_prefix_kernel(QueryArgs a)
{
    const unsigned lane = lane_id();
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
    const uint64_t nbig = a.work_ctr[kCtrBigList];
    const uint64_t G = a.chunk_base[a.m];
    const uint32_t W = a.chunk >> 5;   // mask words per chunk
    for (uint64_t i = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); i < nbig; i += warps) {
        const uint64_t q = a.big_list[i];
        const uint64_t cb = __ldg(a.chunk_base + q), nch = __ldg(a.chunk_base + q + 1) - cb;
        if (!is_big(a, G, cb, nch)) continue;
        // the query's scan length S (its interval lengths), for the last chunk's valid words
        uint32_t len = 0;
        if (lane < a.kint) {
            const uint2 r = __ldg(reinterpret_cast<const uint2*>(a.ranges) + q * a.kint + lane);
            len = r.y - r.x;
        }
        const uint32_t S = __reduce_add_sync(0xffffffffu, len);
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(a.work_ctr + kCtrBigItems, (unsigned long long)nch);
        base = __shfl_sync(0xffffffffu, base, 0);
        // 32 chunks at a time, one per lane: its hit count from its mask words (16-byte loads when
        // a chunk's W words keep 16-byte alignment, i.e. W % 4 == 0; words past the chunk's
        // points, in the last chunk, are not the query's), then a scan
        uint32_t carry = 0;
        for (uint64_t j0 = 0; j0 < nch; j0 += 32) {
            const uint64_t j = j0 + lane;
            uint32_t c = 0;
            if (j < nch) {
                const uint64_t g = cb + j;
                const uint32_t s0 = (uint32_t)j * a.chunk;
                const uint32_t nw = (min(S, s0 + a.chunk) - s0 + 31) >> 5;
                if ((W & 3u) == 0) {
                    const uint4* mp = reinterpret_cast<const uint4*>(a.masks + g * W);
                    for (uint32_t w = 0; w < nw; w += 4) {
                        const uint4 x = __ldcs(mp + (w >> 2));
                        c += __popc(x.x) + (w + 1 < nw ? __popc(x.y) : 0u) + (w + 2 < nw ? __popc(x.z) : 0u) +
                             (w + 3 < nw ? __popc(x.w) : 0u);
                    }
                } else {
                    const uint32_t* mp = a.masks + g * W;
                    for (uint32_t w = 0; w < nw; ++w) c += __popc(__ldcs(mp + w));
                }
                a.big_items[base + j] = (uint32_t)g;
            }
            const uint32_t incl = warp_incl_scan_u32(c);
            if (j < nch) a.chunk_hits[cb + j] = carry + incl - c;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

__global__ void query_keys_kernel(const int32_t* __restrict__ q, uint64_t m, int curve, uint64_t* keys)
{
    __shared__ HilbertTables tb;
    if (curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const int2 c = reinterpret_cast<const int2*>(q)[i];
        // the top 24 of the 60 key bits (cells of side 2^18) order the queries well enough: three
        // radix passes (the sort skips the constant high digits); at 10^7 queries over 10^8
        // points, 32 bits (four passes) gave the same plan and count times and a 0.1 ms longer sort
        keys[i] = point_in_domain(c.x, c.y) ? curve_key(curve, &tb, (uint32_t)c.x, (uint32_t)c.y) >> 36 : ~0ull >> 36;
    }
}

__global__ void gather_u32_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm, uint64_t m,
                                  uint32_t* out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = src[perm[i]];
}

// keys[r] = the input slice of query perm[r]: the number of slice starts floor(m t / S),
// t = 1 .. S - 1, at or below it (so slice t holds queries [floor(m t / S), floor(m (t + 1) / S)))
__global__ void slice_keys_kernel(const uint32_t* __restrict__ perm, uint64_t m, int S, uint64_t* keys)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t q = perm[i];
        uint64_t s = 0;
        for (int t = 1; t < S; ++t) s += q >= m * (uint64_t)t / (uint64_t)S;
        keys[i] = s;
    }
}

int persistent_grid(const void* fn)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms();
}

template <int WPL, int GEOM>
void launch_count_write_geom(const QueryArgs& a, bool write, cudaStream_t st)
{
    if (!write) {
        int g = persistent_grid((const void*)count_kernel<WPL, GEOM>);
        count_kernel<WPL, GEOM><<<g, kThreads, 0, st>>>(a);
    } else {
        if (a.chunk_hits) {
            int gb = persistent_grid((const void*)write_big_kernel<WPL, GEOM>);
            write_big_kernel<WPL, GEOM><<<gb, kThreads, 0, st>>>(a);
            count_launch();
        }
        int g = persistent_grid((const void*)write_kernel<WPL, GEOM>);
        write_kernel<WPL, GEOM><<<g, kThreads, 0, st>>>(a);
    }
}

template <int WPL>
sfc_status launch_count_write(const QueryArgs& a, bool write, cudaStream_t st)
{
    if (a.dim == 3) launch_count_write_geom<WPL, kGeomBall3>(a, write, st);
    else if (a.norm == SFC_NORM_SQUARE) launch_count_write_geom<WPL, kGeomSquare>(a, write, st);
    else launch_count_write_geom<WPL, kGeomDisc>(a, write, st);
    count_launch();
    return launch_status();
}

}  // namespace

// Opts plan_kernel<Bounds, DROP, EXPORT> into its dynamic shared memory (more than 48 KB for
// the finest cover), once per instantiation and device.
template <class Bounds, int DROP, bool EXPORT>
static void allow_plan_smem()
{
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || done[dev]) return;
    cudaFuncSetAttribute(plan_kernel<Bounds, DROP, EXPORT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)plan_smem_bytes<Bounds, DROP>());
    done[dev] = true;
}

template <int DROP, bool EXPORT>
static void plan_dispatch(const QueryArgs& a, const LearnedModelView* lm, const PlanExport& ex, cudaStream_t st)
{
    const unsigned g = (unsigned)((a.m + kThreads - 1) / kThreads);
    if (lm) {
        allow_plan_smem<LearnedBounds, DROP, EXPORT>();
        plan_kernel<LearnedBounds, DROP, EXPORT><<<g, kThreads, plan_smem_bytes<LearnedBounds, DROP>(), st>>>(
            a, LearnedBounds{lm->root, lm->leaf, lm->fence, lm->fence_fine, lm->stats}, ex);
    } else {
        allow_plan_smem<BinaryBounds, DROP, EXPORT>();
        plan_kernel<BinaryBounds, DROP, EXPORT><<<g, kThreads, plan_smem_bytes<BinaryBounds, DROP>(), st>>>(
            a, BinaryBounds{}, ex);
    }
}

template <bool EXPORT>
static sfc_status plan_launch(const QueryArgs& a, const LearnedModelView* lm, const PlanExport& ex, cudaStream_t st)
{
    if (a.m == 0) return SFC_OK;
    if (a.dim == 3) {
        const unsigned g = (unsigned)((a.m + kThreads - 1) / kThreads);
        if (a.drop == 0) plan3_kernel<0, EXPORT><<<g, kThreads, 0, st>>>(a, ex);
        else plan3_kernel<1, EXPORT><<<g, kThreads, 0, st>>>(a, ex);
        count_launch();
        return launch_status();
    }
    if (a.drop == 0) plan_dispatch<0, EXPORT>(a, lm, ex, st);
    else if (a.drop == 1) plan_dispatch<1, EXPORT>(a, lm, ex, st);
    else plan_dispatch<2, EXPORT>(a, lm, ex, st);
    count_launch();
    return launch_status();
}

sfc_status launch_plan(const QueryArgs& a, const LearnedModelView* lm, cudaStream_t st)
{
    return plan_launch<false>(a, lm, PlanExport{}, st);
}

int cover_intervals(int drop) { return drop == 0 ? Cover<0>::K : (drop == 1 ? Cover<1>::K : Cover<2>::K); }

int query_intervals(int dim, int drop)
{
    if (dim == 3) return drop == 0 ? Cover3<0>::K : Cover3<1>::K;
    return cover_intervals(drop);
}

static unsigned flat_grid(uint64_t m)
{
    uint64_t g = (m + kThreads - 1) / kThreads;
    const uint64_t cap = (uint64_t)num_sms() * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

sfc_status launch_query_keys(const int32_t* q, uint64_t m, int curve, uint64_t* keys, cudaStream_t st)
{
    if (m == 0) return SFC_OK;
    query_keys_kernel<<<flat_grid(m), kThreads, 0, st>>>(q, m, curve, keys);
    count_launch();
    return launch_status();
}

sfc_status launch_gather_u32(const uint32_t* src, const uint32_t* perm, uint64_t m, uint32_t* out, cudaStream_t st)
{
    if (m == 0) return SFC_OK;
    gather_u32_kernel<<<flat_grid(m), kThreads, 0, st>>>(src, perm, m, out);
    count_launch();
    return launch_status();
}

sfc_status launch_slice_keys(const uint32_t* perm, uint64_t m, int S, uint64_t* keys, cudaStream_t st)
{
    if (m == 0) return SFC_OK;
    slice_keys_kernel<<<flat_grid(m), kThreads, 0, st>>>(perm, m, S, keys);
    count_launch();
    return launch_status();
}

sfc_status launch_chunk_prefix(const QueryArgs& a, cudaStream_t st)
{
    if (a.m == 0 || !a.chunk_hits) return SFC_OK;
    chunk_prefix_kernel<<<num_sms() * 2, kThreads, 0, st>>>(a);   // a few listed queries
    count_launch();
    return launch_status();
}

sfc_status launch_count(const QueryArgs& a, cudaStream_t st)
{
    if (a.m == 0) return SFC_OK;
    switch (a.chunk >> 10) {
        case 0: case 1: return launch_count_write<1>(a, false, st);
        case 2: return launch_count_write<2>(a, false, st);
        default: return launch_count_write<4>(a, false, st);
    }
}

sfc_status launch_write(const QueryArgs& a, cudaStream_t st)
{
    if (a.m == 0) return SFC_OK;
    switch (a.chunk >> 10) {
        case 0: case 1: return launch_count_write<1>(a, true, st);
        case 2: return launch_count_write<2>(a, true, st);
        default: return launch_count_write<4>(a, true, st);
    }
}

sfc_status launch_ranges(const QueryArgs& a, const LearnedModelView* lm, uint64_t* lo, uint64_t* hi,
                         uint32_t* b, uint32_t* e, uint32_t* cnt, cudaStream_t st)
{
    QueryArgs x = a;
    x.ranges = nullptr;
    x.nchunks = nullptr;
    x.scanned = nullptr;
    x.cells = nullptr;
    return plan_launch<true>(x, lm, PlanExport{lo, hi, b, e, cnt}, st);
}

}  // namespace sfc
