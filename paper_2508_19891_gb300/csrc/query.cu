// Batched distance query (Alg. 1 for m queries at once).
//
//   plan_kernel    one thread per query: bounding square Q of B_delta(q), the level l with
//                  2 delta <= 2^l < 4 delta, the <= 4 cells of cells(Q) and their key
//                  intervals [pi(C)o0, pi(C)o1] (Observation), sorted and with abutting
//                  intervals merged, then lower_bound of both ends of every interval, by
//                  binary search or by the learned model (verified, with fallback).  The
//                  query's scan length S_q is cut into chunks of C points.
//   scan           exclusive scan of the chunk counts -> chunk bases.
//   count_kernel   persistent warps take batches of chunks from a counter (work stealing);
//                  a warp streams the chunk's coordinates, applies the exact int64 filter
//                  dx^2 + dy^2 <= delta^2, keeps the warp ballots as a hit bitmask (one bit
//                  per scanned point) and adds the chunk's popcount to the query's count.
//   scan           exclusive scan of the per-query counts -> the caller's out_offsets.
//   write_kernel   persistent warps take batches of queries; a warp walks its query's
//                  chunks in order, reads the bitmask (or, past the bitmask budget, re-runs
//                  the filter) and writes the ids of the hits with ballot/popc compaction at
//                  out_offsets[q] + rank, so each query's ids come out in array order.
//
// The bitmask makes the second pass read 1 bit instead of 8 bytes per scanned point.
#include "sfc_internal.cuh"
#include "query.cuh"

namespace sfc {

namespace {

constexpr int kThreads = 256;

// ------------------------------------------------------------------------------------
// Ranges (cells(Q) with merged abutting intervals)
// ------------------------------------------------------------------------------------
struct QueryRanges {
    uint64_t lo[4], hi[4];
    int cnt;
};

__device__ __forceinline__ void derive_ranges(int curve, const HilbertTables* tb, int32_t qx,
                                              int32_t qy, int32_t delta, QueryRanges& R)
{
    const int64_t d = delta;
    const int64_t x0 = max((int64_t)0, (int64_t)qx - d), x1 = min((int64_t)kSide - 1, (int64_t)qx + d);
    const int64_t y0 = max((int64_t)0, (int64_t)qy - d), y1 = min((int64_t)kSide - 1, (int64_t)qy + d);
    int l = 0;
    if (d > 0) {
        l = 64 - __clzll((unsigned long long)(2 * d - 1));   // bit length of 2 delta - 1
        if (l > kOmega) l = kOmega;
    }
    const uint64_t span = (l >= kOmega) ? kKeyMax : ((1ull << (2 * l)) - 1);
    int cnt = 0;
    for (int64_t cy = y0 >> l; cy <= (y1 >> l); ++cy) {
        for (int64_t cx = x0 >> l; cx <= (x1 >> l); ++cx) {
            if (cnt == 4) break;   // unreachable: x1 - x0 <= 2 delta <= 2^l gives <= 2 per axis
            uint64_t k = curve_key(curve, tb, (uint32_t)(cx << l), (uint32_t)(cy << l));
            uint64_t lo = k & ~span;
            // insertion in lo order
            int j = cnt;
            while (j > 0 && R.lo[j - 1] > lo) { R.lo[j] = R.lo[j - 1]; R.hi[j] = R.hi[j - 1]; --j; }
            R.lo[j] = lo;
            R.hi[j] = lo | span;
            ++cnt;
        }
    }
    // merge intervals that abut in key order (the scan over them is identical)
    int m = 0;
    for (int i = 0; i < cnt; ++i) {
        if (m > 0 && R.hi[m - 1] + 1 == R.lo[i]) {
            R.hi[m - 1] = R.hi[i];
        } else {
            R.lo[m] = R.lo[i];
            R.hi[m] = R.hi[i];
            ++m;
        }
    }
    R.cnt = m;
}

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

struct BinaryBounds {
    __device__ __forceinline__ void prepare(RootParams*) {}
    __device__ __forceinline__ void operator()(const uint64_t* keys, uint32_t n, const uint64_t* t,
                                               uint32_t* r, int ne) const
    {
        uint32_t lo[8], len[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) { lo[e] = 0; len[e] = e < ne ? n : 0; }
        lower_bounds_window<8>(keys, t, lo, len);
#pragma unroll
        for (int e = 0; e < 8; ++e) r[e] = lo[e];
    }
};

struct LearnedBounds {
    const RootParams* root;      // device; after prepare() the block's shared-memory copy
    const LeafParams* leaf;
    unsigned long long* stats;   // [0] endpoints, [1] misses, [2] window sum
    // every thread of the block calls this, then the block synchronises
    __device__ __forceinline__ void prepare(RootParams* s)
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(root);
        uint32_t* dst = reinterpret_cast<uint32_t*>(s);
        for (unsigned i = threadIdx.x; i < sizeof(RootParams) / 4; i += blockDim.x) dst[i] = src[i];
        root = s;
    }
    __device__ __forceinline__ void operator()(const uint64_t* keys, uint32_t n, const uint64_t* t,
                                               uint32_t* r, int ne) const
    {
        uint32_t lo[8], len[8];
        unsigned long long wsum = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            lo[e] = 0;
            len[e] = 0;
            if (e < ne) {
                const int j = route_leaf(*root, t[e]);
                const LeafParams lp = leaf[j];
                const int64_t p = leaf_predict(lp, t[e]);
                int64_t a = p + lp.err_lo, b = p + (int64_t)lp.err_hi + 1;
                a = max(a, (int64_t)lp.first);
                a = min(a, (int64_t)lp.end);
                b = max(b, a);
                b = min(b, (int64_t)lp.end);
                lo[e] = (uint32_t)a;
                len[e] = (uint32_t)(b - a);
                wsum += len[e];
            }
        }
        lower_bounds_window<8>(keys, t, lo, len);
        // verify: lower_bound is the unique r with keys[r-1] < t <= keys[r]
        uint32_t miss = 0;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            if (e < ne) {
                const uint32_t x = lo[e];
                const bool ok = (x == 0 || __ldg(keys + x - 1) < t[e]) && (x == n || __ldg(keys + x) >= t[e]);
                if (!ok) { miss |= 1u << e; lo[e] = 0; len[e] = n; }
            }
        }
        if (miss) lower_bounds_window<8>(keys, t, lo, len);   // full binary search fallback
#pragma unroll
        for (int e = 0; e < 8; ++e) r[e] = lo[e];
        if (stats) {
            unsigned long long c = ne, mc = __popc(miss);
            // one atomic per warp
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c += __shfl_xor_sync(0xffffffffu, c, o);
                mc += __shfl_xor_sync(0xffffffffu, mc, o);
                wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
            }
            if (lane_id() == 0) {
                atomicAdd(stats + 0, c);
                atomicAdd(stats + 1, mc);
                atomicAdd(stats + 2, wsum);
            }
        }
    }
};

// Range derivation + bound search for one query; returns the merged intervals' bounds.
template <class Bounds>
__device__ __forceinline__ int query_bounds(const Bounds& bounds, int curve, const HilbertTables* tb,
                                            const uint64_t* keys, uint32_t n, bool ok, int32_t qx,
                                            int32_t qy, int32_t delta, QueryRanges& R, uint32_t* b,
                                            uint32_t* e)
{
    R.cnt = 0;
    if (ok) derive_ranges(curve, tb, qx, qy, delta, R);
    uint64_t t[8];
    const int ne = 2 * R.cnt;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        t[2 * i] = i < R.cnt ? R.lo[i] : 0;
        t[2 * i + 1] = i < R.cnt ? R.hi[i] + 1 : 0;
    }
    uint32_t r[8];
    bounds(keys, n, t, r, ne);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        b[i] = i < R.cnt ? r[2 * i] : 0;
        e[i] = i < R.cnt ? r[2 * i + 1] : 0;
    }
    return R.cnt;
}

// ------------------------------------------------------------------------------------
// plan_kernel
// ------------------------------------------------------------------------------------
template <class Bounds>
__global__ void __launch_bounds__(kThreads) plan_kernel(QueryArgs a, Bounds bounds_in)
{
    __shared__ HilbertTables tb;
    __shared__ RootParams s_root;
    Bounds bounds = bounds_in;
    bounds.prepare(&s_root);
    __syncthreads();
    if (a.curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = i < a.m;
    int2 q = make_int2(0, 0);
    int32_t delta = -1;
    if (active) {
        q = reinterpret_cast<const int2*>(a.q)[i];
        delta = a.delta[i];
    }
    const bool ok = active && query_valid(q.x, q.y, delta);
    if (active && !ok) set_status(a.status, SFC_DEV_BAD_QUERY);
    uint32_t b[4], e[4];
    QueryRanges R;
    // every lane calls the bound search (with no endpoints when inactive or invalid), so
    // warp-collective statistics inside it see a converged warp
    query_bounds(bounds, a.curve, &tb, a.keys, a.n, ok, q.x, q.y, delta, R, b, e);
    uint64_t S = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) S += e[k] - b[k];
    if (a.scanned) {   // one atomic per warp
        unsigned long long ws = S;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
        if (lane_id() == 0 && ws) atomicAdd(a.scanned, ws);
    }
    if (!active) return;
    uint4* rp = reinterpret_cast<uint4*>(a.ranges + 8 * i);
    rp[0] = make_uint4(b[0], e[0], b[1], e[1]);
    rp[1] = make_uint4(b[2], e[2], b[3], e[3]);
    a.nchunks[i] = (uint32_t)((S + a.chunk - 1) / a.chunk);
}

// ------------------------------------------------------------------------------------
// Shared helpers of the two scan passes
// ------------------------------------------------------------------------------------
struct QView {
    uint32_t b0, b1, b2, b3;
    uint32_t c1, c2, c3, S;   // cumulative starts of intervals 1..3 and the total
    int2 q;
    int64_t d2;
};

__device__ __forceinline__ QView load_query(const QueryArgs& a, uint64_t qi)
{
    QView v;
    const uint4* rp = reinterpret_cast<const uint4*>(a.ranges + 8 * qi);
    uint4 r0 = __ldg(rp), r1 = __ldg(rp + 1);
    v.b0 = r0.x; v.b1 = r0.z; v.b2 = r1.x; v.b3 = r1.z;
    v.c1 = r0.y - r0.x;
    v.c2 = v.c1 + (r0.w - r0.z);
    v.c3 = v.c2 + (r1.y - r1.x);
    v.S = v.c3 + (r1.w - r1.z);
    v.q = __ldg(reinterpret_cast<const int2*>(a.q) + qi);
    const int64_t d = __ldg(a.delta + qi);
    v.d2 = d * d;
    return v;
}

__device__ __forceinline__ uint32_t map_pos(const QView& v, uint32_t f)
{
    return f < v.c1 ? v.b0 + f : f < v.c2 ? v.b1 + (f - v.c1) : f < v.c3 ? v.b2 + (f - v.c2) : v.b3 + (f - v.c3);
}

// Offset from concatenated index f to array position (mod 2^32) for the interval holding f,
// and the first concatenated index of the next interval.
__device__ __forceinline__ void interval_of(const QView& v, uint32_t f, uint32_t& shift, uint32_t& end)
{
    shift = f < v.c1 ? v.b0 : f < v.c2 ? v.b1 - v.c1 : f < v.c3 ? v.b2 - v.c2 : v.b3 - v.c3;
    end = f < v.c1 ? v.c1 : f < v.c2 ? v.c2 : f < v.c3 ? v.c3 : 0xffffffffu;
}

// Exact closed-ball test: |dx|, |dy| < 2^30, so each square is one signed 32x32 -> 64-bit
// multiply(-add) and the sum stays below 2^61.
__device__ __forceinline__ bool is_hit(const QView& v, int2 p)
{
    const int dx = p.x - v.q.x, dy = p.y - v.q.y;
    const long long s = (long long)dx * dx + (long long)dy * dy;
    return s <= v.d2;
}

// Stores ballot words w0..w3 (points s0 + 32 * (it + u) ...) in lanes it % 32 .. it % 32 + 3 of
// slot it / 32.
template <int WPL>
__device__ __forceinline__ void keep_words(uint32_t (&words)[WPL], uint32_t it, uint32_t w0, uint32_t w1,
                                           uint32_t w2, uint32_t w3)
{
    const uint32_t d = lane_id() - (it & 31);
    if (d < 4) {
        const uint32_t w = d == 0 ? w0 : d == 1 ? w1 : d == 2 ? w2 : w3;
        const uint32_t slot = it >> 5;
#pragma unroll
        for (int s = 0; s < WPL; ++s)
            if (slot == (uint32_t)s) words[s] = w;
    }
}

// Filters points [s0, s1) of the query's concatenated intervals; returns the hit count and
// leaves word w (the ballot of points s0 + 32w ...) in lane w % 32, slot w / 32.  Points go in
// groups of 4 x 32: when the whole group lies inside the chunk and no lane crosses the end of
// its interval (one vote), the group runs without per-point guards; otherwise each point is
// checked and the lane looks its interval up again when it crosses into the next one.
template <int WPL>
__device__ __forceinline__ uint32_t filter_chunk(const QueryArgs& a, const QView& v, uint32_t s0,
                                                 uint32_t s1, uint32_t (&words)[WPL])
{
#pragma unroll
    for (int s = 0; s < WPL; ++s) words[s] = 0;
    const uint32_t nit = (s1 - s0 + 31) >> 5;
    const int2* __restrict__ xy = a.xy;
    uint32_t f = s0 + lane_id();
    uint32_t shift, end;
    interval_of(v, f, shift, end);
    for (uint32_t it = 0; it < nit; it += 4, f += 128) {
        const bool full = s0 + (it + 4) * 32 <= s1;     // warp-uniform
        if (full && __all_sync(0xffffffffu, f + 96 < end)) {
            const int2* p = xy + (f + shift);
            const int2 p0 = __ldg(p), p1 = __ldg(p + 32), p2 = __ldg(p + 64), p3 = __ldg(p + 96);
            const uint32_t w0 = __ballot_sync(0xffffffffu, is_hit(v, p0));
            const uint32_t w1 = __ballot_sync(0xffffffffu, is_hit(v, p1));
            const uint32_t w2 = __ballot_sync(0xffffffffu, is_hit(v, p2));
            const uint32_t w3 = __ballot_sync(0xffffffffu, is_hit(v, p3));
            keep_words<WPL>(words, it, w0, w1, w2, w3);
        } else {
            int2 p[4];
            bool val[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t fu = f + 32u * u;
                val[u] = fu < s1;
                if (fu >= end) interval_of(v, fu, shift, end);
                p[u] = val[u] ? __ldg(xy + (fu + shift)) : make_int2(0, 0);
            }
            uint32_t w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) w[u] = __ballot_sync(0xffffffffu, val[u] && is_hit(v, p[u]));
            keep_words<WPL>(words, it, w[0], w[1], w[2], w[3]);
        }
    }
    uint32_t c = 0;
#pragma unroll
    for (int s = 0; s < WPL; ++s) c += __popc(words[s]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    return c;
}

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
// count_kernel
// ------------------------------------------------------------------------------------
template <int WPL>
__global__ void __launch_bounds__(kThreads) count_kernel(QueryArgs a)
{
    const unsigned lane = lane_id();
    // work items are chunks in processing order: wbase (curve order) or chunk_base (input order)
    const uint64_t* wb = a.wbase ? a.wbase : a.chunk_base;
    const uint64_t G = wb[a.m];
    const uint32_t W = a.chunk >> 5;   // mask words per chunk
    while (true) {
        uint64_t g0 = 0;
        if (lane == 0) g0 = atomicAdd(a.work_ctr, (unsigned long long)a.batch);
        g0 = __shfl_sync(0xffffffffu, g0, 0);
        if (g0 >= G) break;
        const uint64_t g1 = min(G, g0 + a.batch);
        uint64_t r = owner_query(wb, a.m, g0);
        for (uint64_t w = g0; w < g1; ++w) {
            while (__ldg(wb + r + 1) <= w) ++r;
            const uint64_t q = a.perm ? __ldg(a.perm + r) : r;
            const QView v = load_query(a, q);
            const uint32_t j = (uint32_t)(w - __ldg(wb + r));
            const uint64_t g = a.perm ? __ldg(a.chunk_base + q) + j : w;   // mask slot
            const uint32_t s0 = j * a.chunk;
            const uint32_t s1 = min(v.S, s0 + a.chunk);
            uint32_t words[WPL];
            const uint32_t cnt = filter_chunk<WPL>(a, v, s0, s1, words);
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
}

// ------------------------------------------------------------------------------------
// write_kernel
// ------------------------------------------------------------------------------------
template <int WPL>
__global__ void __launch_bounds__(kThreads) write_kernel(QueryArgs a)
{
    // per-warp staging of the array positions of one group of 32 mask words (<= 1024 hits)
    __shared__ uint32_t s_pos[kThreads / 32][1024];
    uint32_t* buf = s_pos[threadIdx.x >> 5];
    const unsigned lane = lane_id();
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.out_offsets[a.m] > a.ids_capacity)
        set_status(a.status, SFC_DEV_CAPACITY);
    const uint32_t W = a.chunk >> 5;
    while (true) {
        uint64_t q0 = 0;
        if (lane == 0) q0 = atomicAdd(a.work_ctr + 1, (unsigned long long)a.qbatch);
        q0 = __shfl_sync(0xffffffffu, q0, 0);
        if (q0 >= a.m) break;
        const uint64_t q1 = min(a.m, q0 + a.qbatch);
        for (uint64_t r = q0; r < q1; ++r) {
            const uint64_t q = a.perm ? __ldg(a.perm + r) : r;
            const uint32_t k = __ldg(a.counts + q);
            if (k == 0) continue;
            const QView v = load_query(a, q);
            const uint64_t off = a.out_offsets[q];
            const uint64_t cb = __ldg(a.chunk_base + q);
            const uint64_t nch = __ldg(a.chunk_base + q + 1) - cb;
            uint32_t rank = 0;
            for (uint64_t j = 0; j < nch && rank < k; ++j) {
                const uint64_t g = cb + j;
                const uint32_t s0 = (uint32_t)j * a.chunk;
                const uint32_t s1 = min(v.S, s0 + a.chunk);
                const uint32_t nw = (s1 - s0 + 31) >> 5;
                uint32_t words[WPL];
                if (g < a.mask_chunks) {
                    const uint32_t* mp = a.masks + g * W;
#pragma unroll
                    for (int s = 0; s < WPL; ++s) {
                        const uint32_t wi = s * 32 + lane;
                        words[s] = wi < nw ? __ldcs(mp + wi) : 0u;
                    }
                } else {
                    filter_chunk<WPL>(a, v, s0, s1, words);
                }
#pragma unroll
                for (int s = 0; s < WPL; ++s) {
                    const uint32_t wl = words[s];
                    const uint32_t pc = __popc(wl);
                    const uint32_t incl = warp_incl_scan_u32(pc);
                    const uint32_t K = __shfl_sync(0xffffffffu, incl, 31);
                    if (K == 0) continue;
                    // each lane lists the positions of its own word's hits
                    uint32_t slot = incl - pc;
                    uint32_t bits = wl;
                    const uint32_t fbase = s0 + ((uint32_t)(s * 32) + lane) * 32u;
                    if (bits) {
                        // one interval lookup per word; a word that crosses an interval end
                        // maps each bit separately
                        uint32_t shift, end;
                        interval_of(v, fbase, shift, end);
                        const bool one = fbase + 31 < end;
                        while (bits) {
                            const uint32_t f = fbase + (uint32_t)(__ffs(bits) - 1);
                            bits &= bits - 1;
                            buf[slot++] = one ? f + shift : map_pos(v, f);
                        }
                    }
                    __syncwarp();
                    // coalesced gather of the ids and write of the output
                    const uint64_t dst0 = off + rank;
#pragma unroll 4
                    for (uint32_t t = lane; t < K; t += 32) {
                        const uint64_t dst = dst0 + t;
                        const uint32_t id = __ldg(a.ids + buf[t]);
                        if (dst < a.ids_capacity) a.out_ids[dst] = id;
                    }
                    __syncwarp();
                    rank += K;
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// ranges export (tests)
// ------------------------------------------------------------------------------------
template <class Bounds>
__global__ void __launch_bounds__(kThreads) ranges_kernel(QueryArgs a, Bounds bounds_in, uint64_t* out_lo,
                                                          uint64_t* out_hi, uint32_t* out_b,
                                                          uint32_t* out_e, uint32_t* out_cnt)
{
    __shared__ HilbertTables tb;
    __shared__ RootParams s_root;
    Bounds bounds = bounds_in;
    bounds.prepare(&s_root);
    __syncthreads();
    if (a.curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    const uint64_t i = (uint64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = i < a.m;
    int2 q = make_int2(0, 0);
    int32_t delta = -1;
    if (active) {
        q = reinterpret_cast<const int2*>(a.q)[i];
        delta = a.delta[i];
    }
    const bool ok = active && query_valid(q.x, q.y, delta);
    QueryRanges R;
    uint32_t b[4], e[4];
    query_bounds(bounds, a.curve, &tb, a.keys, a.n, ok, q.x, q.y, delta, R, b, e);
    if (!active) return;
    for (int k = 0; k < 4; ++k) {
        const bool u = k < R.cnt;
        if (out_lo) out_lo[4 * i + k] = u ? R.lo[k] : 1;
        if (out_hi) out_hi[4 * i + k] = u ? R.hi[k] : 0;
        if (out_b) out_b[4 * i + k] = b[k];
        if (out_e) out_e[4 * i + k] = e[k];
    }
    if (out_cnt) out_cnt[i] = (uint32_t)R.cnt;
}

__global__ void query_keys_kernel(const int32_t* __restrict__ q, uint64_t m, int curve, uint64_t* keys)
{
    __shared__ HilbertTables tb;
    if (curve == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
        const int2 c = reinterpret_cast<const int2*>(q)[i];
        keys[i] = point_in_domain(c.x, c.y) ? curve_key(curve, &tb, (uint32_t)c.x, (uint32_t)c.y) : ~0ull;
    }
}

__global__ void gather_u32_kernel(const uint32_t* __restrict__ src, const uint32_t* __restrict__ perm, uint64_t m,
                                  uint32_t* out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = src[perm[i]];
}

int persistent_grid(const void* fn)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * num_sms();
}

template <int WPL>
sfc_status launch_count_write(const QueryArgs& a, bool write, cudaStream_t st)
{
    if (!write) {
        int g = persistent_grid((const void*)count_kernel<WPL>);
        count_kernel<WPL><<<g, kThreads, 0, st>>>(a);
    } else {
        int g = persistent_grid((const void*)write_kernel<WPL>);
        write_kernel<WPL><<<g, kThreads, 0, st>>>(a);
    }
    count_launch();
    return launch_status();
}

}  // namespace

sfc_status launch_plan(const QueryArgs& a, const LearnedModelView* lm, cudaStream_t st)
{
    if (a.m == 0) return SFC_OK;
    const unsigned g = (unsigned)((a.m + kThreads - 1) / kThreads);
    if (lm) {
        LearnedBounds lb{lm->root, lm->leaf, lm->stats};
        plan_kernel<LearnedBounds><<<g, kThreads, 0, st>>>(a, lb);
    } else {
        plan_kernel<BinaryBounds><<<g, kThreads, 0, st>>>(a, BinaryBounds{});
    }
    count_launch();
    return launch_status();
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
    if (a.m == 0) return SFC_OK;
    const unsigned g = (unsigned)((a.m + kThreads - 1) / kThreads);
    if (lm) {
        LearnedBounds lb{lm->root, lm->leaf, lm->stats};
        ranges_kernel<LearnedBounds><<<g, kThreads, 0, st>>>(a, lb, lo, hi, b, e, cnt);
    } else {
        ranges_kernel<BinaryBounds><<<g, kThreads, 0, st>>>(a, BinaryBounds{}, lo, hi, b, e, cnt);
    }
    count_launch();
    return launch_status();
}

}  // namespace sfc
