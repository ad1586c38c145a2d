// Construction sort: stable LSD radix sort of (key, id) pairs by 60-bit curve key
// ("sort them once", Sec. 3.1.1), one-sweep style (Adinets & Merrill, 2022).
//
//   1. hist_kernel   one read of the input; keys are computed on the fly from the points
//                    (or read), and the 256-bin histograms of all eight 8-bit digits are
//                    accumulated at once.
//   2. plan_kernel   exclusive scan of each histogram (global digit offsets) and the pass
//                    plan: a digit that is the same for every key is skipped, and the
//                    source/destination of each remaining pass is chosen on the device, so
//                    the host never waits (the sort can be captured in a CUDA graph).
//   3. onesweep_kernel, once per digit: each block takes the next tile (4096 keys), ranks
//                    its keys per digit inside each warp with eight ballots (stable: item
//                    order, then lane order), combines warps in shared memory, publishes the
//                    tile's digit counts, reorders the tile in shared memory by digit (the
//                    values are loaded only then, so the ranking holds no registers for them),
//                    learns the tile's global digit offsets by decoupled look-back over earlier
//                    tiles and writes the tile out in contiguous runs.  Every tile but the last
//                    runs without per-key bounds checks, and index arithmetic is 32-bit.  The
//                    first pass reads the points (and computes keys again instead of storing
//                    them); the last pass writes the final arrays and also decodes each key
//                    back into its coordinates, which replaces a random gather xy[id] by a
//                    streaming write.
//
// Look-back words are tagged with a per-pass epoch, so stale words from earlier passes or
// sorts read as "not ready" and the buffer never needs clearing.  The epoch counter lives in
// device memory and is advanced by plan_kernel, so a sort replayed from a CUDA graph still
// gets fresh epochs.  Every wait is bounded (SFC_DEV_TIMEOUT).
#include "sfc_internal.cuh"

namespace sfc {

namespace {

constexpr int kBits = 8;
constexpr int kRadix = 1 << kBits;
constexpr int kPasses = 8;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// keys per thread of a tile, and resident blocks per SM (the register budget) of a pass
#ifndef SFC_SORT_ITEMS
#define SFC_SORT_ITEMS 16
#endif
#ifndef SFC_SORT_BLOCKS
#define SFC_SORT_BLOCKS 3
#endif
constexpr int kItems = SFC_SORT_ITEMS;
constexpr int kTile = kThreads * kItems;        // 4096 keys per tile
constexpr int kWarpSpan = 32 * kItems;          // 512 keys per warp

struct PassPlan {
    uint32_t active;
    uint32_t src;   // 0 = sort source, 1 = tmp 0, 2 = tmp 1
    uint32_t dst;   // 1 = tmp 0, 2 = tmp 1, 3 = final destination
    uint32_t pad;
};

struct Small {
    uint32_t hist[kPasses][kRadix];
    uint32_t offs[kPasses][kRadix];
    PassPlan plan[kPasses];
    uint32_t tile_ctr[kPasses];
    uint32_t epoch_base;   // epoch of pass 0 of this sort (pass p uses epoch_base + p)
};

constexpr uint64_t kFlagAgg = 1ull << 32;
constexpr uint64_t kFlagPrefix = 2ull << 32;

// word = value (32 bits) | flag (2 bits) << 32 | epoch (30 bits) << 34
__device__ __forceinline__ uint64_t lb_word(uint32_t value, uint64_t flag, uint32_t epoch)
{
    return (uint64_t)value | flag | ((uint64_t)epoch << 34);
}

template <int CURVE>
__device__ __forceinline__ uint64_t source_key(const SortSource& s, const HilbertTables* tb, uint64_t i)
{
    if (s.points) {
        int2 p = s.points[i];
        return curve_key(CURVE, tb, (uint32_t)p.x & (kSide - 1), (uint32_t)p.y & (kSide - 1));
    }
    return s.keys[i];
}

template <int CURVE>
__global__ void __launch_bounds__(kThreads) hist_kernel(SortSource src, uint64_t n, Small* sm,
                                                        uint32_t* status)
{
    __shared__ HilbertTables tb;
    __shared__ uint32_t h[kPasses][kRadix];
    if (CURVE == SFC_CURVE_HILBERT && src.points) hilbert_tables_init(&tb);
    for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    // run-length aggregation per digit position: constant digits cost one atomic per run
    uint32_t last[kPasses], run[kPasses];
#pragma unroll
    for (int p = 0; p < kPasses; ++p) { last[p] = 0; run[p] = 0; }
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * kThreads;
    // four elements of the grid stride per iteration, their loads issued together
    for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads + threadIdx.x; i0 < n; i0 += 4 * stride) {
        uint64_t kk[4];
        if (src.points) {
            int2 pt[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + u * stride;
                pt[u] = i < n ? __ldg(src.points + i) : make_int2(0, 0);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                bad |= i0 + u * stride < n && !point_in_domain(pt[u].x, pt[u].y);
                kk[u] = curve_key(CURVE, &tb, (uint32_t)pt[u].x & (kSide - 1), (uint32_t)pt[u].y & (kSide - 1));
            }
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint64_t i = i0 + u * stride;
                kk[u] = i < n ? __ldg(src.keys + i) : 0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u * stride >= n) break;
            const uint64_t k = kk[u];
#pragma unroll
            for (int p = 0; p < kPasses; ++p) {
                uint32_t d = (uint32_t)(k >> (kBits * p)) & (kRadix - 1);
                if (d != last[p] && run[p]) { atomicAdd(&h[p][last[p]], run[p]); run[p] = 0; }
                last[p] = d;
                ++run[p];
            }
        }
    }
#pragma unroll
    for (int p = 0; p < kPasses; ++p)
        if (run[p]) atomicAdd(&h[p][last[p]], run[p]);
    if (bad) set_status(status, SFC_DEV_BAD_POINT);
    __syncthreads();
    for (int i = threadIdx.x; i < kPasses * kRadix; i += kThreads) {
        uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&(&sm->hist[0][0])[i], c);
    }
}

// One block of 256 threads (thread = digit).
__global__ void __launch_bounds__(kRadix) plan_kernel(Small* sm, uint64_t n, uint32_t* epoch_ctr)
{
    if (threadIdx.x == 0) {
        // 30-bit epochs, never 0 (the value of a cleared word); wraps after 2^27 sorts
        uint32_t e = *epoch_ctr;
        if (e + kPasses >= (1u << 30)) e = 0;
        sm->epoch_base = e + 1;
        *epoch_ctr = e + kPasses;
    }
    __shared__ uint32_t s_const[kPasses];
    __shared__ uint32_t s_w[kRadix / 32];
    const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
    for (int p = 0; p < kPasses; ++p) {
        uint32_t c = sm->hist[p][d];
        uint32_t full = __syncthreads_or(c == (uint32_t)n);
        if (d == 0) s_const[p] = full;
        // block exclusive scan of the 256 counts
        uint32_t v = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) s_w[warp] = v;
        __syncthreads();
        uint32_t wo = 0;
        for (int w = 0; w < warp; ++w) wo += s_w[w];
        sm->offs[p][d] = wo + v - c;
        __syncthreads();
    }
    if (d == 0) {
        int act[kPasses], k = 0;
        for (int p = 0; p < kPasses; ++p)
            if (!s_const[p]) act[k++] = p;
        if (k == 0) act[k++] = 0;   // every digit constant: one pass still copies the data
        for (int p = 0; p < kPasses; ++p) sm->plan[p] = PassPlan{0, 0, 0, 0};
        for (int j = 0; j < k; ++j) {
            PassPlan pl;
            pl.active = 1;
            pl.src = j == 0 ? 0u : 1u + ((j - 1) & 1);
            pl.dst = j == k - 1 ? 3u : 1u + (j & 1);
            pl.pad = 0;
            sm->plan[act[j]] = pl;
        }
    }
}

struct PassArgs {
    SortSource src;
    uint64_t* tmp_keys[2];
    uint32_t* tmp_vals[2];
    SortDest dst;
    uint64_t* lookback;   // [tile][digit]
    Small* sm;
    uint64_t n;
    uint32_t* status;
    int pass;
};

constexpr size_t kSortSmem = sizeof(uint64_t) * kTile + sizeof(uint32_t) * kTile +
                             sizeof(uint32_t) * kWarps * kRadix + sizeof(uint32_t) * kRadix +
                             sizeof(uint32_t) * 2 * kWarps + sizeof(HilbertTables);

// One tile of a pass.  FULL: all kTile keys of the tile exist (every tile but the last), so
// no per-key bounds checks.  Index arithmetic is 32-bit (n < 2^32 - 1).
template <int CURVE, bool FULL>
__device__ __forceinline__ void sort_tile(const PassArgs& a, const PassPlan& pl, uint32_t epoch, uint32_t tile,
                                          unsigned char* smem)
{
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + kTile);
    uint32_t* s_hist = s_vals + kTile;                 // [warp][digit]
    uint32_t* s_gbase = s_hist + kWarps * kRadix;      // global start of the digit's run minus its tile-local start
    uint32_t* s_w = s_gbase + kRadix;                  // warp totals of the tile-local scan
    const HilbertTables* tb = reinterpret_cast<const HilbertTables*>(s_w + 2 * kWarps);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n = (uint32_t)a.n;
    const int shift = kBits * a.pass;
    const uint32_t tbase = tile * (uint32_t)kTile;
    const uint32_t wbase = tbase + (uint32_t)(warp * kWarpSpan);

    uint64_t key[kItems];
    uint32_t dr[kItems];   // digit << 16 | rank of the key among the warp's keys of that digit
    const uint64_t* kin = pl.src == 0 ? nullptr : a.tmp_keys[pl.src - 1];
    const uint32_t* vin = pl.src == 0 ? a.src.vals : a.tmp_vals[pl.src - 1];
    if (pl.src == 0) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)(i * 32 + lane);
            key[i] = (FULL || idx < n) ? source_key<CURVE>(a.src, tb, idx) : ~0ull;
        }
    } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)(i * 32 + lane);
            key[i] = (FULL || idx < n) ? kin[idx] : ~0ull;
        }
    }
    // ---- warp-level stable ranking by digit ----
    uint32_t* wh = s_hist + warp * kRadix;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
        const bool valid = FULL || wbase + (uint32_t)(i * 32 + lane) < n;
        const uint32_t d = (uint32_t)(key[i] >> shift) & (kRadix - 1);
        uint32_t peers = FULL ? 0xffffffffu : __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (int b = 0; b < kBits; ++b) {
            const uint32_t bb = __ballot_sync(0xffffffffu, (d >> b) & 1u);
            peers &= ((d >> b) & 1u) ? bb : ~bb;
        }
        const uint32_t before = __popc(peers & lt);
        const uint32_t basec = wh[d];
        __syncwarp();
        if (valid && before == 0) wh[d] = basec + __popc(peers);
        __syncwarp();
        dr[i] = d << 16 | (basec + before);
    }
    __syncthreads();
    // ---- combine warps: thread tid owns digit tid ----
    uint32_t tcount = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tcount += s_hist[w * kRadix + tid];
    uint64_t* lbw = a.lookback + (uint64_t)tile * kRadix + tid;
    atomicExch(reinterpret_cast<unsigned long long*>(lbw),
               lb_word(tcount, tile == 0 ? kFlagPrefix : kFlagAgg, epoch));
    // tile-local exclusive scan over digits; s_hist[w][d] becomes the tile-local position of
    // warp w's first key of digit d
    uint32_t local;
    {
        uint32_t v = tcount;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += t;
        }
        if (lane == 31) s_w[warp] = v;
        __syncthreads();
        uint32_t wo = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) wo += w < warp ? s_w[w] : 0u;
        local = wo + v - tcount;
        uint32_t run = local;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const uint32_t cw = s_hist[w * kRadix + tid];
            s_hist[w * kRadix + tid] = run;
            run += cw;
        }
    }
    __syncthreads();   // every warp's tile-local starts are in s_hist
    // ---- reorder the tile by digit in shared memory: it needs only tile-local positions, so
    // it runs before the look-back, and the values are loaded here rather than with the keys
    // (the ranking then holds no registers for them; 8.62 -> 7.29 ms for 10^8 keys) ----
    {
        uint32_t val[kItems];
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const uint32_t idx = wbase + (uint32_t)(i * 32 + lane);
            val[i] = (FULL || idx < n) ? (pl.src == 0 ? (vin ? vin[idx] : a.src.val_base + idx) : vin[idx]) : 0u;
        }
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            if (FULL || wbase + (uint32_t)(i * 32 + lane) < n) {
                const uint32_t lp = wh[dr[i] >> 16] + (dr[i] & 0xffffu);
                s_keys[lp] = key[i];
                s_vals[lp] = val[i];
            }
        }
    }
    // ---- decoupled look-back for digit tid ----
    uint32_t excl = 0;
    if (tile > 0) {
        int64_t t = (int64_t)tile - 1;
        uint32_t spins = 0;
        while (t >= 0) {
            const uint64_t w = *reinterpret_cast<volatile uint64_t*>(a.lookback + (uint64_t)t * kRadix + tid);
            const uint32_t ep = (uint32_t)(w >> 34);
            const uint32_t fl = (uint32_t)(w >> 32) & 3u;
            if (ep != epoch || fl == 0) {
                if (++spins > kSpinLimit) { set_status(a.status, SFC_DEV_TIMEOUT); break; }
                __nanosleep(32);   // not published yet: leave the issue slots to other warps
                continue;
            }
            excl += (uint32_t)w;
            if (fl == 2) break;
            --t;
        }
        atomicExch(reinterpret_cast<unsigned long long*>(lbw), lb_word(excl + tcount, kFlagPrefix, epoch));
    }
    // global position of tile-local position j of digit d: s_gbase[d] + j (mod 2^32)
    s_gbase[tid] = a.sm->offs[a.pass][tid] + excl - local;
    __syncthreads();
    // ---- write contiguous digit runs ----
    const uint32_t valid_n = FULL ? (uint32_t)kTile : min(n - tbase, (uint32_t)kTile);
    uint64_t* kout = pl.dst == 3 ? a.dst.keys : a.tmp_keys[pl.dst - 1];
    uint32_t* vout = pl.dst == 3 ? a.dst.vals : a.tmp_vals[pl.dst - 1];
    int2* xyout = pl.dst == 3 ? a.dst.xy : nullptr;
#pragma unroll 4
    for (uint32_t j = tid; j < valid_n; j += kThreads) {
        const uint64_t k = s_keys[j];
        const uint32_t d = (uint32_t)(k >> shift) & (kRadix - 1);
        const uint32_t g = s_gbase[d] + j;
        if (g >= n) continue;   // only after a look-back timeout (already flagged)
        kout[g] = k;
        vout[g] = s_vals[j];
        if (xyout) {
            uint32_t x, y;
            if (CURVE == SFC_CURVE_HILBERT) hilbert_decode(tb, k, x, y);
            else morton_decode(k, x, y);
            xyout[g] = make_int2((int)x, (int)y);
        }
    }
}

template <int CURVE>
__global__ void __launch_bounds__(kThreads, SFC_SORT_BLOCKS) onesweep_kernel(PassArgs a)
{
    const PassPlan pl = a.sm->plan[a.pass];
    if (!pl.active) return;
    const uint32_t epoch = a.sm->epoch_base + (uint32_t)a.pass;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ uint32_t s_tile;
    const int tid = threadIdx.x;
    uint32_t* s_hist = reinterpret_cast<uint32_t*>(smem + (sizeof(uint64_t) + sizeof(uint32_t)) * kTile);
    const bool need_tb = CURVE == SFC_CURVE_HILBERT &&
                         ((pl.src == 0 && a.src.points) || (pl.dst == 3 && a.dst.xy));
    if (need_tb) hilbert_tables_init(reinterpret_cast<HilbertTables*>(s_hist + kWarps * kRadix + kRadix + 2 * kWarps));
    for (int i = tid; i < kWarps * kRadix; i += kThreads) s_hist[i] = 0;
    if (tid == 0) s_tile = atomicAdd(&a.sm->tile_ctr[a.pass], 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if ((uint64_t)(tile + 1) * kTile <= a.n)
        sort_tile<CURVE, true>(a, pl, epoch, tile, smem);
    else
        sort_tile<CURVE, false>(a, pl, epoch, tile, smem);
}

}  // namespace

void release_sort_ws(SortWorkspace& ws, cudaStream_t st)
{
    for (int i = 0; i < 2; ++i) {
        ws.tmp_keys[i].release(st);
        ws.tmp_vals[i].release(st);
    }
    ws.lookback.release(st);
    ws.small.release(st);
    ws.epoch_dev.release(st);
}

sfc_status reserve_sort(SortWorkspace& ws, uint64_t n, cudaStream_t st)
{
    const uint64_t tiles = (n + kTile - 1) / kTile;
    for (int i = 0; i < 2; ++i) {
        SFC_TRY(ws.tmp_keys[i].ensure(n * sizeof(uint64_t), st));
        SFC_TRY(ws.tmp_vals[i].ensure(n * sizeof(uint32_t), st));
    }
    const size_t lb_bytes = tiles * kRadix * sizeof(uint64_t);
    if (!ws.epoch_dev.ptr) {
        SFC_TRY(ws.epoch_dev.ensure(sizeof(uint32_t), st));
        SFC_CUDA_TRY(cudaMemsetAsync(ws.epoch_dev.ptr, 0, sizeof(uint32_t), st));
    }
    if (lb_bytes > ws.lookback.bytes) {
        // new words start cleared; older epochs stay distinct from future ones
        SFC_TRY(ws.lookback.ensure(lb_bytes, st));
        SFC_CUDA_TRY(cudaMemsetAsync(ws.lookback.ptr, 0, ws.lookback.bytes, st));
    }
    SFC_TRY(ws.small.ensure(sizeof(Small), st));
    return SFC_OK;
}

sfc_status radix_sort(const SortSource& src, uint64_t n, const SortDest& dst, SortWorkspace& ws,
                      uint32_t* status, cudaStream_t st)
{
    if (n == 0) return SFC_OK;
    if (n >= 0xffffffffull) return SFC_ERR_INVALID;
    if (src.points && dst.curve != src.curve) return SFC_ERR_INVALID;
    const uint64_t tiles = (n + kTile - 1) / kTile;
    SFC_TRY(reserve_sort(ws, n, st));
    Small* sm = ws.small.as<Small>();
    SFC_CUDA_TRY(cudaMemsetAsync(sm, 0, sizeof(Small), st));

    const int curve = src.points ? src.curve : dst.curve;
    int hgrid = (int)((n + kThreads * 8 - 1) / (kThreads * 8));
    if (hgrid > num_sms() * 8) hgrid = num_sms() * 8;
    if (curve == SFC_CURVE_HILBERT)
        hist_kernel<SFC_CURVE_HILBERT><<<hgrid, kThreads, 0, st>>>(src, n, sm, status);
    else
        hist_kernel<SFC_CURVE_Z><<<hgrid, kThreads, 0, st>>>(src, n, sm, status);
    count_launch();
    SFC_TRY(launch_status());
    plan_kernel<<<1, kRadix, 0, st>>>(sm, n, ws.epoch_dev.as<uint32_t>());
    count_launch();
    SFC_TRY(launch_status());

    static bool attr_done[2] = {false, false};
    if (!attr_done[curve]) {
        if (curve == SFC_CURVE_HILBERT)
            SFC_CUDA_TRY(cudaFuncSetAttribute(onesweep_kernel<SFC_CURVE_HILBERT>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem));
        else
            SFC_CUDA_TRY(cudaFuncSetAttribute(onesweep_kernel<SFC_CURVE_Z>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSortSmem));
        attr_done[curve] = true;
    }
    PassArgs a;
    a.src = src;
    a.src.curve = curve;
    for (int i = 0; i < 2; ++i) {
        a.tmp_keys[i] = ws.tmp_keys[i].as<uint64_t>();
        a.tmp_vals[i] = ws.tmp_vals[i].as<uint32_t>();
    }
    a.dst = dst;
    a.lookback = ws.lookback.as<uint64_t>();
    a.sm = sm;
    a.n = n;
    a.status = status;
    for (int p = 0; p < kPasses; ++p) {
        a.pass = p;
        if (curve == SFC_CURVE_HILBERT)
            onesweep_kernel<SFC_CURVE_HILBERT><<<(unsigned)tiles, kThreads, kSortSmem, st>>>(a);
        else
            onesweep_kernel<SFC_CURVE_Z><<<(unsigned)tiles, kThreads, kSortSmem, st>>>(a);
        count_launch();
        SFC_TRY(launch_status());
    }
    return SFC_OK;
}

}  // namespace sfc
