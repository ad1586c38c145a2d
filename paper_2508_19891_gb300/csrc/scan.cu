// Exclusive prefix sum uint32[n] -> uint64[n + 1] in one pass over the data: single-pass
// scan with decoupled look-back (Merrill & Garland, 2016).  Used to turn per-query chunk
// counts into chunk bases and per-query hit counts into output offsets.
//
// Each block takes the next tile index from a counter (so a tile's predecessors are
// already running and will publish), reduces its tile, publishes the aggregate, reads the
// predecessors' words a warp at a time until it meets an inclusive prefix, then publishes
// its own inclusive prefix and writes its outputs.  A word packs a 2-bit flag with a
// 62-bit sum.  The wait on a predecessor is bounded: past kSpinLimit reads it sets
// SFC_DEV_TIMEOUT and continues with the partial sum.
#include <cuda.h>

#include <mutex>

#include "sfc_internal.cuh"

namespace sfc {

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;
constexpr uint64_t kFlagAgg = 1ull << 62;
constexpr uint64_t kFlagPrefix = 2ull << 62;
constexpr uint64_t kValueMask = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v)
{
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane_id() >= o) v += t;
    }
    return v;
}

__global__ void __launch_bounds__(kThreads)
scan_kernel(const uint32_t* __restrict__ in, uint64_t n, uint64_t* __restrict__ out,
            uint64_t* flags /* [0] = tile counter, [1 + t] = tile words */, uint32_t* status,
            int vec)
{
    __shared__ uint32_t s_tile;
    __shared__ uint64_t s_warp[kThreads / 32];
    __shared__ uint64_t s_excl;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(reinterpret_cast<unsigned long long*>(flags), 1ull);
    __syncthreads();
    const uint64_t tile = s_tile;
    const uint64_t base = tile * kTile + (uint64_t)tid * kItems;

    uint32_t v[kItems];
    if (vec && base + kItems <= n) {
        const uint4* p = reinterpret_cast<const uint4*>(in + base);
#pragma unroll
        for (int j = 0; j < kItems / 4; ++j) {
            uint4 u = __ldcs(p + j);
            v[4 * j] = u.x; v[4 * j + 1] = u.y; v[4 * j + 2] = u.z; v[4 * j + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kItems; ++j) v[j] = (base + j < n) ? in[base + j] : 0u;
    }
    uint64_t tsum = 0;
#pragma unroll
    for (int j = 0; j < kItems; ++j) tsum += v[j];

    uint64_t incl = warp_incl_scan(tsum);
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kThreads / 32 ? s_warp[lane] : 0;
        uint64_t wi = warp_incl_scan(w);
        if (lane < kThreads / 32) s_warp[lane] = wi - w;   // exclusive warp offsets
        uint64_t total = __shfl_sync(0xffffffffu, wi, 31);
        // ---- decoupled look-back ----
        uint64_t* words = flags + 1;
        uint64_t excl = 0;
        if (tile == 0) {
            if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(words), kFlagPrefix | total);
        } else {
            if (lane == 0) atomicExch(reinterpret_cast<unsigned long long*>(words + tile), kFlagAgg | total);
            int64_t t = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (true) {
                int64_t idx = t - lane;
                uint64_t wv = kFlagPrefix;   // lanes before tile 0 act as a zero prefix
                if (idx >= 0) wv = *reinterpret_cast<volatile uint64_t*>(words + idx);
                uint32_t notready = __ballot_sync(0xffffffffu, (wv >> 62) == 0);
                if (notready) {
                    if (++spins > kSpinLimit) {
                        if (lane == 0) set_status(status, SFC_DEV_TIMEOUT);
                        break;
                    }
                    continue;
                }
                uint32_t pref = __ballot_sync(0xffffffffu, (wv >> 62) == 2);
                uint64_t val = (idx >= 0) ? (wv & kValueMask) : 0;
                if (pref) {
                    int first = __ffs(pref) - 1;          // nearest predecessor with a prefix
                    if (lane > first) val = 0;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
                excl += val;
                if (pref) break;
                t -= 32;
            }
            if (lane == 0)
                atomicExch(reinterpret_cast<unsigned long long*>(words + tile), kFlagPrefix | (excl + total));
        }
        if (lane == 0) s_excl = excl;
    }
    __syncthreads();
    uint64_t run = s_excl + s_warp[warp] + (incl - tsum);
    uint64_t o[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) { o[j] = run; run += v[j]; }
    if (vec && base + kItems <= n) {
        ulonglong2* q = reinterpret_cast<ulonglong2*>(out + base);
#pragma unroll
        for (int j = 0; j < kItems / 2; ++j) q[j] = make_ulonglong2(o[2 * j], o[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (base + j < n) out[base + j] = o[j];
    }
    // the thread holding element n - 1 also writes the total
    if (base < n && base + kItems >= n) out[n] = run;
}

}  // namespace

sfc_status reserve_scan(ScanWorkspace& ws, uint64_t n, cudaStream_t st)
{
    const uint64_t tiles = (n + kTile - 1) / kTile;
    return ws.flags.ensure((tiles + 1) * sizeof(uint64_t), st);
}

sfc_status exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, ScanWorkspace& ws,
                              uint32_t* status, cudaStream_t st)
{
    if (n == 0) {
        SFC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
        return SFC_OK;
    }
    uint64_t tiles = (n + kTile - 1) / kTile;
    if (tiles > 0x7fffffffull) return SFC_ERR_INVALID;
    SFC_TRY(ws.flags.ensure((tiles + 1) * sizeof(uint64_t), st));
    SFC_CUDA_TRY(cudaMemsetAsync(ws.flags.ptr, 0, (tiles + 1) * sizeof(uint64_t), st));
    int vec = ((((uintptr_t)in) & 15) == 0) && ((((uintptr_t)out) & 15) == 0);
    scan_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(in, n, out, ws.flags.as<uint64_t>(), status, vec);
    count_launch();
    return launch_status();
}

// The standalone scan (sfc_exclusive_scan): its own workspace with a status word in front
// (word 0 status, word 1 tile counter, then the tiles' words), read back once the kernel is
// done so that a look-back wait that gave up is reported by the call itself.
sfc_status exclusive_scan_standalone(const uint32_t* in, uint64_t n, uint64_t* out, cudaStream_t st)
{
    if (n == 0) {
        SFC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), st));
        return SFC_OK;
    }
    const uint64_t tiles = (n + kTile - 1) / kTile;
    if (tiles > 0x7fffffffull) return SFC_ERR_INVALID;
    DevBuf ws;
    SFC_TRY(ws.ensure((tiles + 2) * sizeof(uint64_t), st));
    uint64_t* words = ws.as<uint64_t>();
    sfc_status s = SFC_OK;
    uint32_t bits = 0;
    if (cudaMemsetAsync(words, 0, (tiles + 2) * sizeof(uint64_t), st) != cudaSuccess) s = SFC_ERR_CUDA;
    if (s == SFC_OK) {
        const int vec = ((((uintptr_t)in) & 15) == 0) && ((((uintptr_t)out) & 15) == 0);
        scan_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(in, n, out, words + 1, reinterpret_cast<uint32_t*>(words),
                                                          vec);
        count_launch();
        s = launch_status();
    }
    if (s == SFC_OK && cudaMemcpyAsync(&bits, words, sizeof(bits), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        s = SFC_ERR_CUDA;
    ws.release(st);
    if (cudaStreamSynchronize(st) != cudaSuccess && s == SFC_OK) s = SFC_ERR_CUDA;
    if (s == SFC_OK && (bits & SFC_DEV_TIMEOUT)) s = SFC_ERR_TIMEOUT;
    return s;
}

// ------------------------------------------------------------------------------------
// Scan without allocation (sfc_exclusive_scan_noalloc).
//
// For callers that must not allocate device memory.  Its scratch lives in a file-scope
// device array of fixed size instead of a cudaMallocAsync buffer: word 0 is a status word
// (SFC_DEV_TIMEOUT when a look-back wait of the last call gave up), word 1 the tile counter,
// words 2 .. 2 + tiles the tiles' look-back words.  Host code cannot use the array's name as a
// device address (it is a host-side stand-in), so the address is looked up with
// cudaGetSymbolAddress while the device is current, once per device and CUDA context: a
// context that was torn down and created again (cudaDeviceReset) gets a new id, and the
// address is looked up again for it.
// ------------------------------------------------------------------------------------
constexpr uint64_t kNoAllocMaxTiles = 16384;                       // 131 KB of words
constexpr uint64_t kNoAllocMaxItems = kNoAllocMaxTiles * kTile;     // 67,108,864 elements
static __device__ __align__(256) uint64_t g_noalloc_scan_words[kNoAllocMaxTiles + 2];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
struct NoAllocSlot {
    uint64_t* words = nullptr;
    unsigned long long ctx_id = 0;   // id of the context the address belongs to (0: unknown)
};
NoAllocSlot g_noalloc[kMaxDevices];

// Id of the calling thread's current CUDA context (ids are never reused within a process);
// false if it cannot be had.  The two driver calls are reached through the runtime's
// entry-point lookup, so the library does not link the driver library itself.
bool current_context_id(unsigned long long* id)
{
    using GetCurrentFn = CUresult (*)(CUcontext*);
    using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {   // under g_noalloc_mu
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", reinterpret_cast<void**>(&get_current), 12000,
                                             cudaEnableDefault, &q1) != cudaSuccess || q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", reinterpret_cast<void**>(&get_id), 12000,
                                             cudaEnableDefault, &q2) != cudaSuccess || q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
        looked_up = true;
    }
    if (!get_current || !get_id) return false;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of the array for the current device and context (looked up on first use).
sfc_status noalloc_words(uint64_t** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SFC_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    NoAllocSlot& slot = g_noalloc[dev];
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (!slot.words || (have_id && id != slot.ctx_id)) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_words);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return SFC_ERR_CUDA;
        }
        slot.words = static_cast<uint64_t*>(p);
        // the lookup created the context if there was none yet
        slot.ctx_id = (have_id || current_context_id(&id)) ? id : 0;
    }
    *out = slot.words;
    return SFC_OK;
}

}  // namespace

}  // namespace sfc

extern "C" sfc_status sfc_exclusive_scan_noalloc(const uint32_t* d_in, uint64_t n, uint64_t* d_out, void* stream)
{
    using namespace sfc;
    if (!d_out || (n && !d_in)) return SFC_ERR_INVALID;
    if (n > kNoAllocMaxItems) return SFC_ERR_CAPACITY;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* words = nullptr;
    SFC_TRY(noalloc_words(&words));
    const uint64_t tiles = (n + kTile - 1) / kTile;
    // the status word, the tile counter and the look-back words of this call start at zero
    SFC_CUDA_TRY(cudaMemsetAsync(words, 0, (tiles + 2) * sizeof(uint64_t), st));
    if (n == 0) {
        SFC_CUDA_TRY(cudaMemsetAsync(d_out, 0, sizeof(uint64_t), st));
        return SFC_OK;
    }
    const int vec = ((((uintptr_t)d_in) & 15) == 0) && ((((uintptr_t)d_out) & 15) == 0);
    scan_kernel<<<(unsigned)tiles, kThreads, 0, st>>>(d_in, n, d_out, words + 1, reinterpret_cast<uint32_t*>(words),
                                                      vec);
    count_launch();
    return launch_status();
}

extern "C" sfc_status sfc_exclusive_scan_noalloc_status(uint32_t* h_bits, void* stream)
{
    using namespace sfc;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    uint64_t* words = nullptr;
    SFC_TRY(noalloc_words(&words));
    uint32_t bits = 0;
    SFC_CUDA_TRY(cudaMemcpyAsync(&bits, words, sizeof(bits), cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_bits) *h_bits = bits;
    return (bits & SFC_DEV_TIMEOUT) ? SFC_ERR_TIMEOUT : SFC_OK;
}
