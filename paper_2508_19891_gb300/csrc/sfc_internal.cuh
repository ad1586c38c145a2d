// Internal declarations shared by the library's translation units (device helpers, the
// index structure, launch helpers).  Not part of the public ABI (include/sfc.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/sfc.h"

namespace sfc {

constexpr int kOmega = 30;                       // bits per coordinate
constexpr uint32_t kSide = 1u << kOmega;         // domain [0, 2^30)
constexpr uint64_t kKeyMax = (1ull << 60) - 1;   // largest 60-bit key

// ------------------------------------------------------------------------------------
// Launch bookkeeping
// ------------------------------------------------------------------------------------
extern std::atomic<uint64_t> g_launches;
inline void count_launch(uint64_t k = 1) { g_launches.fetch_add(k, std::memory_order_relaxed); }

#define SFC_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            return e_ == cudaErrorMemoryAllocation ? SFC_ERR_OOM : SFC_ERR_CUDA; \
        }                                                    \
    } while (0)

#define SFC_TRY(expr)                         \
    do {                                      \
        sfc_status s_ = (expr);               \
        if (s_ != SFC_OK) return s_;          \
    } while (0)

inline sfc_status launch_status()
{
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) return SFC_OK;
    return e == cudaErrorMemoryAllocation ? SFC_ERR_OOM : SFC_ERR_CUDA;
}

int num_sms();   // SM count of the current device (cached per device)

// First bit of depth t in the early-termination bitmap (depths stored one after another).
__host__ __device__ __forceinline__ uint64_t occupancy_level_start(int t)
{
    return (((uint64_t)1 << (2 * t)) - 1) / 3;
}

// Device allocation.  Memory comes from the caller's sfc_allocator while a call on an index
// built with one is running on this thread (AllocScope, set by every entry point that takes
// an index), else from the device's stream-ordered pool (cudaMallocAsync).  Each allocation
// remembers where it came from (*owner), and is given back there.
extern thread_local const sfc_allocator* t_alloc;

class AllocScope {
public:
    explicit AllocScope(const sfc_allocator* a) : prev_(t_alloc) { t_alloc = a; }
    ~AllocScope() { t_alloc = prev_; }
    AllocScope(const AllocScope&) = delete;
    AllocScope& operator=(const AllocScope&) = delete;
private:
    const sfc_allocator* prev_;
};

sfc_status dev_alloc(void** p, size_t bytes, cudaStream_t st, const sfc_allocator** owner);
void dev_free(void* p, size_t bytes, cudaStream_t st, const sfc_allocator* owner);

// A grow-only device buffer.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    const sfc_allocator* owner = nullptr;   // allocator the memory came from (NULL: the pool)
    sfc_status ensure(size_t need, cudaStream_t st)
    {
        if (need <= bytes) return SFC_OK;
        if (ptr) dev_free(ptr, bytes, st, owner);
        ptr = nullptr;
        bytes = 0;
        size_t nb = need + need / 8 + 256;
        SFC_TRY(dev_alloc(&ptr, nb, st, &owner));
        bytes = nb;
        return SFC_OK;
    }
    void release(cudaStream_t st)
    {
        if (ptr) dev_free(ptr, bytes, st, owner);
        ptr = nullptr;
        bytes = 0;
    }
    template <class T>
    T* as() const { return reinterpret_cast<T*>(ptr); }
};

// ------------------------------------------------------------------------------------
// Curve keys on the device
// ------------------------------------------------------------------------------------

// Z-curve (Alg. 2): x's bit i goes to key bit 2i, y's bit i to key bit 2i + 1.  Done with
// the magic-mask spread instead of a per-bit loop: each step doubles the gap between
// groups of bits.
__device__ __forceinline__ uint64_t spread_bits(uint32_t v)
{
    uint64_t x = v;
    x = (x | (x << 16)) & 0x0000FFFF0000FFFFull;
    x = (x | (x << 8)) & 0x00FF00FF00FF00FFull;
    x = (x | (x << 4)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}

__device__ __forceinline__ uint32_t gather_bits(uint64_t x)
{
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0F0F0F0F0F0F0F0Full;
    x = (x | (x >> 4)) & 0x00FF00FF00FF00FFull;
    x = (x | (x >> 8)) & 0x0000FFFF0000FFFFull;
    x = (x | (x >> 16)) & 0x00000000FFFFFFFFull;
    return (uint32_t)x;
}

__device__ __forceinline__ uint64_t morton_key(uint32_t x, uint32_t y)
{
    return spread_bits(x) | (spread_bits(y) << 1);
}

__device__ __forceinline__ void morton_decode(uint64_t k, uint32_t& x, uint32_t& y)
{
    x = gather_bits(k);
    y = gather_bits(k >> 1);
}

// Z curve in 3-D (Alg. 2 with a third coordinate): bit i of x, y, z goes to key bit 3i, 3i + 1,
// 3i + 2; 21 bits per coordinate give 63-bit keys.  Magic-mask spread: each step splits the
// bit groups of the previous one and moves them apart, until single bits sit 3 apart.
constexpr int kOmega3 = 21;
constexpr uint32_t kSide3 = 1u << kOmega3;

__host__ __device__ __forceinline__ uint64_t spread3_bits(uint32_t v)
{
    uint64_t x = v & (kSide3 - 1);
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__host__ __device__ __forceinline__ uint32_t gather3_bits(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x | (x >> 8)) & 0x001F0000FF0000FFull;
    x = (x | (x >> 16)) & 0x001F00000000FFFFull;
    x = (x | (x >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)x;
}

__host__ __device__ __forceinline__ uint64_t morton3_key(uint32_t x, uint32_t y, uint32_t z)
{
    return spread3_bits(x) | (spread3_bits(y) << 1) | (spread3_bits(z) << 2);
}

__device__ __forceinline__ bool point3_in_domain(int32_t x, int32_t y, int32_t z)
{
    return (uint32_t)x < kSide3 && (uint32_t)y < kSide3 && (uint32_t)z < kSide3;
}

// Hilbert curve as a finite-state machine.  The orientation of the sub-square being
// refined is one of four symmetries of the square, generated by T (exchange x and y) and
// R (complement both coordinates inside the sub-square); they commute, so a state is two
// bits: bit 0 = T applied, bit 1 = R applied.  At one level, with the raw coordinate bits
// (bx, by) and the state (t, r):
//   (u, v) = (bx ^ r, by ^ r), exchanged if t     -- the bits in the base orientation
//   digit  = 0 for (0,0), 1 for (0,1), 2 for (1,1), 3 for (1,0)
//   if v == 0: t ^= 1, and also r ^= 1 if u == 1  -- lower quadrants flip orientation
// Four levels at a time are tabulated: enc[state][x nibble][y nibble] -> 8 key bits and
// the next state, dec[state][8 key bits] -> both nibbles and the next state.
__device__ __forceinline__ void hilbert_step(int& st, int bx, int by, int& digit)
{
    int t = st & 1, r = st >> 1;
    int u = bx ^ r, v = by ^ r;
    if (t) { int w = u; u = v; v = w; }
    digit = u ? (v ? 2 : 3) : (v ? 1 : 0);
    if (!v) { t ^= 1; if (u) r ^= 1; }
    st = t | (r << 1);
}

__device__ __forceinline__ void hilbert_unstep(int& st, int digit, int& bx, int& by)
{
    int t = st & 1, r = st >> 1;
    int u = (digit == 2 || digit == 3) ? 1 : 0;
    int v = (digit == 1 || digit == 2) ? 1 : 0;
    int a = t ? v : u, b = t ? u : v;
    bx = a ^ r;
    by = b ^ r;
    if (!v) { t ^= 1; if (u) r ^= 1; }
    st = t | (r << 1);
}

struct HilbertTables {
    uint16_t enc[4 * 256];   // [state<<8 | xn<<4 | yn] -> digits8 | next_state << 8
    uint16_t dec[4 * 256];   // [state<<8 | digits8] -> xn | yn << 4 | next_state << 8
};

// Fills the tables in shared memory; every thread of the block must call it (ends with a
// barrier).
__device__ __forceinline__ void hilbert_tables_init(HilbertTables* tb)
{
    for (int e = threadIdx.x; e < 1024; e += blockDim.x) {
        int st0 = e >> 8;
        {   // encode entry: x nibble = bits 7..4 of e, y nibble = bits 3..0
            int xn = (e >> 4) & 15, yn = e & 15, st = st0, d8 = 0;
            for (int b = 3; b >= 0; --b) {
                int dg;
                hilbert_step(st, (xn >> b) & 1, (yn >> b) & 1, dg);
                d8 = (d8 << 2) | dg;
            }
            tb->enc[e] = (uint16_t)(d8 | (st << 8));
        }
        {   // decode entry: 8 key bits = e & 255
            int d8 = e & 255, st = st0, xn = 0, yn = 0;
            for (int b = 3; b >= 0; --b) {
                int bx, by;
                hilbert_unstep(st, (d8 >> (2 * b)) & 3, bx, by);
                xn |= bx << b;
                yn |= by << b;
            }
            tb->dec[e] = (uint16_t)(xn | (yn << 4) | (st << 8));
        }
    }
    __syncthreads();
}

// Coordinates are taken as 32-bit values whose top two bits are 0; the two leading levels
// both select the lower-left quadrant and apply T twice, so the state is back to the start
// and the 64-bit result equals the 60-bit label at w = 30.
__device__ __forceinline__ uint64_t hilbert_key(const HilbertTables* tb, uint32_t x, uint32_t y)
{
    uint64_t k = 0;
    int st = 0;
#pragma unroll
    for (int s = 28; s >= 0; s -= 4) {
        uint32_t e = tb->enc[(st << 8) | (((x >> s) & 15u) << 4) | ((y >> s) & 15u)];
        k = (k << 8) | (e & 255u);
        st = (int)(e >> 8);
    }
    return k;
}

__device__ __forceinline__ void hilbert_decode(const HilbertTables* tb, uint64_t k, uint32_t& x,
                                               uint32_t& y)
{
    uint32_t xx = 0, yy = 0;
    int st = 0;
#pragma unroll
    for (int s = 56; s >= 0; s -= 8) {
        uint32_t e = tb->dec[(st << 8) | (uint32_t)((k >> s) & 255u)];
        xx = (xx << 4) | (e & 15u);
        yy = (yy << 4) | ((e >> 4) & 15u);
        st = (int)(e >> 8);
    }
    x = xx;
    y = yy;
}

__device__ __forceinline__ uint64_t curve_key(int curve, const HilbertTables* tb, uint32_t x,
                                              uint32_t y)
{
    return curve == SFC_CURVE_HILBERT ? hilbert_key(tb, x, y) : morton_key(x, y);
}

__device__ __forceinline__ bool point_in_domain(int32_t x, int32_t y)
{
    return (uint32_t)x < kSide && (uint32_t)y < kSide;
}

// ------------------------------------------------------------------------------------
// Small device utilities
// ------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ void set_status(uint32_t* st, uint32_t bit)
{
    if (st) atomicOr(st, bit);
}

// Bounded spin limit for every device-side wait (look-back, queues).  A wait that reaches
// it sets SFC_DEV_TIMEOUT and gives up instead of hanging the GPU.
constexpr uint32_t kSpinLimit = 1u << 22;

// ------------------------------------------------------------------------------------
// Learned bounds: model layout and the single fp32 predict path
// ------------------------------------------------------------------------------------
// Root, on x = key / 2^60 in [0, 1), one of:
//   piecewise linear (default): K = 256 knots at x = k / K (the key ranges of the 256
//     level-4 quadtree cells), heights h_0 = c, h_{k+1} = h_k + exp(d_k) -- monotone by
//     construction; the initial parameters give f(x) = x;
//   MLP: f(x) = c + sum_k A_k * sigmoid(B_k * x + b_k), A_k = exp(alpha_k), B_k = exp(beta_k).
// Leaf j = floor(f * J) clamped.  Leaf: predicted position first_j + floor(slope_j *
// (key - base_j) + icpt_j); the true lower_bound of every key routed to j lies in
// [pred + err_lo_j, pred + err_hi_j + 1] intersected with [first_j, end_j].  Training-time
// error measurement and query-time prediction both call the functions below, built with
// explicit round-to-nearest intrinsics so no contraction choice can make the two disagree.
constexpr int kHidden = 16;
constexpr int kKnots = 256;
constexpr int kRootPwl = 0;
constexpr int kRootMlp = 1;

// Each leaf also keeps a fence: the keys at kFence equally spaced positions of its range
// (position first + s * (end - first) / kFence, s = 0 .. kFence - 1), one 128-byte line, so
// a search first brackets its target between two fence keys.
constexpr int kFence = 16;
// ... and a fine fence: the keys at kFenceFine equally spaced positions (first + floor(r *
// (end - first) / kFenceFine)), kFence lines of kFence keys; coarse fence key s is fine fence
// key kFence * s, so once the coarse line has bracketed the target between coarse keys s - 1
// and s, fine line s - 1 narrows it to 1 / kFenceFine of the leaf.
constexpr int kFenceFine = kFence * kFence;

struct LeafParams {          // 32 bytes, one sector
    uint64_t base;           // smallest key routed to the leaf
    uint32_t first;          // first position routed to the leaf
    uint32_t end;            // one past the last position routed to the leaf
    float slope;
    float icpt;
    int32_t err_lo;
    int32_t err_hi;
};

struct RootParams {          // derived from the trained parameters
    int kind;
    int leaves;
    float c;
    float A[kHidden];
    float B[kHidden];
    float b[kHidden];
    float h[kKnots + 1];
};

__device__ __forceinline__ float key_to_x(uint64_t key)
{
    return __fmul_rn(__ull2float_rn(key), 8.67361737988403547e-19f /* 2^-60 */);
}

__device__ __forceinline__ float root_eval(const RootParams& r, uint64_t key)
{
    const float x = key_to_x(key);
    if (r.kind == kRootPwl) {
        const float s = __fmul_rn(x, (float)kKnots);
        int k = (int)s;
        k = k < 0 ? 0 : (k > kKnots - 1 ? kKnots - 1 : k);
        const float t = __fsub_rn(s, (float)k);
        return __fmaf_rn(__fsub_rn(r.h[k + 1], r.h[k]), t, r.h[k]);
    }
    float f = r.c;
#pragma unroll
    for (int k = 0; k < kHidden; ++k) {
        const float z = __fmaf_rn(r.B[k], x, r.b[k]);
        const float h = __frcp_rn(__fadd_rn(1.0f, __expf(-z)));
        f = __fmaf_rn(r.A[k], h, f);
    }
    return f;
}

__device__ __forceinline__ int route_leaf(const RootParams& r, uint64_t key)
{
    float s = __fmul_rn(root_eval(r, key), (float)r.leaves);
    int j = (s >= 0.0f) ? ((s < (float)r.leaves) ? (int)s : r.leaves - 1) : 0;   // NaN -> 0
    return j;
}

__device__ __forceinline__ int64_t leaf_predict(const LeafParams& lp, uint64_t key)
{
    float u = __ll2float_rn((long long)(key - lp.base));
    float p = __fmaf_rn(lp.slope, u, lp.icpt);
    p = fminf(fmaxf(p, -2.0e9f), 2.0e9f);
    return (int64_t)lp.first + (int64_t)floorf(p);
}

// ------------------------------------------------------------------------------------
// Host entry points implemented in the various .cu files
// ------------------------------------------------------------------------------------

// keygen.cu
sfc_status launch_keys(const int2* pts, uint64_t n, int curve, uint64_t* keys, uint32_t* status,
                       cudaStream_t st);
sfc_status launch_decode(const uint64_t* keys, uint64_t n, int curve, int2* pts, cudaStream_t st);
// 3-D Z keys of int32[n][3] points (bad coordinates set SFC_DEV_BAD_POINT), and their inverse
// into int4 (x, y, z, 0) records
sfc_status launch_keys3(const int32_t* pts, uint64_t n, uint64_t* keys, uint32_t* status, cudaStream_t st);
sfc_status launch_decode3(const uint64_t* keys, uint64_t n, int4* xyz, cudaStream_t st);

// scan.cu: exclusive scan of uint32 (or a uint32 view) into uint64[n+1].
struct ScanWorkspace {
    DevBuf flags;
};
sfc_status exclusive_scan_u32(const uint32_t* in, uint64_t n, uint64_t* out, ScanWorkspace& ws,
                              uint32_t* status, cudaStream_t st);
sfc_status reserve_scan(ScanWorkspace& ws, uint64_t n, cudaStream_t st);
// the same with its own workspace and status word; synchronises st and returns
// SFC_ERR_TIMEOUT if a look-back wait gave up
sfc_status exclusive_scan_standalone(const uint32_t* in, uint64_t n, uint64_t* out, cudaStream_t st);

// radix.cu: the build sort.
struct SortWorkspace {
    DevBuf tmp_keys[2];
    DevBuf tmp_vals[2];
    DevBuf lookback;      // per (tile, digit) look-back words, epoch-tagged
    DevBuf small;         // histograms, digit offsets, pass plan, tile counters
    DevBuf epoch_dev;     // device epoch counter (advanced on the device per sort)
};
// Source of the keys to sort: either points (keys computed on the fly for `curve`) or
// a key array.  Values: `vals_in` or, when NULL, val_base + index.
struct SortSource {
    const int2* points = nullptr;
    const uint64_t* keys = nullptr;
    const uint32_t* vals = nullptr;
    uint32_t val_base = 0;
    int curve = SFC_CURVE_Z;
};
struct SortDest {
    uint64_t* keys = nullptr;
    uint32_t* vals = nullptr;
    int2* xy = nullptr;   // optional: coordinates decoded from the sorted keys
    int curve = SFC_CURVE_Z;
};
sfc_status radix_sort(const SortSource& src, uint64_t n, const SortDest& dst, SortWorkspace& ws,
                      uint32_t* status, cudaStream_t st);
void release_sort_ws(SortWorkspace& ws, cudaStream_t st);
sfc_status reserve_sort(SortWorkspace& ws, uint64_t n, cudaStream_t st);

}  // namespace sfc
