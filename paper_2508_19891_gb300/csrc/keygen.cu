// Curve keys and their inverse for whole arrays (the key-generation step of the build,
// Sec. 3.1.1 "compute the bit strings pi(A[i])"; Z-curve by Alg. 2, Hilbert per Sec. 2.1).
//
// HBM-bound elementwise kernels: 8 B read + 8 B written per point.  Each thread handles
// two points per iteration through 16-byte vector accesses; the grid is a multiple of the
// SM count and strides over the array.
#include "sfc_internal.cuh"

namespace sfc {

namespace {

constexpr int kThreads = 256;

template <int CURVE>
__global__ void __launch_bounds__(kThreads) keys_kernel(const int2* __restrict__ pts, uint64_t n,
                                                        uint64_t* __restrict__ keys,
                                                        uint32_t* status, int vec)
{
    __shared__ HilbertTables tb;
    if (CURVE == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    if (!vec) {   // operands not 16-byte aligned: one point per thread
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        bool bad = false;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            int2 v = pts[i];
            bad |= !point_in_domain(v.x, v.y);
            keys[i] = curve_key(CURVE, &tb, (uint32_t)v.x & (kSide - 1), (uint32_t)v.y & (kSide - 1));
        }
        if (bad) set_status(status, SFC_DEV_BAD_POINT);
        return;
    }
    const uint64_t pairs = n / 2;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    const int4* p4 = reinterpret_cast<const int4*>(pts);
    ulonglong2* k2 = reinterpret_cast<ulonglong2*>(keys);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += stride) {
        int4 v = __ldcs(p4 + i);
        bad |= !point_in_domain(v.x, v.y) || !point_in_domain(v.z, v.w);
        ulonglong2 o;
        o.x = curve_key(CURVE, &tb, (uint32_t)v.x & (kSide - 1), (uint32_t)v.y & (kSide - 1));
        o.y = curve_key(CURVE, &tb, (uint32_t)v.z & (kSide - 1), (uint32_t)v.w & (kSide - 1));
        __stcs(k2 + i, o);
    }
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
        int2 v = pts[n - 1];
        bad |= !point_in_domain(v.x, v.y);
        keys[n - 1] = curve_key(CURVE, &tb, (uint32_t)v.x & (kSide - 1), (uint32_t)v.y & (kSide - 1));
    }
    if (bad) set_status(status, SFC_DEV_BAD_POINT);
}

template <int CURVE>
__global__ void __launch_bounds__(kThreads) decode_kernel(const uint64_t* __restrict__ keys,
                                                          uint64_t n, int2* __restrict__ pts)
{
    __shared__ HilbertTables tb;
    if (CURVE == SFC_CURVE_HILBERT) hilbert_tables_init(&tb);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t k = keys[i];
        uint32_t x, y;
        if (CURVE == SFC_CURVE_HILBERT) hilbert_decode(&tb, k, x, y);
        else morton_decode(k, x, y);
        pts[i] = make_int2((int)x, (int)y);
    }
}

// 3-D Z keys: points are 12-byte records, read as three 32-bit words (consecutive threads read
// consecutive records, so a warp's loads cover 384 contiguous bytes).
__global__ void __launch_bounds__(kThreads) keys3_kernel(const int32_t* __restrict__ pts, uint64_t n,
                                                         uint64_t* __restrict__ keys, uint32_t* status)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t x = __ldg(pts + 3 * i), y = __ldg(pts + 3 * i + 1), z = __ldg(pts + 3 * i + 2);
        bad |= !point3_in_domain(x, y, z);
        keys[i] = morton3_key((uint32_t)x, (uint32_t)y, (uint32_t)z);
    }
    if (bad) set_status(status, SFC_DEV_BAD_POINT);
}

__global__ void __launch_bounds__(kThreads) decode3_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                           int4* __restrict__ xyz)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        xyz[i] = make_int4((int)gather3_bits(k), (int)gather3_bits(k >> 1), (int)gather3_bits(k >> 2), 0);
    }
}

int grid_for(uint64_t work, int per_block)
{
    uint64_t want = (work + per_block - 1) / per_block;
    uint64_t cap = (uint64_t)num_sms() * 8;
    if (want > cap) want = cap;
    if (want < 1) want = 1;
    return (int)want;
}

}  // namespace

sfc_status launch_keys(const int2* pts, uint64_t n, int curve, uint64_t* keys, uint32_t* status,
                       cudaStream_t st)
{
    if (n == 0) return SFC_OK;
    int vec = (((uintptr_t)pts | (uintptr_t)keys) & 15) == 0;
    int g = grid_for(vec ? (n + 1) / 2 : n, kThreads);
    if (curve == SFC_CURVE_HILBERT)
        keys_kernel<SFC_CURVE_HILBERT><<<g, kThreads, 0, st>>>(pts, n, keys, status, vec);
    else
        keys_kernel<SFC_CURVE_Z><<<g, kThreads, 0, st>>>(pts, n, keys, status, vec);
    count_launch();
    return launch_status();
}

sfc_status launch_decode(const uint64_t* keys, uint64_t n, int curve, int2* pts, cudaStream_t st)
{
    if (n == 0) return SFC_OK;
    int g = grid_for(n, kThreads);
    if (curve == SFC_CURVE_HILBERT)
        decode_kernel<SFC_CURVE_HILBERT><<<g, kThreads, 0, st>>>(keys, n, pts);
    else
        decode_kernel<SFC_CURVE_Z><<<g, kThreads, 0, st>>>(keys, n, pts);
    count_launch();
    return launch_status();
}

sfc_status launch_keys3(const int32_t* pts, uint64_t n, uint64_t* keys, uint32_t* status, cudaStream_t st)
{
    if (n == 0) return SFC_OK;
    keys3_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(pts, n, keys, status);
    count_launch();
    return launch_status();
}

sfc_status launch_decode3(const uint64_t* keys, uint64_t n, int4* xyz, cudaStream_t st)
{
    if (n == 0) return SFC_OK;
    decode3_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(keys, n, xyz);
    count_launch();
    return launch_status();
}

}  // namespace sfc
