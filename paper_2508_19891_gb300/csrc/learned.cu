// Learned bounds: a two-stage CDF model over the sorted keys, trained on the GPU.
//
// The paper locates each interval start with A_P.lower_bound over a static search tree
// (Sec. 2.1, "Storing P twice"); here a model predicts the position and a short search in a
// stored error window finishes it (verified, with the full binary search as fallback, in
// query.cu).  Training, all on the device and without host synchronisation:
//
//   sample_kernel        strided sample of (x = key / 2^60, y = rank / n)
//   train_*_step_kernel  one full-batch Adam step on the mean-squared error of f(x) against
//                        y: forward and backward per sample, per-block partial gradients, and
//                        the last block to finish sums the partials in block order and
//                        applies the update.  Piecewise-linear root: the per-knot gradient is
//                        accumulated in 64-bit fixed point, so the sums are exact and the run
//                        is deterministic; MLP root: fixed-order float reductions.
//   leaf_bounds_kernel   the root is monotone, so every leaf is a contiguous run of positions:
//                        one binary search per leaf boundary over the sorted keys (routing
//                        the probed keys) instead of routing every key; bound_max_kernel
//                        keeps the boundaries in order
//   leaf_stage_kernel    one block per leaf: the leaf's coarse (16) and fine (256) fences,
//                        the least-squares line of position against key offset (one pass of
//                        fp32 sums shifted by the fine fence's mean), and the exact
//                        min / max of (position - prediction) over the leaf's keys with the
//                        same fp32 predict function the queries call
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "sfc_internal.cuh"
#include "index.cuh"

namespace sfc {

namespace {

constexpr int kNPMlp = 3 * kHidden + 1;   // alpha[H], beta[H], b[H], c
constexpr int kNPPwl = kKnots + 1;        // knot heights h[0..K]
constexpr int kMaxNP = kNPPwl > kNPMlp ? kNPPwl : kNPMlp;
constexpr int kTrainThreads = 256;
constexpr int kTrainBlocks = 64;
constexpr int kPartial = kMaxNP + 1;      // per-block partial: gradient entries + loss
constexpr float kFix32 = 536870912.0f;   // 2^29: fixed-point scale of the knot sums

__host__ __device__ constexpr int num_params(int kind) { return kind == kRootPwl ? kNPPwl : kNPMlp; }

struct TrainState {
    float theta[kMaxNP];
    float m[kMaxNP];
    float v[kMaxNP];
    float grad[kMaxNP];
    float loss;
    int t;
    int kind;
    int np;
    RootParams root;
};


// Derived root parameters from theta (one block; every thread calls it).
__device__ void derive_root(TrainState* ts, int leaves)
{
    if (ts->kind == kRootMlp) {
        for (int k = threadIdx.x; k < kHidden; k += blockDim.x) {
            ts->root.A[k] = expf(ts->theta[k]);
            ts->root.B[k] = expf(ts->theta[kHidden + k]);
            ts->root.b[k] = ts->theta[2 * kHidden + k];
        }
        if (threadIdx.x == 0) ts->root.c = ts->theta[3 * kHidden];
    } else {
        for (int k = threadIdx.x; k <= kKnots; k += blockDim.x) ts->root.h[k] = ts->theta[k];
        if (threadIdx.x == 0) ts->root.c = ts->theta[0];
    }
    if (threadIdx.x == 0) {
        ts->root.kind = ts->kind;
        ts->root.leaves = leaves;
    }
}

// Initial parameters (theta0 == NULL).  MLP: H logistic steps of height 1/H centred at
// (k + 1/2)/H with slope 4H.  Piecewise linear: knot heights h_k = k / K, i.e. f(x) = x.
// Both route keys spread evenly over the key space to equal-width leaves.
__device__ float initial_theta(int kind, int j)
{
    if (kind == kRootPwl) return (float)j / (float)kKnots;
    const float s = 4.0f * kHidden;
    if (j < kHidden) return logf(1.0f / kHidden);
    if (j < 2 * kHidden) return logf(s);
    if (j < 3 * kHidden) return -s * ((float)(j - 2 * kHidden) + 0.5f) / kHidden;
    return 0.0f;
}

__global__ void init_state_kernel(TrainState* ts, int kind, const float* theta0, int leaves)
{
    const int np = num_params(kind);
    if (threadIdx.x == 0) {
        ts->kind = kind;
        ts->np = np;
        ts->t = 0;
        ts->loss = 0.0f;
    }
    for (int k = threadIdx.x; k < kMaxNP; k += blockDim.x) {
        ts->theta[k] = k < np ? (theta0 ? theta0[k] : initial_theta(kind, k)) : 0.0f;
        ts->m[k] = 0.0f;
        ts->v[k] = 0.0f;
        ts->grad[k] = 0.0f;
    }
    __syncthreads();
    derive_root(ts, leaves);
}

// Piecewise-linear start from the sample: h_k = rank (y) of the first sample with
// x >= k / K, i.e. the empirical CDF at the knots (0 at k = 0, 1 past the last sample).  The
// sample is sorted by x, so this is one lower_bound per knot; knots over empty regions get
// the flat CDF value there instead of an arbitrary height.
__global__ void pwl_init_from_sample_kernel(TrainState* ts, const float* __restrict__ x,
                                            const float* __restrict__ y, uint32_t N, int leaves)
{
    for (int k = threadIdx.x; k <= kKnots; k += blockDim.x) {
        const float xk = (float)k / (float)kKnots;
        uint32_t lo = 0, len = N;
        while (len > 0) {
            const uint32_t half = len >> 1;
            const bool lt = x[lo + half] < xk;
            lo = lt ? lo + half + 1 : lo;
            len = lt ? len - half - 1 : half;
        }
        ts->theta[k] = k == 0 ? 0.0f : (lo < N ? y[lo] : 1.0f);
    }
    __syncthreads();
    derive_root(ts, leaves);
}

__global__ void sample_kernel(const uint64_t* __restrict__ keys, uint64_t n, uint32_t N, float* x, float* y)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const uint64_t i = (uint64_t)((double)s * (double)n / (double)N);
        x[s] = key_to_x(keys[i]);
        y[s] = (float)((double)i / (double)n);
    }
}

// Converts sample keys to x for sfc_model_loss_grad.
__global__ void keys_to_x_kernel(const uint64_t* __restrict__ keys, uint64_t N, float* x)
{
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < N; s += (uint64_t)gridDim.x * blockDim.x)
        x[s] = key_to_x(keys[s]);
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ void adam_update(TrainState* ts, float lr)
{
    const int t = ts->t + 1;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int j = threadIdx.x; j < ts->np; j += blockDim.x) {
        const float gj = ts->grad[j];
        const float mj = b1 * ts->m[j] + (1.0f - b1) * gj;
        const float vj = b2 * ts->v[j] + (1.0f - b2) * gj * gj;
        ts->m[j] = mj;
        ts->v[j] = vj;
        ts->theta[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
    }
    __syncthreads();
    if (threadIdx.x == 0) ts->t = t;
}

// Returns true in the last block to finish; partial rows are visible to it.
__device__ bool last_block(unsigned* counter)
{
    __shared__ bool s_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last) __threadfence();
    return s_last;
}

// Per-thread gradient (g[0..3H]) and loss (g[3H+1]) of the MLP root over samples i0,
// i0 + stride, ...
__device__ void mlp_accumulate(const float* __restrict__ x, const float* __restrict__ y, uint32_t N, uint32_t i0,
                               uint32_t stride, const float* sA, const float* sB, const float* sb, float sc,
                               float (&g)[kNPMlp + 1])
{
    const float invN = 1.0f / (float)N;
#pragma unroll
    for (int j = 0; j <= kNPMlp; ++j) g[j] = 0.0f;
    for (uint32_t s = i0; s < N; s += stride) {
        const float xi = x[s], yi = y[s];
        float h[kHidden];
        float f = sc;
#pragma unroll
        for (int k = 0; k < kHidden; ++k) {
            const float z = fmaf(sB[k], xi, sb[k]);
            h[k] = 1.0f / (1.0f + __expf(-z));
            f = fmaf(sA[k], h[k], f);
        }
        const float res = f - yi;
        const float r = 2.0f * res * invN;
        g[kNPMlp] += res * res * invN;         // loss
        g[3 * kHidden] += r;                   // dL/dc
#pragma unroll
        for (int k = 0; k < kHidden; ++k) {
            const float ra = r * sA[k];
            const float sk = h[k] * (1.0f - h[k]);
            g[k] += ra * h[k];                             // dL/dalpha_k
            g[2 * kHidden + k] += ra * sk;                 // dL/db_k
            g[kHidden + k] += ra * sk * sB[k] * xi;        // dL/dbeta_k
        }
    }
}

// ---- MLP root: one step (update != 0) or only the loss and gradient ----
__global__ void __launch_bounds__(kTrainThreads)
train_mlp_step_kernel(const float* __restrict__ x, const float* __restrict__ y, uint32_t N, TrainState* ts,
                      float* partial /* [gridDim.x][kPartial] */, unsigned* counter, float lr, int update,
                      int leaves)
{
    __shared__ float sA[kHidden], sB[kHidden], sb[kHidden], sc;
    __shared__ float sred[kTrainThreads / 32][kNPMlp + 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < kHidden) {
        sA[tid] = ts->root.A[tid];
        sB[tid] = ts->root.B[tid];
        sb[tid] = ts->root.b[tid];
    }
    if (tid == 0) sc = ts->root.c;
    __syncthreads();
    float g[kNPMlp + 1];
    mlp_accumulate(x, y, N, blockIdx.x * kTrainThreads + tid, gridDim.x * kTrainThreads, sA, sB, sb, sc, g);
#pragma unroll
    for (int j = 0; j <= kNPMlp; ++j) {
        const float w = warp_sum(g[j]);
        if (lane == 0) sred[warp][j] = w;
    }
    __syncthreads();
    for (int j = tid; j <= kNPMlp; j += kTrainThreads) {
        float acc = 0.0f;
        for (int w = 0; w < kTrainThreads / 32; ++w) acc += sred[w][j];
        partial[blockIdx.x * kPartial + j] = acc;
    }
    if (!last_block(counter)) return;
    for (int j = tid; j <= kNPMlp; j += kTrainThreads) {
        float acc = 0.0f;
        for (unsigned b = 0; b < gridDim.x; ++b) acc += *((volatile float*)partial + b * kPartial + j);
        if (j == kNPMlp) ts->loss = acc;
        else ts->grad[j] = acc;
    }
    __syncthreads();
    if (update) {
        adam_update(ts, lr);
        derive_root(ts, leaves);
    }
    if (tid == 0) *counter = 0;
}

// Accumulates dL/dh of samples i0, i0 + stride, ... into sg[0..K] as 32-bit fixed point
// (scale 2^29: every term is at most 2/N in magnitude and a knot's sum at most 4, so the
// integer sums are exact and independent of the order of the atomics) and returns the thread's
// share of the loss.  The loop bound is uniform across each warp; when all lanes of a warp fall
// in one knot interval (the common case: samples are sorted) the warp adds its sums with one
// atomic per knot.
__device__ float pwl_accumulate(const float* __restrict__ x, const float* __restrict__ y, uint32_t N, uint32_t i0,
                                uint32_t stride, const float* sh, int* sg)
{
    const float invN = 1.0f / (float)N;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wbase = i0 - lane;
    float loss = 0.0f;
    for (uint32_t base = wbase; base < N; base += stride) {
        const uint32_t s = base + lane;
        const bool ok = s < N;
        int k = 0, a = 0, b = 0;
        if (ok) {
            const float xs = x[s] * (float)kKnots;
            k = (int)xs;
            k = k < 0 ? 0 : (k > kKnots - 1 ? kKnots - 1 : k);
            const float t = xs - (float)k;
            const float f = fmaf(sh[k + 1] - sh[k], t, sh[k]);
            const float res = f - y[s];
            const float r = 2.0f * res * invN;
            a = __float2int_rn(r * (1.0f - t) * kFix32);
            b = __float2int_rn(r * t * kFix32);
            loss = fmaf(res * res, invN, loss);
        }
        const int k0 = __shfl_sync(0xffffffffu, k, 0);
        if (__all_sync(0xffffffffu, !ok || k == k0)) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a += __shfl_xor_sync(0xffffffffu, a, o);
                b += __shfl_xor_sync(0xffffffffu, b, o);
            }
            if (lane == 0) {
                atomicAdd(&sg[k0], a);
                atomicAdd(&sg[k0 + 1], b);
            }
        } else if (ok) {
            atomicAdd(&sg[k], a);
            atomicAdd(&sg[k + 1], b);
        }
    }
    return loss;
}

// Block-wide float sum in a fixed order (every thread calls it; result valid in all threads).
__device__ float block_sum_f(float v, float* sh32)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) sh32[warp] = v;
    __syncthreads();
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh32[w];
    return t;
}

// ---- piecewise-linear root: one step (update != 0) or only the loss and gradient ----
// With s = xK, k = floor(s), t = s - k: f = h_k + (h_{k+1} - h_k) t, so dL/dh_k gets
// r (1 - t) and dL/dh_{k+1} gets r t (r = 2 (f - y) / N).  After the Adam update the heights
// are projected back onto non-decreasing sequences (running maximum), which keeps the root
// monotone.
__global__ void __launch_bounds__(kTrainThreads)
train_pwl_step_kernel(const float* __restrict__ x, const float* __restrict__ y, uint32_t N, TrainState* ts,
                      long long* partial /* [gridDim.x][kPartial] fixed point */, unsigned* counter, float lr,
                      int update, int leaves)
{
    __shared__ float sh[kKnots + 1];
    __shared__ int sg[kKnots + 1];
    __shared__ float s32[kTrainThreads / 32];
    const int tid = threadIdx.x;
    for (int j = tid; j <= kKnots; j += kTrainThreads) {
        sh[j] = ts->root.h[j];
        sg[j] = 0;
    }
    __syncthreads();
    const float l = pwl_accumulate(x, y, N, blockIdx.x * kTrainThreads + tid, gridDim.x * kTrainThreads, sh, sg);
    const float bl = block_sum_f(l, s32);
    __syncthreads();
    for (int j = tid; j <= kKnots; j += kTrainThreads) partial[blockIdx.x * kPartial + j] = (long long)sg[j];
    if (tid == 0) partial[blockIdx.x * kPartial + kKnots + 1] = (long long)__float_as_int(bl);
    if (!last_block(counter)) return;
    for (int j = tid; j <= kKnots; j += kTrainThreads) {
        long long acc = 0;
        for (unsigned b = 0; b < gridDim.x; ++b) acc += *((volatile long long*)partial + b * kPartial + j);
        ts->grad[j] = (float)acc / kFix32;
    }
    if (tid == 0) {
        float acc = 0.0f;
        for (unsigned b = 0; b < gridDim.x; ++b)
            acc += __int_as_float((int)*((volatile long long*)partial + b * kPartial + kKnots + 1));
        ts->loss = acc;
    }
    __syncthreads();
    if (update) {
        adam_update(ts, lr);
        if (tid == 0)
            for (int k = 0; k < kKnots; ++k) ts->theta[k + 1] = fmaxf(ts->theta[k + 1], ts->theta[k]);
        __syncthreads();
        derive_root(ts, leaves);
    }
    if (tid == 0) *counter = 0;
}

// ---- the whole training run in one block: per step the same gradient as the step
// kernels, then Adam with a linearly decaying step size (and the monotone projection for the
// piecewise-linear root).  One launch instead of one per step. ----
// Threads of the training-loop block: the piecewise-linear root keeps few registers per
// thread, the MLP root holds a 50-entry gradient per thread.
template <int KIND>
struct LoopThreads { static constexpr int value = KIND == kRootPwl ? 1024 : 512; };

template <int KIND>
__global__ void __launch_bounds__(LoopThreads<KIND>::value)
train_loop_kernel(const float* __restrict__ x, const float* __restrict__ y, uint32_t N, TrainState* ts, int steps,
                  float lr0, int leaves)
{
    constexpr int kLoopThreads = LoopThreads<KIND>::value;
    // optimiser state stays in shared memory for the whole run
    __shared__ float th[kMaxNP], mo[kMaxNP], ve[kMaxNP], gr[kMaxNP];
    __shared__ float sh[kKnots + 1];
    __shared__ int sg[kKnots + 1];
    __shared__ float s32[kLoopThreads / 32];
    __shared__ float sred[kLoopThreads / 32][kNPMlp + 1];
    __shared__ float sA[kHidden], sB[kHidden], sb[kHidden], sc;
    __shared__ float s_loss;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr bool pwl = KIND == kRootPwl;
    const int np = ts->np;
    for (int j = tid; j < kMaxNP; j += kLoopThreads) {
        th[j] = ts->theta[j];
        mo[j] = ts->m[j];
        ve[j] = ts->v[j];
    }
    const int t0 = ts->t;
    __syncthreads();
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int step = 0; step < steps; ++step) {
        const float lr = lr0 * (float)(steps - step) / (float)steps;
        // current root in shared memory
        if constexpr (pwl) {
            for (int j = tid; j <= kKnots; j += kLoopThreads) {
                sh[j] = th[j];
                sg[j] = 0;
            }
        } else {
            if (tid < kHidden) {
                sA[tid] = expf(th[tid]);
                sB[tid] = expf(th[kHidden + tid]);
                sb[tid] = th[2 * kHidden + tid];
            }
            if (tid == 0) sc = th[3 * kHidden];
        }
        __syncthreads();
        if constexpr (pwl) {
            const float l = pwl_accumulate(x, y, N, tid, kLoopThreads, sh, sg);
            const float bl = block_sum_f(l, s32);
            __syncthreads();
            for (int j = tid; j <= kKnots; j += kLoopThreads) gr[j] = (float)sg[j] / kFix32;
            if (tid == 0) s_loss = bl;
        } else {
            float g[kNPMlp + 1];
            mlp_accumulate(x, y, N, tid, kLoopThreads, sA, sB, sb, sc, g);
            (void)s32;
#pragma unroll
            for (int j = 0; j <= kNPMlp; ++j) {
                const float w = warp_sum(g[j]);
                if (lane == 0) sred[warp][j] = w;
            }
            __syncthreads();
            for (int j = tid; j <= kNPMlp; j += kLoopThreads) {
                float acc = 0.0f;
                for (int w = 0; w < kLoopThreads / 32; ++w) acc += sred[w][j];
                if (j == kNPMlp) s_loss = acc;
                else gr[j] = acc;
            }
        }
        __syncthreads();
        // Adam, bias-corrected at step t
        const int t = t0 + step + 1;
        const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
        for (int j = tid; j < np; j += kLoopThreads) {
            const float gj = gr[j];
            const float mj = b1 * mo[j] + (1.0f - b1) * gj;
            const float vj = b2 * ve[j] + (1.0f - b2) * gj * gj;
            mo[j] = mj;
            ve[j] = vj;
            th[j] -= lr * (mj / c1) / (sqrtf(vj / c2) + eps);
        }
        __syncthreads();
        if (pwl) {   // running maximum (Hillis-Steele scan) keeps the knot heights monotone
            for (int o = 1; o <= kKnots; o <<= 1) {
                float v = 0.0f;
                const bool has = tid <= kKnots && tid >= o;
                if (has) v = th[tid - o];
                __syncthreads();
                if (has) th[tid] = fmaxf(th[tid], v);
                __syncthreads();
            }
        }
    }
    for (int j = tid; j < kMaxNP; j += kLoopThreads) {
        ts->theta[j] = th[j];
        ts->m[j] = mo[j];
        ts->v[j] = ve[j];
        ts->grad[j] = gr[j];
    }
    if (tid == 0) {
        ts->t = t0 + steps;
        ts->loss = s_loss;
    }
    __syncthreads();
    derive_root(ts, leaves);
}

// Adam update alone on given state (sfc_model_adam_step).
__global__ void adam_kernel(TrainState* ts, float lr, int t, int np)
{
    if (threadIdx.x == 0) {
        ts->np = np;
        ts->t = t - 1;
    }
    __syncthreads();
    adam_update(ts, lr);
}

// Leaf boundaries.  The root is monotone, so the keys routed to leaf j are the positions
// [bound[j], bound[j + 1]) with bound[j] the first position whose key routes to a leaf >= j
// (bound[0] = 0, bound[leaves] = n): one binary search per boundary over the sorted keys
// instead of routing every key.  A leaf that no key routes to gets bound[j] = bound[j + 1].
__global__ void __launch_bounds__(256) leaf_bounds_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                          const TrainState* ts, int leaves, uint32_t* __restrict__ bound)
{
    __shared__ RootParams s_root;
    for (unsigned w = threadIdx.x; w < sizeof(RootParams) / 4; w += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_root)[w] = reinterpret_cast<const uint32_t*>(&ts->root)[w];
    __syncthreads();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j > leaves) return;
    uint64_t lo = 0, len = n;   // first position with route >= j lies in [lo, lo + len]
    if (j == 0) len = 0;
    else if (j == leaves) lo = n, len = 0;
    while (len > 0) {
        const uint64_t half = len >> 1;
        if (route_leaf(s_root, __ldg(keys + lo + half)) < j) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    bound[j] = (uint32_t)lo;
}

// Running maximum of the boundaries (one block of 1024 threads, each owning a contiguous
// segment), so that the leaves tile [0, n) in order even if fp32 rounding made the root
// step down somewhere.
__global__ void __launch_bounds__(1024) bound_max_kernel(uint32_t* bound, int count)
{
    __shared__ uint32_t s_max[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (count + T - 1) / T;
    const int j0 = t * per, j1 = min(count, j0 + per);
    uint32_t m = 0;
    for (int j = j0; j < j1; ++j) m = max(m, bound[j]);
    s_max[t] = m;
    __syncthreads();
    for (int o = 1; o < T; o <<= 1) {   // inclusive prefix max over the segments
        const uint32_t v = t >= o ? s_max[t - o] : 0u;
        __syncthreads();
        s_max[t] = max(s_max[t], v);
        __syncthreads();
    }
    uint32_t run = t > 0 ? s_max[t - 1] : 0u;
    for (int j = j0; j < j1; ++j) {
        run = max(run, bound[j]);
        bound[j] = run;
    }
}

// Block-wide int min / max (every thread calls it; result valid in all threads).
__device__ int2 block_minmax_i(int lo, int hi, int* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __syncthreads();
    if (lane == 0) {
        sh[2 * warp] = lo;
        sh[2 * warp + 1] = hi;
    }
    __syncthreads();
    int a = 0x7fffffff, b = (int)0x80000000;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        a = min(a, sh[2 * w]);
        b = max(b, sh[2 * w + 1]);
    }
    return make_int2(a, b);
}

// One block per leaf j, over its positions [bound[j], bound[j + 1]):
//   its coarse and fine fences, then the least-squares line of position against key offset
//   (v = position - first against u = key - base, base the leaf's smallest key; fp32 sums of
//   u shifted by the fence keys' mean, fixed-order reductions), then the exact error window:
//   min and max of (position - prediction) over the leaf's keys with the query-time fp32
//   predict function.  The leaf's keys are read twice; the second read mostly comes from L2.
// Threads per leaf block: at 10^8 keys (about 24,000 per leaf) 512 threads take the stage from
// 1.26 ms (256 threads) to 0.99 ms; 1,024 gain another 2%.
#ifndef SFC_LEAF_THREADS
#define SFC_LEAF_THREADS 512
#endif
constexpr int kLeafThreads = SFC_LEAF_THREADS;

__global__ void __launch_bounds__(kLeafThreads) leaf_stage_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                                  const uint32_t* __restrict__ bound, LeafParams* leaf,
                                                                  uint64_t* __restrict__ fence,
                                                                  uint64_t* __restrict__ fence_fine)
{
    __shared__ float sh[kLeafThreads / 32];
    __shared__ int shi[2 * (kLeafThreads / 32)];
    const int j = blockIdx.x;
    LeafParams lp;
    lp.first = bound[j];
    lp.end = bound[j + 1];
    lp.base = lp.first < n ? keys[lp.first] : kKeyMax;
    lp.slope = 0.0f;
    lp.icpt = 0.0f;
    lp.err_lo = 0;
    lp.err_hi = 0;
    const uint32_t cnt = lp.end - lp.first;
    const uint64_t* kp = keys + lp.first;
    const uint32_t B = blockDim.x;
    // the fences first: 256 keys at evenly spaced positions of the leaf, whose mean is the shift
    // of the one-pass sums below (close to the leaf's mean, so the variance keeps its precision)
    float sf = 0.0f;
    for (uint32_t r = threadIdx.x; r < (uint32_t)kFenceFine; r += B) {
        const uint64_t k = cnt ? __ldg(kp + ((uint64_t)r * cnt) / kFenceFine) : ~0ull;
        fence_fine[(size_t)j * kFenceFine + r] = k;
        if (r % kFence == 0) fence[(size_t)j * kFence + r / kFence] = k;
        if (cnt) sf += __ull2float_rn(k - lp.base);
    }
    if (cnt >= 2) {
        // one pass over d = u - mu0 (u = key - base): sum d, sum d^2 and sum d (i - mean i);
        // each thread keeps four loads in flight
        const float mu0 = block_sum_f(sf, sh) / (float)kFenceFine;
        const float mv = 0.5f * (float)(cnt - 1);   // mean of 0 .. cnt - 1
        float s1 = 0.0f, sdd = 0.0f, sdi = 0.0f;
        for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += 4 * B) {
            float d[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t i = i0 + q * B;
                d[q] = i < cnt ? __ull2float_rn(__ldg(kp + i) - lp.base) - mu0 : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t i = i0 + q * B;
                if (i < cnt) {
                    s1 += d[q];
                    sdd = fmaf(d[q], d[q], sdd);
                    sdi = fmaf(d[q], (float)i - mv, sdi);
                }
            }
        }
        s1 = block_sum_f(s1, sh);
        sdd = block_sum_f(sdd, sh);
        sdi = block_sum_f(sdi, sh);
        // sum (i - mean i) = 0, so sdi is already the centred cross sum
        const float dbar = s1 / (float)cnt;
        const float sxx = sdd - (float)cnt * dbar * dbar;
        lp.slope = sxx > 0.0f ? sdi / sxx : 0.0f;
        lp.icpt = mv - lp.slope * (mu0 + dbar);
    }
    if (cnt >= 1) {
        int lo = 0x7fffffff, hi = (int)0x80000000;
        for (uint32_t i = threadIdx.x; i < cnt; i += B) {
            long long e = (long long)(lp.first + i) - leaf_predict(lp, __ldg(kp + i));
            e = e > 0x7fffffffll ? 0x7fffffffll : (e < -0x7fffffffll ? -0x7fffffffll : e);
            lo = min(lo, (int)e);
            hi = max(hi, (int)e);
        }
        const int2 w = block_minmax_i(lo, hi, shi);
        lp.err_lo = w.x;
        lp.err_hi = w.y;
    }
    if (threadIdx.x == 0) leaf[j] = lp;
}

}  // namespace

const RootParams* model_root_device(sfc_index* idx)
{
    TrainState* ts = idx->model.state.as<TrainState>();
    return ts ? &ts->root : nullptr;
}

sfc_status fit_leaves(sfc_index* idx, cudaStream_t st)
{
    ModelState& M = idx->model;
    const int leaves = M.nleaves;
    const uint64_t n = idx->n;
    TrainState* ts = M.state.as<TrainState>();
    SFC_TRY(M.tmp.ensure((size_t)(leaves + 1) * sizeof(uint32_t), st));
    SFC_TRY(M.leaves.ensure((size_t)leaves * sizeof(LeafParams), st));
    SFC_TRY(M.fence.ensure((size_t)leaves * kFence * sizeof(uint64_t), st));
    SFC_TRY(M.fence_fine.ensure((size_t)leaves * kFenceFine * sizeof(uint64_t), st));
    uint32_t* bound = M.tmp.as<uint32_t>();
    const uint64_t* keys = idx->keys.as<uint64_t>();
    leaf_bounds_kernel<<<(leaves + 1 + 255) / 256, 256, 0, st>>>(keys, n, ts, leaves, bound);
    count_launch();
    bound_max_kernel<<<1, 1024, 0, st>>>(bound, leaves + 1);
    count_launch();
    leaf_stage_kernel<<<leaves, kLeafThreads, 0, st>>>(keys, n, bound, M.leaves.as<LeafParams>(),
                                                       M.fence.as<uint64_t>(), M.fence_fine.as<uint64_t>());
    count_launch();
    return launch_status();
}

static uint32_t sample_count(const sfc_index* idx, uint64_t n)
{
    return (uint32_t)std::max<uint64_t>(2, std::min<uint64_t>((uint64_t)idx->opt.train_samples, std::max<uint64_t>(n, 2)));
}

sfc_status reserve_model(sfc_index* idx, uint64_t n, cudaStream_t st)
{
    ModelState& M = idx->model;
    const int leaves = idx->opt.leaves;
    const uint32_t N = sample_count(idx, n);
    SFC_TRY(M.state.ensure(sizeof(TrainState), st));
    SFC_TRY(M.samples.ensure((size_t)N * 2 * sizeof(float), st));
    SFC_TRY(M.partial.ensure((size_t)kTrainBlocks * kPartial * sizeof(long long) + 256, st));
    SFC_TRY(M.tmp.ensure((size_t)(leaves + 1) * sizeof(uint32_t), st));
    SFC_TRY(M.leaves.ensure((size_t)leaves * sizeof(LeafParams), st));
    SFC_TRY(M.fence.ensure((size_t)leaves * kFence * sizeof(uint64_t), st));
    SFC_TRY(M.fence_fine.ensure((size_t)leaves * kFenceFine * sizeof(uint64_t), st));
    return SFC_OK;
}

// Trains the root from its initial parameters (warm: continue from the current ones for
// `steps` more steps), then fits the leaves.
static sfc_status train_root(sfc_index* idx, int steps, bool warm, cudaStream_t st)
{
    ModelState& M = idx->model;
    const int leaves = idx->opt.leaves;
    const int kind = idx->opt.root == SFC_ROOT_MLP ? kRootMlp : kRootPwl;
    const uint64_t n = idx->n;
    const uint32_t N = sample_count(idx, n);
    const bool fresh = !M.state.ptr;
    SFC_TRY(M.state.ensure(sizeof(TrainState), st));
    SFC_TRY(M.samples.ensure((size_t)N * 2 * sizeof(float), st));
    SFC_TRY(M.partial.ensure((size_t)kTrainBlocks * kPartial * sizeof(long long) + 256, st));
    TrainState* ts = M.state.as<TrainState>();
    float* x = M.samples.as<float>();
    float* y = x + N;
    unsigned* counter = reinterpret_cast<unsigned*>(M.partial.as<unsigned char>() +
                                                    (size_t)kTrainBlocks * kPartial * sizeof(long long));
    M.nleaves = leaves;
    SFC_CUDA_TRY(cudaMemsetAsync(counter, 0, 16, st));
    if (!warm || fresh || !M.trained || M.kind != kind) {
        init_state_kernel<<<1, 256, 0, st>>>(ts, kind, nullptr, leaves);
        count_launch();
    }
    M.kind = kind;
    if (n >= 2 && steps > 0) {
        sample_kernel<<<(N + 255) / 256, 256, 0, st>>>(idx->keys.as<uint64_t>(), n, N, x, y);
        count_launch();
        if (kind == kRootPwl && !(warm && !fresh && M.trained)) {
            pwl_init_from_sample_kernel<<<1, 256, 0, st>>>(ts, x, y, N, leaves);
            count_launch();
        }
        // heights live on [0, 1] where a leaf is 1/4096 wide: the piecewise-linear root
        // refines with a twentieth of the MLP's step size
        const float lr0 = idx->opt.learning_rate * (kind == kRootPwl ? 0.05f : 1.0f);
        if (kind == kRootPwl)
            train_loop_kernel<kRootPwl><<<1, LoopThreads<kRootPwl>::value, 0, st>>>(x, y, N, ts, steps, lr0, leaves);
        else
            train_loop_kernel<kRootMlp><<<1, LoopThreads<kRootMlp>::value, 0, st>>>(x, y, N, ts, steps, lr0, leaves);
        count_launch();
    }
    SFC_TRY(launch_status());
    SFC_TRY(fit_leaves(idx, st));
    M.trained = true;
    return SFC_OK;
}

sfc_status train_model(sfc_index* idx, cudaStream_t st)
{
    return train_root(idx, idx->opt.train_steps, false, st);
}

sfc_status refit_model(sfc_index* idx, int steps, cudaStream_t st)
{
    return train_root(idx, steps, true, st);
}

}  // namespace sfc

using namespace sfc;

extern "C" {

int sfc_model_hidden(void) { return kHidden; }

int sfc_model_params(sfc_root root) { return root == SFC_ROOT_MLP ? kNPMlp : (root == SFC_ROOT_PWL ? kNPPwl : -1); }

sfc_status sfc_model_loss_grad(sfc_root root, const float* h_params, const uint64_t* d_keys, const float* d_y,
                               uint64_t s, float* h_loss, float* h_grad, void* stream)
{
    if ((root != SFC_ROOT_PWL && root != SFC_ROOT_MLP) || !h_params || !d_keys || !d_y || s == 0 ||
        s > 0x7fffffffull)
        return SFC_ERR_INVALID;
    const int kind = root == SFC_ROOT_MLP ? kRootMlp : kRootPwl;
    const int np = num_params(kind);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf state, xs, part, th;
    sfc_status rc = SFC_OK;
    do {
        if ((rc = state.ensure(sizeof(TrainState), st)) != SFC_OK) break;
        if ((rc = xs.ensure((size_t)s * sizeof(float), st)) != SFC_OK) break;
        if ((rc = part.ensure((size_t)kTrainBlocks * kPartial * sizeof(long long) + 256, st)) != SFC_OK) break;
        if ((rc = th.ensure(kMaxNP * sizeof(float), st)) != SFC_OK) break;
        TrainState* ts = state.as<TrainState>();
        unsigned* counter = reinterpret_cast<unsigned*>(part.as<unsigned char>() +
                                                        (size_t)kTrainBlocks * kPartial * sizeof(long long));
        if (cudaMemcpyAsync(th.ptr, h_params, np * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemsetAsync(counter, 0, 16, st) != cudaSuccess) { rc = SFC_ERR_CUDA; break; }
        init_state_kernel<<<1, 256, 0, st>>>(ts, kind, th.as<float>(), 1);
        keys_to_x_kernel<<<(unsigned)std::min<uint64_t>((s + 255) / 256, 1024), 256, 0, st>>>(d_keys, s, xs.as<float>());
        if (kind == kRootPwl)
            train_pwl_step_kernel<<<kTrainBlocks, kTrainThreads, 0, st>>>(xs.as<float>(), d_y, (uint32_t)s, ts,
                                                                         part.as<long long>(), counter, 0.0f, 0, 1);
        else
            train_mlp_step_kernel<<<kTrainBlocks, kTrainThreads, 0, st>>>(xs.as<float>(), d_y, (uint32_t)s, ts,
                                                                         part.as<float>(), counter, 0.0f, 0, 1);
        count_launch(3);
        if ((rc = launch_status()) != SFC_OK) break;
        float loss = 0.0f;
        if (cudaMemcpyAsync(h_grad, ts->grad, np * sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(&loss, &ts->loss, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) { rc = SFC_ERR_CUDA; break; }
        if (h_loss) *h_loss = loss;
    } while (0);
    state.release(st);
    xs.release(st);
    part.release(st);
    th.release(st);
    return rc;
}

sfc_status sfc_model_adam_step(float* h_params, float* h_m, float* h_v, const float* h_grad, int np, int t,
                               float lr, void* stream)
{
    if (!h_params || !h_m || !h_v || !h_grad || t < 1 || np < 1 || np > kMaxNP) return SFC_ERR_INVALID;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DevBuf buf;
    SFC_TRY(buf.ensure(sizeof(TrainState), st));
    TrainState* ts = buf.as<TrainState>();
    sfc_status rc = SFC_OK;
    const size_t b = (size_t)np * 4;
    if (cudaMemcpyAsync(ts->theta, h_params, b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ts->m, h_m, b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ts->v, h_v, b, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(ts->grad, h_grad, b, cudaMemcpyHostToDevice, st) != cudaSuccess) {
        rc = SFC_ERR_CUDA;
    } else {
        adam_kernel<<<1, 256, 0, st>>>(ts, lr, t, np);
        count_launch();
        rc = launch_status();
        if (rc == SFC_OK &&
            (cudaMemcpyAsync(h_params, ts->theta, b, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(h_m, ts->m, b, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(h_v, ts->v, b, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaStreamSynchronize(st) != cudaSuccess))
            rc = SFC_ERR_CUDA;
    }
    buf.release(st);
    return rc;
}

sfc_status sfc_model_get(const sfc_index* cidx, int* h_root, float* h_params, int* h_leaves, uint32_t* h_first,
                         uint32_t* h_end, float* h_slope, float* h_icpt, int32_t* h_err_lo, int32_t* h_err_hi,
                         void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx) return SFC_ERR_INVALID;
    if (!idx->model.trained) return SFC_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int L = idx->model.nleaves;
    const int kind = idx->model.kind;
    if (h_leaves) *h_leaves = L;
    if (h_root) *h_root = kind == kRootMlp ? SFC_ROOT_MLP : SFC_ROOT_PWL;
    const TrainState* ts = idx->model.state.as<TrainState>();
    if (h_params)
        SFC_CUDA_TRY(cudaMemcpyAsync(h_params, ts->theta, (size_t)num_params(kind) * 4, cudaMemcpyDeviceToHost, st));
    if (h_first || h_end || h_slope || h_icpt || h_err_lo || h_err_hi) {
        std::vector<LeafParams> lp((size_t)L);
        SFC_CUDA_TRY(cudaMemcpyAsync(lp.data(), idx->model.leaves.ptr, (size_t)L * sizeof(LeafParams),
                                     cudaMemcpyDeviceToHost, st));
        SFC_CUDA_TRY(cudaStreamSynchronize(st));
        for (int j = 0; j < L; ++j) {
            if (h_first) h_first[j] = lp[j].first;
            if (h_end) h_end[j] = lp[j].end;
            if (h_slope) h_slope[j] = lp[j].slope;
            if (h_icpt) h_icpt[j] = lp[j].icpt;
            if (h_err_lo) h_err_lo[j] = lp[j].err_lo;
            if (h_err_hi) h_err_hi[j] = lp[j].err_hi;
        }
    }
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    return SFC_OK;
}

sfc_status sfc_model_fence(const sfc_index* cidx, uint64_t* h_fence, int* h_leaves, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx) return SFC_ERR_INVALID;
    if (!idx->model.trained || !idx->model.fence.ptr) return SFC_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int L = idx->model.nleaves;
    if (h_leaves) *h_leaves = L;
    if (h_fence)
        SFC_CUDA_TRY(cudaMemcpyAsync(h_fence, idx->model.fence.ptr, (size_t)L * kFence * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    return SFC_OK;
}

sfc_status sfc_model_fence_fine(const sfc_index* cidx, uint64_t* h_fence, int* h_leaves, void* stream)
{
    sfc_index* idx = const_cast<sfc_index*>(cidx);
    if (!idx) return SFC_ERR_INVALID;
    if (!idx->model.trained || !idx->model.fence_fine.ptr) return SFC_ERR_STATE;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int L = idx->model.nleaves;
    if (h_leaves) *h_leaves = L;
    if (h_fence)
        SFC_CUDA_TRY(cudaMemcpyAsync(h_fence, idx->model.fence_fine.ptr, (size_t)L * kFenceFine * sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, st));
    SFC_CUDA_TRY(cudaStreamSynchronize(st));
    return SFC_OK;
}

}  // extern "C"
