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
//   route_kernel         leaf of every key (the query-time routing function) and the first /
//                        last position of each leaf
//   leaf_fix_kernel      empty leaves take the position where their keys would start
//   leaf_fit_kernel      one block per leaf: least-squares line of position against key
//                        offset (two passes, fp64 accumulators)
//   leaf_err_kernel      exact min / max of (position - prediction) over each leaf's keys,
//                        with the same fp32 predict function the queries call
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

struct LeafTmp {
    uint32_t first;       // min position routed to the leaf
    uint32_t last;        // max position routed to the leaf
    int32_t err_lo;
    int32_t err_hi;
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

__global__ void leaf_init_kernel(LeafTmp* tmp, int leaves)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < leaves; j += gridDim.x * blockDim.x) {
        tmp[j].first = 0xffffffffu;
        tmp[j].last = 0;
        tmp[j].err_lo = 0x7fffffff;
        tmp[j].err_hi = (int32_t)0x80000000;
    }
}

// Leaf of every key with the query-time routing function; a position starts or ends a
// leaf's run where its neighbour's leaf differs (one atomic per run, not per key).
__global__ void __launch_bounds__(256) route_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                    const TrainState* ts, uint32_t* __restrict__ route,
                                                    LeafTmp* tmp)
{
    __shared__ RootParams s_root;
    for (unsigned w = threadIdx.x; w < sizeof(RootParams) / 4; w += blockDim.x)
        reinterpret_cast<uint32_t*>(&s_root)[w] = reinterpret_cast<const uint32_t*>(&ts->root)[w];
    __syncthreads();
    const unsigned lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // four groups of the grid stride per iteration, their loads issued together (the loop
    // bound is uniform per warp so the shuffles below see the whole warp)
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += 4 * stride) {
        uint64_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * stride + threadIdx.x;
            k[u] = i < n ? __ldg(keys + i) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * stride + threadIdx.x;
            const bool ok = i < n;
            const int j = ok ? route_leaf(s_root, k[u]) : -1;
            int prev = __shfl_up_sync(0xffffffffu, j, 1);
            if (lane == 0 && ok && i > 0) prev = route_leaf(s_root, keys[i - 1]);
            int next = __shfl_down_sync(0xffffffffu, j, 1);
            if ((lane == 31 || i + 1 >= n) && ok) next = (i + 1 < n) ? route_leaf(s_root, keys[i + 1]) : -1;
            if (ok) {
                route[i] = (uint32_t)j;
                if (i == 0 || prev != j) atomicMin(&tmp[j].first, (uint32_t)i);
                if (i + 1 == n || next != j) atomicMax(&tmp[j].last, (uint32_t)i);
            }
        }
    }
}

// One block of 1024 threads: leaf params from the run bounds.  An empty leaf (no key routed
// to it) takes first = end = the start of the next non-empty leaf (n past the last one): a
// suffix minimum over the leaves, each thread owning a contiguous segment.
__global__ void __launch_bounds__(1024) leaf_fix_kernel(const LeafTmp* tmp, int leaves, uint64_t n,
                                                        LeafParams* out, const uint64_t* keys)
{
    __shared__ uint32_t s_min[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (leaves + T - 1) / T;
    const int j0 = t * per, j1 = min(leaves, j0 + per);
    uint32_t m = 0xffffffffu;
    for (int j = j0; j < j1; ++j)
        if (tmp[j].first <= tmp[j].last) m = min(m, tmp[j].first);
    s_min[t] = m;
    __syncthreads();
    // inclusive suffix-min over the threads' segment minima
    for (int o = 1; o < T; o <<= 1) {
        const uint32_t v = (t + o < T) ? s_min[t + o] : 0xffffffffu;
        __syncthreads();
        s_min[t] = min(s_min[t], v);
        __syncthreads();
    }
    uint32_t next_start = (t + 1 < T) ? s_min[t + 1] : 0xffffffffu;
    if (next_start == 0xffffffffu) next_start = (uint32_t)n;
    for (int j = j1 - 1; j >= j0; --j) {
        LeafParams lp;
        if (tmp[j].first > tmp[j].last) {
            lp.first = next_start;
            lp.end = next_start;
            lp.base = next_start < n ? keys[next_start] : kKeyMax;
        } else {
            lp.first = tmp[j].first;
            lp.end = tmp[j].last + 1;
            lp.base = keys[tmp[j].first];
            next_start = min(next_start, tmp[j].first);
        }
        lp.slope = 0.0f;
        lp.icpt = 0.0f;
        lp.err_lo = 0;
        lp.err_hi = 0;
        out[j] = lp;
    }
}

// One block per leaf: v = position - first against u = key - base over [first, end), in
// fp32 with centred second pass and fixed-order tree reductions.  The line only places the
// search window; the window itself is measured exactly afterwards (leaf_err_kernel).
__global__ void __launch_bounds__(256) leaf_fit_kernel(const uint64_t* __restrict__ keys, LeafParams* leaf)
{
    __shared__ float sh[8];
    LeafParams lp = leaf[blockIdx.x];
    const uint32_t cnt = lp.end - lp.first;
    if (cnt < 2) {
        if (threadIdx.x == 0) { leaf[blockIdx.x].slope = 0.0f; leaf[blockIdx.x].icpt = 0.0f; }
        return;
    }
    // two passes (the mean first, for fp32 accuracy); each thread keeps four loads in flight
    const uint64_t* kp = keys + lp.first;
    const uint32_t B = blockDim.x;
    float su = 0.0f;
    for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += 4 * B) {
        float u[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = i0 + q * B;
            u[q] = i < cnt ? __ull2float_rn(__ldg(kp + i) - lp.base) : 0.0f;
        }
        su += (u[0] + u[1]) + (u[2] + u[3]);
    }
    const float mu = block_sum_f(su, sh) / (float)cnt;
    const float mv = 0.5f * (float)(cnt - 1);   // mean of 0 .. cnt - 1
    float sxy = 0.0f, sxx = 0.0f;
    for (uint32_t i0 = threadIdx.x; i0 < cnt; i0 += 4 * B) {
        float du[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = i0 + q * B;
            du[q] = i < cnt ? __ull2float_rn(__ldg(kp + i) - lp.base) - mu : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint32_t i = i0 + q * B;
            if (i < cnt) {
                sxy = fmaf(du[q], (float)i - mv, sxy);
                sxx = fmaf(du[q], du[q], sxx);
            }
        }
    }
    sxy = block_sum_f(sxy, sh);
    sxx = block_sum_f(sxx, sh);
    if (threadIdx.x == 0) {
        const float slope = sxx > 0.0f ? sxy / sxx : 0.0f;
        leaf[blockIdx.x].slope = slope;
        leaf[blockIdx.x].icpt = mv - slope * mu;
    }
}

__global__ void __launch_bounds__(256) leaf_err_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                       const uint32_t* __restrict__ route,
                                                       const LeafParams* __restrict__ leaf, LeafTmp* tmp)
{
    const unsigned lane = threadIdx.x & 31;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    // four groups of the grid stride per iteration, their loads issued together
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < n; base += 4 * stride) {
        uint64_t k[4];
        uint32_t jr[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * stride + threadIdx.x;
            k[u] = i < n ? __ldg(keys + i) : 0;
            jr[u] = i < n ? __ldg(route + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t i = base + u * stride + threadIdx.x;
            const bool ok = i < n;
            int j = -1;
            long long e = 0;
            if (ok) {
                j = (int)jr[u];
                const LeafParams lp = leaf[j];
                e = (long long)i - leaf_predict(lp, k[u]);
                e = e > 0x7fffffffll ? 0x7fffffffll : (e < -0x7fffffffll ? -0x7fffffffll : e);
            }
            // warp-aggregated when the whole warp is in one leaf (the common case)
            const int j0 = __shfl_sync(0xffffffffu, j, 0);
            const bool same = __all_sync(0xffffffffu, j == j0);
            if (same) {
                int lo = (int)e, hi = (int)e;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                    hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
                }
                if (lane == 0 && j0 >= 0) {
                    atomicMin(&tmp[j0].err_lo, lo);
                    atomicMax(&tmp[j0].err_hi, hi);
                }
            } else if (ok) {
                atomicMin(&tmp[j].err_lo, (int)e);
                atomicMax(&tmp[j].err_hi, (int)e);
            }
        }
    }
}

__global__ void leaf_store_err_kernel(const LeafTmp* tmp, LeafParams* leaf, int leaves)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < leaves; j += gridDim.x * blockDim.x) {
        if (tmp[j].err_lo <= tmp[j].err_hi) {
            leaf[j].err_lo = tmp[j].err_lo;
            leaf[j].err_hi = tmp[j].err_hi;
        } else {   // no key routed here: the window is the (empty) leaf range itself
            leaf[j].err_lo = 0;
            leaf[j].err_hi = 0;
        }
    }
}

// The fences of every leaf: the fine fence (kFenceFine keys at equally spaced positions of its
// range) and the coarse one (every kFence-th fine key); a leaf with no keys gets keys that no
// target exceeds.
__global__ void fence_kernel(const uint64_t* __restrict__ keys, const LeafParams* __restrict__ leaf, int leaves,
                             uint64_t* __restrict__ fence, uint64_t* __restrict__ fence_fine)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= leaves * kFenceFine) return;
    const int j = i / kFenceFine, r = i - j * kFenceFine;
    const uint64_t first = leaf[j].first, c = leaf[j].end - leaf[j].first;
    const uint64_t k = c ? keys[first + ((uint64_t)r * c) / kFenceFine] : ~0ull;
    fence_fine[i] = k;
    if (r % kFence == 0) fence[j * kFence + r / kFence] = k;
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
    SFC_TRY(M.tmp.ensure((size_t)leaves * sizeof(LeafTmp), st));
    SFC_TRY(M.leaves.ensure((size_t)leaves * sizeof(LeafParams), st));
    SFC_TRY(M.route.ensure(std::max<uint64_t>(n, 1) * sizeof(uint32_t), st));
    LeafTmp* tmp = M.tmp.as<LeafTmp>();
    LeafParams* lp = M.leaves.as<LeafParams>();
    const uint64_t* keys = idx->keys.as<uint64_t>();
    const int g = (int)std::max<uint64_t>(1, std::min<uint64_t>((n + 255) / 256, (uint64_t)num_sms() * 8));
    leaf_init_kernel<<<(leaves + 255) / 256, 256, 0, st>>>(tmp, leaves);
    count_launch();
    if (n) {
        route_kernel<<<g, 256, 0, st>>>(keys, n, ts, M.route.as<uint32_t>(), tmp);
        count_launch();
    }
    leaf_fix_kernel<<<1, 1024, 0, st>>>(tmp, leaves, n, lp, keys);
    count_launch();
    leaf_fit_kernel<<<leaves, 256, 0, st>>>(keys, lp);
    count_launch();
    if (n) {
        leaf_err_kernel<<<g, 256, 0, st>>>(keys, n, M.route.as<uint32_t>(), lp, tmp);
        count_launch();
    }
    leaf_store_err_kernel<<<(leaves + 255) / 256, 256, 0, st>>>(tmp, lp, leaves);
    count_launch();
    SFC_TRY(M.fence.ensure((size_t)leaves * kFence * sizeof(uint64_t), st));
    SFC_TRY(M.fence_fine.ensure((size_t)leaves * kFenceFine * sizeof(uint64_t), st));
    fence_kernel<<<(leaves * kFenceFine + 255) / 256, 256, 0, st>>>(keys, lp, leaves, M.fence.as<uint64_t>(),
                                                                    M.fence_fine.as<uint64_t>());
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
    SFC_TRY(M.tmp.ensure((size_t)leaves * sizeof(LeafTmp), st));
    SFC_TRY(M.leaves.ensure((size_t)leaves * sizeof(LeafParams), st));
    SFC_TRY(M.fence.ensure((size_t)leaves * kFence * sizeof(uint64_t), st));
    SFC_TRY(M.fence_fine.ensure((size_t)leaves * kFenceFine * sizeof(uint64_t), st));
    SFC_TRY(M.route.ensure(std::max<uint64_t>(n, 1) * sizeof(uint32_t), st));
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
