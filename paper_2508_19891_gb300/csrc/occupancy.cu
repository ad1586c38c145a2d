// Early-termination quadtree (Sec. 2.2, "Early termination"): one boolean per node of the
// complete quadtree of depth D over the domain [0, 2^30)^2, true iff the node's cell holds a
// point.  Node v at depth t is the cell of level 30 - t whose label (the key prefix of
// Def. 2.3, for either curve) is v.  The bits of all depths are stored one after another,
// depth t from bit (4^t - 1) / 3, so D = 12 takes 22.4 M bits (2.8 MB, L2-resident).
//
// Built from the sorted keys in one pass: a point marks the nodes of the depths at which its
// key prefix differs from the previous key's (the common prefix of two keys is the deepest
// node they share), so every non-empty node is marked once, by its first point, and the
// pass reads 8 B per point plus one atomic per non-empty node.  The plan kernel tests each
// cell of a query's cover before searching its bounds and drops empty cells.
#include "index.cuh"

namespace sfc {

namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads) occupancy_kernel(const uint64_t* __restrict__ keys, uint64_t n,
                                                             int D, uint32_t* __restrict__ bits)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint64_t k = keys[i];
        int t0 = 0;
        if (i > 0) {
            const uint64_t x = k ^ keys[i - 1];
            if (x == 0) continue;                       // same unit cell as the previous point
            const int h = 63 - __clzll((long long)x);   // highest differing key bit (< 60)
            t0 = (61 - h) >> 1;                         // prefixes of depth >= t0 differ
        }
        for (int t = t0; t <= D; ++t) {
            const uint64_t b = occupancy_level_start(t) + (k >> (2 * (kOmega - t)));
            atomicOr(bits + (b >> 5), 1u << (b & 31));
        }
    }
}

}  // namespace

uint64_t occupancy_words(int D) { return (occupancy_level_start(D + 1) + 31) / 32; }

sfc_status build_occupancy(sfc_index* idx, cudaStream_t st)
{
    const int D = idx->opt.occupancy_depth;
    if (D <= 0) return SFC_OK;
    const uint64_t words = occupancy_words(D);
    SFC_TRY(idx->occ.ensure(words * sizeof(uint32_t), st));
    SFC_CUDA_TRY(cudaMemsetAsync(idx->occ.ptr, 0, words * sizeof(uint32_t), st));
    if (idx->n == 0) return SFC_OK;
    const uint64_t want = (idx->n + kThreads - 1) / kThreads;
    const unsigned g = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)num_sms() * 8));
    occupancy_kernel<<<g, kThreads, 0, st>>>(idx->keys.as<uint64_t>(), idx->n, D, idx->occ.as<uint32_t>());
    count_launch();
    return launch_status();
}

}  // namespace sfc
