// refine_kernels.cu - one round of the candidate-set refinement on the GPU
// (the support rule of refine.cuh applied to every data vertex).
#include "launch.h"
#include "refine.cuh"

namespace {

constexpr int kThreads = 256;

// nxt starts as a copy of cur; every candidate bit that loses its support is
// cleared in nxt (atomically: 32 vertices share a word), and *changed is set.
__global__ void refine_kernel(DevGraph G, RefineSpec R, const uint32_t* __restrict__ cur, uint32_t* nxt,
                              int32_t* changed) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < G.n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = v >> 5;
        const uint32_t bit = 1u << (v & 31);
        uint32_t in = 0;
        for (int u = 0; u < R.k; ++u)
            if (__ldg(cur + (int64_t)u * G.words + w) & bit) in |= 1u << u;
        if (!in) continue;
        uint32_t drop = in & ~sgm_refine_vertex(G.rowptr, G.col, v, cur, G.words, R.k, R.qadj, in);
        if (!drop) continue;
        atomicOr(changed, 1);
        while (drop) {
            const int u = sgm_low_bit(drop);
            drop &= drop - 1u;
            atomicAnd(nxt + (int64_t)u * G.words + w, ~bit);
        }
    }
}

}  // namespace

cudaError_t sgm_launch_refine(const DevGraph& G, const RefineSpec& R, const uint32_t* cur, uint32_t* nxt,
                              int32_t* changed, cudaStream_t s) {
    if (G.n <= 0 || R.k <= 0) return cudaSuccess;
    int64_t blocks = (G.n + kThreads - 1) / kThreads;
    if (blocks > (1 << 20)) blocks = 1 << 20;
    refine_kernel<<<(int)blocks, kThreads, 0, s>>>(G, R, cur, nxt, changed);
    return cudaGetLastError();
}
