// graph_kernels.cu - per-graph tables built once when G is loaded: degrees,
// CSR validation, 8-bit labels with their histogram, neighbour-label
// frequencies and hub adjacency bitmaps.
#include "launch.h"
#include "sgm_device.cuh"

namespace {

constexpr int kThreads = 256;

inline int grid_for(int64_t items, int per_block = kThreads) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > (1 << 20)) g = 1 << 20;
    return (int)g;
}

__global__ void degrees_kernel(const int64_t* __restrict__ rowptr, int64_t n, int32_t* __restrict__ deg,
                               int32_t* flags) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rowptr[v + 1] - rowptr[v];
        if (d < 0 || d > INT_MAX) {
            atomicOr(flags, SGM_VF_RANGE);
            deg[v] = 0;
        } else {
            deg[v] = (int32_t)d;
        }
    }
}

// One warp per row: every column in range, rows strictly increasing (sorted,
// no duplicates), no self-loop, and the reverse entry present (symmetry).
__global__ void validate_kernel(DevGraph G, int32_t* flags) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    ProbeCount pc;
    for (int64_t v = warp; v < G.n; v += nwarps) {
        const int64_t b = G.rowptr[v];
        const int32_t d = G.deg[v];
        int32_t f = 0;
        for (int32_t j = lane; j < d; j += 32) {
            const int32_t y = G.col[b + j];
            if (y < 0 || y >= G.n) {
                f |= SGM_VF_RANGE;
                continue;
            }
            if (y == v) f |= SGM_VF_SELF_LOOP;
            if (j + 1 < d && G.col[b + j + 1] <= y) f |= SGM_VF_UNSORTED;
        }
        f = __reduce_or_sync(SGM_FULL, f);
        if (f) {
            if (lane == 0) atomicOr(flags, f);
            continue;
        }
        for (int32_t j = lane; j < d; j += 32) {
            const int32_t y = G.col[b + j];
            // bisection in N(y) for v, without the hub bitmaps (not built yet)
            const int32_t* a = G.col + G.rowptr[y];
            int32_t len = G.deg[y];
            bool found = false;
            while (len > 0) {
                const int32_t half = len >> 1;
                const int32_t c = a[half];
                if (c == v) { found = true; break; }
                if (c < v) { a += half + 1; len -= half + 1; } else len = half;
            }
            if (!found) f |= SGM_VF_ASYMMETRIC;
        }
        f = __reduce_or_sync(SGM_FULL, f);
        if (f && lane == 0) atomicOr(flags, f);
    }
    (void)pc;
}

__global__ void labels_kernel(const int32_t* __restrict__ in, int64_t n, int32_t num_labels, uint8_t* __restrict__ out,
                              int32_t* flags, unsigned long long* hist) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t l = in[v];
        if (l < 0 || l >= num_labels) {
            atomicOr(flags, SGM_VF_LABEL);
            out[v] = 0;
        } else {
            out[v] = (uint8_t)l;
            atomicAdd(hist + l, 1ull);
        }
    }
}

// Neighbour-label frequency: nlf[v * L + l] = min(255, #{w in N(v) : L(w) = l}).
// One warp per vertex with a per-warp shared histogram.
__global__ void nlf_kernel(DevGraph G, uint8_t* __restrict__ nlf) {
    extern __shared__ uint32_t hist_all[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int L = G.num_labels;
    uint32_t* hist = hist_all + wib * L;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = warp; v < G.n; v += nwarps) {
        for (int l = lane; l < L; l += 32) hist[l] = 0;
        __syncwarp();
        const int64_t b = G.rowptr[v];
        const int32_t d = G.deg[v];
        for (int32_t j = lane; j < d; j += 32) atomicAdd(hist + G.labels[G.col[b + j]], 1u);
        __syncwarp();
        for (int l = lane; l < L; l += 32) nlf[v * L + l] = (uint8_t)min(hist[l], 255u);
        __syncwarp();
    }
}

// One block per hub: set bit y of the hub's bitmap for every y in N(hub).
__global__ void hub_bits_kernel(DevGraph G, const int32_t* __restrict__ hub_list, uint32_t* __restrict__ bits) {
    const int32_t h = blockIdx.x;
    const int32_t x = hub_list[h];
    uint32_t* row = bits + (int64_t)h * G.words;
    const int64_t b = G.rowptr[x];
    const int32_t d = G.deg[x];
    for (int32_t j = threadIdx.x; j < d; j += blockDim.x) {
        const int32_t y = G.col[b + j];
        atomicOr(row + (y >> 5), 1u << (y & 31));
    }
}

// Upper-rank adjacency N+(w) = {x in N(w) : rank(x) > rank(w)}, rank = (degree,
// id): the candidates of a query vertex that symmetry breaking places above
// its list owner's image. Pass 1 counts, pass 2 copies (order kept, so rows
// stay sorted by id). One warp per vertex.
__global__ void up_count_kernel(DevGraph G, int32_t* __restrict__ updeg) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < G.n; w += nwarps) {
        const int64_t b = G.rowptr[w];
        const int32_t d = G.deg[w];
        int32_t c = 0;
        for (int32_t j = lane; j < d; j += 32) c += sgm_rank_less(G, (int32_t)w, d, G.col[b + j]);
        c = __reduce_add_sync(SGM_FULL, c);
        if (lane == 0) updeg[w] = c;
    }
}

__global__ void up_fill_kernel(DevGraph G, const int64_t* __restrict__ up_rowptr, int32_t* __restrict__ up_col) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp; w < G.n; w += nwarps) {
        const int64_t b = G.rowptr[w];
        const int32_t d = G.deg[w];
        int64_t o = up_rowptr[w];
        for (int32_t j0 = 0; j0 < d; j0 += 32) {
            const int32_t j = j0 + lane;
            const int32_t x = j < d ? G.col[b + j] : 0;
            const bool keep = j < d && sgm_rank_less(G, (int32_t)w, d, x);
            const unsigned m = __ballot_sync(SGM_FULL, keep);
            if (keep) up_col[o + __popc(m & sgm_lanemask_lt())] = x;
            o += __popc(m);
        }
    }
}

}  // namespace

cudaError_t sgm_launch_up_count(const DevGraph& G, int32_t* updeg, cudaStream_t s) {
    if (G.n <= 0) return cudaSuccess;
    up_count_kernel<<<grid_for(G.n * 32), kThreads, 0, s>>>(G, updeg);
    return cudaGetLastError();
}

cudaError_t sgm_launch_up_fill(const DevGraph& G, const int64_t* up_rowptr, int32_t* up_col, cudaStream_t s) {
    if (G.n <= 0) return cudaSuccess;
    up_fill_kernel<<<grid_for(G.n * 32), kThreads, 0, s>>>(G, up_rowptr, up_col);
    return cudaGetLastError();
}

cudaError_t sgm_launch_degrees(const int64_t* rowptr, int64_t n, int32_t* deg, int32_t* flags, cudaStream_t s) {
    degrees_kernel<<<grid_for(n), kThreads, 0, s>>>(rowptr, n, deg, flags);
    return cudaGetLastError();
}

cudaError_t sgm_launch_validate(const DevGraph& G, int32_t* flags, cudaStream_t s) {
    validate_kernel<<<grid_for(G.n * 32), kThreads, 0, s>>>(G, flags);
    return cudaGetLastError();
}

cudaError_t sgm_launch_labels(const int32_t* in, int64_t n, int32_t num_labels, uint8_t* out, int32_t* flags,
                              unsigned long long* hist, cudaStream_t s) {
    labels_kernel<<<grid_for(n), kThreads, 0, s>>>(in, n, num_labels, out, flags, hist);
    return cudaGetLastError();
}

cudaError_t sgm_launch_nlf(const DevGraph& G, uint8_t* nlf, cudaStream_t s) {
    const size_t smem = sizeof(uint32_t) * G.num_labels * (kThreads / 32);
    nlf_kernel<<<grid_for(G.n * 32), kThreads, smem, s>>>(G, nlf);
    return cudaGetLastError();
}

cudaError_t sgm_launch_hub_bits(const DevGraph& G, const int32_t* hub_list, int32_t hubs, uint32_t* bits,
                                cudaStream_t s) {
    if (hubs <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)G.words * hubs, s);
    if (e != cudaSuccess) return e;
    hub_bits_kernel<<<hubs, kThreads, 0, s>>>(G, hub_list, bits);
    return cudaGetLastError();
}
