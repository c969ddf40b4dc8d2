// batch_kernels.cu - breadth-first initialisation of batched runs (Sec. 4.3's
// initialisation phase, for every query of a batch at once, inside the
// captured graph). Each query owns a region of two frontier buffers; one
// launch expands every active query by one level. A query stops expanding
// when its frontier reaches its row target, when the next level would not
// fit its region (the current frontier is kept), or one level short of its
// last query vertex. The extension kernel then takes 32-row tasks from these
// pools, so even a query anchored at one data vertex spreads over the GPU.
#include "launch.h"
#include "sgm_device.cuh"

namespace {

constexpr int kThreads = 256;

// Roots of the queries that start from a breadth-first pool: the root-range
// candidates of phi[0], one block per query.
__global__ void batch_bfs_roots_kernel(BatchArgs B) {
    const int q = blockIdx.x;
    BatchBfs& b = B.bfs[q];
    if (b.depth != 1) return;  // root-chunk queries (depth 0) start elsewhere
    const QueryPlan& P = B.plans[q];
    int32_t* out = B.fr[0] + b.off;
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)P.root_lo + threadIdx.x; v0 - lane < P.root_hi; v0 += blockDim.x) {
        const bool ok = v0 < P.root_hi && sgm_bit(P.lv[0].bits, (int32_t)v0);
        const unsigned m = __ballot_sync(SGM_FULL, ok);
        if (!m) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&b.next_n, (unsigned long long)__popc(m));
        base = __shfl_sync(SGM_FULL, base, 0);
        const unsigned long long pos = base + __popc(m & sgm_lanemask_lt());
        if (ok && pos < (unsigned long long)b.cap_rows) out[pos] = (int32_t)v0;
    }
}

// After the roots: the frontier is the root list (the host sized every
// breadth-first query's region for its whole root range).
__global__ void batch_bfs_start_kernel(BatchArgs B, int32_t nq) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    BatchBfs& b = B.bfs[q];
    if (b.depth != 1) return;
    const int k = B.plans[q].k;
    b.n = min(b.next_n, (unsigned long long)b.cap_rows);
    b.next_n = 0;
    b.cur = 0;
    b.active = (b.n > 0 && b.n < b.tau && 1 < k - 1) ? 1 : 0;
}

// One level d of every active query at depth d: rows of d levels in, rows of
// d + 1 levels out (the per-candidate checks of Alg. 2's Process, as in the
// single-query initialisation). Block row blockIdx.y is query q.
__global__ void batch_bfs_level_kernel(DevGraph G, BatchArgs B, int32_t d) {
    const int q = blockIdx.y;
    BatchBfs& b = B.bfs[q];
    if (!b.active || b.depth != d) return;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const LevelPlan lp = B.plans[q].lv[d];
    const int32_t* in = B.fr[b.cur] + b.off;
    int32_t* out = B.fr[b.cur ^ 1] + b.off;
    const int64_t n_in = (int64_t)b.n;
    const unsigned long long cap = (unsigned long long)b.cap_rows;
    ProbeCount pc;
    for (int64_t r = warp; r < n_in; r += nwarps) {
        const int32_t* row = in + r * d;
        const LocalList L = row_local_list(G, lp, row, d);
        const int besti = L.src & kSrcLevel;
        const uint32_t need = need_mask(lp, L.src);
        const uint32_t sb = (lp.sb_gt | lp.sb_lt) & need;
        for (int32_t j0 = 0; j0 < L.len; j0 += 32) {
            const int32_t j = j0 + lane;
            bool ok = j < L.len;
            int32_t v = 0;
            if (ok) {
                v = L.ptr[j];
                ok = sgm_bit(lp.bits, v);
                const int32_t dv = sb ? __ldg(G.deg + v) : 0;
                for (int i = 0; ok && i < d; ++i) {
                    const uint32_t bit = 1u << i;
                    if (!(need & bit)) continue;
                    const int32_t x = row[i];
                    if ((lp.inj & bit) && x == v) ok = false;
                    else if ((sb & bit) && sgm_rank_less(G, v, dv, x) == ((lp.sb_gt & bit) != 0u)) ok = false;
                    else if ((lp.bwd & bit) && i != besti) ok = sgm_member(G, x, v, pc);
                }
            }
            const unsigned m = __ballot_sync(SGM_FULL, ok);
            if (!m) continue;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(&b.next_n, (unsigned long long)__popc(m));
            base = __shfl_sync(SGM_FULL, base, 0);
            const unsigned long long pos = base + __popc(m & sgm_lanemask_lt());
            if (ok && pos < cap) {
                int32_t* o = out + pos * (d + 1);
                for (int i = 0; i < d; ++i) o[i] = row[i];
                o[d] = v;
            }
        }
    }
}

// Ends level d for every query: take the next frontier if it fit, else keep
// the current one and stop; stop at the row target or one level short of
// the query's last vertex.
__global__ void batch_bfs_commit_kernel(BatchArgs B, int32_t nq, int32_t d) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    BatchBfs& b = B.bfs[q];
    if (!b.active || b.depth != d) return;
    const unsigned long long nn = b.next_n;
    b.next_n = 0;
    if (nn > (unsigned long long)b.cap_rows) {
        b.active = 0;
        return;
    }
    const int k = B.plans[q].k;
    b.cur ^= 1;
    b.n = nn;
    b.depth = d + 1;
    if (nn == 0 || nn >= b.tau || b.depth >= k - 1) b.active = 0;
}

// task_base[q] = sum over earlier queries of ceil(n / 32) pool tasks.
__global__ void batch_tasks_kernel(BatchArgs B, int32_t nq) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    unsigned long long t = 0;
    for (int q = 0; q < nq; ++q) {
        B.task_base[q] = t;
        const BatchBfs& b = B.bfs[q];
        if (b.depth > 0) t += (b.n + 31) / 32;
    }
    B.task_base[nq] = t;
}

}  // namespace

cudaError_t sgm_launch_batch_bfs(const DevGraph& G, const BatchArgs& B, int32_t nq, int32_t max_depth,
                                 int32_t blocks_per_query, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    batch_bfs_roots_kernel<<<nq, kThreads, 0, s>>>(B);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    const int tb = 128, qb = (nq + tb - 1) / tb;
    batch_bfs_start_kernel<<<qb, tb, 0, s>>>(B, nq);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    for (int32_t d = 1; d < max_depth; ++d) {
        batch_bfs_level_kernel<<<dim3(blocks_per_query, nq), kThreads, 0, s>>>(G, B, d);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        batch_bfs_commit_kernel<<<qb, tb, 0, s>>>(B, nq, d);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
    }
    batch_tasks_kernel<<<1, 1, 0, s>>>(B, nq);
    return cudaGetLastError();
}
