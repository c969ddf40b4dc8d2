// batch_kernels.cu - the kernels of a batched run before its persistent
// extension launches (all of them captured in one CUDA graph):
//   batch_filter_kernel   candidate bitmaps of every query in one launch
//   bbfs_roots_kernel     root candidates of every breadth-first query
//   bbfs_scan_kernel      ends a level and lays out the next level's row space
//   bbfs_bound_kernel     per query, the sum of its rows' local-list lengths
//   bbfs_alloc_kernel     hands out the arena for every query's next level
//   bbfs_expand_kernel    one breadth-first level of every expanding query
//   btask_*_kernel        the final frontiers cut into 32-row and range tasks
// The breadth-first phase is Sec. 4.3's initialisation phase (Alg. 2 starts
// from the partial matches of a BFS to tau), run for every query of the batch
// at once: one launch per level covers every query still expanding, so a
// query anchored at one data vertex spreads over the whole GPU before the
// depth-first search starts, and no level needs the host.
#include <algorithm>

#include "launch.h"
#include "sgm_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kScanThreads = 1024;

// ---------------------------------------------------------------------------
// candidate filter of every query (the single-query filter_kernel's rule):
// block row blockIdx.y is query q, whose k bitmaps start at word bits_off[q]
// ---------------------------------------------------------------------------
__global__ void batch_filter_kernel(DevGraph G, const FilterSpec* __restrict__ specs,
                                    const int64_t* __restrict__ bits_off, uint32_t* __restrict__ bits) {
    __shared__ FilterSpec F;
    const int q = blockIdx.y;
    {
        const int32_t* src = (const int32_t*)(specs + q);
        int32_t* dst = (int32_t*)&F;
        for (int i = threadIdx.x; i < (int)(sizeof(FilterSpec) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t* out = bits + bits_off[q];
    const int lane = threadIdx.x & 31;
    const int64_t total = G.words * 32;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v - lane < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const bool in = v < G.n;
        const int32_t lab = (in && G.labels) ? G.labels[v] : 0;
        const int32_t d = in ? G.deg[v] : -1;
        const uint8_t* nlf = (in && G.nlf) ? G.nlf + v * G.num_labels : nullptr;
        for (int u = 0; u < F.k; ++u) {
            bool ok = in && lab == F.label[u];
            if (ok && F.use_filter) {
                ok = d >= F.dq[u];
                if (ok && nlf)
                    for (int t = 0; t < F.nneed[u]; ++t)
                        if (nlf[F.need_label[u][t]] < F.need_cnt[u][t]) { ok = false; break; }
            }
            const unsigned word = __ballot_sync(SGM_FULL, ok);
            if (lane == 0 && v < total) out[(int64_t)u * G.words + (v >> 5)] = word;
        }
    }
}

// ---------------------------------------------------------------------------
// breadth-first phase
// ---------------------------------------------------------------------------
// Roots of every breadth-first query (depth 0, active): the phi[0]
// candidates inside its root range, appended at its host-reserved arena
// offset. Block row blockIdx.y is query q.
__global__ void bbfs_roots_kernel(BatchArgs B) {
    const int q = blockIdx.y;
    BatchBfs& b = B.bfs[q];
    if (b.depth != 0 || !b.active) return;
    const QueryPlan& P = B.plans[q];
    int32_t* out = B.arena + b.off;
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = (int64_t)P.root_lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v0 - lane < P.root_hi;
         v0 += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = v0 < P.root_hi && sgm_bit(P.lv[0].bits, (int32_t)v0);
        const unsigned m = __ballot_sync(SGM_FULL, ok);
        if (!m) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&b.next_n, (unsigned long long)__popc(m));
        base = __shfl_sync(SGM_FULL, base, 0);
        if (ok) out[base + __popc(m & sgm_lanemask_lt())] = (int32_t)v0;
    }
}

// Exclusive scan of one value per thread over a block of at most
// kScanThreads threads; returns the thread's prefix and the block's sum (the
// same value in every thread). Every thread of the block must call it.
__device__ unsigned long long block_excl_scan(unsigned long long x, unsigned long long* total) {
    __shared__ unsigned long long warp_sums[kScanThreads / 32];
    __shared__ unsigned long long block_sum;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = (int)(blockDim.x >> 5);
    unsigned long long incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(SGM_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sums[w] = incl;
    __syncthreads();
    if (w == 0) {
        const unsigned long long s = lane < nw ? warp_sums[lane] : 0ull;
        unsigned long long si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(SGM_FULL, si, o);
            if (lane >= o) si += y;
        }
        if (lane < nw) warp_sums[lane] = si - s;  // exclusive prefix of each warp
        if (lane == 31) block_sum = si;
    }
    __syncthreads();
    const unsigned long long r = warp_sums[w] + incl - x;
    *total = block_sum;
    __syncthreads();
    return r;
}

// Commits level d - 1 of every query that expanded it (d = 1: the roots),
// then lays out the row space of level d: rbase[q] = first global row of
// query q among the queries still expanding at depth d (final = 1: among all
// queries with a frontier, for the task kernels). One block.
__global__ void bbfs_scan_kernel(BatchArgs B, int32_t d, int32_t final_pass) {
    __shared__ unsigned long long carry_s, tile_total;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int q0 = 0; q0 < B.nq; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        unsigned long long cnt = 0;
        if (q < B.nq) {
            BatchBfs& b = B.bfs[q];
            if (b.active && b.depth == d - 1) {
                // level d - 1 was expanded into next_off / next_n
                const int k = B.plans[q].k;
                b.n = b.next_n;
                b.off = b.next_off;
                b.next_n = 0;
                b.bound = 0;
                b.depth = d;
                B.qst[q].level[d - 1] = b.n;
                b.active = (b.n > 0 && b.n < b.tau && d < k - 1) ? 1 : 0;
            }
            if (final_pass ? (b.depth >= 1) : (b.active && b.depth == d)) cnt = b.n;
        }
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl_scan(cnt, &tot);
        if (threadIdx.x == 0) tile_total = tot;
        if (q < B.nq) B.rbase[q] = carry_s + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tile_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.rbase[B.nq] = carry_s;
        B.sc->rows = carry_s;
    }
}

// The query owning global row r of the current row space.
__device__ __forceinline__ int row_query(const unsigned long long* __restrict__ rbase, int nq, unsigned long long r) {
    int lo = 0, hi = nq;  // invariant: rbase[lo] <= r < rbase[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(rbase + mid) <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// bound[q] += the candidates of the local list C^L of every row of q at
// depth d that pass the filter of phi[d] (an upper bound on the rows it adds
// to the next frontier; on a labelled graph far below |C^L|, so the arena
// holds deeper levels). One warp per row, lanes striding over C^L.
// Warps per row of a breadth-first level: when the level has fewer rows than
// the grid has warps, each row's list is shared by up to 64 warps (warp part
// p of K takes the 32-entry chunks p, p + K, p + 2K, ...), so that a hub's
// list does not hold the level on one warp.
__device__ __forceinline__ unsigned long long parts_per_row(unsigned long long rows, unsigned long long nwarps) {
    return rows == 0 ? 1ull : max(1ull, min(64ull, nwarps / rows));
}

__global__ void bbfs_bound_kernel(DevGraph G, BatchArgs B, int32_t d) {
    const int lane = threadIdx.x & 31;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long rows = B.sc->rows;
    const unsigned long long K = parts_per_row(rows, nwarps);
    for (unsigned long long w = warp; w < rows * K; w += nwarps) {
        const unsigned long long r = w / K;
        const int32_t part = (int32_t)(w - r * K);
        const int q = row_query(B.rbase, B.nq, r);
        const BatchBfs& b = B.bfs[q];
        const LevelPlan& lp = B.plans[q].lv[d];
        const int32_t* row = B.arena + b.off + (r - B.rbase[q]) * (unsigned long long)d;
        const LocalList L = row_local_list(G, lp, row, d);
        int32_t c = 0;
        for (int32_t j = part * 32 + lane; j < L.len; j += 32 * (int32_t)K) c += sgm_bit(lp.bits, __ldg(L.ptr + j));
        c = __reduce_add_sync(SGM_FULL, c);
        if (lane == 0 && c) atomicAdd(&B.bfs[q].bound, (unsigned long long)c);
    }
}

// Hands out the arena for level d + 1, query by query in order: a query
// whose bound does not fit stops expanding (its depth-d frontier is kept).
// Then lays out the row space of the queries that got room. One block; the
// per-query values go through shared memory so that one thread can decide
// the allocations in order.
__global__ void bbfs_alloc_kernel(BatchArgs B, int32_t d) {
    __shared__ unsigned long long need_s[kScanThreads];
    __shared__ unsigned long long used_s, carry_s, tile_total;
    if (threadIdx.x == 0) {
        used_s = B.sc->arena_used;
        carry_s = 0;
    }
    __syncthreads();
    for (int q0 = 0; q0 < B.nq; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const bool live = q < B.nq && B.bfs[q].active && B.bfs[q].depth == d;
        need_s[threadIdx.x] = live ? B.bfs[q].bound * (unsigned long long)(d + 1) : 0ull;
        __syncthreads();
        if (threadIdx.x == 0) {
            // in query order; ~0 marks a query that does not fit
            const int nt = min((int)blockDim.x, B.nq - q0);
            unsigned long long used = used_s;
            for (int t = 0; t < nt; ++t) {
                const unsigned long long nd = need_s[t];
                if (nd == 0) {
                    need_s[t] = used;
                } else if (used + nd <= B.arena_cap) {
                    need_s[t] = used;
                    used += nd;
                } else {
                    need_s[t] = ~0ull;
                }
            }
            used_s = used;
        }
        __syncthreads();
        unsigned long long cnt = 0;
        if (live) {
            BatchBfs& b = B.bfs[q];
            if (need_s[threadIdx.x] == ~0ull) {
                b.active = 0;
                B.sc->arena_full = 1;
            } else {
                b.next_off = (int64_t)need_s[threadIdx.x];
                cnt = b.n;
            }
        }
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl_scan(cnt, &tot);
        if (threadIdx.x == 0) tile_total = tot;
        if (q < B.nq) B.rbase[q] = carry_s + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tile_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        B.rbase[B.nq] = carry_s;
        B.sc->rows = carry_s;
        B.sc->arena_used = used_s;
    }
}

// One breadth-first level of every query with room: rows of d levels in,
// rows of d + 1 levels out (Alg. 2's Process checks for every candidate of
// the row's local list, as in the single-query initialisation); one warp per
// row, survivors appended with warp-aggregated atomics.
__global__ void bbfs_expand_kernel(DevGraph G, BatchArgs B, int32_t d) {
    const int lane = threadIdx.x & 31;
    const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nwarps = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    const unsigned long long rows = B.sc->rows;
    const unsigned long long K = parts_per_row(rows, nwarps);
    ProbeCount pc;
    for (unsigned long long w = warp; w < rows * K; w += nwarps) {
        const unsigned long long r = w / K;
        const int32_t part = (int32_t)(w - r * K);
        const int q = row_query(B.rbase, B.nq, r);
        BatchBfs& b = B.bfs[q];
        const LevelPlan& lp = B.plans[q].lv[d];
        const int32_t* row = B.arena + b.off + (r - B.rbase[q]) * (unsigned long long)d;
        int32_t* out = B.arena + b.next_off;
        const LocalList L = row_local_list(G, lp, row, d);
        const int besti = L.src & kSrcLevel;
        const uint32_t need = need_mask(lp, L.src);
        const uint32_t sb = (lp.sb_gt | lp.sb_lt) & need;
        const uint32_t* bits = lp.bits;
        for (int32_t j0 = part * 32; j0 < L.len; j0 += 32 * (int32_t)K) {
            const int32_t j = j0 + lane;
            bool ok = j < L.len;
            int32_t v = 0;
            if (ok) {
                v = L.ptr[j];
                ok = sgm_bit(bits, v);
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
            if (ok) {
                int32_t* o = out + (base + __popc(m & sgm_lanemask_lt())) * (unsigned long long)(d + 1);
                for (int i = 0; i < d; ++i) o[i] = row[i];
                o[d] = v;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// tasks from the final frontiers
// ---------------------------------------------------------------------------
// Does query q's final frontier cut long rows into range tasks? Not when its
// rows are one level short of an arithmetically counted last level (those
// rows are counted without scanning a list).
__device__ __forceinline__ bool splits_rows(const QueryPlan& P, int depth) {
    return P.pool_chunk > 0 && !(P.arith && depth == P.k - 1);
}

// nrange[q] = range tasks of q's rows whose local list for level `depth`
// is longer than the plan's pool_chunk.
__global__ void btask_count_kernel(DevGraph G, BatchArgs B) {
    const unsigned long long rows = B.sc->rows;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < rows;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const int q = row_query(B.rbase, B.nq, r);
        const BatchBfs& b = B.bfs[q];
        const QueryPlan& P = B.plans[q];
        const int d = b.depth;
        if (d >= P.k || !splits_rows(P, d)) continue;
        const int32_t* row = B.arena + b.off + (r - B.rbase[q]) * (unsigned long long)d;
        const int32_t len = row_local_list(G, P.lv[d], row, d).len;
        if (len > P.pool_chunk)
            atomicAdd(&B.bfs[q].nrange, (unsigned long long)((len + P.pool_chunk - 1) / P.pool_chunk));
    }
}

// Per query: its range records get room in the arena (all queries or, when
// they do not fit, none: such queries process their long rows whole), and
// task_base[q] = its first task (exclusive scan over all queries, classes
// contiguous) with range tasks before 32-row tasks; per class, its task
// range. One block.
__global__ void btask_plan_kernel(BatchArgs B, int32_t ncls) {
    __shared__ unsigned long long carry_s;
    __shared__ int32_t fits_s;
    // range records: room for every query's, or for none
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int q0 = 0; q0 < B.nq; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        const unsigned long long nr = q < B.nq ? B.bfs[q].nrange : 0ull;
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl_scan(nr, &tot);
        if (q < B.nq) B.bfs[q].range_off = (int64_t)(B.sc->arena_used + 4ull * (carry_s + ex));
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long need = 4ull * carry_s;
        fits_s = B.sc->arena_used + need <= B.arena_cap ? 1 : 0;
        if (fits_s) B.sc->arena_used += need;
        carry_s = 0;
    }
    __syncthreads();
    // tasks: range tasks, then 32-row tasks, query by query
    for (int q0 = 0; q0 < B.nq; q0 += blockDim.x) {
        const int q = q0 + threadIdx.x;
        unsigned long long cnt = 0;
        if (q < B.nq) {
            BatchBfs& b = B.bfs[q];
            b.split = (fits_s && b.nrange > 0) ? 1 : 0;
            b.range_fill = 0;
            if (b.depth >= 1 && b.depth < B.plans[q].k) cnt = (b.split ? b.nrange : 0ull) + (b.n + 31) / 32;
        }
        unsigned long long tot = 0;
        const unsigned long long ex = block_excl_scan(cnt, &tot);
        if (q < B.nq) B.task_base[q] = carry_s + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry_s += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) B.task_base[B.nq] = carry_s;
    __syncthreads();
    for (int c = threadIdx.x; c < ncls; c += blockDim.x) {
        BatchClass& C = B.cls[c];
        C.task0 = B.task_base[C.q0];
        C.n_tasks = B.task_base[C.q1] - C.task0;
    }
}

// Writes the range records of every long row (queries with split = 1).
__global__ void btask_fill_kernel(DevGraph G, BatchArgs B) {
    const unsigned long long rows = B.sc->rows;
    for (unsigned long long r = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; r < rows;
         r += (unsigned long long)gridDim.x * blockDim.x) {
        const int q = row_query(B.rbase, B.nq, r);
        const BatchBfs& b = B.bfs[q];
        if (!b.split) continue;
        const QueryPlan& P = B.plans[q];
        const int d = b.depth;
        const unsigned long long rr = r - B.rbase[q];
        const int32_t* row = B.arena + b.off + rr * (unsigned long long)d;
        const int32_t len = row_local_list(G, P.lv[d], row, d).len;
        if (len <= P.pool_chunk) continue;
        const int nch = (len + P.pool_chunk - 1) / P.pool_chunk;
        const unsigned long long at = atomicAdd(&B.bfs[q].range_fill, (unsigned long long)nch);
        BatchRange* rec = (BatchRange*)(B.arena + b.range_off) + at;
        for (int j = 0; j < nch; ++j) {
            BatchRange t;
            t.q = q;
            t.row = (int32_t)rr;
            t.lo = j * P.pool_chunk;
            t.hi = min(len, (j + 1) * P.pool_chunk);
            rec[j] = t;
        }
    }
}

inline int grid_rows(int sms) { return 8 * sms; }

}  // namespace

cudaError_t sgm_launch_batch_filter(const DevGraph& G, const FilterSpec* specs, const int64_t* bits_off,
                                    uint32_t* bits, int32_t nq, int32_t sms, cudaStream_t s, size_t bits_words) {
    if (nq <= 0) return cudaSuccess;
    if (G.lab_vert) {
        // labelled: only each query vertex's label bucket, about 16 warps per SM over the batch
        const int wpq = std::max(8, std::min(32 * sms, 16 * sms * 8 / nq));
        return sgm_launch_filter_buckets(G, specs, nullptr, bits_off, bits, bits_words, nq, wpq, s);
    }
    const int64_t items = G.words * 32;
    int64_t gx = (4LL * sms * 8 + nq - 1) / nq;  // about 4 x 8 blocks per SM over the whole batch
    gx = std::max<int64_t>(1, std::min<int64_t>(gx, (items + kThreads - 1) / kThreads));
    batch_filter_kernel<<<dim3((unsigned)gx, nq), kThreads, 0, s>>>(G, specs, bits_off, bits);
    return cudaGetLastError();
}

cudaError_t sgm_launch_batch_bfs(const DevGraph& G, const BatchArgs& B, int32_t max_depth, int32_t root_blocks,
                                 int32_t sms, cudaStream_t s, uint64_t* launches) {
    if (B.nq <= 0) return cudaSuccess;
    cudaError_t err;
    bbfs_roots_kernel<<<dim3(root_blocks, B.nq), kThreads, 0, s>>>(B);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    ++*launches;
    for (int32_t d = 1; d < max_depth; ++d) {
        bbfs_scan_kernel<<<1, kScanThreads, 0, s>>>(B, d, 0);
        bbfs_bound_kernel<<<grid_rows(sms) * 4, kThreads, 0, s>>>(G, B, d);
        bbfs_alloc_kernel<<<1, kScanThreads, 0, s>>>(B, d);
        bbfs_expand_kernel<<<grid_rows(sms) * 4, kThreads, 0, s>>>(G, B, d);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        *launches += 4;
    }
    // commit the last level and lay out the final frontiers
    bbfs_scan_kernel<<<1, kScanThreads, 0, s>>>(B, max_depth, 1);
    ++*launches;
    return cudaGetLastError();
}

cudaError_t sgm_launch_batch_tasks(const DevGraph& G, const BatchArgs& B, int32_t ncls, int32_t sms, cudaStream_t s,
                                   uint64_t* launches) {
    if (B.nq <= 0) return cudaSuccess;
    btask_count_kernel<<<grid_rows(sms) * 4, kThreads, 0, s>>>(G, B);
    btask_plan_kernel<<<1, kScanThreads, 0, s>>>(B, ncls);
    btask_fill_kernel<<<grid_rows(sms) * 4, kThreads, 0, s>>>(G, B);
    *launches += 3;
    return cudaGetLastError();
}
