// coarse_kernels.cu - the coarse-grained parallel model the paper measures
// its fine-grained model against (Alg. 1, DFS-Search with Process; Sec. 2.3
// loop unrolling; the ablation of Sec. 6.3, Table 4), kept as a baseline:
// a warp owns one partial match at a time, scans the match's local candidate
// list C^L with its 32 lanes (Process: label filter, injectivity, membership
// in the other backward neighbours' lists) and materialises the feasible
// candidates C^F of every level in its own execution stack in global memory,
// O(k x d_max) per warp (Issue 1 of Sec. 2.3). With loop unrolling (unroll =
// sigma > 1) the warp takes sigma sibling partial matches per step and its
// lanes scan their concatenated C^L lists, with sigma buffers per level
// (O(k x d_max x sigma)). The leaf level is counted, not stored. Idle lanes
// of every scan round are counted (the idle rate of Table 1).
#include <algorithm>

#include "launch.h"
#include "sgm_device.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxUnroll = 8;  // the unroll factors of Sec. 2.3 and Table 4 go up to 8

// Per-warp state of the depth-first search, in shared memory.
struct CoarseWarp {
    int32_t M[SGM_KMAX];                 // the current partial match, by level
    int32_t nsub[SGM_KMAX];              // sub-buffers at each level (partial matches of its batch)
    int32_t cs[SGM_KMAX];                // current sub-buffer of each level
    int32_t cp[SGM_KMAX];                // position in it
    int32_t cnt[SGM_KMAX][kMaxUnroll];   // feasible candidates in each sub-buffer
    int32_t par[SGM_KMAX][kMaxUnroll];   // the level-(l-1) vertex each sub-buffer extends
    int32_t len[kMaxUnroll];             // scratch: C^L of each partial match of the batch
    int32_t own[32];                     // scratch: owner of each round position where a list starts
    const int32_t* lst[kMaxUnroll];
    int32_t src[kMaxUnroll];
};

// Process (Alg. 1) for a batch of t partial matches that share M[0..l-1] and
// map phi[l] to vs[s] (s < t; for l == D - 1 the batch is the pool row
// itself, t = 1): the feasible candidates of phi[l + 1] of each into
// sub-buffer s of level l + 1 (or, at the last level, only their number).
__device__ unsigned long long coarse_process(const DevGraph& G, const QueryPlan& P, CoarseWarp& W, int l,
                                             const int32_t* vs, int t, int32_t* buf, int64_t dmax, int sigma,
                                             unsigned long long& idle, unsigned long long& rounds,
                                             unsigned long long& cand, ProbeCount& pc) {
    const int lane = threadIdx.x & 31;
    const int nl = l + 1;
    const LevelPlan& lp = P.lv[nl];
    const bool leaf = nl == P.k - 1;
    // the local list of each partial match: the smallest backward list
    if (lane < t) {
        int32_t bestd = INT_MAX, besti = 0, bestx = 0;
        for (int i = 0; i <= l; ++i)
            if ((lp.bwd >> i) & 1u) {
                const int32_t x = i == l ? vs[lane] : W.M[i];
                const int32_t dx = __ldg(G.deg + x);
                if (dx < bestd) { bestd = dx; besti = i; bestx = x; }
            }
        W.len[lane] = bestd == INT_MAX ? 0 : bestd;
        W.lst[lane] = G.col + __ldg(G.rowptr + bestx);
        W.src[lane] = besti;
        if (!leaf) W.cnt[nl][lane] = 0;
    }
    __syncwarp();
    const int ls = lane < t ? W.len[lane] : 0;
    const int incl = sgm_warp_incl_scan(ls);
    const int total = __shfl_sync(SGM_FULL, incl, 31);
    const int excl = incl - ls;
    unsigned long long found = 0;
    for (int base = 0; base < total; base += 32) {
        const int g = base + lane;
        const bool valid = g < total;
        // the partial match owning round position `lane`: the last one whose
        // list starts at or before g (an owner table by round position)
        const bool starts_here = lane < t && ls > 0 && excl > base && excl - base < 32;
        if (starts_here) W.own[excl - base] = lane;
        const unsigned posmask = __reduce_or_sync(SGM_FULL, starts_here ? 1u << (excl - base) : 0u);
        const unsigned carried_m = __ballot_sync(SGM_FULL, lane < t && ls > 0 && excl <= base);
        __syncwarp();
        const unsigned prev = posmask & ((2u << lane) - 1u);
        const int s = prev ? W.own[31 - __clz(prev)] : (carried_m ? 31 - __clz(carried_m) : 0);
        const int32_t ex_s = __shfl_sync(SGM_FULL, excl, s);
        __syncwarp();
        rounds += lane == 0;
        idle += lane == 0 ? (unsigned long long)(32 - min(32, total - base)) : 0ull;
        bool ok = false;
        int32_t v = 0;
        if (valid) {
            const int src = W.src[s];
            v = __ldg(W.lst[s] + (g - ex_s));
            cand += 1;
            pc.filter++;
            ok = sgm_bit(lp.bits, v);
            for (int i = 0; ok && i <= l; ++i) {
                const uint32_t bit = 1u << i;
                const int32_t x = i == l ? vs[s] : W.M[i];
                if ((lp.inj & bit) && x == v) ok = false;
                else if ((lp.bwd & bit) && i != src) ok = sgm_member(G, x, v, pc);
            }
        }
        const unsigned m = __ballot_sync(SGM_FULL, ok);
        if (leaf) {
            found += lane == 0 ? (unsigned long long)__popc(m) : 0ull;  // summed over the warp at the end
            continue;
        }
        // append the survivors of each partial match to its sub-buffer
        const unsigned peers = __match_any_sync(SGM_FULL, ok ? s : -1 - lane);
        if (ok) {
            const int leader = __ffs(peers) - 1;
            int at = 0;
            if (lane == leader) at = atomicAdd(&W.cnt[nl][s], __popc(peers));
            at = __shfl_sync(peers, at, leader) + __popc(peers & sgm_lanemask_lt());
            buf[((int64_t)nl * sigma + s) * dmax + at] = v;
        }
        __syncwarp();
    }
    if (!leaf && lane < t) W.par[nl][lane] = vs[lane];
    if (lane == 0) {
        W.nsub[nl] = leaf ? 0 : t;
        W.cs[nl] = 0;
        W.cp[nl] = 0;
    }
    __syncwarp();
    return found;
}

__global__ void __launch_bounds__(kThreads) coarse_kernel(DevGraph G, const QueryPlan* __restrict__ Pg, PoolArgs pa,
                                                          RunState* st, int32_t* __restrict__ stack, int64_t dmax,
                                                          int32_t sigma, unsigned long long cap_ns) {
    __shared__ QueryPlan P;
    __shared__ CoarseWarp Ws[kWarps];
    __shared__ int32_t vsb[kWarps][kMaxUnroll];
    {
        const int32_t* src = (const int32_t*)Pg;
        int32_t* dst = (int32_t*)&P;
        for (int i = threadIdx.x; i < (int)(sizeof(QueryPlan) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * kWarps + wib;
    CoarseWarp& W = Ws[wib];
    int32_t* vs = vsb[wib];
    int32_t* buf = stack + gw * (int64_t)P.k * sigma * dmax;
    const int D = P.D, k = P.k;
    unsigned long long count = 0, idle = 0, rounds = 0, cand = 0, groups = 0;
    ProbeCount pc;
    const unsigned long long t0 = sgm_globaltimer();
    unsigned iter = 0;
    bool stop = false;
    while (!stop) {
        unsigned long long r = 0;
        if (lane == 0) r = atomicAdd(&st->pool_head, 1ull);
        r = __shfl_sync(SGM_FULL, r, 0);
        if (r >= (unsigned long long)pa.n_short) break;
        const int64_t row = pa.short_idx ? (int64_t)__ldg(pa.short_idx + r) : (int64_t)r;
        if (lane < D) W.M[lane] = pa.rows[row * D + lane];
        if (lane == 0) vs[0] = pa.rows[row * D + D - 1];
        __syncwarp();
        // the pool row is a batch of one partial match at level D - 1
        count += coarse_process(G, P, W, D - 1, vs, 1, buf, dmax, sigma, idle, rounds, cand, pc);
        groups += lane == 0;
        int l = D;
        while (l >= D) {
            // every 256 steps: stop when the run is stopped or past its time cap
            if ((++iter & 255u) == 0u) {
                int f = 0;
                if (lane == 0) {
                    if (*(volatile int32_t*)&st->status != 0) f = 1;
                    else if (cap_ns && sgm_globaltimer() - t0 > cap_ns) {
                        atomicCAS(&st->status, 0, SGM_E_TIME_CAP);
                        f = 1;
                    }
                }
                if (__shfl_sync(SGM_FULL, f, 0)) {
                    stop = true;
                    break;
                }
            }
            if (l >= k - 1 || W.cs[l] >= W.nsub[l]) {
                --l;  // level done
                continue;
            }
            const int s = W.cs[l];
            const int c = W.cnt[l][s];
            const int p = W.cp[l];
            if (p >= c) {
                if (lane == 0) {
                    W.cs[l] = s + 1;
                    W.cp[l] = 0;
                }
                __syncwarp();
                continue;
            }
            // the next batch: up to sigma siblings of sub-buffer s
            const int t = min(sigma, c - p);
            if (lane < t) vs[lane] = buf[((int64_t)l * sigma + s) * dmax + p + lane];
            if (lane == 0) {
                W.cp[l] = p + t;
                W.M[l - 1] = W.par[l][s];
            }
            __syncwarp();
            count += coarse_process(G, P, W, l, vs, t, buf, dmax, sigma, idle, rounds, cand, pc);
            groups += lane == 0 ? (unsigned long long)t : 0ull;
            if (l + 1 < k - 1) ++l;
        }
    }
    count = sgm_warp_sum_u64(count);
    const unsigned long long cc = sgm_warp_sum_u64(cand);
    const unsigned long long sp = sgm_warp_sum_u64(pc.search), bp = sgm_warp_sum_u64(pc.bitmap);
    const unsigned long long fp = sgm_warp_sum_u64(pc.filter), al = sgm_warp_sum_u64(pc.alg);
    if (lane == 0) {
        sgm_add_checked(&st->count, count, &st->overflow);
        atomicAdd(&st->cand_checked, cc);
        atomicAdd(&st->list_elems, cc);
        atomicAdd(&st->search_probes, sp);
        atomicAdd(&st->bitmap_probes, bp);
        atomicAdd(&st->filter_probes, fp);
        atomicAdd(&st->alg_bytes, al + 4ull * cc);
        atomicAdd(&st->task_groups, groups);
        atomicAdd(&st->scatter_rounds, rounds);
        atomicAdd(&st->idle_lanes, idle);
    }
}

}  // namespace

int32_t sgm_coarse_warps(int32_t sms, int32_t k, int32_t sigma, int64_t dmax, int64_t budget_bytes) {
    const int64_t per_warp = (int64_t)k * sigma * std::max<int64_t>(dmax, 1) * 4;
    const int64_t by_memory = std::max<int64_t>(kWarps, budget_bytes / per_warp);
    const int64_t by_occupancy = (int64_t)sms * 32;  // 32 resident warps per SM at most
    return (int32_t)(std::min(by_memory, by_occupancy) / kWarps * kWarps);
}

cudaError_t sgm_launch_coarse(const DevGraph& G, const QueryPlan* P, const PoolArgs& pa, RunState* st,
                              int32_t* stack, int64_t dmax, int32_t sigma, int32_t warps, uint64_t cap_ns,
                              cudaStream_t s) {
    if (sigma < 1 || sigma > kMaxUnroll || warps < kWarps) return cudaErrorInvalidValue;
    coarse_kernel<<<warps / kWarps, kThreads, 0, s>>>(G, P, pa, st, stack, dmax, sigma, cap_ns);
    return cudaGetLastError();
}
