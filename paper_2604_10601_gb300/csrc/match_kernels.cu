// match_kernels.cu - the matching hot path on sm_103a:
//   filter_kernel      candidate bitmaps (label, degree, neighbour-label frequency)
//   roots_kernel       root candidates of phi[0] (first level of Alg. 1 BFS-Search)
//   bfs_*_kernel       initialization phase: breadth-first expansion to tau
//                      partial matches (Sec. 4.3; Alg. 2 line 1)
//   extend_kernel      persistent fine-grained search (Alg. 2) with warp-level
//                      batch exploration (Sec. 4.2) and a queue of stealable
//                      candidate ranges (Sec. 4.3, dynamic balancing)
#include <algorithm>
#include <cstring>

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

// ---------------------------------------------------------------------------
// candidate filter: bit v of bitmap u set iff v may be the image of u
// ---------------------------------------------------------------------------
__global__ void filter_kernel(DevGraph G, FilterSpec F, uint32_t* __restrict__ bits) {
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
            if (lane == 0 && v < total) bits[(int64_t)u * G.words + (v >> 5)] = word;
        }
    }
}

// The same filter on a labelled graph, visiting only the vertices that carry
// the label of the query vertex (its bucket: ascending ids), into bitmaps
// cleared beforehand. One warp per 1024 bucket entries of one query vertex;
// lanes with a passing vertex in the same bitmap word combine their bits and
// one of them ORs the word in. Block row blockIdx.y is query q (spec
// specs[q], bitmaps from word bits_off[q]; specs == nullptr: the one spec F0).
__global__ void filter_bucket_kernel(DevGraph G, const FilterSpec* __restrict__ specs,
                                     const int64_t* __restrict__ bits_off, uint32_t* __restrict__ bits, FilterSpec F0) {
    __shared__ FilterSpec F;
    const int q = blockIdx.y;
    {
        const int32_t* src = specs ? (const int32_t*)(specs + q) : (const int32_t*)&F0;
        int32_t* dst = (int32_t*)&F;
        for (int i = threadIdx.x; i < (int)(sizeof(FilterSpec) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    uint32_t* out = bits + (bits_off ? bits_off[q] : 0);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int u = 0; u < F.k; ++u) {
        const int lab = F.label[u];
        if (lab < 0 || lab >= G.num_labels) continue;
        // one pass over the bucket serves every query vertex of this label:
        // the first of them makes it, the others are skipped
        bool first = true;
        for (int u0 = 0; u0 < u; ++u0) first = first && F.label[u0] != lab;
        if (!first) continue;
        uint32_t group = 0;
        int dmin = INT_MAX;
        for (int u2 = u; u2 < F.k; ++u2)
            if (F.label[u2] == lab) {
                group |= 1u << u2;
                dmin = min(dmin, (int)F.dq[u2]);
            }
        // only the bucket's prefix of vertices whose degree can reach dmin
        const int c = F.use_filter ? min(dmin, kDegClasses - 1) : 0;
        const int64_t base = __ldg(G.lab_off + lab);
        const int64_t cnt = __ldg(G.lab_ge + (int64_t)lab * kDegClasses + c);
        for (int64_t seg = warp; seg * 1024 < cnt; seg += nwarps) {
            for (int t = 0; t < 32; ++t) {
                const int64_t idx = seg * 1024 + t * 32 + lane;
                const bool in = idx < cnt;
                const int32_t v = in ? __ldg(G.lab_vert + base + idx) : 0;
                const int32_t dv = (in && F.use_filter) ? __ldg(G.deg + v) : 0;
                const uint8_t* nlf = (in && F.use_filter && G.nlf) ? G.nlf + (int64_t)v * G.num_labels : nullptr;
                for (uint32_t gm = group; gm; gm &= gm - 1u) {
                    const int u2 = __ffs(gm) - 1;
                    bool ok = in;
                    if (ok && F.use_filter) {
                        ok = dv >= F.dq[u2];
                        if (ok && nlf)
                            for (int j = 0; j < F.nneed[u2]; ++j)
                                if (nlf[F.need_label[u2][j]] < F.need_cnt[u2][j]) { ok = false; break; }
                    }
                    if (!__any_sync(SGM_FULL, ok)) continue;
                    const int key = ok ? (v >> 5) : -1 - lane;
                    const unsigned peers = __match_any_sync(SGM_FULL, key);
                    if (ok) {
                        const unsigned word = __reduce_or_sync(peers, 1u << (v & 31));
                        if (lane == __ffs(peers) - 1) atomicOr(out + (int64_t)u2 * G.words + (v >> 5), word);
                    }
                }
                if (seg * 1024 + (t + 1) * 32 >= cnt) break;
            }
        }
    }
}

// The count-table entries of the hub vertices: cnt_last[w] = #{y in N(w) :
// y passes the filter of phi[k-1]} for every hub w that passes the filter of
// phi[arith_b] (every image of that level does). One warp per (plan, hub),
// lanes striding over N(w), so that no warp of the search has to scan a
// hub's list alone. Block row blockIdx.y is plan idx[blockIdx.y].
__global__ void cnt_hubs_kernel(DevGraph G, const QueryPlan* __restrict__ plans, const int32_t* __restrict__ idx) {
    const QueryPlan& P = plans[idx ? idx[blockIdx.y] : blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t* gate = P.lv[P.arith_b].bits;
    const uint32_t* bits = P.lv[P.k - 1].bits;
    for (int h = warp; h < G.hubs; h += nwarps) {
        const int32_t w = __ldg(G.hub_list + h);
        if (!sgm_bit(gate, w)) continue;
        const int32_t* a = G.col + __ldg(G.rowptr + w);
        const int32_t d = __ldg(G.deg + w);
        int32_t c = 0;
        for (int32_t j = lane; j < d; j += 32) c += sgm_bit(bits, __ldg(a + j));
        c = __reduce_add_sync(SGM_FULL, c);
        if (lane == 0) P.cnt_last[w] = c;
    }
}

// Appends every v in [lo, hi) with bit v set to out (order not kept).
__global__ void roots_kernel(const uint32_t* __restrict__ bits0, int64_t lo, int64_t hi, int32_t* __restrict__ out,
                             RunState* st) {
    const int lane = threadIdx.x & 31;
    for (int64_t v0 = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v0 - lane < hi;
         v0 += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = v0 < hi && sgm_bit(bits0, (int32_t)v0);
        const unsigned m = __ballot_sync(SGM_FULL, ok);
        if (!m) continue;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&st->frontier_n, (unsigned long long)__popc(m));
        base = __shfl_sync(SGM_FULL, base, 0);
        if (ok) out[base + __popc(m & sgm_lanemask_lt())] = (int32_t)v0;
    }
}

// Upper bound on the next BFS frontier: sum of local candidate list sizes.
__global__ void bfs_bound_kernel(DevGraph G, const QueryPlan* __restrict__ P, const int32_t* __restrict__ rows,
                                 int64_t n_rows, int32_t d, RunState* st) {
    const LevelPlan lp = P->lv[d];
    unsigned long long acc = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_rows; r += (int64_t)gridDim.x * blockDim.x)
        acc += (unsigned long long)row_local_list(G, lp, rows + r * d, d).len;
    acc = sgm_warp_sum_u64(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&st->frontier_bound, acc);
}

// One BFS level (Alg. 1 BFS-Search, Process): every row of depth d is
// extended by every feasible candidate of phi[d]; one warp per row, one lane
// per candidate, survivors appended with warp-aggregated atomics.
__global__ void bfs_expand_kernel(DevGraph G, const QueryPlan* __restrict__ P, const int32_t* __restrict__ in,
                                  int64_t n_in, int32_t d, int32_t* __restrict__ out, int64_t cap_rows, RunState* st) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const LevelPlan lp = P->lv[d];
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
            if (lane == 0) base = atomicAdd(&st->frontier_n, (unsigned long long)__popc(m));
            base = __shfl_sync(SGM_FULL, base, 0);
            const unsigned long long pos = base + __popc(m & sgm_lanemask_lt());
            if (ok && pos < (unsigned long long)cap_rows) {
                int32_t* o = out + pos * (d + 1);
                for (int i = 0; i < d; ++i) o[i] = row[i];
                o[d] = v;
            }
        }
    }
}

// Splits the initial pool (rows of depth d): a row whose local list for
// level d has at most `chunk` candidates goes to short_idx, a longer list is
// cut into range tasks of `chunk` candidates. Counts in st->frontier_n
// (short rows) and st->frontier_bound (tasks); warp-aggregated appends.
__global__ void chunk_pool_kernel(DevGraph G, const QueryPlan* __restrict__ P, const int32_t* __restrict__ rows,
                                  int64_t n_rows, int32_t d, int32_t chunk, int32_t* __restrict__ short_idx,
                                  PoolTask* __restrict__ tasks, int64_t task_cap, RunState* st) {
    const int lane = threadIdx.x & 31;
    const LevelPlan lp = P->lv[d];
    for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r0 - lane < n_rows;
         r0 += (int64_t)gridDim.x * blockDim.x) {
        const bool in = r0 < n_rows;
        const int32_t len = in ? row_local_list(G, lp, rows + r0 * d, d).len : 0;
        const bool shrt = in && len <= chunk;
        const unsigned ms = __ballot_sync(SGM_FULL, shrt);
        unsigned long long sbase = 0;
        if (lane == 0 && ms) sbase = atomicAdd(&st->frontier_n, (unsigned long long)__popc(ms));
        sbase = __shfl_sync(SGM_FULL, sbase, 0);
        if (shrt) short_idx[sbase + __popc(ms & sgm_lanemask_lt())] = (int32_t)r0;
        const int nch = (in && !shrt) ? (len + chunk - 1) / chunk : 0;
        const int incl = sgm_warp_incl_scan(nch);
        const int tot = __shfl_sync(SGM_FULL, incl, 31);
        unsigned long long tbase = 0;
        if (lane == 0 && tot) tbase = atomicAdd(&st->frontier_bound, (unsigned long long)tot);
        tbase = __shfl_sync(SGM_FULL, tbase, 0) + (unsigned long long)(incl - nch);
        for (int j = 0; j < nch; ++j)
            if (tbase + j < (unsigned long long)task_cap) {
                PoolTask t;
                t.row = (int32_t)r0;
                t.lo = j * chunk;
                t.hi = min(len, (j + 1) * chunk);
                tasks[tbase + j] = t;
            }
    }
}

// Pool rows that are already complete embeddings (k <= init depth), each
// standing for its orbit under the automorphisms kept for symmetry breaking.
__global__ void pool_leaf_kernel(int32_t mode, const QueryPlan* __restrict__ P, const int32_t* __restrict__ rows,
                                 int64_t n_rows, int32_t k, RunState* st, int32_t* __restrict__ out, uint64_t cap) {
    const int lane = threadIdx.x & 31;
    const int na = P->aut_n;
    unsigned long long h = 0, c = 0;
    for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r0 - lane < n_rows;
         r0 += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = r0 < n_rows;
        int32_t Mu[SGM_KMAX];
        if (ok) for (int i = 0; i < k; ++i) Mu[P->lv[i].u] = rows[r0 * k + i];
        unsigned long long base = 0;
        if (mode == SGM_KMODE_ENUM) {
            const unsigned m = __ballot_sync(SGM_FULL, ok);
            if (lane == 0 && m) base = atomicAdd(&st->rows, (unsigned long long)__popc(m) * na);
            base = __shfl_sync(SGM_FULL, base, 0) + (unsigned long long)__popc(m & sgm_lanemask_lt()) * na;
        }
        if (!ok) continue;
        if (mode == SGM_KMODE_COUNT) {
            c++;
            continue;
        }
        c += na;
        for (int a = 0; a < na; ++a) {
            int32_t Ma[SGM_KMAX];
            for (int u = 0; u < k; ++u) Ma[u] = Mu[P->aut[a * k + u]];
            h += sgm_embedding_hash(Ma, k);
            if (mode == SGM_KMODE_ENUM && base + a < cap)
                for (int u = 0; u < k; ++u) out[(base + a) * k + u] = Ma[u];
        }
    }
    c = sgm_warp_sum_u64(c);
    h = sgm_warp_sum_u64(h);
    if (lane == 0) {
        sgm_add_checked(&st->count, c, &st->overflow);
        if (h) atomicAdd(&st->hash, h);
    }
}

// ---------------------------------------------------------------------------
// persistent fine-grained extension (Alg. 2)
// ---------------------------------------------------------------------------
// Per-warp execution stack in shared memory (Sec. 5.1, S of size |V(Q)| x 32).
// Slot (l, s) holds the candidate v mapped to phi[l], its parent slot pid at
// level l-1 (Sec. 4.2: partial matches are rebuilt by walking pid links),
// and, once valid, the local candidate list for level l+1 (C^L = N(w) or
// N+(w), w = the image of the backward neighbour of phi[l+1] with the
// shortest list): its first entry, length and the level it came from. Levels
// below the task's root level R come from a base row (the initial partial
// match fetched from the pool or the queue).
struct WarpStack {
    unsigned long long* lvl;  // [kcap] partial matches found per level
    const int32_t** lst;      // [kcap][32] first entry of the slot's local list
    int32_t* v;               // [kcap][32]
    int32_t* len;             // [kcap][32], 0 = slot carries no task group
    int32_t* cur;             // [kcap][2] saved cursor (parent i, position j) of each level
    int32_t* base;            // [32][kcap] base rows
    int32_t* tmp;             // [32] scatter owner table
    uint8_t* pid;             // [kcap][32]
    uint8_t* src;             // [kcap][32]
};

__host__ __device__ inline size_t warp_stack_bytes(int kcap) {
    return (size_t)kcap * (8 + 256 + 2 * 128 + 8 + 128 + 64) + 128;
}

__device__ inline WarpStack carve_stack(unsigned char* p, int kcap) {
    WarpStack s;
    s.lvl = (unsigned long long*)p;
    p += 8 * kcap;
    s.lst = (const int32_t**)p;
    p += 256 * kcap;
    s.v = (int32_t*)p;
    p += 128 * kcap;
    s.len = (int32_t*)p;
    p += 128 * kcap;
    s.cur = (int32_t*)p;
    p += 8 * kcap;
    s.base = (int32_t*)p;
    p += 128 * kcap;
    s.tmp = (int32_t*)p;
    p += 128;
    s.pid = (uint8_t*)p;
    p += 32 * kcap;
    s.src = (uint8_t*)p;
    return s;
}

// Visits M[l], M[l-1], ..., M[0] of the partial match ending in slot (l, s),
// calling f(level, vertex) until f returns false (Alg. 2, GenerateTask and
// Process walk the stack from level l-1 down to 0 the same way).
template <class F>
__device__ __forceinline__ void walk(const WarpStack& S, int R, int kcap, int l, int s, F&& f) {
    int i = l;
    for (; i >= R; --i) {
        if (!f(i, S.v[i * 32 + s])) return;
        s = S.pid[i * 32 + s];
    }
    const int32_t* row = S.base + s * kcap;
    for (; i >= 0; --i)
        if (!f(i, row[i])) return;
}

struct Ctx {
    DevGraph G;
    const QueryPlan* P;  // shared-memory copy
    WarpStack S;
    int kcap;
    int R;
};

// GenerateTask for slot (l, s): choose C^L for level l+1.
__device__ __forceinline__ void gen_task(const Ctx& c, int l, int s) {
    if (c.G.cg) {
        // on G': the shortest candidate-edge list N(M[i]) ∩ C(phi[l+1]) over
        // the backward neighbours i (its entries pass the level's filter)
        const uint32_t B = c.P->lv[l + 1].bwd;
        int32_t bestd = INT_MAX, besti = 0;
        const int32_t* bestp = nullptr;
        walk(c.S, c.R, c.kcap, l, s, [&](int i, int32_t x) {
            const uint32_t bit = 1u << i;
            if (B & bit) {
                const CgEdge* e = c.G.cg + i * 32 + (l + 1);
                const uint32_t w = __ldg(e->bits + (x >> 5));
                const int32_t r = __ldg(e->rank + (x >> 5)) + __popc(w & ((1u << (x & 31)) - 1u));
                const int64_t a = __ldg(e->ptr + r);
                const int32_t d = (int32_t)(__ldg(e->ptr + r + 1) - a);
                if (d < bestd) { bestd = d; besti = i; bestp = e->adj + a; }
            }
            return (B & (bit - 1u)) != 0u;
        });
        c.S.lst[l * 32 + s] = bestp;
        c.S.len[l * 32 + s] = bestd == INT_MAX ? 0 : bestd;
        c.S.src[l * 32 + s] = (uint8_t)besti;
        return;
    }
    const uint32_t B = c.P->lv[l + 1].bwd;
    const uint32_t U = c.P->lv[l + 1].up;
    int32_t bestd = INT_MAX, besti = 0, bestx = 0;
    walk(c.S, c.R, c.kcap, l, s, [&](int i, int32_t x) {
        const uint32_t bit = 1u << i;
        if (B & bit) {
            const int32_t d = (U & bit) ? __ldg(c.G.updeg + x) : __ldg(c.G.deg + x);
            if (d < bestd) { bestd = d; besti = i; bestx = x; }
        }
        return (B & (bit - 1u)) != 0u;
    });
    const LocalList L = local_list_of(c.G, besti, bestx, (U >> besti) & 1u);
    c.S.lst[l * 32 + s] = L.ptr;
    c.S.len[l * 32 + s] = L.len;
    c.S.src[l * 32 + s] = (uint8_t)L.src;
}

// Process (Alg. 2): can phi[l] map to v, the candidate taken from the list
// of level `src`, given the partial match ending in slot (l-1, p)?
// The candidate filter (bit v of the level's bitmap) has been passed already.
__device__ __forceinline__ bool check(const Ctx& c, int l, int p, int32_t v, int src, ProbeCount& pc) {
    const LevelPlan& lp = c.P->lv[l];
    const uint32_t need = need_mask(lp, src);
    if (!need) return true;
    const uint32_t sb = (lp.sb_gt | lp.sb_lt) & need;
    src &= kSrcLevel;
    const int32_t dv = sb ? __ldg(c.G.deg + v) : 0;
    bool ok = true;
    walk(c.S, c.R, c.kcap, l - 1, p, [&](int i, int32_t x) {
        const uint32_t bit = 1u << i;
        if (need & bit) {
            if ((lp.inj & bit) && x == v) { ok = false; return false; }
            // here v != x: a backward neighbour's image is adjacent to v and
            // a vertex of another label never shares v's bitmap
            if ((sb & bit) && (sgm_rank_less(c.G, v, dv, x) == ((lp.sb_gt & bit) != 0u))) {
                ok = false;
                return false;
            }
            if ((lp.bwd & bit) && i != src && !sgm_member(c.G, x, v, pc)) {
                ok = false;
                return false;
            }
        }
        return (need & (bit - 1u)) != 0u;
    });
    return ok;
}

// Arithmetic last level (count mode): phi[k-1] has the single backward
// neighbour at level b, so its feasible candidates given the match M ending
// in slot (l, s) are N(M[b]) minus the filtered-out vertices and the
// vertices of M: count = cnt_last[M[b]] - #{i : M[i] in N(M[b]), M[i] passes
// the filter of phi[k-1]}. Called by the whole warp; lanes with need = false
// only help. Returns the lane's count.
__device__ __forceinline__ unsigned long long arith_count(const Ctx& c, int l, int s, bool need, ProbeCount& pc) {
    const int lane = threadIdx.x & 31;
    const int b = c.P->arith_b;
    int32_t xb = -1;
    if (need)
        walk(c.S, c.R, c.kcap, l, s, [&](int i, int32_t x) {
            if (i == b) { xb = x; return false; }
            return true;
        });
    const uint32_t* bits = c.P->lv[c.P->k - 1].bits;
    int32_t* tab = c.P->cnt_last;
    int32_t cnt = need ? tab[xb] : 0;
    if (c.P->cnt_lazy) {
        // entries still at -1: the warp counts N(x) against the last level's
        // bitmap, once per distinct x, and records it (every writer of an
        // entry writes the same value)
        unsigned todo = __ballot_sync(SGM_FULL, need && cnt < 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            const int32_t x = __shfl_sync(SGM_FULL, xb, src);
            const int32_t* a = c.G.col + __ldg(c.G.rowptr + x);
            const int32_t d = __ldg(c.G.deg + x);
            int32_t part = 0;
            for (int32_t j = lane; j < d; j += 32) {
                part += sgm_bit(bits, __ldg(a + j));
                pc.filter++;
            }
            const int32_t tot = __reduce_add_sync(SGM_FULL, part);
            const unsigned same = __ballot_sync(SGM_FULL, need && xb == x);
            if ((same >> lane) & 1u) cnt = tot;
            if (lane == src) tab[x] = tot;
            todo &= ~same;
        }
    }
    if (!need) return 0;
    long long total = cnt;
    const uint32_t known = c.P->arith_known;
    walk(c.S, c.R, c.kcap, l, s, [&](int i, int32_t x) {
        if (i != b) {
            pc.filter++;
            if (sgm_bit(bits, x) && (((known >> i) & 1u) || sgm_member(c.G, xb, x, pc))) --total;
        }
        return true;
    });
    return (unsigned long long)total;
}

struct LaneAcc {
    unsigned long long count = 0, hash = 0, last_level = 0;
    unsigned long long cand = 0, groups = 0, rounds = 0, idle = 0, steals = 0;
    unsigned long long row_bytes = 0;  // 8 B per backward neighbour of every task group
    ProbeCount pc;
};

template <int MODE>
__device__ __forceinline__ void leaf(const Ctx& c, int l, int p, int32_t v, bool ok, unsigned mask, LaneAcc& acc,
                                     RunState* st, int32_t* out, uint64_t cap) {
    const int lane = threadIdx.x & 31;
    if (MODE == SGM_KMODE_COUNT) {
        if (lane == 0) acc.count += __popc(mask);
        return;
    }
    // each visited embedding stands for its orbit {M o sigma : sigma in Aut(Q)}
    int32_t Mu[SGM_KMAX];
    const int k = c.P->k;
    const int na = c.P->aut_n;
    if (ok) {
        walk(c.S, c.R, c.kcap, l - 1, p, [&](int i, int32_t x) {
            Mu[c.P->lv[i].u] = x;
            return true;
        });
        Mu[c.P->lv[l].u] = v;
    }
    unsigned long long base = 0;
    if (MODE == SGM_KMODE_ENUM) {
        if (lane == 0) base = atomicAdd(&st->rows, (unsigned long long)__popc(mask) * na);
        base = __shfl_sync(SGM_FULL, base, 0) + (unsigned long long)__popc(mask & sgm_lanemask_lt()) * na;
    }
    if (!ok) return;
    acc.count += na;
    for (int a = 0; a < na; ++a) {
        int32_t Ma[SGM_KMAX];
        const int8_t* sg = c.P->aut + a * k;
        for (int u = 0; u < k; ++u) Ma[u] = Mu[sg[u]];
        acc.hash += sgm_embedding_hash(Ma, k);
        if (MODE == SGM_KMODE_ENUM && base + a < cap)
            for (int u = 0; u < k; ++u) out[(base + a) * k + u] = Ma[u];
    }
}

// Pushes the stealable task (prefix of the match ending in slot (L-1, p) at
// level L, candidate positions [lo, hi)) to the work queue.
__device__ bool push_task(const Ctx& c, RunState* st, QueueTask* queue, int qcap, int L, int p, int lo, int hi,
                          int qid) {
    const int lane = threadIdx.x & 31;
    unsigned long long slot = 0;
    bool ok = false;
    if (lane == 0) {
        // reserve a slot only if the ring has room (head..tail < qcap)
        unsigned long long t = *(volatile unsigned long long*)&st->q_tail;
        for (int tries = 0; tries < 64; ++tries) {
            const unsigned long long h = *(volatile unsigned long long*)&st->q_head;
            if (t - h >= (unsigned long long)qcap) break;
            const unsigned long long seen = atomicCAS(&st->q_tail, t, t + 1);
            if (seen == t) { slot = t; ok = true; break; }
            t = seen;
        }
    }
    ok = __shfl_sync(SGM_FULL, ok, 0);
    if (!ok) return false;
    slot = __shfl_sync(SGM_FULL, slot, 0);
    QueueTask* q = queue + (slot % (unsigned long long)qcap);
    // wait until the previous user of this ring slot has released it
    if (lane == 0) {
        int spins = 0;
        while (*(volatile int32_t*)&q->ready != 0 && ++spins < (1 << 22)) __nanosleep(64);
        if (spins >= (1 << 22)) atomicCAS(&st->status, 0, SGM_E_DEVICE_TIMEOUT);
    }
    __syncwarp();
    int32_t x = 0;
    if (lane < L) {
        // lane i fetches M[i] by walking from slot (L-1, p)
        walk(c.S, c.R, c.kcap, L - 1, p, [&](int i, int32_t y) {
            if (i == lane) { x = y; return false; }
            return true;
        });
        q->prefix[lane] = x;
    }
    if (lane == 0) {
        q->L = L;
        q->lo = lo;
        q->hi = hi;
        q->qid = qid;
    }
    sgm_fence_acq_rel();
    __syncwarp();
    if (lane == 0) atomicExch(&q->ready, 1);
    return true;
}

// Two-level stealing, block level (Sec. 4.3): hands the candidate range
// [lo, hi) at level L of the match ending in slot (L-1, p) to an idle warp of
// this block through its shared-memory box. The claimed warp is counted as
// active on its behalf until it takes the range. False when no idle warp of
// the block could be claimed.
__device__ bool hand_to_idle_warp(const Ctx& c, RunState* st, BlockMail* bm, int L, int p, int lo, int hi) {
    const int lane = threadIdx.x & 31;
    int target = -1;
    if (lane == 0) {
        unsigned m = *(volatile unsigned*)&bm->idle_mask;
        for (int tries = 0; m && tries < 32; ++tries) {
            const int w = __ffs(m) - 1;
            const unsigned old = atomicAnd(&bm->idle_mask, ~(1u << w));
            if (old & (1u << w)) {
                target = w;
                break;
            }
            m = old & ~(1u << w);
        }
        if (target >= 0) atomicAdd(&st->active, 1);
    }
    target = __shfl_sync(SGM_FULL, target, 0);
    if (target < 0) return false;
    QueueTask* q = &bm->box[target];
    if (lane < L) {
        int32_t x = 0;
        walk(c.S, c.R, c.kcap, L - 1, p, [&](int i, int32_t y) {
            if (i == lane) { x = y; return false; }
            return true;
        });
        q->prefix[lane] = x;
    }
    if (lane == 0) {
        q->L = L;
        q->lo = lo;
        q->hi = hi;
        q->qid = 0;
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) atomicExch(&bm->ready[target], 1);
    return true;
}

// The fine-grained model without batching (one partial match's tasks per
// scatter round, the "Fine" row of the ablation of Sec. 6.3): keep only the
// pending candidates of the first parent slot that has any.
__device__ __forceinline__ int first_parent_only(int rem) {
    const unsigned nz = __ballot_sync(SGM_FULL, rem > 0);
    return nz && (int)(threadIdx.x & 31) == __ffs(nz) - 1 ? rem : 0;
}

// Position of the (r+1)-th set bit of w (r < popc(w)), by halving.
__device__ __forceinline__ int nth_set_bit(uint32_t w, int r) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int c = __popc(w & ((1u << s) - 1u));
        if (c <= r) {
            r -= c;
            w >>= s;
            pos += s;
        }
    }
    return pos;
}

// Copies the plan of one query into this warp's shared-memory plan: the
// 64-byte header and the query's k levels (the copy holds kcap >= k levels).
__device__ __forceinline__ void load_plan(QueryPlan* dst, const QueryPlan* __restrict__ src) {
    const int lane = threadIdx.x & 31;
    const int32_t* a = (const int32_t*)src;
    int32_t* b = (int32_t*)dst;
    const int n = (int)(offsetof(QueryPlan, lv) + sizeof(LevelPlan) * __ldg(&src->k)) / 4;
    for (int i = lane; i < n; i += 32) b[i] = a[i];
    __syncwarp();
}

// Adds this warp's per-query results (count, hash, per-level counts) to the
// query's run state and clears them.
template <int MODE>
__device__ void flush_query(LaneAcc& acc, const WarpStack& S, int kcap, int k, int from_level, RunState* qs) {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    const unsigned long long cnt = sgm_warp_sum_u64(acc.count);
    const unsigned long long hsh = sgm_warp_sum_u64(acc.hash);
    const unsigned long long last = sgm_warp_sum_u64(acc.last_level);
    if (lane == 0) {
        if (MODE != SGM_KMODE_ENUM) sgm_add_checked(&qs->count, cnt, &qs->overflow);
        if (hsh) atomicAdd(&qs->hash, hsh);
        if (last) sgm_add_checked(&qs->level[k - 1], last, &qs->overflow);
    }
    for (int i = lane; i < kcap; i += 32) {
        if (i < k && i >= from_level && S.lvl[i]) sgm_add_checked(&qs->level[i], S.lvl[i], &qs->overflow);
        S.lvl[i] = 0;
    }
    acc.count = acc.hash = acc.last_level = 0;
    __syncwarp();
}

// A task a warp has run for this many scatter rounds offers half of its
// shallowest pending candidate range to the other warps, idle or not: in a
// busy batch no warp is ever idle until the end, and a heavy subtree would
// otherwise stay on one warp.
constexpr unsigned kLongTaskRounds = 128;

// Takes the task in ring slot `slot` of the work queue (claimed by this warp):
// waits (bounded) until its producer has published it, copies it into the
// warp's base row 0 and releases the slot.
__device__ __forceinline__ void take_queue_slot(QueueTask* queue, int qcap, unsigned long long slot, RunState* st,
                                                const WarpStack& S, int& r_L, int& r_lo, int& r_hi, int& r_q) {
    const int lane = threadIdx.x & 31;
    QueueTask* q = queue + (slot % (unsigned long long)qcap);
    if (lane == 0) {
        int spins = 0;
        while (*(volatile int32_t*)&q->ready == 0 && ++spins < (1 << 22)) __nanosleep(64);
        if (spins >= (1 << 22)) atomicCAS(&st->status, 0, SGM_E_DEVICE_TIMEOUT);
    }
    __syncwarp();
    sgm_fence_acq_rel();
    r_L = *(volatile int32_t*)&q->L;
    r_lo = *(volatile int32_t*)&q->lo;
    r_hi = *(volatile int32_t*)&q->hi;
    r_q = *(volatile int32_t*)&q->qid;
    if (lane < r_L) S.base[lane] = *(volatile int32_t*)&q->prefix[lane];
    __syncwarp();
    if (lane == 0) atomicExch(&q->ready, 0);
}

// Has query q of a batched run stopped (its work cap, or a failure)? Warp-uniform.
__device__ __forceinline__ bool query_stopped(const BatchArgs& B, int q) {
    int32_t dead = 0;
    if ((threadIdx.x & 31) == 0) dead = *(volatile int32_t*)&B.qst[q].status;
    return __shfl_sync(SGM_FULL, dead, 0) != 0;
}

// The persistent extension kernel. One warp runs Alg. 2's Search over a
// batch of up to 32 partial matches at a time, fetched from the initial
// pool (BATCH = false: the rows of one query's BFS initialisation) or from
// the root candidates of many queries (BATCH = true: chunks of consecutive
// bitmap words of phi[0], each chunk belonging to one query), and steals
// candidate ranges from the work queue once the pool is empty.
template <int MODE, bool BATCH, bool GATHER>
__global__ void __launch_bounds__(1024) extend_kernel(DevGraph G, const QueryPlan* __restrict__ Pg,
                                                      PoolArgs pa, RunState* st,
                                                      QueueTask* queue, int32_t qcap, int32_t* __restrict__ out,
                                                      uint64_t cap, int32_t kcap, uint64_t time_cap_ns,
                                                      uint64_t work_cap, BatchArgs B) {
    __shared__ QueryPlan Pblock;
    extern __shared__ __align__(16) unsigned char dyn[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    QueryPlan* Pw = &Pblock;
    if (BATCH) {
        Pw = (QueryPlan*)(dyn + warp_stack_bytes(kcap) * (blockDim.x >> 5) + (size_t)B.plan_bytes * wib);
    }
    BlockMail* bm = (!BATCH && pa.block_mail)
                        ? (BlockMail*)(dyn + warp_stack_bytes(kcap) * (blockDim.x >> 5))
                        : nullptr;
    if (!BATCH) {
        const int32_t* src = (const int32_t*)Pg;
        int32_t* dst = (int32_t*)&Pblock;
        for (int i = threadIdx.x; i < (int)(sizeof(QueryPlan) / 4); i += blockDim.x) dst[i] = src[i];
        if (bm) {
            if (threadIdx.x == 0) bm->idle_mask = 0u;
            if (threadIdx.x < 32) bm->ready[threadIdx.x] = 0;
        }
        __syncthreads();
    }
    const QueryPlan& P = *Pw;
    Ctx c;
    c.G = G;
    c.P = Pw;
    c.kcap = kcap;
    c.S = carve_stack(dyn + warp_stack_bytes(kcap) * wib, kcap);
    c.R = BATCH ? 1 : P.D;
    const WarpStack& S = c.S;
    int cq = -1;                                     // query of the warp's current work (BATCH)
    RunState* qs = BATCH ? nullptr : st;             // per-query results
    int k = BATCH ? 0 : P.k;
    const int D = BATCH ? 1 : P.D;
    for (int i = lane; i < kcap; i += 32) S.lvl[i] = 0;
    LaneAcc acc;
    const unsigned long long t0 = sgm_globaltimer();
    bool abort = false;
    unsigned iter = 0;
    unsigned long long wcand = 0;  // candidates since the last work-cap report (warp-uniform)
    bool pool_done = false;
    bool tasks_done = false;
    bool bfs_done = !BATCH;  // batched runs: the tasks cut from the breadth-first pools
    bool counted = true;  // this warp is counted in st->active
    if (lane == 0) atomicAdd(&st->active, 1);
    // BATCH: current chunk [cw, cend) of bitmap words; window of 32 words
    // starting at wbase, lane j holding what is left of word wbase + j
    long long cw = 0, cend = 0, wbase = 0;
    uint32_t wword = 0, wmask = 0;
    int gq = -1;  // BATCH: query of the current root chunk (a queue task may switch away from it)
    // BATCH: the tasks of this launch's size class (written by the task
    // kernels that run before it in the captured graph)
    unsigned long long n_tasks = 0, task0 = 0;
    int cls_q0 = 0, cls_q1 = 0;
    if (BATCH) {
        const BatchClass& C = B.cls[B.cls_id];
        n_tasks = C.n_tasks;
        task0 = C.task0;
        cls_q0 = C.q0;
        cls_q1 = C.q1;
    }

    auto switch_query = [&](int q) {
        if (q == cq) return;
        if (cq >= 0) {
            flush_query<MODE>(acc, S, kcap, k, 0, qs);
            // candidates checked for the previous query count against its own cap
            if (work_cap && wcand && lane == 0) atomicAdd(&qs->work, wcand);
            wcand = 0;
        }
        load_plan(Pw, B.plans + q);
        cq = q;
        qs = B.qst + q;
        k = Pw->k;
    };

    while (!abort) {
        // ---- fetch: up to 32 initial partial matches, else a stolen range
        int ci = 0, cj = 0;
        int nvalid = 0;
        // a single-parent candidate range [r_lo, r_hi) at level r_L (from the
        // initial pool's range tasks or from the work queue)
        bool have_range = false;
        int r_L = 0, r_lo = 0, r_hi = 0, r_q = 0;
        if (queue) {
            // ranges offered by other warps come before new initial work: they
            // are the pending parts of the heaviest subtrees
            unsigned long long slot = 0;
            bool got = false;
            if (lane == 0) {
                const unsigned long long h = *(volatile unsigned long long*)&st->q_head;
                const unsigned long long t = *(volatile unsigned long long*)&st->q_tail;
                if (h < t && atomicCAS(&st->q_head, h, h + 1) == h) {
                    got = true;
                    slot = h;
                }
            }
            if (__shfl_sync(SGM_FULL, got, 0)) {
                take_queue_slot(queue, qcap, __shfl_sync(SGM_FULL, slot, 0), st, S, r_L, r_lo, r_hi, r_q);
                have_range = true;
                acc.steals += (lane == 0);
            }
        }
        if (!BATCH && !pool_done && !have_range) {
            unsigned long long start = 0;
            if (lane == 0) start = atomicAdd(&st->pool_head, 32ull);
            start = __shfl_sync(SGM_FULL, start, 0);
            if (start < (unsigned long long)pa.n_short) {
                nvalid = (int)min((unsigned long long)32, (unsigned long long)pa.n_short - start);
                for (int idx = lane; idx < nvalid * D; idx += 32) {
                    const int s = idx / D, i = idx - s * D;
                    const int64_t r = pa.short_idx ? (int64_t)__ldg(pa.short_idx + start + s) : (int64_t)(start + s);
                    S.base[s * kcap + i] = pa.rows[r * D + i];
                }
                c.R = D;
            } else {
                pool_done = true;
            }
        }
        if (!BATCH && pool_done && nvalid == 0 && !tasks_done && !have_range) {
            unsigned long long t = 0;
            if (lane == 0) t = atomicAdd(&st->task_head, 1ull);
            t = __shfl_sync(SGM_FULL, t, 0);
            if (t < (unsigned long long)pa.n_tasks) {
                const PoolTask pt = pa.tasks[t];
                if (lane < D) S.base[lane] = pa.rows[(int64_t)pt.row * D + lane];
                have_range = true;
                r_L = D;
                r_lo = pt.lo;
                r_hi = pt.hi;
            } else {
                tasks_done = true;
            }
        }
        bool skip_long = false;  // BATCH: rows with long lists are covered by range tasks
        if (BATCH && !bfs_done && !have_range) {
            // the next task of the class, query by query: a range task cut
            // from a long row of the query's final frontier, or 32 of its
            // rows; the tasks of a query that has stopped (its work cap) are
            // passed over before the warp switches to it
            while (true) {
                unsigned long long t = 0;
                if (lane == 0) t = atomicAdd(&st->pool_head, 1ull);
                t = __shfl_sync(SGM_FULL, t, 0);
                if (t >= n_tasks) {
                    bfs_done = true;
                    break;
                }
                const unsigned long long gt = task0 + t;
                // the last query of the class whose first task is <= gt
                int q = cls_q0, hi = cls_q1;
                while (hi - q > 1) {
                    const int mid = (q + hi) >> 1;
                    if (B.task_base[mid] <= gt) q = mid;
                    else hi = mid;
                }
                if (query_stopped(B, q)) continue;
                switch_query(q);
                const BatchBfs& bq = B.bfs[q];
                const int Dq = bq.depth;
                const unsigned long long local = gt - B.task_base[q];
                const unsigned long long nr = bq.split ? bq.nrange : 0ull;
                if (local < nr) {
                    const BatchRange rec = ((const BatchRange*)(B.arena + bq.range_off))[local];
                    const int32_t* row = B.arena + bq.off + (int64_t)rec.row * Dq;
                    if (lane < Dq) S.base[lane] = row[lane];
                    have_range = true;
                    r_L = Dq;
                    r_lo = rec.lo;
                    r_hi = rec.hi;
                    r_q = q;
                } else {
                    const unsigned long long r0 = 32ull * (local - nr);
                    nvalid = (int)min(32ull, bq.n - r0);
                    const int32_t* rows = B.arena + bq.off + (int64_t)r0 * Dq;
                    for (int idx = lane; idx < nvalid * Dq; idx += 32) {
                        const int s = idx / Dq, i = idx - s * Dq;
                        S.base[s * kcap + i] = rows[idx];
                    }
                    c.R = Dq;
                    skip_long = bq.split != 0;
                }
                break;
            }
        }
        if (BATCH && bfs_done && !have_range && nvalid == 0 && !pool_done) {
            // gather up to 32 root candidates of one query from its chunk
            if (gq >= 0) switch_query(gq);
            while (nvalid < 32) {
                if (wmask == 0) {
                    if (wbase + 32 < cend) {
                        wbase += 32;
                    } else {
                        if (nvalid > 0) break;  // never mix queries in one batch
                        long long ch = 0;
                        if (lane == 0) ch = (long long)atomicAdd(&st->chunk_head, 1ull);
                        ch = __shfl_sync(SGM_FULL, ch, 0);
                        if (ch >= B.nchunks) {
                            pool_done = true;
                            break;
                        }
                        gq = __ldg(B.chunk_q + ch);
                        switch_query(gq);
                        cw = __ldg(B.chunk_w + ch);
                        cend = min((long long)B.words, cw + B.chunk_words);
                        wbase = cw;
                    }
                    const long long w = wbase + lane;
                    wword = w < cend ? __ldg(P.lv[0].bits + w) : 0u;
                    // keep the roots inside the query's root range
                    const long long v0 = w * 32;
                    if (v0 < P.root_lo) wword &= P.root_lo - v0 >= 32 ? 0u : ~((1u << (P.root_lo - v0)) - 1u);
                    if (v0 + 32 > P.root_hi) wword &= P.root_hi <= v0 ? 0u : ((1u << (P.root_hi - v0)) - 1u);
                    wmask = __ballot_sync(SGM_FULL, wword != 0u);
                    continue;
                }
                const int j = __ffs(wmask) - 1;
                const uint32_t word = __shfl_sync(SGM_FULL, wword, j);
                const int pc = __popc(word);
                const int t = min(pc, 32 - nvalid);
                if (lane >= nvalid && lane < nvalid + t)
                    S.base[lane * kcap] = (int32_t)((wbase + j) * 32 + nth_set_bit(word, lane - nvalid));
                const uint32_t rest = t == pc ? 0u : (word & ~((1u << nth_set_bit(word, t)) - 1u));
                if (lane == j) wword = rest;
                if (rest == 0u) wmask &= ~(1u << j);
                nvalid += t;
            }
            if (nvalid > 0) {
                c.R = 1;
                if (lane == 0) S.lvl[0] += nvalid;
                if (k == 1) {
                    // single-vertex query: every root is an embedding
                    const bool ok = lane < nvalid;
                    leaf<MODE>(c, 0, 0, ok ? S.base[lane * kcap] : 0, ok, __ballot_sync(SGM_FULL, ok), acc, qs, out,
                               cap);
                    continue;
                }
            }
        }
        if (nvalid == 0 && !have_range) {
            // pool exhausted: take a stolen range from the queue or finish.
            // A waiting warp is not counted in st->active; the run is over
            // when the queue is empty and no warp is active. The wait gives
            // up (SGM_E_DEVICE_TIMEOUT) only if no active warp has shown
            // progress on the heartbeat for 2^24 polls.
            if (!queue) break;
            if (lane == 0) {
                sgm_fence_acq_rel();
                atomicSub(&st->active, 1);
            }
            counted = false;
            bool got = false, done = false, registered = false, mail = false, claimed = false;
            unsigned long long slot = 0, last_hb = 0;
            int spins = 0;
            unsigned nap = 128;
            const unsigned mybit = 1u << wib;
            // two-level stealing: offer this warp to the busy warps of its block
            if (bm && lane == 0) atomicOr(&bm->idle_mask, mybit);
            while (!got && !done && !mail) {
                if (lane == 0) {
                    // plain (volatile) reads while polling; a fence only once a
                    // task is in sight, so that a warp that sees the queue
                    // drained also sees this warp counted as active
                    const unsigned long long h = *(volatile unsigned long long*)&st->q_head;
                    const unsigned long long t = *(volatile unsigned long long*)&st->q_tail;
                    if (bm && *(volatile int32_t*)&bm->ready[wib] != 0) {
                        mail = true;  // a warp of this block handed over a range (and counted this warp)
                    } else if (h < t && !claimed) {
                        bool mine = true;
                        if (bm) {
                            // leave the block's idle set before taking from the queue;
                            // a warp already claimed waits for its box instead
                            const unsigned old = atomicAnd(&bm->idle_mask, ~mybit);
                            if (!(old & mybit)) {
                                claimed = true;
                                mine = false;
                            }
                        }
                        if (mine) {
                            atomicAdd(&st->active, 1);
                            sgm_fence_acq_rel();
                            if (atomicCAS(&st->q_head, h, h + 1) == h) {
                                got = true;
                                slot = h;
                            } else {
                                atomicSub(&st->active, 1);
                                if (bm) atomicOr(&bm->idle_mask, mybit);
                            }
                        }
                        nap = 128;
                    } else {
                        const int32_t act = *(volatile int32_t*)&st->active;
                        const int32_t stt = *(volatile int32_t*)&st->status;
                        const unsigned long long hb = *(volatile unsigned long long*)&st->heartbeat;
                        if (hb != last_hb) {
                            last_hb = hb;
                            spins = 0;
                        }
                        if (act == 0 || stt != 0) {
                            done = true;
                        } else if (++spins > (1 << 22)) {
                            // no progress signal for 2^22 polls of >= 128 ns each
                            atomicCAS(&st->status, 0, SGM_E_DEVICE_TIMEOUT);
                            done = true;
                        } else {
                            if (!registered) {
                                atomicAdd(&st->idle, 1);
                                registered = true;
                            }
                            __nanosleep(nap);
                            nap = min(nap * 2, 1024u);
                        }
                    }
                }
                got = __shfl_sync(SGM_FULL, got, 0);
                done = __shfl_sync(SGM_FULL, done, 0);
                mail = __shfl_sync(SGM_FULL, mail, 0);
            }
            if (lane == 0 && registered) atomicSub(&st->idle, 1);
            if (mail) {
                // the range in this warp's box (the hand-over counted it as active)
                __threadfence_block();
                const QueueTask* q = &bm->box[wib];
                r_L = *(volatile const int32_t*)&q->L;
                r_lo = *(volatile const int32_t*)&q->lo;
                r_hi = *(volatile const int32_t*)&q->hi;
                r_q = 0;
                if (lane < r_L) S.base[lane] = *(volatile const int32_t*)&q->prefix[lane];
                __syncwarp();
                if (lane == 0) atomicExch(&bm->ready[wib], 0);
                counted = true;
                have_range = true;
                acc.steals += (lane == 0);
            } else {
                if (bm && lane == 0) atomicAnd(&bm->idle_mask, ~mybit);  // (leaving: no longer offered)
                if (!got) break;
                counted = true;
                slot = __shfl_sync(SGM_FULL, slot, 0);
                take_queue_slot(queue, qcap, slot, st, S, r_L, r_lo, r_hi, r_q);
                have_range = true;
                acc.steals += (lane == 0);
            }
        }
        if (BATCH && (have_range || nvalid > 0)) {
            // a query stopped by its work cap (or a failure) drops its remaining tasks
            if (query_stopped(B, have_range ? r_q : cq)) continue;
            if (have_range) switch_query(r_q);
        }
        if (have_range) {
            c.R = r_L;
            nvalid = 1;
            // the slot at level L-1 is base row 0; its list is recomputed here,
            // then clipped to [lo, hi)
            if (lane == 0) {
                gen_task(c, r_L - 1, 0);
                acc.row_bytes += 8u * __popc(P.lv[r_L].bwd);
            }
            __syncwarp();
            if (lane == 0) S.len[(r_L - 1) * 32] = r_hi;
            if (lane > 0) S.len[(r_L - 1) * 32 + lane] = 0;
            ci = 0;
            cj = r_lo;
            acc.groups += (lane == 0);
            __syncwarp();
        } else {
            __syncwarp();
            // GenerateTask for the base level R-1
            const int Rb = c.R;
            const bool arith_base = P.arith && Rb == k - 1;
            if (lane < nvalid) {
                gen_task(c, Rb - 1, lane);
                acc.row_bytes += 8u * __popc(P.lv[Rb].bwd);
                if (BATCH && skip_long && !arith_base && S.len[(Rb - 1) * 32 + lane] > P.pool_chunk)
                    S.len[(Rb - 1) * 32 + lane] = 0;
            } else {
                S.len[(Rb - 1) * 32 + lane] = 0;
            }
            acc.groups += lane < nvalid;
            __syncwarp();
            if (arith_base) {
                // the initial matches are one level short: count arithmetically
                const unsigned long long a = arith_count(c, Rb - 1, lane, lane < nvalid, acc.pc);
                acc.count += a;
                acc.last_level += a;
                continue;
            }
        }

        // ---- depth-first search over levels R..k-1 (Alg. 2, Search)
        const int R = c.R;
        int l = R;
        unsigned task_rounds = 0;  // rounds since the task started or last offered a range
        while (true) {
            ++iter;  // warp-uniform round counter
            ++task_rounds;
            // report every 256 rounds, or every 8192 candidates (a round may
            // take several scatter rounds when it gathers filtered candidates)
            if ((time_cap_ns || work_cap) && ((iter & 255u) == 0u || wcand >= 8192u)) {
                int32_t stop = 0;
                if (lane == 0) {
                    if (*(volatile int32_t*)&st->status != 0) stop = 1;
                    else if (time_cap_ns && sgm_globaltimer() - t0 > time_cap_ns) stop = SGM_E_TIME_CAP;
                    else if (work_cap && BATCH) {
                        // batched runs cap each query: a query past its cap
                        // stops (its tasks are dropped), the others go on
                        const unsigned long long done = atomicAdd(&qs->work, wcand) + wcand;
                        if (done > work_cap) atomicCAS(&qs->status, 0, SGM_E_WORK_CAP);
                        if (*(volatile int32_t*)&qs->status != 0) stop = 2;
                    } else if (work_cap) {
                        // candidates since the last report (fewer than 16384)
                        const unsigned long long done = atomicAdd(&st->work, wcand) + wcand;
                        if (done > work_cap) stop = SGM_E_WORK_CAP;
                    }
                }
                wcand = 0;
                stop = __shfl_sync(SGM_FULL, stop, 0);
                if (BATCH && stop == 2) break;  // abandon this task of a stopped query
                if (stop) {
                    if (lane == 0 && stop != 1) atomicCAS(&st->status, 0, stop);
                    abort = true;
                    break;
                }
            }
            // ScatterTask: fill the 32 lanes from the concatenated lists of the
            // valid parent slots at level l-1, starting at cursor (ci, cj).
            const int pl = (l - 1) * 32;
            const int ls = S.len[pl + lane];
            // pending candidates of the cursor's parent slot; when they fill a
            // whole round (and the round is not gathered), the lanes take them
            // in order and the prefix scan over the slots is skipped
            const int head = __shfl_sync(SGM_FULL, ls, ci) - cj;
            const bool single = !GATHER && head >= 32;
            int rem = 0, incl = 0, total = head;
            if (!single) {
                rem = lane > ci ? ls : (lane == ci ? ls - cj : 0);
                if (pa.one_parent) rem = first_parent_only(rem);
                incl = sgm_warp_incl_scan(rem);
                total = __shfl_sync(SGM_FULL, incl, 31);
            }
            if (total == 0) {
                if (l == R) break;  // task finished
                --l;
                ci = S.cur[2 * l];
                cj = S.cur[2 * l + 1];
                continue;
            }
            // a long-running task offers half of its shallowest pending range
            // (lane i looks at level R + i; the current level's cursor is in
            // registers, the shallower ones were saved on the way down)
            if (queue && P.split_min > 0 && task_rounds >= kLongTaskRounds) {
                task_rounds = 0;
                const int li = R + lane;
                int p_i = 0, c_i = 0, e_i = 0;
                if (li < l) {
                    p_i = S.cur[2 * li];
                    c_i = S.cur[2 * li + 1];
                    e_i = S.len[(li - 1) * 32 + p_i];
                } else if (li == l) {
                    p_i = ci;
                    c_i = cj;
                    e_i = S.len[pl + ci];
                }
                const int thr_i = max(2, (2 * P.split_min) >> min(k - 1 - li, 16));
                const unsigned cand = __ballot_sync(SGM_FULL, li <= l && e_i - c_i > thr_i);
                if (cand) {
                    const int src = __ffs(cand) - 1;
                    const int Ld = R + src;
                    const int pd = __shfl_sync(SGM_FULL, p_i, src);
                    const int mid = __shfl_sync(SGM_FULL, c_i + (e_i - c_i) / 2, src);
                    const int end = __shfl_sync(SGM_FULL, e_i, src);
                    if (push_task(c, st, queue, qcap, Ld, pd, mid, end, BATCH ? cq : 0)) {
                        if (lane == 0) S.len[(Ld - 1) * 32 + pd] = mid;
                        __syncwarp();
                        if (Ld == l) continue;  // recompute the round with the shortened range
                    }
                }
            }
            // offer half of a long candidate range to idle warps (Sec. 4.3).
            // At a task's root level the range must exceed 2 x split_min; at
            // deeper levels (split_depth > 1) the threshold halves with every
            // query level still below, since each candidate there roots a
            // larger subtree (never below 2)
            if (bm && P.split_min > 0 && l < R + P.split_depth) {
                // block level first: an idle warp of this block gets half of
                // the range straight into its shared-memory box
                const int thr = P.split_depth > 1 ? max(2, (2 * P.split_min) >> min(k - 1 - l, 16)) : 2 * P.split_min;
                if (head > thr) {
                    int any = 0;
                    if (lane == 0) any = *(volatile unsigned*)&bm->idle_mask != 0u;
                    if (__shfl_sync(SGM_FULL, any, 0)) {
                        const int end = S.len[pl + ci];
                        const int mid = cj + head / 2;
                        if (hand_to_idle_warp(c, st, bm, l, ci, mid, end)) {
                            if (lane == 0) S.len[pl + ci] = mid;
                            __syncwarp();
                            continue;  // recompute the round with the shortened range
                        }
                    }
                }
            }
            if (queue && P.split_min > 0 && l < R + P.split_depth && (iter & 7u) == 0u) {
                const int cur_rem = head;  // (the first slot with pending candidates is the cursor's)
                const int thr = P.split_depth > 1 ? max(2, (2 * P.split_min) >> min(k - 1 - l, 16)) : 2 * P.split_min;
                if (cur_rem > thr) {
                    int idle = 0;
                    if (lane == 0) idle = *(volatile int32_t*)&st->idle;
                    idle = __shfl_sync(SGM_FULL, idle, 0);
                    if (idle > 0) {
                        const int end = S.len[pl + ci];
                        const int mid = cj + cur_rem / 2;
                        if (push_task(c, st, queue, qcap, l, ci, mid, end, BATCH ? cq : 0)) {
                            if (lane == 0) S.len[pl + ci] = mid;
                            __syncwarp();
                            continue;  // recompute the round with the shortened range
                        }
                    }
                }
            }
            // ScatterTask with the candidate filter first: a scatter round
            // fills the lanes from the parents' lists and tests each
            // candidate's filter bit. When at least half of them pass (or the
            // graph is unlabelled), the round goes on as it is. Otherwise the passing candidates are
            // packed into lanes 0..nacc-1 and further scatter rounds add to
            // them until 32 are gathered or the level's parents run out, so
            // that the membership tests run on full lanes (a selective label
            // filter leaves most lanes idle otherwise). When a round brings
            // more passing candidates than there is room for, the cursor
            // resumes at the first one left out; every candidate is counted
            // once, when it is consumed.
            const uint32_t* fbits = P.lv[l].bits;
            int nacc = 0, p = 0;
            int32_t v = -1;
            bool gathered = false;  // lanes hold packed candidates (else their own, valid = filter passed)
            bool fpass = false;
            if (single) {
                // a whole round from the cursor's slot
                p = ci;
                v = __ldg(S.lst[pl + ci] + cj + lane);
                cj += 32;
                acc.cand += 1;
                acc.pc.filter += 1;
                wcand += 32ull;
                if (lane == 0) {
                    acc.rounds++;
                    if (queue && (acc.rounds & 255u) == 0) atomicAdd(&st->heartbeat, 1ull);
                }
                fpass = sgm_bit(fbits, v);
                nacc = 1;
            } else if constexpr (!GATHER) {
                // one scatter round: lane i takes the i-th pending candidate
                const int excl = incl - rem;
                const bool owner = rem > 0 && excl < 32;
                const unsigned starts = __reduce_or_sync(SGM_FULL, owner ? (1u << excl) : 0u);
                if (owner) S.tmp[excl] = lane;
                __syncwarp();
                const int take = min(total, 32);
                const bool valid = lane < take;
                int pos = 0;
                if (valid) {
                    const int first = 31 - __clz(starts & ((2u << lane) - 1u));
                    p = S.tmp[first];
                    pos = (p == ci ? cj : 0) + (lane - first);
                    v = __ldg(S.lst[pl + p] + pos);
                }
                ci = __shfl_sync(SGM_FULL, p, take - 1);
                cj = __shfl_sync(SGM_FULL, pos, take - 1) + 1;
                __syncwarp();
                acc.cand += valid;
                acc.pc.filter += valid;
                wcand += (unsigned long long)take;
                if (lane == 0) {
                    acc.rounds++;
                    acc.idle += 32 - take;
                    if (queue && (acc.rounds & 255u) == 0) atomicAdd(&st->heartbeat, 1ull);
                }
                fpass = valid && sgm_bit(fbits, v);
                nacc = 1;
            } else {
                int r_incl = incl, r_rem = rem, r_total = total;
                int round_consumed = 0;  // a round gathers from at most 4096 candidates
                while (true) {
                    const int excl = r_incl - r_rem;
                    const bool owner = r_rem > 0 && excl < 32;
                    const unsigned starts = __reduce_or_sync(SGM_FULL, owner ? (1u << excl) : 0u);
                    if (owner) S.tmp[excl] = lane;
                    __syncwarp();
                    const int take = min(r_total, 32);
                    const bool valid = lane < take;
                    int sp = 0, pos = 0;
                    int32_t sv = -1;
                    if (valid) {
                        const int first = 31 - __clz(starts & ((2u << lane) - 1u));
                        sp = S.tmp[first];
                        pos = (sp == ci ? cj : 0) + (lane - first);
                        sv = __ldg(S.lst[pl + sp] + pos);
                    }
                    __syncwarp();
                    const bool f = valid && sgm_bit(fbits, sv);
                    const unsigned m = __ballot_sync(SGM_FULL, f);
                    const int cnt = __popc(m);
                    const int room = 32 - nacc;
                    int consumed = take;
                    if (cnt > room) {
                        const int ov = nth_set_bit(m, room);
                        consumed = ov;
                        ci = __shfl_sync(SGM_FULL, sp, ov);
                        cj = __shfl_sync(SGM_FULL, pos, ov);
                    } else {
                        ci = __shfl_sync(SGM_FULL, sp, take - 1);
                        cj = __shfl_sync(SGM_FULL, pos, take - 1) + 1;
                    }
                    acc.cand += lane < consumed;
                    acc.pc.filter += lane < consumed;
                    wcand += (unsigned long long)consumed;
                    if (lane == 0) {
                        acc.rounds++;
                        acc.idle += 32 - take;
                        if (queue && (acc.rounds & 255u) == 0) atomicAdd(&st->heartbeat, 1ull);
                    }
                    if (!gathered && (2 * cnt >= take || pa.one_parent)) {
                        // the first round is at least half full: no packing
                        v = sv;
                        p = sp;
                        fpass = f;
                        nacc = cnt;
                        break;
                    }
                    gathered = true;
                    const int got = min(cnt, room);
                    if (got > 0) {
                        const int rank = min(max(lane - nacc, 0), got - 1);
                        const int from = nth_set_bit(m, rank);
                        const int32_t rv = __shfl_sync(SGM_FULL, sv, from);
                        const int rp = __shfl_sync(SGM_FULL, sp, from);
                        if (lane >= nacc && lane < nacc + got) {
                            v = rv;
                            p = rp;
                        }
                        nacc += got;
                    }
                    round_consumed += consumed;
                    if (nacc == 32 || round_consumed >= 4096) break;
                    // the next scatter round from the advanced cursor
                    const int ls2 = S.len[pl + lane];
                    r_rem = lane > ci ? ls2 : (lane == ci ? ls2 - cj : 0);
                    if (pa.one_parent) r_rem = first_parent_only(r_rem);
                    r_incl = sgm_warp_incl_scan(r_rem);
                    r_total = __shfl_sync(SGM_FULL, r_incl, 31);
                    if (r_total == 0) break;
                }
            }
            if (nacc == 0) continue;  // no candidate passed: the next round moves on or backtracks
            const bool valid = gathered ? lane < nacc : fpass;
            // Process: one lane per task T_M(u, v)
            const bool ok = valid && check(c, l, p, v, S.src[pl + p], acc.pc);
            const unsigned mask = __ballot_sync(SGM_FULL, ok);
            if (lane == 0) S.lvl[l] += __popc(mask);
            if (l == k - 1) {
                leaf<MODE>(c, l, p, v, ok, mask, acc, qs, out, cap);
                continue;
            }
            if (!mask) continue;
            // push the surviving lanes as the next level's parents
            S.v[l * 32 + lane] = v;
            S.pid[l * 32 + lane] = (uint8_t)p;
            __syncwarp();
            if (P.arith && l + 1 == k - 1) {
                const unsigned long long a = arith_count(c, l, lane, ok, acc.pc);
                acc.count += a;
                acc.last_level += a;
                __syncwarp();
                continue;
            }
            if (ok) {
                gen_task(c, l, lane);
                acc.groups++;
                acc.row_bytes += 8u * __popc(P.lv[l + 1].bwd);
            } else {
                S.len[l * 32 + lane] = 0;
            }
            if (lane == 0) {
                S.cur[2 * l] = ci;
                S.cur[2 * l + 1] = cj;
            }
            __syncwarp();
            ++l;
            ci = 0;
            cj = 0;
        }
    }
    if (lane == 0 && counted) atomicSub(&st->active, 1);
    // the last query's checks since its last report (batched runs count each query's work)
    if (BATCH && work_cap && qs && wcand && lane == 0) atomicAdd(&qs->work, wcand);

    // ---- flush per-warp results
    if (qs) flush_query<MODE>(acc, S, kcap, k, BATCH ? 0 : D, qs);
    const unsigned long long cand = sgm_warp_sum_u64(acc.cand);
    const unsigned long long sp = sgm_warp_sum_u64(acc.pc.search);
    const unsigned long long bp = sgm_warp_sum_u64(acc.pc.bitmap);
    const unsigned long long fp = sgm_warp_sum_u64(acc.pc.filter);
    const unsigned long long grp = sgm_warp_sum_u64(acc.groups);
    const unsigned long long alg = sgm_warp_sum_u64(acc.pc.alg + acc.row_bytes + 4ull * acc.cand);
    if (lane == 0) {
        atomicAdd(&st->alg_bytes, alg);
        atomicAdd(&st->cand_checked, cand);
        atomicAdd(&st->list_elems, cand);
        atomicAdd(&st->search_probes, sp);
        atomicAdd(&st->bitmap_probes, bp);
        atomicAdd(&st->filter_probes, fp);
        atomicAdd(&st->task_groups, grp);
        atomicAdd(&st->scatter_rounds, acc.rounds);
        atomicAdd(&st->idle_lanes, acc.idle);
        atomicAdd(&st->steals, acc.steals);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t sgm_launch_filter_buckets(const DevGraph& G, const FilterSpec* specs, const FilterSpec* F0,
                                      const int64_t* bits_off, uint32_t* bits, size_t bits_words, int32_t nq,
                                      int32_t warps_per_query, cudaStream_t s) {
    if (nq <= 0) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(bits, 0, sizeof(uint32_t) * bits_words, s);
    if (err != cudaSuccess) return err;
    FilterSpec f0;
    memset(&f0, 0, sizeof(f0));
    if (F0) f0 = *F0;
    const int blocks = std::max(1, (warps_per_query + 7) / 8);
    filter_bucket_kernel<<<dim3(blocks, nq), kThreads, 0, s>>>(G, specs, bits_off, bits, f0);
    return cudaGetLastError();
}

cudaError_t sgm_launch_filter(const DevGraph& G, const FilterSpec& F, uint32_t* bits, cudaStream_t s) {
    if (G.lab_vert) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        return sgm_launch_filter_buckets(G, nullptr, &F, nullptr, bits, (size_t)F.k * G.words, 1, 32 * sms, s);
    }
    filter_kernel<<<grid_for(G.words * 32), kThreads, 0, s>>>(G, F, bits);
    return cudaGetLastError();
}

cudaError_t sgm_launch_cnt_hubs(const DevGraph& G, const QueryPlan* plans, const int32_t* idx, int32_t nq,
                                int32_t sms, cudaStream_t s) {
    if (nq <= 0 || G.hubs <= 0) return cudaSuccess;
    // about 4 warps per SM per plan, at least one warp per 64 hubs
    const int warps = std::max(1, std::min((G.hubs + 63) / 64 * 8, 4 * sms / std::max(1, nq / 8 + 1) + 8));
    const int blocks = (warps + 7) / 8;
    cnt_hubs_kernel<<<dim3(blocks, nq), kThreads, 0, s>>>(G, plans, idx);
    return cudaGetLastError();
}

cudaError_t sgm_launch_roots(const uint32_t* bits0, int64_t lo, int64_t hi, int32_t* out, RunState* st,
                             cudaStream_t s) {
    if (hi <= lo) return cudaSuccess;
    roots_kernel<<<grid_for(hi - lo), kThreads, 0, s>>>(bits0, lo, hi, out, st);
    return cudaGetLastError();
}

cudaError_t sgm_launch_bfs_bound(const DevGraph& G, const QueryPlan* P, const int32_t* rows, int64_t n_rows,
                                 int32_t d, RunState* st, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    bfs_bound_kernel<<<grid_for(n_rows), kThreads, 0, s>>>(G, P, rows, n_rows, d, st);
    return cudaGetLastError();
}

cudaError_t sgm_launch_bfs_expand(const DevGraph& G, const QueryPlan* P, const int32_t* in, int64_t n_in, int32_t d,
                                  int32_t* out, int64_t cap_rows, RunState* st, cudaStream_t s) {
    if (n_in <= 0) return cudaSuccess;
    bfs_expand_kernel<<<grid_for(n_in * 32), kThreads, 0, s>>>(G, P, in, n_in, d, out, cap_rows, st);
    return cudaGetLastError();
}

cudaError_t sgm_launch_chunk_pool(const DevGraph& G, const QueryPlan* P, const int32_t* rows, int64_t n_rows,
                                  int32_t d, int32_t chunk, int32_t* short_idx, PoolTask* tasks, int64_t task_cap,
                                  RunState* st, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    chunk_pool_kernel<<<grid_for(n_rows), kThreads, 0, s>>>(G, P, rows, n_rows, d, chunk, short_idx, tasks, task_cap,
                                                            st);
    return cudaGetLastError();
}

cudaError_t sgm_launch_pool_leaf(int32_t mode, const QueryPlan* P, const int32_t* rows, int64_t n_rows, int32_t k,
                                 RunState* st, int32_t* out, uint64_t cap, cudaStream_t s) {
    if (n_rows <= 0) return cudaSuccess;
    pool_leaf_kernel<<<grid_for(n_rows), kThreads, 0, s>>>(mode, P, rows, n_rows, k, st, out, cap);
    return cudaGetLastError();
}

int32_t sgm_batch_plan_bytes(int32_t kcap) { return (int32_t)(offsetof(QueryPlan, lv) + sizeof(LevelPlan) * kcap); }

size_t sgm_extend_smem_bytes(int32_t kcap, int32_t warps_per_block, bool batch) {
    return (warp_stack_bytes(kcap) + (batch ? (size_t)sgm_batch_plan_bytes(kcap) : 0)) * (size_t)warps_per_block;
}

template <int MODE, bool BATCH, bool GATHER>
static void* extend_fn() {
    return (void*)extend_kernel<MODE, BATCH, GATHER>;
}

template <bool GATHER>
static void* extend_ptr_g(int32_t mode, bool batch) {
    if (batch)
        return mode == SGM_KMODE_HASH ? extend_fn<SGM_KMODE_HASH, true, GATHER>()
                                      : extend_fn<SGM_KMODE_COUNT, true, GATHER>();
    switch (mode) {
        case SGM_KMODE_HASH: return extend_fn<SGM_KMODE_HASH, false, GATHER>();
        case SGM_KMODE_ENUM: return extend_fn<SGM_KMODE_ENUM, false, GATHER>();
        default: return extend_fn<SGM_KMODE_COUNT, false, GATHER>();
    }
}

static void* extend_ptr(int32_t mode, bool batch, bool gather) {
    return gather ? extend_ptr_g<true>(mode, batch) : extend_ptr_g<false>(mode, batch);
}

int sgm_extend_max_blocks_per_sm(int32_t mode, bool batch, bool gather, int32_t warps_per_block, size_t smem_bytes) {
    void* f = extend_ptr(mode, batch, gather);
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, f, warps_per_block * 32, smem_bytes) != cudaSuccess)
        return 0;
    return blocks;
}

cudaError_t sgm_launch_extend(const ExtendLaunch& L, const DevGraph& G, const QueryPlan* P, const PoolArgs& pa,
                              RunState* st, QueueTask* queue, int32_t qcap, int32_t* out, uint64_t cap,
                              uint64_t time_cap_ns, uint64_t work_cap, const BatchArgs* batch, cudaStream_t s) {
    const dim3 grid(L.blocks), block(L.warps_per_block * 32);
    const bool b = batch != nullptr;
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    if (b) B = *batch;
    void* f = extend_ptr(L.mode, b, L.gather != 0);
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
    // the kernel's parameters in order, for the variant chosen at run time
    DevGraph Gv = G;
    PoolArgs pav = pa;
    int32_t kcap = L.kcap;
    void* args[] = {&Gv, (void*)&P, &pav, &st, &queue, &qcap, &out, &cap, &kcap, &time_cap_ns, &work_cap, &B};
    return cudaLaunchKernel(f, grid, block, args, L.smem_bytes, s);
}
