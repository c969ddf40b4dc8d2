// sgm_device.cuh - device helpers of the matching kernels: candidate-bitmap
// tests, neighbour-list membership, the embedding hash and warp primitives.
#pragma once

#include <climits>

#include "sgm_internal.cuh"

// Bit v of a vertex bitmap (candidate bitmaps, hub adjacency bitmaps).
__device__ __forceinline__ bool sgm_bit(const uint32_t* __restrict__ bits, int32_t v) {
    return (__ldg(bits + (v >> 5)) >> (v & 31)) & 1u;
}

struct ProbeCount {
    unsigned long long search = 0;  // binary-search probes into sorted rows
    unsigned long long bitmap = 0;  // hub adjacency-bitmap probes
    unsigned long long filter = 0;  // candidate-bitmap probes
    unsigned long long alg = 0;     // algorithmic bytes of the membership tests (see sgm_member)
};

// Algorithmic bytes of one membership test into a sorted row of len entries:
// streaming the row (4 B per entry) or searching it, whichever is cheaper; a
// search touches one 32-byte sector per halving until 8 entries (one
// sector) remain: max(1, ceil(log2(len / 8))) sectors.
__device__ __forceinline__ unsigned member_bytes(int32_t len) {
    const int lg = len > 1 ? 32 - __clz(len - 1) : 0;  // ceil(log2(len))
    const unsigned sectors = (unsigned)max(1, lg - 3);
    return min(4u * (unsigned)len, 32u * sectors);
}

// Is v in N(x)? The edge test of Process (Alg. 2, "v not in N(v')"). A hub
// (a vertex with an adjacency bitmap) answers with one bit probe; any other
// row is searched by bisection over its sorted entries (Sec. 5.2 costs one
// such search O(log |N(x)|) per backward neighbour and candidate).
__device__ __forceinline__ bool sgm_member(const DevGraph& G, int32_t x, int32_t v, ProbeCount& pc) {
    if (G.hubs) {
        const int32_t h = __ldg(G.hub_id + x);
        if (h >= 0) {
            pc.bitmap++;
            pc.alg += 32;
            return sgm_bit(G.hub_bits + (int64_t)h * G.words, v);
        }
    }
    const int32_t* a = G.col + __ldg(G.rowptr + x);
    int32_t len = __ldg(G.deg + x);
    pc.alg += member_bytes(len);
    while (len > 0) {
        const int32_t half = len >> 1;
        const int32_t c = __ldg(a + half);
        pc.search++;
        if (c == v) return true;
        if (c < v) {
            a += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return false;
}

// Symmetry-breaking order on data vertices: (degree, id), lexicographic.
// Is vertex a (degree da) before vertex b?
__device__ __forceinline__ bool sgm_rank_less(const DevGraph& G, int32_t a, int32_t da, int32_t b) {
    const int32_t db = __ldg(G.deg + b);
    return da < db || (da == db && a < b);
}

// SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ unsigned long long sgm_mix64(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// h(M) over an embedding indexed by query-vertex id (the ABI's embedding hash).
__device__ __forceinline__ unsigned long long sgm_embedding_hash(const int32_t* Mu, int k) {
    unsigned long long x = 0x243F6A8885A308D3ull;
    for (int u = 0; u < k; ++u)
        x = sgm_mix64(x ^ (((unsigned long long)(uint32_t)u << 32) | (unsigned long long)(uint32_t)Mu[u]));
    return sgm_mix64(x);
}

__device__ __forceinline__ int sgm_warp_incl_scan(int x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(SGM_FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long sgm_warp_sum_u64(unsigned long long x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(SGM_FULL, x, o);
    return x;
}

__device__ __forceinline__ unsigned sgm_lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Acquire-release fence at GPU scope: orders this thread's earlier memory
// operations before its later ones for every thread of the device that
// synchronises with it. Lighter than the sequentially consistent
// __threadfence(), and all the work-queue protocol needs (publishing a task
// before its ready flag, reading it after the flag, counting a warp active
// before it takes a task).
__device__ __forceinline__ void sgm_fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned long long sgm_globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Adds to a 64-bit result counter and flags wrap-around instead of hiding it.
__device__ __forceinline__ void sgm_add_checked(unsigned long long* dst, unsigned long long x, int32_t* overflow) {
    if (x == 0) return;
    const unsigned long long old = atomicAdd(dst, x);
    if (old + x < old) atomicExch(overflow, 1);
}

// The local candidate list C^L_M(u) of Sec. 4.1: the smallest neighbour list
// among the mapped backward neighbours of the level's query vertex. A backward
// neighbour whose image symmetry breaking puts below the candidate (bit i of
// `up`) offers its upper-rank list N+(M[i]) instead of N(M[i]).
struct LocalList {
    const int32_t* ptr;  // first entry
    int32_t len;
    int32_t src;         // level of the owner, | kSrcUpper when ptr is in N+
};
constexpr int kSrcUpper = 0x40;
constexpr int kSrcLevel = 0x1f;

__device__ __forceinline__ LocalList local_list_of(const DevGraph& G, int i, int32_t x, bool upper) {
    LocalList L;
    if (upper) {
        L.ptr = G.up_col + __ldg(G.up_rowptr + x);
        L.len = __ldg(G.updeg + x);
        L.src = i | kSrcUpper;
    } else {
        L.ptr = G.col + __ldg(G.rowptr + x);
        L.len = __ldg(G.deg + x);
        L.src = i;
    }
    return L;
}

__device__ __forceinline__ LocalList row_local_list(const DevGraph& G, const LevelPlan& lp, const int32_t* row,
                                                    int d) {
    int32_t bestd = INT_MAX, besti = 0, bestx = 0;
    bool bestu = false;
    for (int i = 0; i < d; ++i)
        if ((lp.bwd >> i) & 1u) {
            const int32_t x = row[i];
            const bool up = (lp.up >> i) & 1u;
            const int32_t dx = up ? __ldg(G.updeg + x) : __ldg(G.deg + x);
            if (dx < bestd) { bestd = dx; besti = i; bestx = x; bestu = up; }
        }
    return local_list_of(G, besti, bestx, bestu);
}

// Checks still needed for a candidate taken from list L: injectivity,
// symmetry breaking and membership in every other backward list; the owner's
// own membership (and its rank test, for N+) hold by construction.
__device__ __forceinline__ uint32_t need_mask(const LevelPlan& lp, int src) {
    const uint32_t own = 1u << (src & kSrcLevel);
    const uint32_t sb = lp.sb_gt | lp.sb_lt;
    return lp.inj | (sb & ~((src & kSrcUpper) ? own : 0u)) | (lp.bwd & ~own);
}
