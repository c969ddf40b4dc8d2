// refine.cuh - the support rule of the candidate-set refinement (the
// candidate sets of the candidate graph G' that the paper's large-query
// workloads search on, Sec. 6.1, Methods Under Study). One round keeps v as
// a candidate of query vertex u only if, for every query neighbour u' of u,
// some data neighbour of v is a candidate of u' in the previous round.
// Host and device compile the same rule: the kernel applies it to every
// vertex of a round; a host build of it is tested against the oracle.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define SGM_HD __host__ __device__ __forceinline__
#else
#define SGM_HD inline
#endif

SGM_HD int sgm_low_bit(uint32_t x) {
#if defined(__CUDA_ARCH__)
    return __ffs(x) - 1;
#else
    return __builtin_ctz(x);
#endif
}

// The query vertices whose candidate v stays after one round. `in`: bit u set
// iff v is a candidate of u in `cur` (k bitmaps of `words` uint32 words,
// bitmap u at cur + u * words); qadj[u]: bit u' set iff {u, u'} is a query
// edge. The scan of N(v) stops as soon as every needed neighbour set has a
// member among v's neighbours.
SGM_HD uint32_t sgm_refine_vertex(const int64_t* rowptr, const int32_t* col, int64_t v, const uint32_t* cur,
                                  int64_t words, int32_t k, const uint32_t* qadj, uint32_t in) {
    uint32_t need = 0;
    for (int u = 0; u < k; ++u)
        if ((in >> u) & 1u) need |= qadj[u];
    uint32_t has = 0;
    const int64_t end = rowptr[v + 1];
    for (int64_t j = rowptr[v]; j < end && (need & ~has) != 0u; ++j) {
        const int32_t x = col[j];
        uint32_t left = need & ~has;
        while (left) {
            const int u2 = sgm_low_bit(left);
            left &= left - 1u;
            if ((cur[(int64_t)u2 * words + (x >> 5)] >> (x & 31)) & 1u) has |= 1u << u2;
        }
    }
    uint32_t out = 0;
    for (int u = 0; u < k; ++u)
        if (((in >> u) & 1u) && (qadj[u] & ~has) == 0u) out |= 1u << u;
    return out;
}
