/* closed_forms.c - test-only counts that pin the engine's full-graph results
 * to closed forms, written independently of both the oracle and the engine.
 *
 *   cf_triangles: triangles of a symmetric CSR graph, each counted once:
 *       every edge is oriented from the lower to the higher (degree, id)
 *       rank (an oriented CSR is built first), and for each vertex v the
 *       out-neighbours of each out-neighbour w of v are looked up in a mark
 *       array holding v's out-neighbours.
 *       K3 has 6 embeddings per triangle.
 *   cf_trace_a4: tr(A^4) = sum over ordered vertex pairs (u, v) of
 *       c(u, v)^2, c = the number of common neighbours (closed 4-walks),
 *       by counting the 2-walks out of each u in a dense array. C4 has
 *       tr(A^4) - 2 sum_v d(v)^2 + 2|E| embeddings.
 * Built with gcc by the tests that use it. */
#include <stdint.h>
#include <stdlib.h>

static int rank_less(const int64_t* rowptr, int32_t a, int32_t b) {
    const int64_t da = rowptr[a + 1] - rowptr[a], db = rowptr[b + 1] - rowptr[b];
    return da < db || (da == db && a < b);
}

int64_t cf_triangles(int64_t n, const int64_t* rowptr, const int32_t* col) {
    /* the oriented graph: out(v) = neighbours of higher rank (a hub has few) */
    int64_t* orp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* mark = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!orp || !mark) {
        free(orp);
        free(mark);
        return -1;
    }
    orp[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t c = 0;
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; ++j) c += rank_less(rowptr, (int32_t)v, col[j]);
        orp[v + 1] = orp[v] + c;
    }
    int32_t* ocol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(orp[n] > 0 ? orp[n] : 1));
    if (!ocol) {
        free(orp);
        free(mark);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) {
        int64_t at = orp[v];
        for (int64_t j = rowptr[v]; j < rowptr[v + 1]; ++j)
            if (rank_less(rowptr, (int32_t)v, col[j])) ocol[at++] = col[j];
        mark[v] = -1;
    }
    int64_t t = 0;
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t j = orp[v]; j < orp[v + 1]; ++j) mark[ocol[j]] = v;
        for (int64_t j = orp[v]; j < orp[v + 1]; ++j) {
            const int32_t w = ocol[j];
            for (int64_t i = orp[w]; i < orp[w + 1]; ++i) t += mark[ocol[i]] == v;
        }
    }
    free(orp);
    free(ocol);
    free(mark);
    return t;
}

int64_t cf_trace_a4(int64_t n, const int64_t* rowptr, const int32_t* col) {
    int64_t* cnt = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!cnt || !touched) {
        free(cnt);
        free(touched);
        return -1;
    }
    int64_t s = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t nt = 0;
        for (int64_t j = rowptr[u]; j < rowptr[u + 1]; ++j) {
            const int32_t w = col[j];
            for (int64_t i = rowptr[w]; i < rowptr[w + 1]; ++i) {
                const int32_t v = col[i];
                if (cnt[v]++ == 0) touched[nt++] = v;
            }
        }
        for (int64_t i = 0; i < nt; ++i) {
            s += cnt[touched[i]] * cnt[touched[i]];
            cnt[touched[i]] = 0;
        }
    }
    free(cnt);
    free(touched);
    return s;
}
