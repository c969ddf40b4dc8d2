/*
 * graphgen.c - seeded synthetic inputs for the subgraph-matching engine and
 * its oracle: Erdos-Renyi and R-MAT data graphs, uniform and Zipf vertex
 * labels, and random-walk query extraction.
 *
 * This module is input generation only. It holds none of the matching
 * arithmetic (no candidate checks, no embedding hash); both the CUDA engine
 * and the CPU oracle consume what it produces.
 *
 * Random numbers come from one counter-based generator, so every value is a
 * pure function of (seed, stream, counter) and the output is identical for
 * any thread count and on any host architecture:
 *     fmix(z)            = MurmurHash3 64-bit finaliser (Appleby, public domain)
 *     rand(seed, s, i)   = fmix(fmix(fmix(seed) ^ s) + (i + 1) * 0x9E3779B97F4A7C15)
 *     uniform01          = (rand >> 11) * 2^-53
 *
 * Workload shapes follow the paper's experimental setup:
 *   - R-MAT graphs as produced by PaRMAT (Sec. 6.1, "Datasets"): every edge
 *     picks one of four quadrants per bit with probabilities a, b, c, d;
 *     self-loops dropped, symmetrised, duplicates removed.
 *   - uniform labels (Sec. 6.1, "each vertex is assigned a label uniformly").
 *   - Zipf labels P(l) proportional to (l+1)^-alpha (Appendix A, label skew).
 *   - random queries grown from a seed vertex by random neighbours, keeping
 *     the connecting edges (Sec. 6.1, "Query Sets").
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_GOLDEN 0x9E3779B97F4A7C15ULL

enum { GG_STREAM_ER = 1, GG_STREAM_RMAT = 2, GG_STREAM_LABEL = 3, GG_STREAM_WALK = 4 };

static inline uint64_t gg_fmix(uint64_t z) {
    z ^= z >> 33;
    z *= 0xff51afd7ed558ccdULL;
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ULL;
    z ^= z >> 33;
    return z;
}

uint64_t gg_rand64(uint64_t seed, uint64_t stream, uint64_t i) {
    return gg_fmix(gg_fmix(gg_fmix(seed) ^ stream) + (i + 1) * GG_GOLDEN);
}

static inline double gg_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------------------ */
/* CSR construction: undirected, sorted, no self-loops, no duplicates.        */
/* ------------------------------------------------------------------------ */

static int gg_cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

static void gg_sort_row(int32_t* a, int64_t len) {
    if (len < 32) {
        for (int64_t i = 1; i < len; i++) {
            int32_t x = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
            a[j + 1] = x;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), gg_cmp_i32);
    }
}

/*
 * Builds the symmetric CSR of the undirected simple graph spanned by the m
 * edge pairs (src[i], dst[i]) over vertices [0, n). Self-loops are dropped,
 * both directions are stored, rows are sorted ascending and deduplicated.
 * rowptr must hold n+1 entries, col at least 2*m. Returns nnz (directed
 * entries) or -1 on a vertex id out of range, -2 on allocation failure.
 */
int64_t gg_csr_from_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                          int64_t* rowptr, int32_t* col) {
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) return -2;
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int64_t i = 0; i < m; i++) {
        int32_t s = src[i], d = dst[i];
        if (s < 0 || d < 0 || s >= n || d >= n) { bad = 1; continue; }
        if (s == d) continue;
        __atomic_fetch_add(&deg[s], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&deg[d], 1, __ATOMIC_RELAXED);
    }
    if (bad) { free(deg); return -1; }
    rowptr[0] = 0;
    for (int64_t v = 0; v < n; v++) rowptr[v + 1] = rowptr[v] + deg[v];
    int64_t* pos = deg; /* reuse as write cursors */
    for (int64_t v = 0; v < n; v++) pos[v] = rowptr[v];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++) {
        int32_t s = src[i], d = dst[i];
        if (s == d) continue;
        col[__atomic_fetch_add(&pos[s], 1, __ATOMIC_RELAXED)] = d;
        col[__atomic_fetch_add(&pos[d], 1, __ATOMIC_RELAXED)] = s;
    }
    /* sort + dedupe each row in place; pos[v] becomes the deduplicated length */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t v = 0; v < n; v++) {
        int32_t* a = col + rowptr[v];
        int64_t len = rowptr[v + 1] - rowptr[v];
        gg_sort_row(a, len);
        int64_t w = 0;
        for (int64_t i = 0; i < len; i++)
            if (w == 0 || a[i] != a[w - 1]) a[w++] = a[i];
        pos[v] = w;
    }
    /* compact rows to the front (forward moves never overlap a later row) */
    int64_t out = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t start = rowptr[v], len = pos[v];
        if (out != start && len) memmove(col + out, col + start, (size_t)len * sizeof(int32_t));
        rowptr[v] = out;
        out += len;
    }
    rowptr[n] = out;
    free(deg);
    return out;
}

/* ------------------------------------------------------------------------ */
/* Erdos-Renyi G(n, p): every unordered pair {i<j} is an edge with prob. p.   */
/* Returns nnz; col needs capacity for every sampled pair twice.              */
/* ------------------------------------------------------------------------ */
int64_t gg_er_edges(int64_t n, double p, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap) {
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            if (gg_unit(gg_rand64(seed, GG_STREAM_ER, (uint64_t)(i * n + j))) < p) {
                if (m >= cap) return -3;
                src[m] = (int32_t)i;
                dst[m] = (int32_t)j;
                m++;
            }
        }
    return m;
}

/* ------------------------------------------------------------------------ */
/* R-MAT edge sampling (PaRMAT-style, no noise, no permutation).              */
/* Edge e descends `scale` levels; at level t (most significant bit first) it */
/* picks quadrant 0..3 with probabilities a, b, c, 1-a-b-c using the 32-bit   */
/* half t%2 of rand(seed, RMAT, e*ceil(scale/2) + t/2).                       */
/* ------------------------------------------------------------------------ */
void gg_rmat_edges(int32_t scale, int64_t m, double a, double b, double c, uint64_t seed,
                   int32_t* src, int32_t* dst) {
    const double t_ab = a + b, t_abc = a + b + c;
    const int64_t words = (scale + 1) / 2;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; e++) {
        uint32_t s = 0, d = 0;
        uint64_t r = 0;
        for (int32_t t = 0; t < scale; t++) {
            if ((t & 1) == 0) r = gg_rand64(seed, GG_STREAM_RMAT, (uint64_t)(e * words + t / 2));
            uint32_t half = (t & 1) ? (uint32_t)(r >> 32) : (uint32_t)r;
            double x = (double)half * (1.0 / 4294967296.0);
            uint32_t sb, db;
            if (x < a) { sb = 0; db = 0; }
            else if (x < t_ab) { sb = 0; db = 1; }
            else if (x < t_abc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
}

/* ------------------------------------------------------------------------ */
/* Vertex labels.                                                             */
/* ------------------------------------------------------------------------ */
void gg_labels_uniform(int64_t n, int32_t num_labels, uint64_t seed, int32_t* out) {
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; v++) {
        int32_t l = (int32_t)(gg_unit(gg_rand64(seed, GG_STREAM_LABEL, (uint64_t)v)) * num_labels);
        out[v] = l < num_labels ? l : num_labels - 1;
    }
}

/* Zipf: P(l) = (l+1)^-alpha / sum_{i=1..L} i^-alpha, l = 0..L-1 (Appendix A),
 * sampled by inverse CDF on one 53-bit uniform per vertex. */
void gg_labels_zipf(int64_t n, int32_t num_labels, double alpha, uint64_t seed, int32_t* out) {
    double* cdf = (double*)malloc(sizeof(double) * (size_t)num_labels);
    double z = 0.0;
    for (int32_t l = 0; l < num_labels; l++) z += pow((double)(l + 1), -alpha);
    double acc = 0.0;
    for (int32_t l = 0; l < num_labels; l++) {
        acc += pow((double)(l + 1), -alpha) / z;
        cdf[l] = acc;
    }
    cdf[num_labels - 1] = 1.0;
#pragma omp parallel for schedule(static)
    for (int64_t v = 0; v < n; v++) {
        double x = gg_unit(gg_rand64(seed, GG_STREAM_LABEL, (uint64_t)v));
        int32_t lo = 0, hi = num_labels - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if (x < cdf[mid]) hi = mid; else lo = mid + 1;
        }
        out[v] = lo;
    }
    free(cdf);
}

/* ------------------------------------------------------------------------ */
/* Random-walk query extraction (Sec. 6.1 "Query Sets").                      */
/* ------------------------------------------------------------------------ */
static int gg_adjacent(const int64_t* rowptr, const int32_t* col, int32_t x, int32_t y) {
    int64_t lo = rowptr[x], hi = rowptr[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < y) lo = mid + 1; else hi = mid;
    }
    return lo < rowptr[x + 1] && col[lo] == y;
}

/*
 * Grows a k-vertex query from the data graph. A walk starts at a uniformly
 * drawn vertex of degree >= 1, steps to a uniform neighbour of the current
 * vertex each time and keeps the vertex if it is new; after 64*k steps
 * without completing it restarts from a new seed vertex.
 *   dense != 0: the query holds every edge of G among the walked vertices.
 *   dense == 0: the discovery-tree edges plus n_extra further edges of G
 *               among the walked vertices, drawn uniformly (fewer if fewer exist).
 * verts_out[k]: data vertex of local query vertex i (discovery order), so
 * verts_out is itself one embedding of the query. edges_out holds m pairs
 * (i < j), sorted. Returns m >= 0, or -1 when no vertex has an edge or the
 * walk never reaches k distinct vertices.
 */
int32_t gg_walk_query_bounded(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t k,
                              int32_t dense, int32_t n_extra, uint64_t seed, int64_t min_deg, int64_t max_deg,
                              int32_t* verts_out, int32_t* edges_out);

int32_t gg_walk_query(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t k,
                      int32_t dense, int32_t n_extra, uint64_t seed,
                      int32_t* verts_out, int32_t* edges_out) {
    return gg_walk_query_bounded(n, rowptr, col, k, dense, n_extra, seed, 1, INT64_MAX, verts_out, edges_out);
}

/* As gg_walk_query, but the walk only visits vertices whose degree lies in
 * [min_deg, max_deg]: the seed is redrawn and a step to a neighbour outside
 * the range is skipped (it still counts as a step). With min_deg <= 1 and
 * max_deg >= the maximum degree the draws are the same as gg_walk_query's. */
int32_t gg_walk_query_bounded(int64_t n, const int64_t* rowptr, const int32_t* col, int32_t k,
                              int32_t dense, int32_t n_extra, uint64_t seed, int64_t min_deg, int64_t max_deg,
                              int32_t* verts_out, int32_t* edges_out) {
    uint64_t ctr = 0;
    int32_t cnt = 0;
    int32_t tree_a[64], tree_b[64];
    int32_t ntree = 0;
    if (k < 1 || k > 64) return -1;
    for (int32_t restart = 0; restart < 1000 && cnt < k; restart++) {
        int32_t v = -1;
        for (int32_t tries = 0; tries < 100000; tries++) {
            int64_t c = (int64_t)(gg_rand64(seed, GG_STREAM_WALK, ctr++) % (uint64_t)n);
            const int64_t dc = rowptr[c + 1] - rowptr[c];
            if (dc > 0 && dc >= min_deg && dc <= max_deg) { v = (int32_t)c; break; }
        }
        if (v < 0) return -1;
        cnt = 0;
        ntree = 0;
        verts_out[cnt++] = v;
        int32_t cur_local = 0;
        int32_t cur = v;
        for (int64_t step = 0; step < 64LL * k && cnt < k; step++) {
            int64_t d = rowptr[cur + 1] - rowptr[cur];
            int32_t w = col[rowptr[cur] + (int64_t)(gg_rand64(seed, GG_STREAM_WALK, ctr++) % (uint64_t)d)];
            if (rowptr[w + 1] - rowptr[w] > max_deg || rowptr[w + 1] - rowptr[w] < min_deg) continue;
            int32_t wl = -1;
            for (int32_t i = 0; i < cnt; i++)
                if (verts_out[i] == w) { wl = i; break; }
            if (wl < 0) {
                wl = cnt;
                verts_out[cnt++] = w;
                tree_a[ntree] = cur_local;
                tree_b[ntree] = wl;
                ntree++;
            }
            cur = w;
            cur_local = wl;
        }
    }
    if (cnt < k) return -1;
    /* adjacency among the walked vertices, as an upper-triangular bit matrix */
    uint64_t adj[64], in_tree[64];
    for (int32_t i = 0; i < k; i++) { adj[i] = 0; in_tree[i] = 0; }
    for (int32_t i = 0; i < k; i++)
        for (int32_t j = i + 1; j < k; j++)
            if (gg_adjacent(rowptr, col, verts_out[i], verts_out[j])) adj[i] |= 1ULL << j;
    for (int32_t t = 0; t < ntree; t++) {
        int32_t i = tree_a[t] < tree_b[t] ? tree_a[t] : tree_b[t];
        int32_t j = tree_a[t] < tree_b[t] ? tree_b[t] : tree_a[t];
        in_tree[i] |= 1ULL << j;
    }
    if (!dense) {
        /* candidate extra edges: induced, not in the tree; pick n_extra uniformly */
        int32_t ca[2048], cb[2048];
        int32_t nc = 0;
        for (int32_t i = 0; i < k; i++)
            for (int32_t j = i + 1; j < k; j++)
                if (((adj[i] >> j) & 1) && !((in_tree[i] >> j) & 1) && nc < 2048) {
                    ca[nc] = i; cb[nc] = j; nc++;
                }
        int32_t take = n_extra < nc ? n_extra : nc;
        for (int32_t t = 0; t < take; t++) {
            int32_t r = t + (int32_t)(gg_rand64(seed, GG_STREAM_WALK, ctr++) % (uint64_t)(nc - t));
            int32_t xa = ca[t], xb = cb[t];
            ca[t] = ca[r]; cb[t] = cb[r];
            ca[r] = xa; cb[r] = xb;
            in_tree[ca[t]] |= 1ULL << cb[t];
        }
        for (int32_t i = 0; i < k; i++) adj[i] = in_tree[i];
    }
    int32_t m = 0;
    for (int32_t i = 0; i < k; i++)
        for (int32_t j = i + 1; j < k; j++)
            if ((adj[i] >> j) & 1) {
                edges_out[2 * m] = i;
                edges_out[2 * m + 1] = j;
                m++;
            }
    return m;
}

int32_t gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
