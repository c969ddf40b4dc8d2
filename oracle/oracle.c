/*
 * oracle.c - plain, slow, single-threaded CPU reference for subgraph matching.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the engine links, imports or calls
 * this file; only the tests, the package's smoke check and the benchmark's
 * CPU-baseline leg do. It shares no code with the CUDA path.
 *
 * What it computes (Definition 1, Sec. 2.1): every injective map
 * M : V(Q) -> V(G) with L(M[u]) = L(u) for each query vertex u and
 * {M[u], M[u']} in E(G) for each query edge {u, u'} (non-induced). Outputs:
 *   count = number of such maps (uint64),
 *   hash  = sum over maps of h(M) mod 2^64, where
 *           h(M) = mix(x_k),  x_0 = 0x243F6A8885A308D3,
 *           x_{u+1} = mix(x_u XOR ((u << 32) | (uint32)M[u])),  u = 0..k-1,
 *           and mix is the SplitMix64 output function (Steele, Lea, Flood,
 *           OOPSLA 2014). The map is indexed by query-vertex id, so the hash
 *           does not depend on the matching order or on emission order.
 *   level_counts[i] = number of partial matches over the first i+1 vertices
 *           of the matching order (embeddings of the prefix-induced query),
 *           optionally with every vertex restricted to a candidate set.
 *
 * How: the depth-first search of Alg. 1 (Search/Process) run sequentially -
 * extend the partial match one query vertex at a time along the order phi,
 * take as local candidates the neighbour list of the first backward
 * neighbour's image, and keep a candidate v when its label equals L(u), it is
 * not already used, and it lies in the neighbour list of every other backward
 * neighbour's image (plain binary search over the sorted CSR row).
 * With no order given it uses its own simple rule: the smallest-id vertex of
 * maximum query degree first, then repeatedly the smallest-id vertex adjacent
 * to those already chosen (the smallest unchosen id if none is adjacent).
 *
 * Root slicing: with root_u >= 0 the order starts at root_u and only maps
 * with root_lo <= M[root_u] < root_hi are produced.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXK 32

enum {
    OR_OK = 0,
    OR_E_ARG = -1,
    OR_E_ORDER = -2,
    OR_E_BUDGET = -3,
    OR_E_OOM = -4,
};

uint64_t oracle_mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t oracle_embedding_hash(int32_t k, const int32_t* M) {
    uint64_t x = 0x243F6A8885A308D3ULL;
    for (int32_t u = 0; u < k; u++)
        x = oracle_mix64(x ^ (((uint64_t)(uint32_t)u << 32) | (uint64_t)(uint32_t)M[u]));
    return oracle_mix64(x);
}

typedef struct {
    /* data graph */
    int64_t n;
    const int64_t* rowptr;
    const int32_t* col;
    const int32_t* labels; /* NULL: every vertex has label 0 */
    /* query */
    int32_t k;
    uint32_t qadj[OR_MAXK]; /* bit j of qadj[u]: query edge {u, j} */
    int32_t qlab[OR_MAXK];
    int32_t order[OR_MAXK];
    /* candidate restriction: bit v of cand[u * words ...], or NULL */
    const uint32_t* cand;
    int64_t words;
    /* root slice */
    int64_t root_lo, root_hi;
    /* state */
    int32_t M[OR_MAXK];
    unsigned char* used;
    /* outputs */
    uint64_t count, hash;
    uint64_t* level_counts;
    int32_t* rows;
    uint64_t cap;
    uint64_t steps, max_steps;
    int aborted;
} or_ctx;

static int or_label(const or_ctx* c, int64_t v) { return c->labels ? c->labels[v] : 0; }

static int or_in_row(const or_ctx* c, int32_t x, int32_t v) {
    int64_t lo = c->rowptr[x], hi = c->rowptr[x + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (c->col[mid] < v) lo = mid + 1;
        else hi = mid;
    }
    return lo < c->rowptr[x + 1] && c->col[lo] == v;
}

static void or_emit(or_ctx* c) {
    if (c->rows && c->count < c->cap) memcpy(c->rows + c->count * (uint64_t)c->k, c->M, sizeof(int32_t) * c->k);
    c->count++;
    c->hash += oracle_embedding_hash(c->k, c->M);
}

/* accept v as the image of u = order[i]; first_b is the position of the
 * backward neighbour whose row supplied v (-1 when v came from a vertex scan) */
static int or_accept(const or_ctx* c, int32_t i, int32_t u, int32_t v, int32_t first_b) {
    if (or_label(c, v) != c->qlab[u]) return 0;
    if (c->used[v]) return 0;
    if (c->cand && !((c->cand[(int64_t)u * c->words + (v >> 5)] >> (v & 31)) & 1u)) return 0;
    for (int32_t j = 0; j < i; j++) {
        int32_t w = c->order[j];
        if (j == first_b || !((c->qadj[u] >> w) & 1u)) continue;
        if (!or_in_row(c, c->M[w], v)) return 0;
    }
    return 1;
}

static void or_rec(or_ctx* c, int32_t i) {
    if (c->aborted) return;
    if (i == c->k) {
        or_emit(c);
        return;
    }
    if (c->max_steps && ++c->steps > c->max_steps) {
        c->aborted = 1;
        return;
    }
    int32_t u = c->order[i];
    int32_t first_b = -1;
    for (int32_t j = 0; j < i; j++)
        if ((c->qadj[u] >> c->order[j]) & 1u) { first_b = j; break; }
    int64_t lo, hi;
    const int32_t* src = NULL;
    if (first_b >= 0) {
        int32_t x = c->M[c->order[first_b]];
        lo = c->rowptr[x];
        hi = c->rowptr[x + 1];
        src = c->col;
    } else if (i == 0) {
        lo = c->root_lo;
        hi = c->root_hi;
    } else {
        lo = 0;
        hi = c->n;
    }
    for (int64_t t = lo; t < hi; t++) {
        int32_t v = src ? src[t] : (int32_t)t;
        if (!or_accept(c, i, u, v, first_b)) continue;
        c->M[u] = v;
        c->used[v] = 1;
        if (c->level_counts) c->level_counts[i]++;
        or_rec(c, i + 1);
        c->used[v] = 0;
        if (c->aborted) return;
    }
}

static int or_setup_query(or_ctx* c, int32_t k, int32_t m, const int32_t* qedges, const int32_t* qlabels) {
    if (k < 1 || k > OR_MAXK || m < 0) return OR_E_ARG;
    c->k = k;
    memset(c->qadj, 0, sizeof(c->qadj));
    for (int32_t e = 0; e < m; e++) {
        int32_t a = qedges[2 * e], b = qedges[2 * e + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return OR_E_ARG;
        c->qadj[a] |= 1u << b;
        c->qadj[b] |= 1u << a;
    }
    for (int32_t u = 0; u < k; u++) c->qlab[u] = qlabels ? qlabels[u] : 0;
    return OR_OK;
}

static void or_own_order(or_ctx* c, int32_t start) {
    uint32_t chosen = 0;
    int32_t first = start;
    if (first < 0) {
        int32_t best = -1;
        for (int32_t u = 0; u < c->k; u++)
            if (best < 0 || __builtin_popcount(c->qadj[u]) > __builtin_popcount(c->qadj[best])) best = u;
        first = best;
    }
    c->order[0] = first;
    chosen = 1u << first;
    for (int32_t i = 1; i < c->k; i++) {
        int32_t pick = -1;
        for (int32_t u = 0; u < c->k && pick < 0; u++)
            if (!((chosen >> u) & 1u) && (c->qadj[u] & chosen)) pick = u;
        for (int32_t u = 0; u < c->k && pick < 0; u++)
            if (!((chosen >> u) & 1u)) pick = u;
        c->order[i] = pick;
        chosen |= 1u << pick;
    }
}

/*
 * Enumerates all embeddings of Q in G (see the file header).
 *   order: NULL for the oracle's own order, else a permutation of 0..k-1 in
 *          which every vertex but the first has an earlier neighbour.
 *   root_u: -1 for the full set, else only maps with M[root_u] in
 *           [root_lo, root_hi); the order must then start at root_u.
 *   cand: NULL, or k bitmaps of ceil(n/32) words restricting M[u].
 *   rows: NULL or a buffer of cap*k int32 receiving the first cap maps.
 *   level_counts: NULL or k uint64 (zeroed here).
 *   max_steps: 0 for no limit, else abort with OR_E_BUDGET after that many
 *          search-tree nodes.
 */
int32_t oracle_match(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* labels,
                     int32_t k, int32_t m, const int32_t* qedges, const int32_t* qlabels,
                     const int32_t* order, int32_t root_u, int64_t root_lo, int64_t root_hi,
                     const uint32_t* cand, int32_t* rows, uint64_t cap,
                     uint64_t* count, uint64_t* hash, uint64_t* level_counts, uint64_t max_steps) {
    or_ctx c;
    memset(&c, 0, sizeof(c));
    if (n < 0 || !rowptr || (n > 0 && !col)) return OR_E_ARG;
    int32_t st = or_setup_query(&c, k, m, qedges, qlabels);
    if (st) return st;
    c.n = n;
    c.rowptr = rowptr;
    c.col = col;
    c.labels = labels;
    c.cand = cand;
    c.words = (n + 31) / 32;
    c.rows = rows;
    c.cap = rows ? cap : 0;
    c.max_steps = max_steps;
    c.level_counts = level_counts;
    if (level_counts) memset(level_counts, 0, sizeof(uint64_t) * k);
    if (root_u >= k) return OR_E_ARG;
    if (order) {
        uint32_t seen = 0;
        for (int32_t i = 0; i < k; i++) {
            int32_t u = order[i];
            if (u < 0 || u >= k || ((seen >> u) & 1u)) return OR_E_ORDER;
            if (i > 0 && !(c.qadj[u] & seen)) return OR_E_ORDER;
            seen |= 1u << u;
            c.order[i] = u;
        }
        if (root_u >= 0 && order[0] != root_u) return OR_E_ORDER;
    } else {
        or_own_order(&c, root_u);
    }
    c.root_lo = 0;
    c.root_hi = n;
    if (root_u >= 0) {
        c.root_lo = root_lo < 0 ? 0 : root_lo;
        c.root_hi = root_hi > n ? n : root_hi;
    }
    c.used = (unsigned char*)calloc((size_t)n + 1, 1);
    if (!c.used) return OR_E_OOM;
    if (c.root_lo < c.root_hi || root_u < 0) or_rec(&c, 0);
    free(c.used);
    *count = c.count;
    if (hash) *hash = c.hash;
    return c.aborted ? OR_E_BUDGET : OR_OK;
}

/* The order the oracle picks for itself (see the file header). */
int32_t oracle_own_order(int32_t k, int32_t m, const int32_t* qedges, int32_t root_u, int32_t* order_out) {
    or_ctx c;
    memset(&c, 0, sizeof(c));
    int32_t st = or_setup_query(&c, k, m, qedges, NULL);
    if (st) return st;
    or_own_order(&c, root_u);
    memcpy(order_out, c.order, sizeof(int32_t) * k);
    return OR_OK;
}

/*
 * Brute force over every injective map (n!/(n-k)! of them, in lexicographic
 * order of (M[0], ..., M[k-1])), testing Definition 1 directly with a dense
 * adjacency matrix. Only for tiny graphs: n <= 64.
 */
int32_t oracle_brute(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* labels,
                     int32_t k, int32_t m, const int32_t* qedges, const int32_t* qlabels,
                     int32_t* rows, uint64_t cap, uint64_t* count, uint64_t* hash) {
    if (n < 0 || n > 64 || k < 1 || k > OR_MAXK) return OR_E_ARG;
    uint64_t adj[64];
    memset(adj, 0, sizeof(adj));
    for (int64_t v = 0; v < n; v++)
        for (int64_t t = rowptr[v]; t < rowptr[v + 1]; t++) adj[v] |= 1ULL << col[t];
    int32_t M[OR_MAXK];
    uint64_t cnt = 0, h = 0;
    /* odometer over all k-tuples of distinct vertices */
    int32_t depth = 0;
    M[0] = -1;
    while (depth >= 0) {
        M[depth]++;
        if (M[depth] >= n) {
            depth--;
            continue;
        }
        int dup = 0;
        for (int32_t j = 0; j < depth; j++)
            if (M[j] == M[depth]) dup = 1;
        if (dup) continue;
        if (depth + 1 < k) {
            depth++;
            M[depth] = -1;
            continue;
        }
        int ok = 1;
        for (int32_t u = 0; u < k && ok; u++) {
            int32_t lu = qlabels ? qlabels[u] : 0;
            int32_t lv = labels ? labels[M[u]] : 0;
            if (lu != lv) ok = 0;
        }
        for (int32_t e = 0; e < m && ok; e++) {
            int32_t a = qedges[2 * e], b = qedges[2 * e + 1];
            if (!((adj[M[a]] >> M[b]) & 1ULL)) ok = 0;
        }
        if (ok) {
            if (rows && cnt < cap) memcpy(rows + cnt * (uint64_t)k, M, sizeof(int32_t) * k);
            cnt++;
            h += oracle_embedding_hash(k, M);
        }
    }
    *count = cnt;
    if (hash) *hash = h;
    return OR_OK;
}

/*
 * Candidate sets by definition: v is a candidate of query vertex u iff
 *   L(v) = L(u),  d_G(v) >= d_Q(u),  and for every label l the number of
 *   neighbours of v with label l is at least the number of neighbours of u
 *   with label l (neighbour-label frequency).
 * Each condition is necessary for M[u] = v in any embedding, so restricting
 * candidates never removes an embedding. bits_out: k bitmaps of ceil(n/32)
 * words, bit v of bitmap u set iff v is a candidate of u.
 */
int32_t oracle_filter(int64_t n, const int64_t* rowptr, const int32_t* col, const int32_t* labels,
                      int32_t num_labels, int32_t k, int32_t m, const int32_t* qedges,
                      const int32_t* qlabels, uint32_t* bits_out) {
    or_ctx c;
    memset(&c, 0, sizeof(c));
    if (num_labels < 1) return OR_E_ARG;
    int32_t st = or_setup_query(&c, k, m, qedges, qlabels);
    if (st) return st;
    int64_t words = (n + 31) / 32;
    memset(bits_out, 0, sizeof(uint32_t) * (size_t)(words * k));
    int64_t* qnlf = (int64_t*)calloc((size_t)k * num_labels, sizeof(int64_t));
    int64_t* vnlf = (int64_t*)calloc((size_t)num_labels, sizeof(int64_t));
    if (!qnlf || !vnlf) {
        free(qnlf);
        free(vnlf);
        return OR_E_OOM;
    }
    for (int32_t u = 0; u < k; u++)
        for (int32_t w = 0; w < k; w++)
            if ((c.qadj[u] >> w) & 1u) {
                int32_t lw = c.qlab[w];
                if (lw < 0 || lw >= num_labels) continue; /* such a u has no candidate */
                qnlf[(int64_t)u * num_labels + lw]++;
            }
    for (int64_t v = 0; v < n; v++) {
        memset(vnlf, 0, sizeof(int64_t) * num_labels);
        for (int64_t t = rowptr[v]; t < rowptr[v + 1]; t++) vnlf[labels ? labels[col[t]] : 0]++;
        int64_t dv = rowptr[v + 1] - rowptr[v];
        int32_t lv = labels ? labels[v] : 0;
        for (int32_t u = 0; u < k; u++) {
            if (lv != c.qlab[u]) continue;
            if (dv < __builtin_popcount(c.qadj[u])) continue;
            int ok = 1;
            for (int32_t l = 0; l < num_labels && ok; l++)
                if (vnlf[l] < qnlf[(int64_t)u * num_labels + l]) ok = 0;
            /* a query neighbour with an out-of-range label can never be matched */
            for (int32_t w = 0; w < k && ok; w++)
                if (((c.qadj[u] >> w) & 1u) && (c.qlab[w] < 0 || c.qlab[w] >= num_labels)) ok = 0;
            if (ok) bits_out[(int64_t)u * words + (v >> 5)] |= 1u << (v & 31);
        }
    }
    free(qnlf);
    free(vnlf);
    return OR_OK;
}
