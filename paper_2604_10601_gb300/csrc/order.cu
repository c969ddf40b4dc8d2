// order.cu - the learned matching order (host side): prefix features for the
// cost model and a beam search over connected orders scored by the model's
// predicted partial-match counts, with the rule-based greedy order as the
// fallback. The paper generates phi with a rule-based method on the CPU
// (Sec. 3); the model is this library's addition. The model's forward pass
// runs in mlp.cu's kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "objects.h"

extern "C" sgm_status sgm_model_forward(sgm_model* m, const float* X, int64_t n, float* y);
extern "C" sgm_status sgm_model_info(const sgm_model* m, int32_t* in_dim, int32_t* hidden, int64_t* n_params,
                                     int64_t* steps);

namespace {

struct QueryView {
    int k = 0;
    int m = 0;
    uint32_t adj[SGM_KMAX];
    int32_t label[SGM_KMAX];
};

double selectivity(const sgm_graph_stats& gs, int32_t label) {
    // -log2 of the fraction of data vertices carrying the label (floored at 1/n)
    const double n = gs.n > 0 ? (double)gs.n : 1.0;
    double p = (label >= 0 && label < gs.num_labels && label < 256) ? gs.label_frac[label] : 0.0;
    p = std::max(p, 1.0 / n);
    return -std::log2(p);
}

double moment(const sgm_graph_stats& gs, int j) { return j <= 0 ? 0.0 : gs.log2_deg_moment[std::min(j, 4) - 1]; }

// Features of the prefix phi[0..i] (see include/sgm.h for the list).
void prefix_features(const sgm_graph_stats& gs, const QueryView& q, const int32_t* phi, int i, int64_t anchor_deg,
                     float* f) {
    const int k = q.k;
    uint32_t P = 0;
    for (int t = 0; t <= i; ++t) P |= 1u << phi[t];
    const int u = phi[i];
    int eP = 0, degc[5] = {0, 0, 0, 0, 0};
    double sel_sum = 0.0, mom_sum = 0.0;
    for (int t = 0; t <= i; ++t) {
        const int v = phi[t];
        const int dv = popc32(q.adj[v] & P);
        eP += dv;
        degc[std::min(dv, 4)]++;
        sel_sum += selectivity(gs, q.label[v]);
        mom_sum += moment(gs, std::min(dv, 4));
    }
    eP /= 2;
    const int s = i + 1;
    double entropy = 0.0, pmax = 0.0;
    for (int l = 0; l < gs.num_labels && l < 256; ++l) {
        const double p = gs.label_frac[l];
        if (p > 0) entropy -= p * std::log2(p);
        pmax = std::max(pmax, p);
    }
    const double n = std::max<double>((double)gs.n, 1.0);
    const double nnz = std::max<double>((double)gs.nnz, 1.0);
    float* o = f;
    *o++ = anchor_deg >= 0 ? (float)(std::log2(1.0 + (double)anchor_deg) / 32.0) : 0.0f;
    *o++ = (float)(s / 32.0);
    *o++ = (float)(eP / 64.0);
    *o++ = (float)((eP - s + 1) / 32.0);
    *o++ = (float)(popc32(q.adj[u]) / 32.0);
    *o++ = (float)(popc32(q.adj[u] & P & ~(1u << u)) / 32.0);
    *o++ = (float)(selectivity(gs, q.label[u]) / 16.0);
    *o++ = (float)(sel_sum / 128.0);
    for (int d = 1; d <= 4; ++d) *o++ = (float)(degc[d] / 32.0);
    *o++ = (float)(mom_sum / 256.0);
    *o++ = (float)(std::log2(n) / 32.0);
    *o++ = (float)(std::log2(nnz) / 32.0);
    for (int j = 1; j <= 4; ++j) *o++ = (float)(moment(gs, j) / (16.0 * j));
    *o++ = (float)(entropy / 8.0);
    *o++ = (float)(gs.num_labels / 64.0);
    *o++ = (float)pmax;
    *o++ = (float)(k / 32.0);
    *o++ = (float)(q.m / 64.0);
    for (int b = 0; b < 8; ++b) *o++ = (float)gs.deg_hist[b];
}

sgm_status check_phi(const QueryView& q, const int32_t* phi) {
    uint32_t seen = 0;
    for (int i = 0; i < q.k; ++i) {
        const int u = phi[i];
        if (u < 0 || u >= q.k || ((seen >> u) & 1u)) return sgm_fail(SGM_E_INVALID_ARG, "order is not a permutation");
        if (i > 0 && !(q.adj[u] & seen))
            return sgm_fail(SGM_E_ORDER_NOT_CONNECTED, "order vertex %d (position %d) has no earlier neighbour", u, i);
        seen |= 1u << u;
    }
    return SGM_OK;
}

QueryView view_of(const sgm_query* q) {
    QueryView v;
    v.k = q->k;
    v.m = q->m;
    memcpy(v.adj, q->adj, sizeof(v.adj));
    memcpy(v.label, q->label, sizeof(v.label));
    return v;
}

// Does the order end in a vertex with exactly one earlier neighbour? A count
// then takes its last level arithmetically (no candidate is visited there),
// so that prefix costs no search work.
bool arith_last_level(const QueryView& q, const int32_t* phi) {
    if (q.k < 2) return false;
    uint32_t before = 0;
    for (int i = 0; i < q.k - 1; ++i) before |= 1u << phi[i];
    return __builtin_popcount(q.adj[phi[q.k - 1]] & before) == 1;
}

// Predicted work of each order in `orders` (each k long): the sum over its
// first `upto` prefixes of the predicted partial matches, the last prefix
// left out when it is counted arithmetically.
sgm_status predict_work(sgm_model* md, const sgm_graph_stats& gs, const QueryView& q,
                        const std::vector<std::vector<int32_t>>& orders, int upto, int64_t anchor_deg,
                        std::vector<double>& work) {
    const int n_ord = (int)orders.size();
    std::vector<float> X((size_t)n_ord * upto * SGM_FEATURES);
    for (int o = 0; o < n_ord; ++o)
        for (int i = 0; i < upto; ++i)
            prefix_features(gs, q, orders[o].data(), i, anchor_deg, X.data() + ((size_t)o * upto + i) * SGM_FEATURES);
    std::vector<float> y((size_t)n_ord * upto);
    SGM_TRY(sgm_model_forward(md, X.data(), (int64_t)y.size(), y.data()));
    work.assign(n_ord, 0.0);
    for (int o = 0; o < n_ord; ++o)
        for (int i = 0; i < upto; ++i)
            if (!(i == q.k - 1 && arith_last_level(q, orders[o].data())))
                work[o] += std::pow(10.0, std::min<double>(y[(size_t)o * upto + i], 30.0));
    return SGM_OK;
}

}  // namespace

// Degree of data vertex v of g (one value read back from the device), or -1.
static int64_t anchor_degree(const sgm_graph* g, int64_t v) {
    if (v < 0 || v >= g->G.n) return -1;
    int32_t d = 0;
    if (cudaMemcpy(&d, g->G.deg + v, sizeof(int32_t), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return d;
}

extern "C" sgm_status sgm_features_from_stats(const sgm_graph_stats* gs, int32_t k, int32_t m, const int32_t* edges,
                                              const int32_t* labels, const int32_t* phi, int64_t anchor_deg,
                                              float* out) {
    if (!gs || !phi || !out || (m > 0 && !edges)) return sgm_fail(SGM_E_INVALID_ARG, "sgm_features_from_stats: NULL argument");
    if (k < 1 || k > SGM_KMAX || m < 0) return sgm_fail(SGM_E_INVALID_ARG, "bad k = %d or m = %d", k, m);
    if (gs->num_labels < 1 || gs->num_labels > 256) return sgm_fail(SGM_E_INVALID_ARG, "num_labels %d", gs->num_labels);
    QueryView q;
    q.k = k;
    q.m = m;
    memset(q.adj, 0, sizeof(q.adj));
    for (int i = 0; i < m; ++i) {
        const int a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b) return sgm_fail(SGM_E_QUERY_INVALID, "query edge %d invalid", i);
        q.adj[a] |= 1u << b;
        q.adj[b] |= 1u << a;
    }
    for (int u = 0; u < k; ++u) q.label[u] = labels ? labels[u] : 0;
    SGM_TRY(check_phi(q, phi));
    for (int i = 0; i < k; ++i) prefix_features(*gs, q, phi, i, anchor_deg, out + (size_t)i * SGM_FEATURES);
    return SGM_OK;
}

extern "C" sgm_status sgm_prefix_features(const sgm_query* q, const sgm_graph* g, const int32_t* phi, int64_t anchor,
                                          float* out) {
    if (!q || !g || !out) return sgm_fail(SGM_E_INVALID_ARG, "sgm_prefix_features: NULL argument");
    const QueryView v = view_of(q);
    const int32_t* order = phi;
    if (!order) {
        if (!q->has_order) return sgm_fail(SGM_E_INVALID_ARG, "the query has no order yet");
        order = q->order;
    }
    SGM_TRY(check_phi(v, order));
    const int64_t ad = anchor >= 0 ? anchor_degree(g, anchor) : -1;
    if (anchor >= 0 && ad < 0) return sgm_fail(SGM_E_INVALID_ARG, "anchor %lld outside the graph", (long long)anchor);
    for (int i = 0; i < v.k; ++i) prefix_features(g->gstats, v, order, i, ad, out + (size_t)i * SGM_FEATURES);
    return SGM_OK;
}

extern "C" sgm_status sgm_query_order_learned(sgm_query* q, const sgm_graph* g, sgm_model* md, int32_t beam,
                                              int32_t root, int64_t anchor, double* pred_learned,
                                              double* pred_greedy, int32_t* used_learned) {
    if (!q || !g || !md) return sgm_fail(SGM_E_INVALID_ARG, "sgm_query_order_learned: NULL argument");
    if (beam < 1) return sgm_fail(SGM_E_INVALID_ARG, "beam must be >= 1");
    if (root >= q->k) return sgm_fail(SGM_E_INVALID_ARG, "root %d outside [0, %d)", root, q->k);
    const int64_t ad = anchor >= 0 ? anchor_degree(g, anchor) : -1;
    if (anchor >= 0 && ad < 0) return sgm_fail(SGM_E_INVALID_ARG, "anchor %lld outside the graph", (long long)anchor);
    int32_t in_dim = 0;
    SGM_TRY(sgm_model_info(md, &in_dim, nullptr, nullptr, nullptr));
    if (in_dim != SGM_FEATURES) return sgm_fail(SGM_E_INVALID_ARG, "model input %d != SGM_FEATURES", in_dim);
    const QueryView v = view_of(q);
    const sgm_graph_stats& gs = g->gstats;
    const int k = v.k;
    // beam search: states are prefixes; the score of a state is the predicted
    // work of its prefixes so far (a full order's last prefix is free when a
    // count takes that level arithmetically)
    struct State {
        std::vector<int32_t> phi;
        uint32_t set;
        double work;
    };
    std::vector<State> states;
    for (int u = 0; u < k; ++u)
        if (root < 0 || u == root) states.push_back({{u}, 1u << u, 0.0});
    for (int len = 1; len <= k; ++len) {
        // score the current states' last prefix
        std::vector<std::vector<int32_t>> pre;
        for (const State& st : states) {
            std::vector<int32_t> full = st.phi;
            full.resize(k, 0);
            pre.push_back(full);
        }
        // features of prefix len-1 only: pass orders padded, score index len-1
        std::vector<float> X(states.size() * SGM_FEATURES);
        for (size_t o = 0; o < states.size(); ++o)
            prefix_features(gs, v, pre[o].data(), len - 1, ad, X.data() + o * SGM_FEATURES);
        std::vector<float> y(states.size());
        SGM_TRY(sgm_model_forward(md, X.data(), (int64_t)y.size(), y.data()));
        for (size_t o = 0; o < states.size(); ++o)
            if (!(len == k && arith_last_level(v, states[o].phi.data())))
                states[o].work += std::pow(10.0, std::min<double>(y[o], 30.0));
        std::sort(states.begin(), states.end(), [](const State& a, const State& b) {
            return a.work != b.work ? a.work < b.work : a.phi < b.phi;
        });
        if ((int)states.size() > beam) states.resize(beam);
        if (len == k) break;
        std::vector<State> next;
        for (const State& st : states) {
            uint32_t frontier = 0;
            for (int32_t u : st.phi) frontier |= v.adj[u];
            frontier &= ~st.set;
            for (int u = 0; u < k; ++u)
                if ((frontier >> u) & 1u) {
                    State ns = st;
                    ns.phi.push_back(u);
                    ns.set |= 1u << u;
                    next.push_back(ns);
                }
        }
        if (next.empty()) return sgm_fail(SGM_E_QUERY_DISCONNECTED, "query graph is not connected");
        states.swap(next);
    }
    const State& best = states.front();
    // the greedy order, scored the same way
    sgm_query tmp = *q;
    sgm_greedy_order(&tmp, g, root >= 0 ? root : -1);
    std::vector<std::vector<int32_t>> greedy = {std::vector<int32_t>(tmp.order, tmp.order + k)};
    std::vector<double> gw;
    SGM_TRY(predict_work(md, gs, v, greedy, k, ad, gw));
    const bool take = best.work < gw[0];
    memcpy(q->order, take ? best.phi.data() : tmp.order, sizeof(int32_t) * k);
    q->has_order = true;
    if (pred_learned) *pred_learned = best.work;
    if (pred_greedy) *pred_greedy = gw[0];
    if (used_learned) *used_learned = take ? 1 : 0;
    return SGM_OK;
}
