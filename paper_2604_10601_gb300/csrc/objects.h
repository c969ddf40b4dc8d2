// objects.h - the engine, graph and query objects behind the opaque handles
// of include/sgm.h, shared by the host-side translation units of libsgm.
#pragma once

#include <cstdarg>
#include <vector>

#include "launch.h"

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

sgm_status buf_ensure(DevBuf& b, size_t bytes);
void buf_free(DevBuf& b);
// Records a printf-style message for sgm_last_error() and returns st.
sgm_status sgm_fail(sgm_status st, const char* fmt, ...);

struct sgm_engine {
    int32_t device = 0;
    cudaStream_t stream = nullptr;
    int32_t sms = 0;
    DevBuf bits, cnt, poolA, poolB, queue, state, plan, aut, short_idx, tasks, refine, coarse, cgtab;
    std::vector<CgEdge> h_cgtab;  // host copy of the G' edge table of the last search on G'
    RunState* h_state = nullptr;  // pinned
    QueryPlan h_plan;
    sgm_stats stats;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    int32_t live_graphs = 0;
    int32_t live_queries = 0;
};

struct sgm_graph {
    sgm_engine* e = nullptr;
    DevGraph G;
    std::vector<void*> owned;  // device allocations freed with the graph
    std::vector<unsigned long long> label_hist;
    int32_t dmax = 0;
    sgm_graph_stats gstats;    // label and degree statistics (cost-model features)
};

struct sgm_query {
    sgm_engine* e = nullptr;
    int32_t k = 0;
    int32_t m = 0;
    uint32_t adj[SGM_KMAX];
    int32_t label[SGM_KMAX];
    int32_t order[SGM_KMAX];
    bool has_order = false;
    // label-preserving automorphisms of Q (identity first); empty when there
    // are more than kAutCap of them (symmetry breaking is then skipped)
    std::vector<std::vector<int8_t>> aut;
};

// The candidate graph G' of one query (sgm_cgraph_build), on the device.
struct sgm_cgraph {
    sgm_engine* e = nullptr;
    const sgm_graph* g = nullptr;
    const sgm_query* q = nullptr;
    int32_t k = 0;
    int64_t words = 0;
    DevBuf bits;                   // uint32 [k][words]: C(u)
    DevBuf rank;                   // int32 [k][words + 1]: set bits of C(u) before each word
    DevBuf ptr;                    // int64: the offset arrays of the directed edges, concatenated
    DevBuf adj;                    // int32: their lists, concatenated
    int32_t edge_of[SGM_KMAX][SGM_KMAX];  // directed edge index of (u, u2); -1: not a query edge
    std::vector<int32_t> eu, ev;          // per directed edge: (u, u2)
    std::vector<int64_t> rows, entries;   // |C(u)| and the total list length
    std::vector<int64_t> ptr_off, adj_off;  // offsets into ptr and adj (elements)
};

static const size_t kAutCap = 4096;

static inline int popc32(uint32_t x) { return __builtin_popcount(x); }

// Rule-based greedy order (sgm_query_order_greedy); root < 0 picks phi[0].
void sgm_greedy_order(sgm_query* q, const sgm_graph* g, int32_t root);

sgm_status sgm_resolve_opts(const sgm_opts* user_opts, sgm_opts& o);
sgm_status sgm_check_order(const sgm_query* q, const int32_t* phi);
sgm_status sgm_build_filter_spec(const sgm_graph* g, const sgm_query* q, int32_t use_filter, FilterSpec& F);
void sgm_build_plan(const sgm_graph* g, const sgm_query* q, const sgm_opts& o, int32_t kmode, bool full_range,
                    uint32_t* bits, QueryPlan& P, std::vector<int8_t>& aut_flat, int& aut_n);
