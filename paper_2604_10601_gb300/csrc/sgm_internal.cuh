// sgm_internal.cuh - structures shared by the host side of libsgm and its
// sm_103a kernels. Nothing here is part of the public ABI (include/sgm.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sgm.h"

#define SGM_KMAX 32
#define SGM_FULL 0xffffffffu

// Data graph G on the device (Sec. 2.1): symmetric sorted CSR plus the
// per-graph tables used by the filter and the membership tests.
struct DevGraph {
    int64_t n;
    int64_t nnz;
    int64_t words;            // ceil(n / 32): words of one vertex bitmap
    const int64_t* rowptr;    // [n + 1]
    const int32_t* col;       // [nnz], rows strictly increasing
    const int32_t* deg;       // [n]
    const uint8_t* labels;    // [n] or nullptr (unlabelled)
    const uint8_t* nlf;       // [n * num_labels] neighbour-label counts (saturating), or nullptr
    int32_t num_labels;
    const int64_t* up_rowptr; // [n + 1] upper-rank adjacency N+(v) = {x in N(v) : rank(x) > rank(v)},
    const int32_t* up_col;    //   rank = (degree, id); rows sorted by id
    const int32_t* updeg;     // [n] |N+(v)|
    int32_t hubs;             // number of hub bitmaps
    const int32_t* hub_id;    // [n], -1 = no bitmap; nullptr when hubs == 0
    const uint32_t* hub_bits; // [hubs * words]: bit y of hub h set iff y in N(hub)
};

// One level l of the matching order phi (Sec. 2.2), as the kernels see it.
struct LevelPlan {
    uint32_t bwd;            // bit i (i < l): phi[i] is a backward neighbour of phi[l]
    uint32_t inj;            // bit i (i < l): M[i] may equal a candidate of phi[l] (same label,
                             // not a backward neighbour), so injectivity must be tested
    uint32_t sb_gt;          // bit i: symmetry breaking needs rank(M[l]) > rank(M[i])
    uint32_t sb_lt;          // bit i: symmetry breaking needs rank(M[l]) < rank(M[i])
    uint32_t up;             // bit i (backward, in sb_gt): the candidates may come from N+(M[i])
    int32_t u;               // query vertex phi[l]
    const uint32_t* bits;    // candidate bitmap of phi[l] (words per graph)
};

enum { SGM_KMODE_COUNT = 0, SGM_KMODE_HASH = 1, SGM_KMODE_ENUM = 2 };

struct QueryPlan {
    int32_t k;
    int32_t D;               // levels 0..D-1 come from the initial task pool
    int32_t arith;           // 1: level k-1 is counted arithmetically from level k-2
    int32_t arith_b;         // the level of the single backward neighbour of phi[k-1]
    uint32_t arith_known;    // bit i: phi[i] ~ phi[arith_b] in Q, so M[i] in N(M[arith_b])
    int32_t split_min;       // offer half of a candidate range longer than this (0 = never)
    int32_t split_depth;     // ... at levels R .. R + split_depth - 1 of a task (R = its root level)
    int32_t pool_chunk;      // candidates per range task of the initial pool
    int32_t root_lo;         // batched runs: M[phi[0]] restricted to [root_lo, root_hi)
    int32_t root_hi;
    const int32_t* cnt_last; // [n]: #{y in N(w) : y passes the filter of phi[k-1]}
    int32_t aut_n;           // automorphisms expanded at the leaves (hash / enumerate), 1 = none
    int32_t pad2;
    const int8_t* aut;       // [aut_n][k]: sigma(u) of every automorphism (identity first)
    LevelPlan lv[SGM_KMAX];
};

// Device-side results and counters of one run (one query, or the shared
// part of a batched run). The words that many warps poll or update while the
// kernel runs (pool and queue cursors, progress, warp counts) sit on their
// own 128-byte lines, apart from each other and from the results that are
// written once per warp.
struct alignas(128) RunState {
    unsigned long long count;
    unsigned long long hash;
    unsigned long long level[SGM_KMAX];
    unsigned long long rows;          // enumerate: rows claimed
    unsigned long long cand_checked;
    unsigned long long list_elems;
    unsigned long long search_probes;
    unsigned long long bitmap_probes;
    unsigned long long filter_probes;
    unsigned long long task_groups;
    unsigned long long steals;
    unsigned long long idle_lanes;
    unsigned long long scatter_rounds;
    unsigned long long frontier_n;    // BFS: rows written to the next frontier
    unsigned long long frontier_bound;
    int32_t status;                   // first device error (sgm_status), 0 = none
    int32_t overflow;
    alignas(128) unsigned long long pool_head;  // next initial row (or chunk of roots) to fetch
    alignas(128) unsigned long long task_head;  // next candidate-range task of the initial pool
    // work queue of stealable sub-ranges
    alignas(128) unsigned long long q_head;
    alignas(128) unsigned long long q_tail;
    alignas(128) unsigned long long heartbeat;  // bumped by warps holding work (progress signal)
    alignas(128) unsigned long long work;       // candidate tasks reported against the work cap
    alignas(128) int32_t active;                // warps holding work
    alignas(128) int32_t idle;                  // warps waiting for work
};

// One stealable sub-task: extend the partial match prefix[0..L-1] at level L
// over the candidate positions [lo, hi) of its local candidate list.
struct QueueTask {
    int32_t L;
    int32_t lo;
    int32_t hi;
    int32_t ready;
    int32_t qid;             // query of the task (batched runs; 0 otherwise)
    int32_t pad;
    int32_t prefix[SGM_KMAX];
};

// Initial work of a single-query run: the BFS rows of depth D (Sec. 4.3's
// initial pool). Rows whose local list for level D is short are fetched 32
// at a time (through short_idx, or every row in order when short_idx is
// null); the longer lists are cut into candidate ranges [lo, hi) of at most
// one chunk, fetched one range at a time, so that a few rows with very long
// lists cannot hold the launch up.
struct PoolTask {
    int32_t row;
    int32_t lo;
    int32_t hi;
};

struct PoolArgs {
    const int32_t* rows;       // [n_rows][D]
    const int32_t* short_idx;  // [n_short] or nullptr (= rows 0 .. n_short - 1)
    int64_t n_short;
    const PoolTask* tasks;     // [n_tasks]
    int64_t n_tasks;
};

// Batched runs: many queries in one persistent launch. The initial work is
// the root candidates of every query, cut into chunks of consecutive words
// of the query's phi[0] candidate bitmap.
// Breadth-first initialisation of one query of a batched run (Sec. 4.3's
// initial pool, for all queries of the batch at once, inside the captured
// graph): the current frontier holds n rows of `depth` mapped levels in
// frontier buffer `cur`, within the query's own region of each buffer.
struct BatchBfs {
    int64_t off;                // first int32 of the query's region in each frontier buffer
    int64_t cap_rows;           // rows the region holds at any depth (cap_rows * k int32)
    unsigned long long tau;     // stop expanding once the frontier holds this many rows
    unsigned long long n;       // rows of the current frontier
    unsigned long long next_n;  // rows appended to the next frontier (atomic)
    int32_t depth;              // levels per row of the current frontier; 0 = query starts from root chunks
    int32_t active;             // 1 while the query still expands
    int32_t cur;                // frontier buffer holding the current rows (0 or 1)
    int32_t pad;
};

struct BatchArgs {
    const QueryPlan* plans;  // [nq]
    RunState* qst;           // [nq] per-query results (count, hash, levels, overflow)
    const int32_t* chunk_q;  // [nchunks] query of each chunk
    const int64_t* chunk_w;  // [nchunks] first bitmap word of each chunk
    int64_t nchunks;
    int64_t words;           // words per bitmap
    int32_t chunk_words;     // words per chunk (task granularity)
    int32_t nq;
    BatchBfs* bfs;           // [nq] or nullptr: queries that start from a breadth-first pool
    int32_t* fr[2];          // frontier buffers
    unsigned long long* task_base;  // [nq + 1] first 32-row pool task of each query (exclusive scan)
};

// ---------------------------------------------------------------------------
// host-side helpers
// ---------------------------------------------------------------------------
void sgm_set_error(const char* fmt, ...);

#define SGM_CUDA_TRY(expr)                                                          \
    do {                                                                            \
        cudaError_t err__ = (expr);                                                 \
        if (err__ != cudaSuccess) {                                                 \
            cudaGetLastError(); /* a later launch must not report this error */    \
            sgm_set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(err__), \
                          __FILE__, __LINE__);                                      \
            return err__ == cudaErrorMemoryAllocation ? SGM_E_OOM : SGM_E_CUDA;     \
        }                                                                           \
    } while (0)

#define SGM_TRY(expr)                    \
    do {                                 \
        sgm_status st__ = (expr);        \
        if (st__ < 0) return st__;       \
    } while (0)
