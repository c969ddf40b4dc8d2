// sgm_internal.cuh - structures shared by the host side of libsgm and its
// sm_103a kernels. Nothing here is part of the public ABI (include/sgm.h).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "sgm.h"

#define SGM_KMAX 32
#define SGM_BATCH_MAX_CLASSES 8  // size classes of a batched run (one persistent launch each)
#define SGM_FULL 0xffffffffu

// Data graph G on the device (Sec. 2.1): symmetric sorted CSR plus the
// per-graph tables used by the filter and the membership tests.
// Degree classes of the label buckets: min(degree, 8).
constexpr int kDegClasses = 9;

// One directed query edge of the candidate graph G' as the extension kernel
// reads it (App. C): the list N(x) ∩ C(u2) of a candidate x of u is
// adj[ptr[r] .. ptr[r+1]), r = the rank of x in C(u) = rank[x >> 5] + the set
// bits of bits[x >> 5] below x.
struct CgEdge {
    const int64_t* ptr;    // [|C(u)| + 1]
    const int32_t* adj;
    const int32_t* rank;   // [words + 1] set bits of C(u) before each word
    const uint32_t* bits;  // C(u)
};

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
    const int32_t* hub_list;  // [hubs]: the vertex of each hub bitmap
    const int64_t* lab_off;   // [num_labels + 1] labelled graphs: vertices of label l are
    const int32_t* lab_vert;  //   lab_vert[lab_off[l] .. lab_off[l + 1]), nullptr otherwise; ordered
                              //   by degree class min(deg, kDegClasses - 1) descending, ids ascending
                              //   within a class
    const int64_t* lab_ge;    // [num_labels][kDegClasses]: vertices of label l with class >= c, i.e.
                              //   the bucket's prefix holding every vertex of degree >= c (c < 8)
    const uint32_t* hub_bits; // [hubs * words]: bit y of hub h set iff y in N(hub)
    const CgEdge* cg;         // searches on G': [32 x 32], entry (i, j) = the edge (phi[i], phi[j])
                              // for backward neighbours i < j; nullptr otherwise
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
    int32_t* cnt_last;       // [n]: #{y in N(w) : y passes the filter of phi[k-1]} for the images w
                             // of phi[arith_b]; the degrees when every neighbour passes
    int32_t aut_n;           // automorphisms expanded at the leaves (hash / enumerate), 1 = none
    int32_t cnt_lazy;        // 1: cnt_last starts as -1 everywhere and a warp fills an entry the
                             // first time a partial match needs it
    const int8_t* aut;       // [aut_n][k]: sigma(u) of every automorphism (identity first)
    LevelPlan lv[SGM_KMAX];
};
// A batched run keeps, per warp, the plan's header and its first kcap levels.
static_assert(offsetof(QueryPlan, lv) == 64, "QueryPlan header is 64 bytes");
static_assert(sizeof(LevelPlan) == 32, "LevelPlan is 32 bytes");

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
    unsigned long long alg_bytes;     // algorithmic bytes of the extension kernel (cost model below)
    unsigned long long frontier_n;    // BFS: rows written to the next frontier
    unsigned long long frontier_bound;
    int32_t status;                   // first device error (sgm_status), 0 = none
    int32_t overflow;
    alignas(128) unsigned long long pool_head;  // next initial row (or chunk of roots) to fetch
    alignas(128) unsigned long long task_head;  // next candidate-range task of the initial pool
    alignas(128) unsigned long long chunk_head; // batched runs: next root chunk
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
    int32_t one_parent;        // 1: a scatter round takes tasks from one partial match only
    int32_t block_mail;        // 1: two-level stealing, the block level first (BlockMail)
};

// Two-level work stealing, block level (Sec. 4.3): an idle warp sets its bit
// in idle_mask; a busy warp of the same block claims the bit and writes half
// of a candidate range into the idle warp's box, then sets ready. Lives in
// shared memory after the warp stacks.
struct BlockMail {
    uint32_t idle_mask;
    int32_t ready[32];
    int32_t pad[3];
    QueueTask box[32];
};

// Batched runs: many queries in one captured CUDA graph. Every query first
// expands breadth-first (Sec. 4.3's initialisation phase, for all queries at
// once, one launch per level over every query still expanding) into one
// arena of int32 rows; the arena is handed out on the device, per query and
// level, from the sum of the rows' local-list lengths (an upper bound on the
// next frontier). A query stops expanding at its row target, one level short
// of its last vertex, or when the arena cannot hold its next level (its
// current frontier stays valid: the arena is never reused within a run). Its
// final frontier then becomes tasks: 32 consecutive rows per task, and rows
// whose local list is longer than the plan's pool_chunk are cut into range
// tasks instead. Queries are grouped into size classes by k (the per-warp
// stack is laid out for the class's largest k), one persistent extension
// kernel per class, the classes on parallel branches of the graph.
struct BatchBfs {
    int64_t off;                    // arena int32 offset of the current frontier (rows of `depth` ints)
    int64_t next_off;               // arena int32 offset of the next frontier
    unsigned long long n;           // rows of the current frontier
    unsigned long long next_n;      // rows appended to the next frontier (atomic)
    unsigned long long bound;       // sum of the current rows' local-list lengths (atomic)
    unsigned long long tau;         // stop expanding once the frontier holds this many rows
    unsigned long long nrange;      // range tasks cut from the final frontier's long rows
    unsigned long long range_fill;  // range tasks written so far (atomic)
    int64_t range_off;              // arena int32 offset of the query's BatchRange records
    int32_t depth;                  // levels per row; 0 = the query starts from root chunks
    int32_t active;                 // 1 while the query still expands
    int32_t cls;                    // size class
    int32_t split;                  // 1: the final frontier's long rows become range tasks
};

// Range task of a batched run: candidate positions [lo, hi) of the local list
// of row `row` of query q's final frontier.
struct BatchRange {
    int32_t q;
    int32_t row;
    int32_t lo;
    int32_t hi;
};

// One size class: queries [q0, q1) (ordered by class on the host), one
// persistent launch. A query's tasks are its range tasks (when split) and
// then its 32-row tasks, and the tasks of a class run query by query:
// global task ids [task0, task0 + n_tasks), query q owning
// [task_base[q], task_base[q + 1]). The warps of a launch thus work on a few
// queries at a time, whose bitmaps and neighbourhoods stay in L2. The counts
// are written on the device before the launch reads them.
struct BatchClass {
    int32_t q0;
    int32_t q1;
    int32_t kcap;                   // per-warp stack depth of the launch
    int32_t pad;
    unsigned long long task0;
    unsigned long long n_tasks;
};

// Device scalars of the breadth-first phase.
struct BatchScalars {
    unsigned long long arena_used;  // int32 elements of the arena in use
    unsigned long long rows;        // rows of the current global row space
    int32_t arena_full;             // some query stopped for lack of arena
    int32_t pad;
};

struct BatchArgs {
    const QueryPlan* plans;          // [nq]
    RunState* qst;                   // [nq] per-query results (count, hash, levels, overflow)
    BatchBfs* bfs;                   // [nq]
    BatchClass* cls;                 // [ncls]
    BatchScalars* sc;
    unsigned long long* rbase;       // [nq + 1] row space: first global row of each query (exclusive scan)
    unsigned long long* task_base;   // [nq + 1] first task of each query (exclusive scan)
    int32_t* arena;
    unsigned long long arena_cap;    // int32 elements
    const int32_t* chunk_q;          // [nchunks] root chunks of the launch's class: query of each chunk
    const int64_t* chunk_w;          //   and its first bitmap word
    int64_t nchunks;
    int64_t words;                   // words per bitmap
    int32_t chunk_words;             // words per root chunk
    int32_t nq;
    int32_t cls_id;                  // size class of the launch
    int32_t plan_bytes;              // bytes of each warp's shared-memory copy of a plan
};
static_assert(sizeof(BatchRange) == 16, "BatchRange is four int32");

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
