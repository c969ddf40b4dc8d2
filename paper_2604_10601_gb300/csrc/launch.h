// launch.h - host launchers of the libsgm kernels (internal to the library).
#pragma once

#include "sgm_internal.cuh"

// ---- data-graph tables (graph_kernels.cu) ----------------------------------
enum {
    SGM_VF_RANGE = 1,       // column outside [0, n)
    SGM_VF_UNSORTED = 2,    // row not strictly increasing
    SGM_VF_SELF_LOOP = 4,
    SGM_VF_ASYMMETRIC = 8,
    SGM_VF_LABEL = 16,      // label outside [0, num_labels)
};

cudaError_t sgm_launch_degrees(const int64_t* rowptr, int64_t n, int32_t* deg, int32_t* flags, cudaStream_t s);
cudaError_t sgm_launch_validate(const DevGraph& G, int32_t* flags, cudaStream_t s);
cudaError_t sgm_launch_labels(const int32_t* in, int64_t n, int32_t num_labels, uint8_t* out, int32_t* flags,
                              unsigned long long* hist, cudaStream_t s);
cudaError_t sgm_launch_nlf(const DevGraph& G, uint8_t* nlf, cudaStream_t s);
cudaError_t sgm_launch_up_count(const DevGraph& G, int32_t* updeg, cudaStream_t s);
cudaError_t sgm_launch_up_fill(const DevGraph& G, const int64_t* up_rowptr, int32_t* up_col, cudaStream_t s);
cudaError_t sgm_launch_hub_bits(const DevGraph& G, const int32_t* hub_list, int32_t hubs, uint32_t* bits,
                                cudaStream_t s);

// ---- matching (match_kernels.cu) --------------------------------------------
// Per-query description of the candidate filter (label, degree and
// neighbour-label frequency), one entry per query vertex.
struct FilterSpec {
    int32_t k;
    int32_t use_filter;
    int32_t label[SGM_KMAX];
    int32_t dq[SGM_KMAX];
    int32_t nneed[SGM_KMAX];
    uint8_t need_label[SGM_KMAX][SGM_KMAX];
    uint8_t need_cnt[SGM_KMAX][SGM_KMAX];
};

cudaError_t sgm_launch_filter(const DevGraph& G, const FilterSpec& F, uint32_t* bits, cudaStream_t s);
// Labelled graphs (G.lab_vert): clears bits[0 .. bits_words) and sets the
// candidates of nq queries (specs[q] in device memory, or the one host spec
// F0 when specs is null) by visiting only each query vertex's label bucket.
cudaError_t sgm_launch_filter_buckets(const DevGraph& G, const FilterSpec* specs, const FilterSpec* F0,
                                      const int64_t* bits_off, uint32_t* bits, size_t bits_words, int32_t nq,
                                      int32_t warps_per_query, cudaStream_t s);

// ---- candidate-set refinement (refine_kernels.cu) ----------------------------
struct RefineSpec {
    int32_t k;
    uint32_t qadj[SGM_KMAX];  // bit u' of qadj[u]: {u, u'} is a query edge
};
// One round: nxt (a copy of cur on entry) loses every candidate bit without
// support in cur; *changed is set to 1 if any bit was cleared.
cudaError_t sgm_launch_refine(const DevGraph& G, const RefineSpec& R, const uint32_t* cur, uint32_t* nxt,
                              int32_t* changed, cudaStream_t s);

// Arithmetic last level: cnt_last[w] for every hub vertex w that is a
// candidate of phi[arith_b], for the nq plans (plans[idx[j]], or plans[j]
// when idx is null) whose table is filled on demand.
cudaError_t sgm_launch_cnt_hubs(const DevGraph& G, const QueryPlan* plans, const int32_t* idx, int32_t nq,
                                int32_t sms, cudaStream_t s);
cudaError_t sgm_launch_roots(const uint32_t* bits0, int64_t lo, int64_t hi, int32_t* out, RunState* st,
                             cudaStream_t s);
cudaError_t sgm_launch_bfs_bound(const DevGraph& G, const QueryPlan* P, const int32_t* rows, int64_t n_rows,
                                 int32_t d, RunState* st, cudaStream_t s);
cudaError_t sgm_launch_bfs_expand(const DevGraph& G, const QueryPlan* P, const int32_t* in, int64_t n_in,
                                  int32_t d, int32_t* out, int64_t cap_rows, RunState* st, cudaStream_t s);
cudaError_t sgm_launch_pool_leaf(int32_t mode, const QueryPlan* P, const int32_t* rows, int64_t n_rows,
                                 int32_t k, RunState* st, int32_t* out, uint64_t cap, cudaStream_t s);

struct ExtendLaunch {
    int32_t mode;            // SGM_KMODE_*
    int32_t gather = 0;      // 1: gather filter-passing candidates before the membership tests
                             //    (labelled graphs, whose label filter is selective)
    int32_t kcap;            // stack depth the shared memory is laid out for
    int32_t warps_per_block;
    int32_t blocks;
    size_t smem_bytes;
};
size_t sgm_extend_smem_bytes(int32_t kcap, int32_t warps_per_block, bool batch);
// bytes of a batched launch's per-warp copy of a plan (header + kcap levels)
int32_t sgm_batch_plan_bytes(int32_t kcap);
int sgm_extend_max_blocks_per_sm(int32_t mode, bool batch, bool gather, int32_t warps_per_block, size_t smem_bytes);
// batch == nullptr: one query (plan P, initial pool); else many queries (B).
cudaError_t sgm_launch_extend(const ExtendLaunch& L, const DevGraph& G, const QueryPlan* P, const PoolArgs& pa,
                              RunState* st, QueueTask* queue, int32_t qcap, int32_t* out, uint64_t cap,
                              uint64_t time_cap_ns, uint64_t work_cap, const BatchArgs* batch, cudaStream_t s);
// batched runs (batch_kernels.cu)
// candidate bitmaps of nq queries in one launch; query q's bitmaps start at word bits_off[q]
cudaError_t sgm_launch_batch_filter(const DevGraph& G, const FilterSpec* specs, const int64_t* bits_off,
                                    uint32_t* bits, int32_t nq, int32_t sms, cudaStream_t s, size_t bits_words);
// breadth-first phase of every query (levels 1 .. max_depth - 1), then the final row space
cudaError_t sgm_launch_batch_bfs(const DevGraph& G, const BatchArgs& B, int32_t max_depth, int32_t root_blocks,
                                 int32_t sms, cudaStream_t s, uint64_t* launches);
// 32-row and range tasks from the final frontiers, per size class
cudaError_t sgm_launch_batch_tasks(const DevGraph& G, const BatchArgs& B, int32_t ncls, int32_t sms, cudaStream_t s,
                                   uint64_t* launches);
cudaError_t sgm_launch_chunk_pool(const DevGraph& G, const QueryPlan* P, const int32_t* rows, int64_t n_rows,
                                  int32_t d, int32_t chunk, int32_t* short_idx, PoolTask* tasks, int64_t task_cap,
                                  RunState* st, cudaStream_t s);

// ---- coarse-grained baseline (coarse_kernels.cu) ------------------------------
// Warps (a multiple of 8) the coarse model can run with stacks of
// k x sigma x dmax int32 each within budget_bytes.
int32_t sgm_coarse_warps(int32_t sms, int32_t k, int32_t sigma, int64_t dmax, int64_t budget_bytes);
cudaError_t sgm_launch_coarse(const DevGraph& G, const QueryPlan* P, const PoolArgs& pa, RunState* st,
                              int32_t* stack, int64_t dmax, int32_t sigma, int32_t warps, uint64_t cap_ns,
                              cudaStream_t s);
