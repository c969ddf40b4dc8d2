/*
 * sgm.h - C ABI of libsgm, an exact subgraph-matching engine for one GB300
 * (sm_103a).
 *
 * The problem (Definition 1, Sec. 2.1 of "gMatch: Fine-Grained and
 * Hardware-Efficient Subgraph Matching on GPUs"): given an undirected
 * labelled data graph G and a connected query graph Q, find every injective
 * map M : V(Q) -> V(G) with L(M[u]) = L(u) for every query vertex and
 * {M[u], M[u']} in E(G) for every query edge (non-induced embeddings). The
 * engine extends partial matches along a matching order phi (Sec. 2.2): each
 * step checks candidates v from the neighbour list of one mapped backward
 * neighbour against the candidate filter, injectivity and the neighbour lists
 * of the other mapped backward neighbours (Alg. 2, Process).
 *
 * Conventions for every call:
 *   - Return value: sgm_status; 0 = success, > 0 = success with a warning,
 *     < 0 = error. A thread-local message is available from sgm_last_error().
 *     No C++ exception crosses this boundary.
 *   - All device work runs on the engine's stream (sgm_create / sgm_set_stream)
 *     and every call returns only after that work has finished.
 *   - Pointers marked "device" are CUDA device pointers of the engine's device;
 *     "host" pointers are ordinary host memory. Sizes are element counts.
 *   - Vertex ids are int32 in [0, n). Query vertex ids are 0..k-1, k <= 32.
 *   - Counts are uint64. An embedding count that would pass 2^64 - 1 returns
 *     SGM_E_COUNT_OVERFLOW, never a wrapped value.
 *   - Embedding hash (project-defined; the paper has none): for one embedding,
 *         h(M) = mix(x_k), x_0 = 0x243F6A8885A308D3,
 *         x_{u+1} = mix(x_u XOR ((u << 32) | (uint32)M[u])), u = 0..k-1,
 *     with mix the SplitMix64 output function (Steele, Lea, Flood, OOPSLA
 *     2014); the hash of a set of embeddings is the sum of h(M) mod 2^64. It
 *     does not depend on the matching order or on the order of emission.
 */
#ifndef SGM_H
#define SGM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t sgm_status;

#define SGM_OK 0
#define SGM_W_TRUNCATED 1            /* enumerate: more embeddings than the output capacity */
#define SGM_E_INVALID_ARG (-1)       /* null pointer, bad size, bad flag combination */
#define SGM_E_GRAPH_UNSORTED (-2)    /* a CSR row is not strictly increasing (or has duplicates) */
#define SGM_E_GRAPH_SELF_LOOP (-3)   /* v appears in its own neighbour list */
#define SGM_E_GRAPH_ASYMMETRIC (-4)  /* u in N(v) but v not in N(u) */
#define SGM_E_QUERY_DISCONNECTED (-5)
#define SGM_E_QUERY_TOO_LARGE (-6)   /* k > 32 */
#define SGM_E_ORDER_NOT_CONNECTED (-7)
#define SGM_E_LABEL_RANGE (-8)       /* a label outside [0, num_labels) */
#define SGM_E_OOM (-9)               /* device allocation failed */
#define SGM_E_COUNT_OVERFLOW (-10)
#define SGM_E_DEVICE_TIMEOUT (-11)   /* a bounded device wait ran out */
#define SGM_E_QUEUE_OVERFLOW (-12)   /* reserved: a full work queue only stops warps offering ranges */
#define SGM_E_TIME_CAP (-13)         /* opts.time_cap_s elapsed: query unsolved (Sec. 6.1, Metrics) */
#define SGM_E_CUDA (-14)             /* a CUDA runtime call failed */
#define SGM_E_GRAPH_RANGE (-15)      /* a column index outside [0, n) or rowptr not monotone */
#define SGM_E_QUERY_INVALID (-16)    /* self-loop, duplicate edge or vertex id out of range in Q */
#define SGM_E_WORK_CAP (-17)         /* opts.work_cap candidate tasks checked: query unsolved */

/* sgm_graph_load_csr flags */
#define SGM_HOST_PTRS 0u      /* rowptr/col/labels are host pointers (copied to the device) */
#define SGM_DEVICE_PTRS 1u    /* rowptr/col/labels are device pointers */
#define SGM_BORROW 2u         /* with SGM_DEVICE_PTRS: use the caller's rowptr/col in place; the
                                 caller keeps them alive and unchanged until sgm_graph_free */
#define SGM_VALIDATE 4u       /* check the CSR on the device (range, sortedness, loops, symmetry) */

/* sgm_opts.mode for sgm_count */
#define SGM_MODE_COUNT 0      /* count only; the last level may be counted arithmetically */
#define SGM_MODE_HASH 1       /* count + embedding hash; every embedding is visited */

typedef struct sgm_engine sgm_engine;
typedef struct sgm_graph sgm_graph;
typedef struct sgm_query sgm_query;

/* Run options. Fill with sgm_opts_default() and change what you need. */
typedef struct sgm_opts {
    uint32_t struct_size;      /* sizeof(sgm_opts) */
    int32_t mode;              /* SGM_MODE_COUNT or SGM_MODE_HASH (sgm_count only) */
    int64_t tau;               /* initial task pool threshold of the BFS initialization phase
                                  (Sec. 4.3; default 10^6) */
    int64_t pool_cap_bytes;    /* device bytes the initial pool may use (default 1 GiB) */
    int32_t use_filter;        /* 1: label + degree + neighbour-label-frequency candidate
                                  filter; 0: label filter only (default 1) */
    int32_t arith_last;        /* 1: in SGM_MODE_COUNT, count the last level arithmetically when
                                  its query vertex has one backward neighbour (default 1) */
    int32_t warps_per_block;   /* extension kernel block size in warps (default 8) */
    int32_t blocks_per_sm;     /* 0 = as many as fit (default 0) */
    int32_t split_min;         /* candidate-range length above which a warp offers half of
                                  a range to idle warps through the work queue (default 256;
                                  0 = no queue) */
    int32_t sym_break;         /* 1: symmetry breaking (default 1). The engine finds the label-
                                  preserving automorphisms Aut(Q), constrains M[u] < M[v] for the
                                  pairs a stabiliser chain of Aut(Q) gives (order on data vertices:
                                  degree, then id), visits one embedding per Aut(Q)-orbit and
                                  multiplies by |Aut(Q)| (hash and enumerate expand each visited
                                  embedding over Aut(Q)). In SGM_MODE_COUNT with an arithmetic
                                  last level, only the automorphisms fixing the last query
                                  vertex of phi are used, so that level keeps its arithmetic
                                  count. Results are identical either way. 1 applies it to
                                  full root ranges only; 2 also to root slices, where a slice
                                  then holds the embeddings whose visited orbit representative
                                  has its root in the slice (slices of a partition of [0, n)
                                  still sum to the full count and hash: the sharding mode). */
    double time_cap_s;         /* per-query search time cap in seconds; 0 = none */
    int32_t chunk_words;       /* batched runs: words of 32 root candidates per initial task
                                  (task granularity; default 4) */
    int32_t split_depth;       /* ranges may be offered at the first split_depth levels of a task
                                  (1 = its root level only; default 1). A range is offered when longer than
                                  2 x split_min, or, with split_depth > 1, than
                                  max(2, 2 x split_min / 2^(levels left below it)). */
    int32_t pool_chunk;        /* initial pool: local lists longer than this many candidates are
                                  cut into range tasks of this size (0 = never; default 512) */
    int32_t refine_rounds;     /* candidate-set refinement after the filter (sgm_refine): at most
                                  this many rounds, stopping early at the fixed point (0 = off,
                                  the default; not supported by sgm_batch_create). Counts,
                                  hashes and listings are unchanged: no embedding loses a
                                  candidate. */
    uint64_t work_cap;         /* stop with SGM_E_WORK_CAP once more than this many candidate
                                  tasks T_M(u, v) have been reported by the extension kernel's
                                  warps (each reports every 256 rounds or 8192 candidates; 0 =
                                  none). A run that needs at most work_cap checks always
                                  completes, whatever the scheduling; one needing more than
                                  work_cap + 16384 x (resident warps) always stops. Batched runs apply the cap to each query
                                  on its own: a query past it stops (status SGM_E_WORK_CAP,
                                  unsolved, Sec. 6.1 Metrics) and the others go on. */
    int32_t exec_model;        /* sgm_count's execution model (the ablation of Sec. 6.3, Table 4):
                                  SGM_EXEC_FINE_BATCH (default): one candidate per thread, a warp's
                                  32 tasks drawn from many partial matches (warp-level batch
                                  exploration, Sec. 4.2); SGM_EXEC_FINE_NAIVE: one candidate per
                                  thread, a round's tasks from one partial match only;
                                  SGM_EXEC_COARSE: Alg. 1's coarse-grained model, a warp per
                                  partial match with its feasible candidates materialised in a
                                  per-warp stack of k x unroll x d_max int32 in device memory.
                                  The coarse model counts only (SGM_MODE_COUNT) and runs without
                                  symmetry breaking and without the arithmetic last level; the
                                  counts are the same in every model. Batched runs use the default. */
    int32_t unroll;            /* SGM_EXEC_COARSE: partial matches a warp processes per step (loop
                                  unrolling, Sec. 2.3; 1 = the naive model, at most 8; default 1) */
    int32_t steal_mode;        /* dynamic balancing (Sec. 4.3) of the fine-grained models with
                                  split_min > 0: 0 (default) = one device-wide queue of candidate
                                  ranges that idle warps poll; 1 = two-level: an idle warp first
                                  offers itself to the busy warps of its own block, which hand it
                                  half of a range through a shared-memory box (about 5 KB per
                                  block), and the device-wide queue serves as the second level.
                                  Results are identical; batched runs use 0. */
} sgm_opts;

#define SGM_EXEC_FINE_BATCH 0
#define SGM_EXEC_FINE_NAIVE 1
#define SGM_EXEC_COARSE 2

/* Per-call statistics of the last count/enumerate on this engine. */
typedef struct sgm_stats {
    double ms_filter;          /* candidate filter + per-query tables */
    double ms_init;            /* BFS initialization phase */
    double ms_search;          /* persistent extension kernel */
    int32_t init_depth;        /* number of query vertices mapped by the initialization phase */
    int32_t grid_blocks;
    int64_t pool_size;         /* partial matches in the initial pool */
    uint64_t cand_checked;     /* candidate tasks T_M(u, v) processed (Sec. 4.1) */
    uint64_t list_elems;       /* adjacency-list elements read to produce those candidates */
    uint64_t search_probes;    /* binary-search probes into neighbour lists */
    uint64_t bitmap_probes;    /* hub adjacency-bitmap probes */
    uint64_t filter_probes;    /* candidate-bitmap probes */
    uint64_t task_groups;      /* task groups T^G_M(u) generated */
    uint64_t steals;           /* sub-ranges handed to other warps through the work queue */
    uint64_t idle_lanes;       /* task slots left empty in scatter rounds (idle rate, Sec. 2.3) */
    uint64_t scatter_rounds;   /* warp scatter rounds */
    uint64_t launches;         /* kernels launched by the call */
    uint64_t aut_size;         /* |Aut(Q)| used for symmetry breaking (1 = none) */
    uint64_t alg_bytes;        /* algorithmic bytes the extension kernel moved: per task group
                                  8 B per backward neighbour (row offsets); 4 B per local-list
                                  element; per membership test 32 B into a hub bitmap, else
                                  min(4 |N|, 32 max(1, ceil(log2(|N| / 8)))) B into a sorted
                                  row of |N| entries (streamed or searched, whichever is
                                  cheaper; the last 8 entries share one 32-byte sector) */
    uint64_t stack_bytes;      /* execution stacks of the search: shared memory of the fine-grained
                                  launch, or the device buffers of the coarse model */
} sgm_stats;

void sgm_opts_default(sgm_opts* opts);

/* Thread-local text of the last error on this thread ("" if none). */
const char* sgm_last_error(void);

/* Creates an engine on CUDA device `device` using `cuda_stream` (a cudaStream_t,
 * NULL for the default stream). *out receives the handle. */
sgm_status sgm_create(sgm_engine** out, int32_t device, void* cuda_stream);
sgm_status sgm_set_stream(sgm_engine* e, void* cuda_stream);
/* Frees the engine and its device scratch. Graphs and queries must be freed first. */
sgm_status sgm_destroy(sgm_engine* e);

/*
 * Loads the data graph G (Sec. 2.1) as symmetric CSR: rowptr int64[n+1],
 * col int32[rowptr[n]] with each row strictly increasing, both directions of
 * every undirected edge present and no self-loops. labels: int32[n] with
 * values in [0, num_labels), or NULL for an unlabelled graph (num_labels = 1).
 * num_labels <= 256. Builds the per-graph tables (degrees, neighbour-label
 * frequencies, hub adjacency bitmaps). *out belongs to the caller until
 * sgm_graph_free. With SGM_VALIDATE a malformed CSR returns its error code.
 */
sgm_status sgm_graph_load_csr(sgm_engine* e, int64_t n, const int64_t* rowptr, const int32_t* col,
                              const int32_t* labels, int32_t num_labels, uint32_t flags,
                              sgm_graph** out);
sgm_status sgm_graph_free(sgm_graph* g);
/* n, directed entries (rowptr[n]), maximum degree, number of hub bitmaps. Any out may be NULL. */
sgm_status sgm_graph_info(const sgm_graph* g, int64_t* n, int64_t* nnz, int32_t* dmax, int32_t* hubs);

/*
 * Registers the query graph Q: k vertices (1 <= k <= 32), m undirected
 * edges given as host int32 pairs edges[2*i], edges[2*i+1], and host labels
 * int32[k] (NULL = all 0). Q must be simple and connected. The query starts
 * with the rule-based order (sgm_query_order_greedy) computed against the
 * first graph it is run on unless an order is set.
 */
sgm_status sgm_query_register(sgm_engine* e, int32_t k, int32_t m, const int32_t* edges,
                              const int32_t* labels, sgm_query** out);
sgm_status sgm_query_free(sgm_query* q);
/* Sets the matching order phi (Sec. 2.2): a host permutation of 0..k-1 in
 * which every vertex but phi[0] has an earlier neighbour. */
sgm_status sgm_query_set_order(sgm_query* q, const int32_t* phi, int32_t k);
/*
 * Rule-based greedy order in the spirit of RI (Sec. 3, which generates phi
 * with RI on the CPU): phi[0] = the vertex of maximum degree (ties: the
 * rarer label in G, then the smaller id); then repeatedly the unordered
 * vertex with the most ordered neighbours, ties by the most neighbours
 * adjacent to the ordered set, then by the most remaining neighbours, then
 * the smaller id.
 */
sgm_status sgm_query_order_greedy(sgm_query* q, const sgm_graph* g);
/* Greedy order as above but forced to start at query vertex `root`. */
sgm_status sgm_query_order_greedy_from(sgm_query* q, const sgm_graph* g, int32_t root);
/* Copies the current order into phi_out[k] (host). */
sgm_status sgm_query_get_order(const sgm_query* q, int32_t* phi_out);

/*
 * Candidate bitmaps of the filter kernel: bit v of word v/32 of bitmap u is
 * set iff L(v) = L(u), d(v) >= d_Q(u) and, for every label l, v has at least
 * as many neighbours labelled l as u has (with use_filter = 0 only the label
 * test). dev_bits: device uint32[k * ceil(n/32)], owned by the caller.
 */
sgm_status sgm_filter(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                      uint32_t* dev_bits);

/*
 * Candidate sets of the candidate graph G' (Sec. 6.1, Methods Under Study:
 * the large-query workloads search on a G' built from labels and query
 * structure). The filter's bitmaps as in sgm_filter, then rounds of the
 * support rule: v stays a candidate of u only if, for every query neighbour
 * u' of u, some neighbour of v was a candidate of u' after the previous
 * round. Stops after max_rounds rounds or at the first round that clears
 * nothing (the fixed point). Every embedding keeps its candidates.
 * dev_bits: device uint32[k * ceil(n/32)], owned by the caller, layout as in
 * sgm_filter. rounds: host int32 or NULL, receives the number of rounds that
 * cleared at least one candidate. Synchronous on return; errors:
 * SGM_E_INVALID_ARG (NULL handle, max_rounds < 0, objects of another
 * engine), SGM_E_LABEL_RANGE, SGM_E_CUDA.
 */
sgm_status sgm_refine(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                      int32_t max_rounds, uint32_t* dev_bits, int32_t* rounds);

/*
 * The candidate graph G' of a query on the device (Sec. 6.1, Methods Under
 * Study; App. C): the candidate sets C(u) (the filter, then refine_rounds
 * rounds of sgm_refine's support rule; 0 = the filter alone) and, for every
 * query edge in both directions (u, u2), the candidate edges: for each v of
 * C(u), ascending, the sorted list N(v) ∩ C(u2). Row i of edge (u, u2)
 * belongs to the i-th smallest vertex of C(u). The object holds its own
 * device memory (the bitmaps, a per-word rank of each bitmap, and one
 * int64 offset array and one int32 entry array per directed edge) and keeps
 * g and q referenced: destroy it before either. Synchronous on return.
 * Errors: SGM_E_INVALID_ARG (NULL handle, refine_rounds < 0, objects of
 * another engine), SGM_E_LABEL_RANGE, SGM_E_OOM, SGM_E_CUDA.
 */
typedef struct sgm_cgraph sgm_cgraph;
sgm_status sgm_cgraph_build(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                            int32_t refine_rounds, sgm_cgraph** out);
sgm_status sgm_cgraph_destroy(sgm_cgraph* c);

/*
 * Sizes of directed query edge (u, u2) of G': rows = |C(u)|, entries = the
 * total length of its lists. SGM_E_INVALID_ARG when u and u2 are not
 * adjacent in the query (or out of range).
 */
sgm_status sgm_cgraph_edge_size(const sgm_cgraph* c, int32_t u, int32_t u2, int64_t* rows, int64_t* entries);

/*
 * Copies directed edge (u, u2) of G' out: vs int32[rows] (the vertices of
 * C(u), ascending), ptr int64[rows + 1] (ptr[0] = 0; list i is
 * adj[ptr[i] .. ptr[i+1])), adj int32[entries]. Each pointer may be host or
 * device memory (or NULL to skip that array), sized from
 * sgm_cgraph_edge_size and owned by the caller. Synchronous.
 */
sgm_status sgm_cgraph_edge_copy(const sgm_cgraph* c, int32_t u, int32_t u2, int32_t* vs, int64_t* ptr,
                                int32_t* adj);

/*
 * As sgm_count, searching on G': the candidate sets are c's, and the local
 * candidate list of a level (Sec. 4.1) is the shortest of the candidate-edge
 * lists N(M[i]) ∩ C(phi[l]) over its mapped backward neighbours i, instead of
 * the shortest plain neighbour list. c must have been built for q and the
 * graph g. opts->refine_rounds is ignored (c's sets are used as they are) and
 * the initial pool is not cut into range tasks. root_lo, root_hi restrict
 * M[phi[0]] as in sgm_count_root_range (0, n: every root). Counts, hashes
 * and level counts are those of sgm_count with the same candidate sets.
 */
sgm_status sgm_count_cgraph(sgm_engine* e, const sgm_graph* g, sgm_query* q, const sgm_cgraph* c,
                            const sgm_opts* opts, int64_t root_lo, int64_t root_hi, uint64_t* count,
                            uint64_t* hash, uint64_t* level_counts);

/*
 * Counts the embeddings of Q in G (Definition 1) along the query's order.
 *   opts: NULL = defaults.  count: host uint64 out.
 *   hash: host uint64 out or NULL; a non-NULL hash visits every embedding
 *         (as SGM_MODE_HASH) and returns the embedding hash described above.
 *   level_counts: host uint64[k] or NULL; level_counts[i] = partial matches
 *         over phi[0..i] whose vertices all pass the candidate filter (and
 *         keep their candidacy through the refinement when
 *         opts->refine_rounds > 0).
 */
sgm_status sgm_count(sgm_engine* e, const sgm_graph* g, const sgm_query* q, const sgm_opts* opts,
                     uint64_t* count, uint64_t* hash, uint64_t* level_counts);

/*
 * As sgm_count, restricted to embeddings with root_lo <= M[phi[0]] < root_hi
 * (a root slice). Slices over a partition of [0, n) sum to the full count
 * and hash.
 */
sgm_status sgm_count_root_range(sgm_engine* e, const sgm_graph* g, const sgm_query* q,
                                const sgm_opts* opts, int64_t root_lo, int64_t root_hi,
                                uint64_t* count, uint64_t* hash, uint64_t* level_counts);

/*
 * Lists the embeddings of Q in G. dev_out: device int32[cap * k]; row r holds
 * one embedding indexed by query-vertex id (dev_out[r*k + u] = M[u]). Rows
 * come in no particular order. *written = min(total, cap) rows are filled,
 * *total and *hash cover every embedding; returns SGM_W_TRUNCATED when
 * total > cap.
 */
sgm_status sgm_enumerate(sgm_engine* e, const sgm_graph* g, const sgm_query* q, const sgm_opts* opts,
                         int32_t* dev_out, uint64_t cap, uint64_t* written, uint64_t* total,
                         uint64_t* hash);

/* Statistics of the last count or enumerate call on this engine. */
sgm_status sgm_get_stats(const sgm_engine* e, sgm_stats* out);

/*
 * Host-only views of the query preprocessing (no engine, no device; for
 * inspection and tests). Query given as in sgm_query_register.
 *
 * sgm_query_automorphisms: the label-preserving automorphisms of Q, each a
 * row aut_out[a * k + u] = sigma(u), identity first; *n_out = their number
 * (0 when there are more than 4096: symmetry breaking is then skipped);
 * at most `cap` rows are written.
 *
 * sgm_query_symmetry_plan: the symmetry-breaking constraints the engine uses
 * along the order phi (Appendix A mentions symmetry breaking; the stabiliser
 * chain is this library's construction): sb_gt_out[l] bit i means the
 * embedding visited must have rank(M[phi[l]]) > rank(M[phi[i]]), rank =
 * (degree, id) of the data vertex; up_out[l] (may be NULL) marks the backward
 * neighbours whose upper-rank list N+ serves level l; group_out (group_cap
 * rows of k, may be NULL) receives the subgroup H of Aut(Q) whose orbits the
 * constraints pick one embedding from, *group_n = |H|. count_mode = 1 gives
 * the plan of a count (where H fixes the last vertex when the last level is
 * counted arithmetically; *arith_out = 1 then), 0 that of hash / enumerate.
 */
sgm_status sgm_query_automorphisms(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                   int32_t* aut_out, int32_t cap, int32_t* n_out);
/* The rule-based greedy order of sgm_query_order_greedy (or _from when root >= 0)
 * given the data graph's label counts (label_count[num_labels], host; the
 * rule's only input from G), into phi_out[k]. Q must be connected. */
sgm_status sgm_query_greedy_order_host(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                       const unsigned long long* label_count, int32_t num_labels, int32_t root,
                                       int32_t* phi_out);
sgm_status sgm_query_symmetry_plan(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                   const int32_t* phi, int32_t count_mode, uint32_t* sb_gt_out, uint32_t* up_out,
                                   int32_t* group_out, int32_t group_cap, int32_t* group_n, int32_t* arith_out);

/* ------------------------------------------------------------------------
 * Counting without allocation. The paper has no counterpart to this entry
 * point; it exists for callers that cannot allocate device memory while a
 * query runs: services whose device memory belongs to another framework's
 * caching allocator (a direct cudaMalloc can fail although that pool still
 * has room), latency-bound servers that must not stall other streams
 * (cudaFree synchronises the whole device), and deployments that reserve all
 * memory at start-up so that a query never fails for lack of memory.
 *
 * sgm_count_noalloc counts the embeddings of Q in G like sgm_count, but
 * calls no cudaMalloc, cudaFree or other allocating routine. All of its
 * scratch lives in one static device array of SGM_NOALLOC_SCRATCH_BYTES
 * inside libsgm. The CUDA runtime places that array on a device when it
 * loads the module holding it: when the library loads under eager module
 * loading, or, under lazy loading (CUDA's default), during the first call on
 * that device, which looks up the array's device address. That first call
 * therefore allocates the array: make it at start-up on every device you
 * will use (n = 0 with k = 1 is enough). From then on the device holds the
 * array until the process exits. The call blocks until the count is on the
 * host (it synchronises its stream), so it cannot be captured into a CUDA
 * graph. A call needs about 9 n + k ceil(n/32) 4 + 160 KB bytes of it;
 * larger sizes return SGM_E_INVALID_ARG with a message. Every call shares
 * the array and it keeps the last call's contents (the call clears what must
 * start at zero), so calls that overlap on the GPU - from two threads, or on
 * two streams of one device - race: serialise them. The call returns when
 * the count is done, and leaves the caller's current device as it found it.
 *
 *   device, cuda_stream: the CUDA device and stream (cudaStream_t, NULL =
 *           default stream) to run on.
 *   n, rowptr, col, labels, num_labels: the data graph as in
 *           sgm_graph_load_csr, all three arrays DEVICE pointers owned by the
 *           caller (labels may be NULL: unlabelled, num_labels = 1). The
 *           CSR is NOT validated: only rowptr's monotonicity and the label
 *           range are checked, so a column index outside [0, n) makes the
 *           kernels read outside the caller's arrays. Validate untrusted
 *           graphs first (sgm_graph_load_csr with SGM_VALIDATE).
 *   k, m, edges, qlabels: the query as in sgm_query_register (HOST).
 *   phi: HOST order int32[k], or NULL for the rule-based greedy order
 *           (without the graph's label frequencies).
 *   count: HOST uint64 out.
 * Candidate filter: label and degree; no symmetry breaking, no arithmetic
 * last level; the same stealable sub-ranges as sgm_count's defaults; the
 * count equals sgm_count's.
 * ---------------------------------------------------------------------- */
#define SGM_NOALLOC_SCRATCH_BYTES (32u << 20)

sgm_status sgm_count_noalloc(int32_t device, void* cuda_stream, int64_t n, const int64_t* rowptr,
                             const int32_t* col, const int32_t* labels, int32_t num_labels, int32_t k, int32_t m,
                             const int32_t* edges, const int32_t* qlabels, const int32_t* phi, uint64_t* count);

/* ------------------------------------------------------------------------
 * Batched execution: many queries in one captured CUDA graph (not in the
 * paper, which runs one query at a time). A batch fixes, at creation, every
 * query's order, plan and candidate-bitmap storage, and captures the whole
 * run as one CUDA graph on a private stream:
 *   1. clear the run states; the candidate filter of every query (one launch);
 *   2. the initialisation phase of Sec. 4.3 for every query whose root range
 *      holds at most 2^20 vertices (anchored queries and other narrow
 *      ranges), all queries together: one launch per breadth-first level
 *      over every query still expanding, into one device arena of
 *      4 x opts.pool_cap_bytes (at most max(256 MiB, 16 MiB per query))
 *      handed out on the device by the filter-passing candidates of each
 *      level. A query expands
 *      until its frontier holds max(256, opts.tau / (queries expanding))
 *      rows, until one level short of its last vertex, or until the arena
 *      cannot hold its next level;
 *   3. tasks from the final frontiers: 32 consecutive rows, and, for a row
 *      whose local list is longer than opts.pool_chunk, ranges of that many
 *      candidates;
 *   4. one persistent extension kernel per size class of k (k <= 8, <= 16,
 *      <= 24, <= 32; the per-warp stack is laid out for the class's largest
 *      k), the classes on parallel branches of the graph, each with its own
 *      queue of stealable ranges. Queries with wider root ranges start from
 *      chunks of opts.chunk_words bitmap words of root candidates.
 * Each run replays the graph. Counts and hashes equal those of separate
 * sgm_count calls. opts.work_cap applies to each query separately. The
 * graph, the queries and the engine must outlive the batch; queries without
 * an order get the greedy one. At most 65535 queries. Device memory: the
 * bitmaps (sum over queries of k * ceil(n/32) * 4 bytes), the arena, and
 * about 1.5 KB per query.
 * ---------------------------------------------------------------------- */
typedef struct sgm_batch sgm_batch;

/* root_ranges: host int64[2 * nq], query i restricted to root_lo <= M[phi[0]] < root_hi
 * (ranges[2i], ranges[2i+1]; an anchored query when the range is one vertex), or NULL
 * for full ranges. Symmetry breaking (sym_break = 1) applies to full ranges only. */
sgm_status sgm_batch_create(sgm_engine* e, const sgm_graph* g, sgm_query* const* qs, int32_t nq,
                            const int64_t* root_ranges, const sgm_opts* opts, int32_t want_hash, sgm_batch** out);
sgm_status sgm_batch_free(sgm_batch* b);
/* Runs the batch. counts: host uint64[nq]; hashes: host uint64[nq] (only with
 * want_hash at creation) or NULL; statuses: host sgm_status[nq] or NULL; ms:
 * host double or NULL, the device time of the captured graph. A query that
 * passed opts.work_cap reports SGM_E_WORK_CAP and count 0; on a device
 * timeout or the time cap every query reports that status (and count 0).
 * Returns the first failing query's status, or SGM_OK. */
sgm_status sgm_batch_run(sgm_batch* b, uint64_t* counts, uint64_t* hashes, sgm_status* statuses, double* ms);
/* Candidate checks of each query (host uint64[nq], the caller's order) in
 * the last sgm_batch_run, counted only when the batch was created with
 * opts.work_cap > 0. For a query that finished, the figure is exact and the
 * same whatever the scheduling (each candidate of each task group counted
 * once), so "finished with at most W checks" is a deterministic rule: a
 * query needing at most work_cap checks always finishes. */
sgm_status sgm_batch_query_work(const sgm_batch* b, uint64_t* work);
/* Create, run once, free. */
sgm_status sgm_count_batch(sgm_engine* e, const sgm_graph* g, sgm_query* const* qs, int32_t nq,
                           const int64_t* root_ranges, const sgm_opts* opts, uint64_t* counts, uint64_t* hashes,
                           sgm_status* statuses);

/* ------------------------------------------------------------------------
 * Learned matching order. The paper builds phi with a rule-based method on
 * the CPU (Sec. 3); this cost model is an addition of this library. Every
 * connected order yields the same embeddings, so a learned order changes
 * only the search time, never a result.
 *
 * A small MLP (in_dim -> hidden -> hidden -> 1, ReLU, FP32) predicts
 * log10(1 + number of partial matches) of each prefix phi[0..i] from the
 * SGM_FEATURES features below. Training (mean squared error, full-batch
 * Adam) and inference run in the library's own CUDA kernels.
 * ---------------------------------------------------------------------- */
typedef struct sgm_model sgm_model;

#define SGM_MODEL_MAX_IN 128
#define SGM_FEATURES 32

/* Label and degree statistics of a data graph (filled at load time). */
typedef struct sgm_graph_stats {
    int64_t n;                  /* vertices */
    int64_t nnz;                /* directed CSR entries */
    int32_t num_labels;
    int32_t reserved;
    double label_frac[256];     /* fraction of vertices with each label */
    double log2_deg_moment[4];  /* log2 E[d^j], j = 1..4, over all vertices (0 if E = 0) */
    double deg_hist[8];         /* fraction of vertices with floor(log2(d + 1)) = b (b = 7: >= 7) */
} sgm_graph_stats;

sgm_status sgm_graph_get_stats(const sgm_graph* g, sgm_graph_stats* out);

/*
 * Features of every prefix of an order (host computation, no device work):
 * out[i * SGM_FEATURES + f] for prefix phi[0..i], i = 0..k-1. Query given as
 * in sgm_query_register (edges int32[2m], labels int32[k] or NULL); phi a
 * connected order. Returns SGM_E_INVALID_ARG / SGM_E_ORDER_NOT_CONNECTED on
 * bad input. The features are: log2(1 + degree of the anchor) for an
 * anchored query (phi[0] mapped to one given data vertex; anchor_deg < 0:
 * not anchored, feature 0); prefix size, edges and cycle
 * rank; the new vertex's query degree, backward-neighbour count and label
 * selectivity -log2 p(L); the prefix's summed label selectivity; how many
 * prefix vertices have prefix degree 1, 2, 3, >= 4; the prefix's summed
 * degree-moment term log2 E[d^min(deg,4)]; log2 n, log2 nnz, the four
 * log2 degree moments, label entropy, label count, largest label fraction,
 * k and m of Q; the 8-bin degree histogram. Each is scaled to about [0, 1].
 */
sgm_status sgm_features_from_stats(const sgm_graph_stats* gs, int32_t k, int32_t m, const int32_t* edges,
                                   const int32_t* labels, const int32_t* phi, int64_t anchor_deg, float* out);
/* The same for a registered query and loaded graph; phi NULL = the query's current
 * order; anchor = the data vertex phi[0] is fixed to, or -1. */
sgm_status sgm_prefix_features(const sgm_query* q, const sgm_graph* g, const int32_t* phi, int64_t anchor,
                               float* out);

/* Creates a model on the engine's device from host float32 parameters packed as
 * [W1 (in_dim x hidden, row-major), b1 (hidden), W2 (hidden x hidden), b2 (hidden),
 *  w3 (hidden), b3 (1)]. in_dim in [1, SGM_MODEL_MAX_IN]; hidden a multiple of 32 in [32, 256]. */
sgm_status sgm_model_create(sgm_engine* e, int32_t in_dim, int32_t hidden, const float* init_params,
                            sgm_model** out);
sgm_status sgm_model_free(sgm_model* m);
sgm_status sgm_model_info(const sgm_model* m, int32_t* in_dim, int32_t* hidden, int64_t* n_params, int64_t* steps);
/* Copies the packed parameters to / from host float32[n_params]; set also clears the Adam moments. */
sgm_status sgm_model_get_params(const sgm_model* m, float* params_out);
sgm_status sgm_model_set_params(sgm_model* m, const float* params);
/* y[i] = MLP(X[i]) for host float32 X[n * in_dim], host y[n]. */
sgm_status sgm_model_forward(sgm_model* m, const float* X, int64_t n, float* y);
/* Gradient of L = (1/n) sum (MLP(X[i]) - t[i])^2 with respect to the packed
 * parameters (host grad[n_params] or NULL) and L itself (host or NULL). The
 * gradient is kept on the device for sgm_model_adam_step. */
sgm_status sgm_model_gradient(sgm_model* m, const float* X, const float* t, int64_t n, float* grad, float* loss);
/* One Adam update (Kingma and Ba, ICLR 2015) with the last gradient. */
sgm_status sgm_model_adam_step(sgm_model* m, float lr, float beta1, float beta2, float eps);
/* `steps` full-batch Adam updates (beta1 0.9, beta2 0.999, eps 1e-8) on host
 * X[n * in_dim], t[n]; losses (host float[steps] or NULL) receives L before each update. */
sgm_status sgm_model_train(sgm_model* m, const float* X, const float* t, int64_t n, int32_t steps, float lr,
                           float* losses);

/*
 * Learned order: a beam search (width `beam`, >= 1) over connected orders that
 * minimises the predicted search work sum_i 10^pred(prefix i), where the last
 * prefix counts nothing when its query vertex has exactly one earlier
 * neighbour (a count takes that level arithmetically). The rule-based
 * greedy order (sgm_query_order_greedy, or sgm_query_order_greedy_from when
 * root >= 0) is scored the same way and kept when its predicted work is not
 * larger (fallback). root >= 0 fixes phi[0] = root (anchored queries; the
 * features then carry the anchor's degree, see sgm_prefix_features). The
 * chosen order is set on q.
 * pred_learned / pred_greedy (host, may be NULL) receive both predicted works;
 * *used_learned (may be NULL) = 1 when the learned order was taken.
 */
sgm_status sgm_query_order_learned(sgm_query* q, const sgm_graph* g, sgm_model* m, int32_t beam, int32_t root,
                                   int64_t anchor, double* pred_learned, double* pred_greedy,
                                   int32_t* used_learned);

#ifdef __cplusplus
}
#endif

#endif /* SGM_H */
