// noalloc.cu - a count entry point that allocates nothing.
//
// Some callers cannot allocate device memory at call time: a service whose
// device memory belongs to another framework's caching allocator (a direct
// cudaMalloc can fail although that pool has room), a latency-bound server
// that must not stall its other streams (cudaFree synchronises the whole
// device), or a deployment that reserves all of its memory when it starts so
// that a query can never fail for lack of memory later.
// sgm_count_noalloc serves them: the caller passes the graph
// already in device memory and the query on the host, and every piece of
// scratch (degrees, 8-bit labels, candidate bitmaps, the root list, the run
// state, the plan and the work queue) lives in one file-scope device array of
// SGM_NOALLOC_SCRATCH_BYTES. The CUDA runtime places that array on a device
// when it loads this file's module there: at library load with eager module
// loading, or, with lazy loading (CUDA's default), at the first call on that
// device, which looks up the array's address. From then on the device holds
// it until the process exits, so a caller that must never allocate later
// makes one call per device at start-up (n = 0 and k = 1 is enough).
#include <algorithm>
#include <cstring>
#include <mutex>

#include "objects.h"

static __device__ __align__(256) unsigned char g_noalloc_scratch[SGM_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 256;
std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {nullptr};  // device address of the array, per device

// Device address of g_noalloc_scratch on `device` (which must be current).
// In host code the array's name is only a stand-in, so the address is looked
// up with cudaGetSymbolAddress, once per device, and cached.
sgm_status noalloc_scratch(int device, unsigned char** out) {
    if (device < 0 || device >= kMaxDevices) return sgm_fail(SGM_E_INVALID_ARG, "device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[device]) {
        void* p = nullptr;
        const cudaError_t err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess)
            return sgm_fail(SGM_E_CUDA, "cudaGetSymbolAddress(scratch) failed: %s", cudaGetErrorString(err));
        g_noalloc_addr[device] = p;
    }
    *out = (unsigned char*)g_noalloc_addr[device];
    return SGM_OK;
}

inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Puts the caller's current device back on every return path: the entry
// point runs inside host frameworks (torch, for one) that keep their own
// notion of the current device.
struct DeviceGuard {
    int saved = -1;
    DeviceGuard() {
        if (cudaGetDevice(&saved) != cudaSuccess) {
            saved = -1;
            cudaGetLastError();
        }
    }
    ~DeviceGuard() {
        if (saved >= 0) cudaSetDevice(saved);
    }
};

// The same rule-based order as sgm_query_order_greedy, without the label
// frequencies of a loaded graph: the vertex of maximum degree first (ties:
// smaller id), then repeatedly the vertex with the most ordered neighbours
// (ties: most frontier neighbours, most unvisited neighbours, smaller id).
void simple_order(int k, const uint32_t* adj, int32_t* order) {
    int first = 0;
    for (int u = 1; u < k; ++u)
        if (popc32(adj[u]) > popc32(adj[first])) first = u;
    uint32_t ordered = 1u << first;
    order[0] = first;
    for (int i = 1; i < k; ++i) {
        uint32_t frontier = 0;
        for (int u = 0; u < k; ++u)
            if ((ordered >> u) & 1u) frontier |= adj[u];
        frontier &= ~ordered;
        int best = -1, bv = -1, bn = -1, bu = -1;
        for (int u = 0; u < k; ++u) {
            if (!((frontier >> u) & 1u)) continue;
            const int vis = popc32(adj[u] & ordered), nb = popc32(adj[u] & frontier);
            const int unv = popc32(adj[u] & ~ordered & ~frontier);
            if (vis > bv || (vis == bv && (nb > bn || (nb == bn && unv > bu)))) {
                best = u;
                bv = vis;
                bn = nb;
                bu = unv;
            }
        }
        order[i] = best;
        ordered |= 1u << best;
    }
}

}  // namespace

extern "C" sgm_status sgm_count_noalloc(int32_t device, void* cuda_stream, int64_t n, const int64_t* rowptr,
                                        const int32_t* col, const int32_t* labels, int32_t num_labels, int32_t k,
                                        int32_t m, const int32_t* edges, const int32_t* qlabels, const int32_t* phi,
                                        uint64_t* count) {
    if (!rowptr || !count || (m > 0 && !edges)) return sgm_fail(SGM_E_INVALID_ARG, "sgm_count_noalloc: NULL argument");
    if (n < 0 || n > INT32_MAX) return sgm_fail(SGM_E_INVALID_ARG, "n = %lld outside [0, 2^31)", (long long)n);
    if (k > SGM_KMAX) return sgm_fail(SGM_E_QUERY_TOO_LARGE, "k = %d > %d", k, SGM_KMAX);
    if (k < 1 || m < 0) return sgm_fail(SGM_E_INVALID_ARG, "bad k = %d or m = %d", k, m);
    if (num_labels < 1 || num_labels > 256 || (!labels && num_labels != 1))
        return sgm_fail(SGM_E_INVALID_ARG, "num_labels = %d (1 without labels, at most 256)", num_labels);
    // query: simple, connected, labels in range
    uint32_t adj[SGM_KMAX];
    int32_t qlab[SGM_KMAX];
    memset(adj, 0, sizeof(adj));
    for (int32_t i = 0; i < m; ++i) {
        const int32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b || ((adj[a] >> b) & 1u))
            return sgm_fail(SGM_E_QUERY_INVALID, "query edge %d = (%d, %d) invalid or repeated", i, a, b);
        adj[a] |= 1u << b;
        adj[b] |= 1u << a;
    }
    for (int32_t u = 0; u < k; ++u) {
        qlab[u] = qlabels ? qlabels[u] : 0;
        if (qlab[u] < 0 || qlab[u] >= num_labels) return sgm_fail(SGM_E_LABEL_RANGE, "query label %d", qlab[u]);
    }
    int32_t order[SGM_KMAX];
    if (phi) {
        memcpy(order, phi, sizeof(int32_t) * k);
    } else {
        uint32_t seen = 1u, frontier = 1u;
        while (frontier) {
            uint32_t next = 0;
            for (int u = 0; u < k; ++u)
                if ((frontier >> u) & 1u) next |= adj[u];
            next &= ~seen;
            seen |= next;
            frontier = next;
        }
        if (seen != (k == 32 ? 0xffffffffu : ((1u << k) - 1u)))
            return sgm_fail(SGM_E_QUERY_DISCONNECTED, "query graph is not connected");
        simple_order(k, adj, order);
    }
    {
        uint32_t seen = 0;
        for (int i = 0; i < k; ++i) {
            const int u = order[i];
            if (u < 0 || u >= k || ((seen >> u) & 1u)) return sgm_fail(SGM_E_INVALID_ARG, "order is not a permutation");
            if (i > 0 && !(adj[u] & seen)) return sgm_fail(SGM_E_ORDER_NOT_CONNECTED, "order position %d", i);
            seen |= 1u << u;
        }
    }
    // scratch layout; every piece starts on a 256-byte boundary
    const int64_t words = (n + 31) / 32;
    const int32_t qcap = 1024;
    size_t off = 0;
    const size_t o_state = off;
    off += up256(sizeof(RunState));
    const size_t o_plan = off;
    off += up256(sizeof(QueryPlan));
    const size_t o_flags = off;
    off += up256(16 + sizeof(unsigned long long) * 256);
    const size_t o_aut = off;
    off += up256(SGM_KMAX);
    const size_t o_queue = off;
    off += up256(sizeof(QueueTask) * qcap);
    const size_t o_deg = off;
    off += up256(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1));
    const size_t o_lab = off;
    off += up256((size_t)std::max<int64_t>(n, 1));
    const size_t o_roots = off;
    off += up256(sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1));
    const size_t o_bits = off;
    off += up256(sizeof(uint32_t) * (size_t)std::max<int64_t>(words, 1) * k);
    if (off > (size_t)SGM_NOALLOC_SCRATCH_BYTES)
        return sgm_fail(SGM_E_INVALID_ARG,
                        "sgm_count_noalloc: n = %lld and k = %d need %zu scratch bytes, more than the %u available",
                        (long long)n, k, off, (unsigned)SGM_NOALLOC_SCRATCH_BYTES);
    DeviceGuard restore_device;
    SGM_CUDA_TRY(cudaSetDevice(device));
    unsigned char* base = nullptr;
    SGM_TRY(noalloc_scratch(device, &base));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    RunState* st = (RunState*)(base + o_state);
    QueryPlan* dP = (QueryPlan*)(base + o_plan);
    int32_t* d_flags = (int32_t*)(base + o_flags);
    unsigned long long* d_hist = (unsigned long long*)(base + o_flags + 16);
    int8_t* d_aut = (int8_t*)(base + o_aut);
    QueueTask* queue = (QueueTask*)(base + o_queue);
    int32_t* deg = (int32_t*)(base + o_deg);
    uint8_t* lab8 = (uint8_t*)(base + o_lab);
    int32_t* roots = (int32_t*)(base + o_roots);
    uint32_t* bits = (uint32_t*)(base + o_bits);
    // the array keeps the previous call's contents: clear what starts at zero
    SGM_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));
    SGM_CUDA_TRY(cudaMemsetAsync(d_flags, 0, 16 + sizeof(unsigned long long) * 256, s));
    SGM_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(QueueTask) * qcap, s));
    // per-graph tables the kernels read: degrees and 8-bit labels
    DevGraph G;
    memset(&G, 0, sizeof(G));
    G.n = n;
    G.words = words;
    G.rowptr = rowptr;
    G.col = col;
    G.deg = deg;
    G.num_labels = num_labels;
    SGM_CUDA_TRY(sgm_launch_degrees(rowptr, n, deg, d_flags, s));
    if (labels) {
        SGM_CUDA_TRY(sgm_launch_labels(labels, n, num_labels, lab8, d_flags, d_hist, s));
        G.labels = lab8;
    }
    int32_t h_flags = 0;
    SGM_CUDA_TRY(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_flags & SGM_VF_RANGE) return sgm_fail(SGM_E_GRAPH_RANGE, "rowptr is not non-decreasing");
    if (h_flags & SGM_VF_LABEL) return sgm_fail(SGM_E_LABEL_RANGE, "a data label is outside [0, %d)", num_labels);
    // candidate bitmaps: label and degree (no neighbour-label table here)
    FilterSpec F;
    memset(&F, 0, sizeof(F));
    F.k = k;
    F.use_filter = 1;
    for (int u = 0; u < k; ++u) {
        F.label[u] = qlab[u];
        F.dq[u] = popc32(adj[u]);
    }
    SGM_CUDA_TRY(sgm_launch_filter(G, F, bits, s));
    // plan: backward neighbours and injectivity tests; no symmetry breaking,
    // no arithmetic level, no initialisation beyond the root level
    QueryPlan P;
    memset(&P, 0, sizeof(P));
    P.k = k;
    P.D = 1;
    P.aut_n = 1;
    P.aut = d_aut;  // identity permutation, written below
    // the same stealable sub-ranges as sgm_count's defaults: a warp offers
    // half of a root-level range longer than 2 x 256 candidates to idle warps
    P.split_min = 256;
    P.split_depth = 1;
    for (int l = 0; l < k; ++l) {
        const int u = order[l];
        LevelPlan& lp = P.lv[l];
        lp.u = u;
        lp.bits = bits + (size_t)u * words;
        for (int i = 0; i < l; ++i) {
            const int w = order[i];
            if ((adj[u] >> w) & 1u) lp.bwd |= 1u << i;
            else if (qlab[w] == qlab[u]) lp.inj |= 1u << i;
        }
    }
    int8_t ident[SGM_KMAX];
    for (int u = 0; u < k; ++u) ident[u] = (int8_t)u;
    SGM_CUDA_TRY(cudaMemcpyAsync(d_aut, ident, (size_t)k, cudaMemcpyHostToDevice, s));
    SGM_CUDA_TRY(cudaMemcpyAsync(dP, &P, sizeof(QueryPlan), cudaMemcpyHostToDevice, s));
    // root candidates of phi[0]
    SGM_CUDA_TRY(sgm_launch_roots(P.lv[0].bits, 0, n, roots, st, s));
    unsigned long long n_roots = 0;
    SGM_CUDA_TRY(cudaMemcpyAsync(&n_roots, &st->frontier_n, sizeof(n_roots), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    if (k == 1 || n_roots == 0) {
        *count = k == 1 ? n_roots : 0;
        return SGM_OK;
    }
    int sms = 0;
    SGM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    ExtendLaunch L;
    L.mode = SGM_KMODE_COUNT;
    L.gather = labels ? 1 : 0;
    L.kcap = k;
    L.warps_per_block = 8;
    L.smem_bytes = sgm_extend_smem_bytes(k, L.warps_per_block, false);
    const int bps = sgm_extend_max_blocks_per_sm(SGM_KMODE_COUNT, false, L.gather != 0, L.warps_per_block,
                                                   L.smem_bytes);
    if (bps < 1) return sgm_fail(SGM_E_CUDA, "extension kernel does not fit on an SM");
    L.blocks = bps * sms;
    PoolArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.rows = roots;
    pa.n_short = (int64_t)n_roots;
    SGM_CUDA_TRY(sgm_launch_extend(L, G, dP, pa, st, queue, qcap, nullptr, 0, 0, 0, nullptr, s));
    RunState hs;
    SGM_CUDA_TRY(cudaMemcpyAsync(&hs, st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.status) return sgm_fail(hs.status, "device error %d", hs.status);
    if (hs.overflow) return sgm_fail(SGM_E_COUNT_OVERFLOW, "embedding count exceeds 2^64 - 1");
    *count = hs.count;
    return SGM_OK;
}
