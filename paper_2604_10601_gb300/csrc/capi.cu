// capi.cu - the C ABI of libsgm (include/sgm.h): engine, graph and query
// objects, the rule-based matching order, and the host orchestration of one
// run: filter -> root candidates -> BFS initialization to tau -> persistent
// extension kernel -> results.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <tuple>
#include <vector>

#include "objects.h"

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512];

void sgm_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static sgm_status fail(sgm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

extern "C" const char* sgm_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// device buffers
// ---------------------------------------------------------------------------
sgm_status buf_ensure(DevBuf& b, size_t bytes) {
    if (bytes <= b.bytes && b.p) return SGM_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    SGM_CUDA_TRY(cudaMalloc(&b.p, bytes));
    b.bytes = bytes;
    return SGM_OK;
}

void buf_free(DevBuf& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

sgm_status sgm_fail(sgm_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

// ---------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------
extern "C" void sgm_opts_default(sgm_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->struct_size = sizeof(sgm_opts);
    o->mode = SGM_MODE_COUNT;
    o->tau = 1000000;
    o->pool_cap_bytes = (int64_t)1 << 30;
    o->use_filter = 1;
    o->arith_last = 1;
    o->warps_per_block = 8;
    o->blocks_per_sm = 0;
    o->split_min = 256;
    o->sym_break = 1;
    o->time_cap_s = 0.0;
    o->chunk_words = 4;
    o->split_depth = 1;
    o->pool_chunk = 512;
    o->exec_model = SGM_EXEC_FINE_BATCH;
    o->unroll = 1;
    o->steal_mode = 0;
}

extern "C" sgm_status sgm_create(sgm_engine** out, int32_t device, void* cuda_stream) {
    if (!out) return fail(SGM_E_INVALID_ARG, "sgm_create: out is NULL");
    *out = nullptr;
    int ndev = 0;
    SGM_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(SGM_E_INVALID_ARG, "sgm_create: device %d of %d", device, ndev);
    SGM_CUDA_TRY(cudaSetDevice(device));
    sgm_engine* e = new (std::nothrow) sgm_engine();
    if (!e) return fail(SGM_E_OOM, "sgm_create: host allocation failed");
    e->device = device;
    e->stream = (cudaStream_t)cuda_stream;
    cudaDeviceProp prop;
    cudaError_t err = cudaGetDeviceProperties(&prop, device);
    if (err != cudaSuccess) {
        delete e;
        return fail(SGM_E_CUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(err));
    }
    e->sms = prop.multiProcessorCount;
    err = cudaMallocHost((void**)&e->h_state, sizeof(RunState));
    for (int i = 0; i < 4 && err == cudaSuccess; ++i) err = cudaEventCreate(&e->ev[i]);
    if (err != cudaSuccess) {
        delete e;
        return fail(SGM_E_CUDA, "sgm_create: %s", cudaGetErrorString(err));
    }
    memset(&e->stats, 0, sizeof(e->stats));
    *out = e;
    return SGM_OK;
}

int32_t sgm_engine_device(const sgm_engine* e) { return e->device; }
cudaStream_t sgm_engine_stream(const sgm_engine* e) { return e->stream; }

extern "C" sgm_status sgm_set_stream(sgm_engine* e, void* cuda_stream) {
    if (!e) return fail(SGM_E_INVALID_ARG, "sgm_set_stream: engine is NULL");
    e->stream = (cudaStream_t)cuda_stream;
    return SGM_OK;
}

extern "C" sgm_status sgm_destroy(sgm_engine* e) {
    if (!e) return SGM_OK;
    if (e->live_graphs || e->live_queries)
        return fail(SGM_E_INVALID_ARG, "sgm_destroy: %d graphs and %d queries still alive", e->live_graphs,
                    e->live_queries);
    cudaSetDevice(e->device);
    cudaStreamSynchronize(e->stream);
    DevBuf* bufs[] = {&e->bits,  &e->cnt,  &e->poolA, &e->poolB,     &e->queue,
                      &e->state, &e->plan, &e->aut,   &e->short_idx, &e->tasks, &e->refine, &e->coarse,
                      &e->cgtab};
    for (DevBuf* b : bufs) buf_free(*b);
    if (e->h_state) cudaFreeHost(e->h_state);
    for (int i = 0; i < 4; ++i)
        if (e->ev[i]) cudaEventDestroy(e->ev[i]);
    delete e;
    return SGM_OK;
}

extern "C" sgm_status sgm_get_stats(const sgm_engine* e, sgm_stats* out) {
    if (!e || !out) return fail(SGM_E_INVALID_ARG, "sgm_get_stats: NULL argument");
    *out = e->stats;
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// data graph
// ---------------------------------------------------------------------------
static sgm_status graph_alloc(sgm_graph* g, void** p, size_t bytes) {
    *p = nullptr;
    SGM_CUDA_TRY(cudaMalloc(p, bytes ? bytes : 16));
    g->owned.push_back(*p);
    return SGM_OK;
}

static void graph_release(sgm_graph* g) {
    for (void* p : g->owned) cudaFree(p);
    g->owned.clear();
}

static int env_int(const char* name, int dflt) {
    const char* s = getenv(name);
    return s && *s ? atoi(s) : dflt;
}

static sgm_status graph_build(sgm_engine* e, sgm_graph* g, int64_t n, const int64_t* rowptr, const int32_t* col,
                              const int32_t* labels, int32_t num_labels, uint32_t flags) {
    const bool dev = flags & SGM_DEVICE_PTRS;
    const bool borrow = dev && (flags & SGM_BORROW);
    cudaStream_t s = e->stream;
    DevGraph& G = g->G;
    memset(&G, 0, sizeof(G));
    int64_t ends[2] = {0, 0};
    if (dev) {
        SGM_CUDA_TRY(cudaMemcpy(&ends[0], rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost));
        SGM_CUDA_TRY(cudaMemcpy(&ends[1], rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost));
    } else {
        ends[0] = rowptr[0];
        ends[1] = rowptr[n];
    }
    if (ends[0] != 0 || ends[1] < 0) return fail(SGM_E_GRAPH_RANGE, "rowptr[0]=%lld rowptr[n]=%lld", (long long)ends[0], (long long)ends[1]);
    const int64_t nnz = ends[1];
    G.n = n;
    G.nnz = nnz;
    G.words = (n + 31) / 32;
    G.num_labels = num_labels;
    if (nnz > 0 && !col) return fail(SGM_E_INVALID_ARG, "col is NULL with %lld entries", (long long)nnz);
    // rowptr / col
    void* p = nullptr;
    if (borrow) {
        G.rowptr = rowptr;
        G.col = col;
    } else {
        SGM_TRY(graph_alloc(g, &p, sizeof(int64_t) * (n + 1)));
        SGM_CUDA_TRY(cudaMemcpyAsync(p, rowptr, sizeof(int64_t) * (n + 1),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        G.rowptr = (const int64_t*)p;
        SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * nnz));
        if (nnz)
            SGM_CUDA_TRY(cudaMemcpyAsync(p, col, sizeof(int32_t) * nnz,
                                         dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
        G.col = (const int32_t*)p;
    }
    // scratch flags word + label histogram
    void* scratch = nullptr;
    SGM_TRY(graph_alloc(g, &scratch, 16 + sizeof(unsigned long long) * 256));
    int32_t* d_flags = (int32_t*)scratch;
    unsigned long long* d_hist = (unsigned long long*)((char*)scratch + 16);
    SGM_CUDA_TRY(cudaMemsetAsync(scratch, 0, 16 + sizeof(unsigned long long) * 256, s));
    // degrees
    SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * (n ? n : 1)));
    G.deg = (const int32_t*)p;
    SGM_CUDA_TRY(sgm_launch_degrees(G.rowptr, n, (int32_t*)p, d_flags, s));
    int32_t h_flags = 0;
    SGM_CUDA_TRY(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_flags & SGM_VF_RANGE) return fail(SGM_E_GRAPH_RANGE, "rowptr is not non-decreasing");
    // labels
    g->label_hist.assign(num_labels, 0);
    if (labels) {
        const int32_t* lab_dev = labels;
        void* tmp = nullptr;
        if (!dev) {
            SGM_CUDA_TRY(cudaMalloc(&tmp, sizeof(int32_t) * (n ? n : 1)));
            cudaError_t ce = cudaMemcpyAsync(tmp, labels, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
            if (ce != cudaSuccess) {
                cudaFree(tmp);
                return fail(SGM_E_CUDA, "label copy: %s", cudaGetErrorString(ce));
            }
            lab_dev = (const int32_t*)tmp;
        }
        SGM_TRY(graph_alloc(g, &p, n ? n : 1));
        G.labels = (const uint8_t*)p;
        cudaError_t ce = sgm_launch_labels(lab_dev, n, num_labels, (uint8_t*)p, d_flags, d_hist, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(g->label_hist.data(), d_hist, sizeof(unsigned long long) * num_labels,
                                                   cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (tmp) cudaFree(tmp);
        if (ce != cudaSuccess) return fail(SGM_E_CUDA, "labels: %s", cudaGetErrorString(ce));
        if (h_flags & SGM_VF_LABEL) return fail(SGM_E_LABEL_RANGE, "a data label is outside [0, %d)", num_labels);
    } else {
        g->label_hist[0] = (unsigned long long)n;
    }
    // validation
    if (flags & SGM_VALIDATE) {
        SGM_CUDA_TRY(sgm_launch_validate(G, d_flags, s));
        SGM_CUDA_TRY(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        if (h_flags & SGM_VF_RANGE) return fail(SGM_E_GRAPH_RANGE, "a column index is outside [0, n)");
        if (h_flags & SGM_VF_SELF_LOOP) return fail(SGM_E_GRAPH_SELF_LOOP, "the CSR holds a self-loop");
        if (h_flags & SGM_VF_UNSORTED) return fail(SGM_E_GRAPH_UNSORTED, "a CSR row is not strictly increasing");
        if (h_flags & SGM_VF_ASYMMETRIC) return fail(SGM_E_GRAPH_ASYMMETRIC, "the CSR is not symmetric");
    }
    // degrees to the host: maximum degree and hub selection
    std::vector<int32_t> deg(n);
    if (n) SGM_CUDA_TRY(cudaMemcpy(deg.data(), G.deg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
    int32_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) dmax = std::max(dmax, deg[v]);
    g->dmax = dmax;
    // label and degree statistics for the cost model
    {
        sgm_graph_stats& gs = g->gstats;
        memset(&gs, 0, sizeof(gs));
        gs.n = n;
        gs.nnz = nnz;
        gs.num_labels = num_labels;
        for (int l = 0; l < num_labels; ++l) gs.label_frac[l] = n ? (double)g->label_hist[l] / (double)n : 0.0;
        double mom[4] = {0, 0, 0, 0}, hist[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int64_t v = 0; v < n; ++v) {
            const double x = (double)deg[v];
            double pw = x;
            for (int j = 0; j < 4; ++j, pw *= x) mom[j] += pw;
            hist[std::min(7, 31 - __builtin_clz((unsigned)deg[v] + 1u))] += 1.0;
        }
        for (int j = 0; j < 4; ++j) gs.log2_deg_moment[j] = (n && mom[j] > 0) ? std::log2(mom[j] / (double)n) : 0.0;
        for (int b = 0; b < 8; ++b) gs.deg_hist[b] = n ? hist[b] / (double)n : 0.0;
    }
    // vertices bucketed by label (the candidate filter visits only the bucket
    // of a query vertex's label); within a bucket by degree class min(d, 8)
    // descending and ids ascending within a class, so that the vertices of
    // degree >= c (c < 8) are a prefix of the bucket
    if (G.labels && num_labels >= 2 && n > 0) {
        std::vector<uint8_t> lab(n);
        SGM_CUDA_TRY(cudaMemcpy(lab.data(), G.labels, (size_t)n, cudaMemcpyDeviceToHost));
        const int C = kDegClasses;
        auto cls = [&](int64_t v) { return std::min<int64_t>(deg[v], C - 1); };
        std::vector<int64_t> cnt((size_t)num_labels * C, 0);
        for (int64_t v = 0; v < n; ++v) cnt[(size_t)lab[v] * C + cls(v)]++;
        std::vector<int64_t> off(num_labels + 1, 0), ge((size_t)num_labels * C, 0), at((size_t)num_labels * C, 0);
        for (int l = 0; l < num_labels; ++l) {
            off[l + 1] = off[l] + (int64_t)g->label_hist[l];
            int64_t run = 0;
            for (int c = C - 1; c >= 0; --c) {
                at[(size_t)l * C + c] = off[l] + run;  // class c starts after the higher classes
                run += cnt[(size_t)l * C + c];
                ge[(size_t)l * C + c] = run;
            }
        }
        std::vector<int32_t> vert(n);
        for (int64_t v = 0; v < n; ++v) vert[at[(size_t)lab[v] * C + cls(v)]++] = (int32_t)v;
        SGM_TRY(graph_alloc(g, &p, sizeof(int64_t) * (num_labels + 1)));
        SGM_CUDA_TRY(cudaMemcpy(p, off.data(), sizeof(int64_t) * (num_labels + 1), cudaMemcpyHostToDevice));
        G.lab_off = (const int64_t*)p;
        SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * (size_t)n));
        SGM_CUDA_TRY(cudaMemcpy(p, vert.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice));
        G.lab_vert = (const int32_t*)p;
        SGM_TRY(graph_alloc(g, &p, sizeof(int64_t) * ge.size()));
        SGM_CUDA_TRY(cudaMemcpy(p, ge.data(), sizeof(int64_t) * ge.size(), cudaMemcpyHostToDevice));
        G.lab_ge = (const int64_t*)p;
    }
    // neighbour-label frequencies (labelled graphs with 2..64 labels)
    if (G.labels && num_labels >= 2 && num_labels <= 64) {
        SGM_TRY(graph_alloc(g, &p, (size_t)n * num_labels));
        SGM_CUDA_TRY(sgm_launch_nlf(G, (uint8_t*)p, s));
        G.nlf = (const uint8_t*)p;
    }
    // upper-rank adjacency N+(v) for symmetry-broken levels
    {
        SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * (n ? n : 1)));
        G.updeg = (const int32_t*)p;
        SGM_CUDA_TRY(sgm_launch_up_count(G, (int32_t*)p, s));
        std::vector<int32_t> updeg(n);
        if (n) SGM_CUDA_TRY(cudaMemcpyAsync(updeg.data(), G.updeg, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        std::vector<int64_t> up_rowptr(n + 1);
        up_rowptr[0] = 0;
        for (int64_t v = 0; v < n; ++v) up_rowptr[v + 1] = up_rowptr[v] + updeg[v];
        SGM_TRY(graph_alloc(g, &p, sizeof(int64_t) * (n + 1)));
        G.up_rowptr = (const int64_t*)p;
        SGM_CUDA_TRY(cudaMemcpy(p, up_rowptr.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice));
        SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * (size_t)std::max<int64_t>(up_rowptr[n], 1)));
        G.up_col = (const int32_t*)p;
        SGM_CUDA_TRY(sgm_launch_up_fill(G, G.up_rowptr, (int32_t*)p, s));
    }
    // hub adjacency bitmaps: the highest-degree vertices with degree >= hub_min,
    // as many as fit the budget
    const int hub_min = env_int("SGM_HUB_MIN_DEG", 128);
    const long long budget = (long long)env_int("SGM_HUB_BUDGET_MB", 1024) << 20;
    const long long per_hub = (long long)G.words * 4;
    std::vector<int32_t> cand;
    for (int64_t v = 0; v < n; ++v)
        if (deg[v] >= hub_min) cand.push_back((int32_t)v);
    std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) { return deg[a] != deg[b] ? deg[a] > deg[b] : a < b; });
    long long max_hubs = per_hub > 0 ? budget / per_hub : 0;
    if ((long long)cand.size() > max_hubs) cand.resize((size_t)max_hubs);
    G.hubs = (int32_t)cand.size();
    if (G.hubs > 0) {
        std::vector<int32_t> hub_id(n, -1);
        for (int32_t h = 0; h < G.hubs; ++h) hub_id[cand[h]] = h;
        SGM_TRY(graph_alloc(g, &p, sizeof(int32_t) * n));
        SGM_CUDA_TRY(cudaMemcpy(p, hub_id.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice));
        G.hub_id = (const int32_t*)p;
        void* list = nullptr;
        SGM_TRY(graph_alloc(g, &list, sizeof(int32_t) * G.hubs));
        SGM_CUDA_TRY(cudaMemcpy(list, cand.data(), sizeof(int32_t) * G.hubs, cudaMemcpyHostToDevice));
        G.hub_list = (const int32_t*)list;
        SGM_TRY(graph_alloc(g, &p, (size_t)per_hub * G.hubs));
        G.hub_bits = (const uint32_t*)p;
        SGM_CUDA_TRY(sgm_launch_hub_bits(G, (const int32_t*)list, G.hubs, (uint32_t*)p, s));
    }
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    return SGM_OK;
}

extern "C" sgm_status sgm_graph_load_csr(sgm_engine* e, int64_t n, const int64_t* rowptr, const int32_t* col,
                                         const int32_t* labels, int32_t num_labels, uint32_t flags, sgm_graph** out) {
    if (!e || !out || !rowptr) return fail(SGM_E_INVALID_ARG, "sgm_graph_load_csr: NULL argument");
    *out = nullptr;
    if (n < 0 || n > INT32_MAX) return fail(SGM_E_INVALID_ARG, "n = %lld outside [0, 2^31)", (long long)n);
    if (num_labels < 1 || num_labels > 256) return fail(SGM_E_INVALID_ARG, "num_labels = %d outside [1, 256]", num_labels);
    if (!labels && num_labels != 1) return fail(SGM_E_INVALID_ARG, "unlabelled graph needs num_labels = 1");
    if ((flags & SGM_BORROW) && !(flags & SGM_DEVICE_PTRS))
        return fail(SGM_E_INVALID_ARG, "SGM_BORROW needs SGM_DEVICE_PTRS");
    if (flags & ~(SGM_DEVICE_PTRS | SGM_BORROW | SGM_VALIDATE)) return fail(SGM_E_INVALID_ARG, "unknown flags 0x%x", flags);
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    sgm_graph* g = new (std::nothrow) sgm_graph();
    if (!g) return fail(SGM_E_OOM, "host allocation failed");
    g->e = e;
    sgm_status st = graph_build(e, g, n, rowptr, col, labels, num_labels, flags);
    if (st < 0) {
        cudaStreamSynchronize(e->stream);
        graph_release(g);
        delete g;
        return st;
    }
    e->live_graphs++;
    *out = g;
    return SGM_OK;
}

extern "C" sgm_status sgm_graph_free(sgm_graph* g) {
    if (!g) return SGM_OK;
    cudaSetDevice(g->e->device);
    cudaStreamSynchronize(g->e->stream);
    graph_release(g);
    g->e->live_graphs--;
    delete g;
    return SGM_OK;
}

extern "C" sgm_status sgm_graph_get_stats(const sgm_graph* g, sgm_graph_stats* out) {
    if (!g || !out) return fail(SGM_E_INVALID_ARG, "sgm_graph_get_stats: NULL argument");
    *out = g->gstats;
    return SGM_OK;
}

extern "C" sgm_status sgm_graph_info(const sgm_graph* g, int64_t* n, int64_t* nnz, int32_t* dmax, int32_t* hubs) {
    if (!g) return fail(SGM_E_INVALID_ARG, "sgm_graph_info: graph is NULL");
    if (n) *n = g->G.n;
    if (nnz) *nnz = g->G.nnz;
    if (dmax) *dmax = g->dmax;
    if (hubs) *hubs = g->G.hubs;
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// query graph and matching order
// ---------------------------------------------------------------------------
// Every bijection sigma of V(Q) with L(sigma(u)) = L(u) and
// {u, w} in E(Q) <=> {sigma(u), sigma(w)} in E(Q), by backtracking in vertex
// order with label and degree pruning. Stops (clearing the list) past kAutCap.
static void enumerate_automorphisms(sgm_query& q) {
    const int k = q.k;
    q.aut.clear();
    int8_t map[SGM_KMAX];
    uint32_t used = 0;
    bool over = false;
    std::vector<std::pair<int, int>> stack;  // (vertex, next candidate)
    int u = 0, w = 0;
    while (true) {
        if (u == k) {
            q.aut.emplace_back(map, map + k);
            if (q.aut.size() > kAutCap) { over = true; break; }
            if (stack.empty()) break;
            std::tie(u, w) = stack.back();
            stack.pop_back();
            used &= ~(1u << map[u]);
            continue;
        }
        bool placed = false;
        for (; w < k; ++w) {
            if ((used >> w) & 1u) continue;
            if (q.label[w] != q.label[u] || popc32(q.adj[w]) != popc32(q.adj[u])) continue;
            bool ok = true;
            for (int x = 0; x < u && ok; ++x)
                ok = (((q.adj[u] >> x) & 1u) != 0) == (((q.adj[w] >> map[x]) & 1u) != 0);
            if (!ok) continue;
            map[u] = (int8_t)w;
            used |= 1u << w;
            stack.emplace_back(u, w + 1);
            ++u;
            w = 0;
            placed = true;
            break;
        }
        if (placed) continue;
        if (stack.empty()) break;
        std::tie(u, w) = stack.back();
        stack.pop_back();
        used &= ~(1u << map[u]);
    }
    if (over) q.aut.clear();
}

extern "C" sgm_status sgm_query_register(sgm_engine* e, int32_t k, int32_t m, const int32_t* edges,
                                         const int32_t* labels, sgm_query** out) {
    if (!e || !out) return fail(SGM_E_INVALID_ARG, "sgm_query_register: NULL argument");
    *out = nullptr;
    if (k > SGM_KMAX) return fail(SGM_E_QUERY_TOO_LARGE, "k = %d > %d", k, SGM_KMAX);
    if (k < 1 || m < 0 || (m > 0 && !edges)) return fail(SGM_E_INVALID_ARG, "bad k = %d or m = %d", k, m);
    sgm_query q;
    q.e = e;
    q.k = k;
    q.m = m;
    memset(q.adj, 0, sizeof(q.adj));
    for (int32_t i = 0; i < m; ++i) {
        const int32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b)
            return fail(SGM_E_QUERY_INVALID, "query edge %d = (%d, %d) invalid", i, a, b);
        if ((q.adj[a] >> b) & 1u) return fail(SGM_E_QUERY_INVALID, "duplicate query edge (%d, %d)", a, b);
        q.adj[a] |= 1u << b;
        q.adj[b] |= 1u << a;
    }
    for (int32_t u = 0; u < k; ++u) {
        q.label[u] = labels ? labels[u] : 0;
        if (q.label[u] < 0) return fail(SGM_E_LABEL_RANGE, "query label %d of vertex %d", q.label[u], u);
    }
    // connectivity
    uint32_t seen = 1u, frontier = 1u;
    while (frontier) {
        uint32_t next = 0;
        for (int32_t u = 0; u < k; ++u)
            if ((frontier >> u) & 1u) next |= q.adj[u];
        next &= ~seen;
        seen |= next;
        frontier = next;
    }
    const uint32_t all = k == 32 ? 0xffffffffu : ((1u << k) - 1u);
    if (seen != all) return fail(SGM_E_QUERY_DISCONNECTED, "query graph is not connected");
    enumerate_automorphisms(q);
    sgm_query* qq = new (std::nothrow) sgm_query(q);
    if (!qq) return fail(SGM_E_OOM, "host allocation failed");
    e->live_queries++;
    *out = qq;
    return SGM_OK;
}

extern "C" sgm_status sgm_query_free(sgm_query* q) {
    if (!q) return SGM_OK;
    q->e->live_queries--;
    delete q;
    return SGM_OK;
}

sgm_status sgm_check_order(const sgm_query* q, const int32_t* phi) {
    uint32_t seen = 0;
    for (int32_t i = 0; i < q->k; ++i) {
        const int32_t u = phi[i];
        if (u < 0 || u >= q->k || ((seen >> u) & 1u)) return fail(SGM_E_INVALID_ARG, "order is not a permutation");
        if (i > 0 && !(q->adj[u] & seen))
            return fail(SGM_E_ORDER_NOT_CONNECTED, "order vertex %d (position %d) has no earlier neighbour", u, i);
        seen |= 1u << u;
    }
    return SGM_OK;
}

extern "C" sgm_status sgm_query_set_order(sgm_query* q, const int32_t* phi, int32_t k) {
    if (!q || !phi) return fail(SGM_E_INVALID_ARG, "sgm_query_set_order: NULL argument");
    if (k != q->k) return fail(SGM_E_INVALID_ARG, "order length %d != k = %d", k, q->k);
    SGM_TRY(sgm_check_order(q, phi));
    memcpy(q->order, phi, sizeof(int32_t) * k);
    q->has_order = true;
    return SGM_OK;
}

void sgm_greedy_order(sgm_query* q, const sgm_graph* g, int32_t root) {
    const int k = q->k;
    auto freq = [&](int u) -> unsigned long long {
        const int32_t l = q->label[u];
        return (g && l < (int32_t)g->label_hist.size()) ? g->label_hist[l] : 0ull;
    };
    int first = root;
    if (first < 0) {
        first = 0;
        for (int u = 1; u < k; ++u) {
            const int du = popc32(q->adj[u]), df = popc32(q->adj[first]);
            if (du > df || (du == df && freq(u) < freq(first))) first = u;
        }
    }
    uint32_t ordered = 1u << first;
    q->order[0] = first;
    for (int i = 1; i < k; ++i) {
        uint32_t frontier = 0;
        for (int u = 0; u < k; ++u)
            if ((ordered >> u) & 1u) frontier |= q->adj[u];
        frontier &= ~ordered;
        int best = -1, bv = -1, bn = -1, bu = -1;
        for (int u = 0; u < k; ++u) {
            if (!((frontier >> u) & 1u)) continue;
            const int vis = popc32(q->adj[u] & ordered);
            const int neig = popc32(q->adj[u] & frontier);
            const int unv = popc32(q->adj[u] & ~ordered & ~frontier);
            if (vis > bv || (vis == bv && (neig > bn || (neig == bn && unv > bu)))) {
                best = u;
                bv = vis;
                bn = neig;
                bu = unv;
            }
        }
        q->order[i] = best;
        ordered |= 1u << best;
    }
    q->has_order = true;
}

extern "C" sgm_status sgm_query_order_greedy(sgm_query* q, const sgm_graph* g) {
    if (!q) return fail(SGM_E_INVALID_ARG, "sgm_query_order_greedy: query is NULL");
    sgm_greedy_order(q, g, -1);
    return SGM_OK;
}

extern "C" sgm_status sgm_query_order_greedy_from(sgm_query* q, const sgm_graph* g, int32_t root) {
    if (!q) return fail(SGM_E_INVALID_ARG, "sgm_query_order_greedy_from: query is NULL");
    if (root < 0 || root >= q->k) return fail(SGM_E_INVALID_ARG, "root %d outside [0, %d)", root, q->k);
    sgm_greedy_order(q, g, root);
    return SGM_OK;
}

extern "C" sgm_status sgm_query_get_order(const sgm_query* q, int32_t* phi_out) {
    if (!q || !phi_out) return fail(SGM_E_INVALID_ARG, "sgm_query_get_order: NULL argument");
    if (!q->has_order) return fail(SGM_E_INVALID_ARG, "the query has no order yet");
    memcpy(phi_out, q->order, sizeof(int32_t) * q->k);
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// filter
// ---------------------------------------------------------------------------
sgm_status sgm_build_filter_spec(const sgm_graph* g, const sgm_query* q, int32_t use_filter, FilterSpec& F) {
    memset(&F, 0, sizeof(F));
    F.k = q->k;
    F.use_filter = use_filter ? 1 : 0;
    for (int u = 0; u < q->k; ++u) {
        if (q->label[u] >= g->G.num_labels)
            return fail(SGM_E_LABEL_RANGE, "query label %d outside [0, %d)", q->label[u], g->G.num_labels);
        F.label[u] = q->label[u];
        F.dq[u] = popc32(q->adj[u]);
        if (g->G.nlf) {
            int cnt[256] = {0};
            for (int w = 0; w < q->k; ++w)
                if ((q->adj[u] >> w) & 1u) cnt[q->label[w]]++;
            for (int l = 0; l < g->G.num_labels; ++l)
                if (cnt[l]) {
                    F.need_label[u][F.nneed[u]] = (uint8_t)l;
                    F.need_cnt[u][F.nneed[u]] = (uint8_t)cnt[l];
                    F.nneed[u]++;
                }
        }
    }
    return SGM_OK;
}

// Candidate-set refinement of the k bitmaps at `bits` (indexed by query
// vertex), in place: at most max_rounds rounds of the support rule
// (refine.cuh), stopping after the first round that clears nothing;
// *rounds_out = the rounds that cleared at least one candidate.
static sgm_status refine_bits(sgm_engine* e, const sgm_graph* g, const sgm_query* q, uint32_t* bits,
                              int32_t max_rounds, int32_t* rounds_out, uint64_t& launches) {
    const DevGraph& G = g->G;
    RefineSpec R;
    memset(&R, 0, sizeof(R));
    R.k = q->k;
    for (int u = 0; u < q->k; ++u) R.qadj[u] = q->adj[u];
    const size_t bytes = sizeof(uint32_t) * (size_t)G.words * (size_t)q->k;
    const size_t flag_off = (bytes + 255) & ~(size_t)255;
    SGM_TRY(buf_ensure(e->refine, flag_off + 256));
    int32_t* flag = (int32_t*)((char*)e->refine.p + flag_off);
    cudaStream_t s = e->stream;
    uint32_t* cur = bits;
    uint32_t* nxt = (uint32_t*)e->refine.p;
    int32_t rounds = 0;
    for (int32_t r = 0; r < max_rounds; ++r) {
        SGM_CUDA_TRY(cudaMemcpyAsync(nxt, cur, bytes, cudaMemcpyDeviceToDevice, s));
        SGM_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int32_t), s));
        SGM_CUDA_TRY(sgm_launch_refine(G, R, cur, nxt, flag, s));
        ++launches;
        int32_t changed = 0;
        SGM_CUDA_TRY(cudaMemcpyAsync(&changed, flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        if (!changed) break;
        ++rounds;
        std::swap(cur, nxt);
    }
    if (cur != bits) SGM_CUDA_TRY(cudaMemcpyAsync(bits, cur, bytes, cudaMemcpyDeviceToDevice, s));
    if (rounds_out) *rounds_out = rounds;
    return SGM_OK;
}

extern "C" sgm_status sgm_refine(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                                 int32_t max_rounds, uint32_t* dev_bits, int32_t* rounds) {
    if (!e || !g || !q || !dev_bits || max_rounds < 0) return fail(SGM_E_INVALID_ARG, "sgm_refine: bad argument");
    if (g->e != e || q->e != e) return fail(SGM_E_INVALID_ARG, "graph or query belongs to another engine");
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    FilterSpec F;
    SGM_TRY(sgm_build_filter_spec(g, q, use_filter, F));
    SGM_CUDA_TRY(sgm_launch_filter(g->G, F, dev_bits, e->stream));
    uint64_t launches = 1;
    int32_t r = 0;
    SGM_TRY(refine_bits(e, g, q, dev_bits, max_rounds, &r, launches));
    SGM_CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (rounds) *rounds = r;
    return SGM_OK;
}

extern "C" sgm_status sgm_filter(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                                 uint32_t* dev_bits) {
    if (!e || !g || !q || !dev_bits) return fail(SGM_E_INVALID_ARG, "sgm_filter: NULL argument");
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    FilterSpec F;
    SGM_TRY(sgm_build_filter_spec(g, q, use_filter, F));
    SGM_CUDA_TRY(sgm_launch_filter(g->G, F, dev_bits, e->stream));
    SGM_CUDA_TRY(cudaStreamSynchronize(e->stream));
    return SGM_OK;
}

// ---------------------------------------------------------------------------
// one run: filter -> roots -> BFS init -> persistent extension
// ---------------------------------------------------------------------------
struct RunResult {
    uint64_t count = 0, hash = 0, rows = 0;
    uint64_t level[SGM_KMAX] = {0};
};

// Defaults, or the caller's options after checking them.
sgm_status sgm_resolve_opts(const sgm_opts* user_opts, sgm_opts& o) {
    sgm_opts_default(&o);
    if (user_opts) {
        if (user_opts->struct_size != sizeof(sgm_opts)) return fail(SGM_E_INVALID_ARG, "sgm_opts.struct_size mismatch");
        o = *user_opts;
    }
    if (o.warps_per_block < 1 || o.warps_per_block > 8) return fail(SGM_E_INVALID_ARG, "warps_per_block must be 1..8");
    if (o.sym_break < 0 || o.sym_break > 2) return fail(SGM_E_INVALID_ARG, "sym_break must be 0, 1 or 2");
    if (o.tau < 1 || o.pool_cap_bytes < 0 || o.split_min < 0 || o.time_cap_s < 0 || o.chunk_words < 1 ||
        o.blocks_per_sm < 0 || o.split_depth < 1 || o.pool_chunk < 0 || o.refine_rounds < 0 ||
        o.exec_model < SGM_EXEC_FINE_BATCH || o.exec_model > SGM_EXEC_COARSE || o.unroll < 1 || o.unroll > 8 ||
        o.steal_mode < 0 || o.steal_mode > 1)
        return fail(SGM_E_INVALID_ARG,
                    "bad tau / pool_cap_bytes / split_min / time_cap_s / chunk_words / refine_rounds / "
                    "exec_model / unroll / steal_mode");
    return SGM_OK;
}

// The per-level plan of one query along its order (Sec. 2.2: backward
// neighbours; injectivity tests only against same-label earlier vertices),
// with symmetry-breaking constraints and the arithmetic last level. The
// automorphisms the leaves expand (hash / enumerate) go to aut_flat
// (aut_n rows of k); P.aut and P.cnt_last are left for the caller.
void sgm_build_plan(const sgm_graph* g, const sgm_query* q, const sgm_opts& o, int32_t kmode, bool full_range,
                    uint32_t* bits, QueryPlan& P, std::vector<int8_t>& aut_flat, int& aut_n) {
    const int k = q->k;
    const DevGraph& G = g->G;
    memset(&P, 0, sizeof(P));
    P.k = k;
    for (int l = 0; l < k; ++l) {
        const int u = q->order[l];
        LevelPlan& lp = P.lv[l];
        lp.u = u;
        lp.bits = bits + (size_t)u * G.words;
        for (int i = 0; i < l; ++i) {
            const int w = q->order[i];
            if ((q->adj[u] >> w) & 1u) lp.bwd |= 1u << i;
            else if (q->label[w] == q->label[u]) lp.inj |= 1u << i;
        }
    }
    // symmetry breaking (stabiliser chain of Aut(Q)): repeatedly take the
    // earliest vertex u of phi that some remaining automorphism moves,
    // require M[u] < M[v] for every other v of its orbit, and keep only the
    // automorphisms fixing u. By default only over the full root range: a
    // root slice is defined on every embedding, not on orbit representatives
    // (sym_break = 2 applies it to slices too, with representative slices).
    aut_flat.clear();
    aut_n = 1;
    // The constraints come from a subgroup H of Aut(Q) acting freely on the
    // embeddings: one embedding per H-orbit is visited and the count is
    // multiplied by |H|. In count mode, when the last query vertex of phi has
    // a single backward neighbour, H is the stabiliser of that vertex, so the
    // last level stays free of constraints and is counted arithmetically
    // (removing a whole level beats removing a factor of |Aut(Q)| / |H|).
    const bool arith_eligible = kmode == SGM_KMODE_COUNT && o.arith_last && k >= 2 && popc32(P.lv[k - 1].bwd) == 1;
    std::vector<const std::vector<int8_t>*> group;
    if ((o.sym_break == 2 || (o.sym_break == 1 && full_range)) && q->aut.size() > 1) {
        const int ulast = q->order[k - 1];
        for (const auto& a : q->aut)
            if (!arith_eligible || a[ulast] == ulast) group.push_back(&a);
    }
    if (group.size() > 1) {
        int pos[SGM_KMAX];
        for (int l = 0; l < k; ++l) pos[q->order[l]] = l;
        std::vector<const std::vector<int8_t>*> alive = group;
        while (alive.size() > 1) {
            int u = -1;
            for (int l = 0; l < k && u < 0; ++l) {
                const int x = q->order[l];
                for (const auto* a : alive)
                    if ((*a)[x] != x) { u = x; break; }
            }
            uint32_t orbit = 0;
            for (const auto* a : alive) orbit |= 1u << (*a)[u];
            for (int v = 0; v < k; ++v)
                if (v != u && ((orbit >> v) & 1u)) P.lv[pos[v]].sb_gt |= 1u << pos[u];
            std::vector<const std::vector<int8_t>*> keep;
            for (const auto* a : alive)
                if ((*a)[u] == u) keep.push_back(a);
            alive.swap(keep);
        }
        aut_n = (int)group.size();
        for (const auto* a : group) aut_flat.insert(aut_flat.end(), a->begin(), a->end());
    } else {
        for (int u = 0; u < k; ++u) aut_flat.push_back((int8_t)u);
    }
    // a backward neighbour that the candidate must outrank offers N+ instead of N
    for (int l = 0; l < k; ++l) P.lv[l].up = P.lv[l].bwd & P.lv[l].sb_gt;
    P.aut_n = aut_n;
    P.arith = (arith_eligible && (P.lv[k - 1].sb_gt | P.lv[k - 1].sb_lt) == 0) ? 1 : 0;
    if (P.arith) {
        P.arith_b = __builtin_ctz(P.lv[k - 1].bwd);
        const int ub = q->order[P.arith_b];
        for (int i = 0; i < k - 1; ++i)
            if (i != P.arith_b && ((q->adj[ub] >> q->order[i]) & 1u)) P.arith_known |= 1u << i;
    }
    P.split_min = o.split_min;
    P.split_depth = o.split_depth;
    P.pool_chunk = o.pool_chunk;
}

static sgm_status run(sgm_engine* e, const sgm_graph* g, sgm_query* q, const sgm_opts* user_opts, int32_t kmode,
                      int64_t root_lo, int64_t root_hi, int32_t* out, uint64_t cap, RunResult& res,
                      const sgm_cgraph* cg = nullptr) {
    sgm_opts o;
    SGM_TRY(sgm_resolve_opts(user_opts, o));
    const bool coarse = o.exec_model == SGM_EXEC_COARSE;
    if (cg) {
        // a search on G': its candidate sets as they are; pool rows are not
        // cut into range tasks (those index plain neighbour lists)
        if (cg->g != g || cg->q != q || cg->k != q->k)
            return fail(SGM_E_INVALID_ARG, "the candidate graph was built for another graph or query");
        if (coarse) return fail(SGM_E_INVALID_ARG, "the coarse model does not search on the candidate graph");
        o.refine_rounds = 0;
        o.pool_chunk = 0;
    }
    if (coarse) {
        // the coarse model of Alg. 1 counts only, over the plain search space
        if (kmode != SGM_KMODE_COUNT) return fail(SGM_E_INVALID_ARG, "the coarse model counts only (no hash, no listing)");
        o.sym_break = 0;
        o.arith_last = 0;
        o.pool_chunk = 0;
    }
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    if (!q->has_order) sgm_greedy_order(q, g, -1);
    SGM_TRY(sgm_check_order(q, q->order));
    const DevGraph& G = g->G;
    const int k = q->k;
    const int64_t n = G.n;
    cudaStream_t s = e->stream;
    memset(&e->stats, 0, sizeof(e->stats));
    uint64_t launches = 0;
    root_lo = std::max<int64_t>(0, root_lo);
    root_hi = std::min<int64_t>(n, root_hi);

    // candidate bitmaps of every query vertex
    FilterSpec F;
    SGM_TRY(sgm_build_filter_spec(g, q, o.use_filter, F));
    SGM_TRY(buf_ensure(e->bits, sizeof(uint32_t) * (size_t)G.words * k));
    uint32_t* bits = (uint32_t*)e->bits.p;
    // plan
    QueryPlan& P = e->h_plan;
    std::vector<int8_t> aut_flat;
    int aut_n = 1;
    const bool full_range = root_lo <= 0 && root_hi >= n;
    sgm_build_plan(g, q, o, kmode, full_range, bits, P, aut_flat, aut_n);
    SGM_TRY(buf_ensure(e->aut, aut_flat.size()));
    SGM_CUDA_TRY(cudaMemcpyAsync(e->aut.p, aut_flat.data(), aut_flat.size(), cudaMemcpyHostToDevice, s));
    P.aut = (const int8_t*)e->aut.p;

    SGM_CUDA_TRY(cudaEventRecord(e->ev[0], s));
    if (cg) {
        SGM_CUDA_TRY(cudaMemcpyAsync(bits, cg->bits.p, sizeof(uint32_t) * (size_t)G.words * k,
                                     cudaMemcpyDeviceToDevice, s));
    } else {
        SGM_CUDA_TRY(sgm_launch_filter(G, F, bits, s));
        ++launches;
    }
    if (o.refine_rounds > 0) SGM_TRY(refine_bits(e, g, q, bits, o.refine_rounds, nullptr, launches));
    if (P.arith) {
        if (!G.labels) {
            // unlabelled: every neighbour y of w has d(y) >= 1 = d_Q(phi[k-1])
            P.cnt_last = const_cast<int32_t*>(G.deg);
        } else {
            // filled by the extension kernel for the images of phi[arith_b] it meets
            SGM_TRY(buf_ensure(e->cnt, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1)));
            SGM_CUDA_TRY(cudaMemsetAsync(e->cnt.p, 0xff, sizeof(int32_t) * (size_t)n, s));
            P.cnt_last = (int32_t*)e->cnt.p;
            P.cnt_lazy = 1;
            // the hub entries up front, by the whole GPU (a hub's list is too long for one warp)
            SGM_TRY(buf_ensure(e->plan, sizeof(QueryPlan)));
            SGM_CUDA_TRY(cudaMemcpyAsync(e->plan.p, &P, sizeof(QueryPlan), cudaMemcpyHostToDevice, s));
            SGM_CUDA_TRY(sgm_launch_cnt_hubs(G, (const QueryPlan*)e->plan.p, nullptr, 1, e->sms, s));
            ++launches;
        }
    }
    SGM_CUDA_TRY(cudaEventRecord(e->ev[1], s));

    // state
    SGM_TRY(buf_ensure(e->state, sizeof(RunState)));
    RunState* st = (RunState*)e->state.p;
    SGM_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(RunState), s));
    SGM_TRY(buf_ensure(e->plan, sizeof(QueryPlan)));
    QueryPlan* dP = (QueryPlan*)e->plan.p;

    // initialization phase (Sec. 4.3): root candidates, then BFS levels until
    // the pool holds at least tau partial matches
    const int64_t nroots_max = std::max<int64_t>(root_hi - root_lo, 0);
    SGM_TRY(buf_ensure(e->poolA, sizeof(int32_t) * (size_t)std::max<int64_t>(nroots_max, 1)));
    int32_t* cur = (int32_t*)e->poolA.p;
    SGM_CUDA_TRY(sgm_launch_roots(P.lv[0].bits, root_lo, root_hi, cur, st, s));
    ++launches;
    unsigned long long counters[2];
    SGM_CUDA_TRY(cudaMemcpyAsync(counters, &st->frontier_n, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t n_cur = (int64_t)counters[0];
    res.level[0] = (uint64_t)n_cur;
    int D = 1;
    const int Dmax = k >= 2 ? k - 1 : 1;
    bool cur_is_A = true;
    while (D < Dmax && n_cur > 0 && n_cur < o.tau) {
        P.D = D;  // only lv[] is read by the BFS kernels
        SGM_CUDA_TRY(cudaMemcpyAsync(dP, &P, sizeof(QueryPlan), cudaMemcpyHostToDevice, s));
        SGM_CUDA_TRY(cudaMemsetAsync(&st->frontier_n, 0, 2 * sizeof(unsigned long long), s));
        SGM_CUDA_TRY(sgm_launch_bfs_bound(G, dP, cur, n_cur, D, st, s));
        ++launches;
        SGM_CUDA_TRY(cudaMemcpyAsync(counters, &st->frontier_n, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        const unsigned long long bound = counters[1];
        const double bytes = (double)bound * (D + 1) * sizeof(int32_t);
        if (bytes > (double)o.pool_cap_bytes) break;
        DevBuf& nb = cur_is_A ? e->poolB : e->poolA;
        SGM_TRY(buf_ensure(nb, (size_t)std::max(bytes, 4.0)));
        int32_t* next = (int32_t*)nb.p;
        SGM_CUDA_TRY(sgm_launch_bfs_expand(G, dP, cur, n_cur, D, next, (int64_t)bound, st, s));
        ++launches;
        SGM_CUDA_TRY(cudaMemcpyAsync(counters, &st->frontier_n, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        n_cur = (int64_t)counters[0];
        cur = next;
        cur_is_A = !cur_is_A;
        res.level[D] = (uint64_t)n_cur;
        ++D;
    }
    P.D = D;
    SGM_CUDA_TRY(cudaMemcpyAsync(dP, &P, sizeof(QueryPlan), cudaMemcpyHostToDevice, s));
    // cut the long local lists of the pool rows into range tasks
    PoolArgs pa;
    memset(&pa, 0, sizeof(pa));
    pa.rows = cur;
    pa.n_short = n_cur;
    // (rows one level short of an arithmetic last level are counted per row)
    if (n_cur > 0 && D < k && o.pool_chunk > 0 && !(P.arith && D == k - 1)) {
        SGM_CUDA_TRY(cudaMemsetAsync(&st->frontier_n, 0, 2 * sizeof(unsigned long long), s));
        SGM_CUDA_TRY(sgm_launch_bfs_bound(G, dP, cur, n_cur, D, st, s));
        ++launches;
        SGM_CUDA_TRY(cudaMemcpyAsync(counters, &st->frontier_n, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        SGM_CUDA_TRY(cudaStreamSynchronize(s));
        const unsigned long long bound = counters[1];
        if (bound > (unsigned long long)o.pool_chunk) {
            const int64_t task_cap = (int64_t)(bound / (unsigned long long)o.pool_chunk) + n_cur;
            SGM_TRY(buf_ensure(e->short_idx, sizeof(int32_t) * (size_t)n_cur));
            SGM_TRY(buf_ensure(e->tasks, sizeof(PoolTask) * (size_t)task_cap));
            SGM_CUDA_TRY(cudaMemsetAsync(&st->frontier_n, 0, 2 * sizeof(unsigned long long), s));
            SGM_CUDA_TRY(sgm_launch_chunk_pool(G, dP, cur, n_cur, D, o.pool_chunk, (int32_t*)e->short_idx.p,
                                               (PoolTask*)e->tasks.p, task_cap, st, s));
            ++launches;
            SGM_CUDA_TRY(cudaMemcpyAsync(counters, &st->frontier_n, 2 * sizeof(unsigned long long),
                                         cudaMemcpyDeviceToHost, s));
            SGM_CUDA_TRY(cudaStreamSynchronize(s));
            pa.short_idx = (const int32_t*)e->short_idx.p;
            pa.n_short = (int64_t)counters[0];
            pa.tasks = (const PoolTask*)e->tasks.p;
            pa.n_tasks = std::min<int64_t>((int64_t)counters[1], task_cap);
        }
        SGM_CUDA_TRY(cudaMemsetAsync(&st->frontier_n, 0, 2 * sizeof(unsigned long long), s));
    }
    SGM_CUDA_TRY(cudaEventRecord(e->ev[2], s));

    // search
    int blocks = 0;
    if (n_cur > 0) {
        if (D >= k) {
            SGM_CUDA_TRY(sgm_launch_pool_leaf(kmode, dP, cur, n_cur, k, st, out, cap, s));
            ++launches;
        } else {
            ExtendLaunch L;
            L.mode = kmode;
            L.gather = G.labels ? 1 : 0;
            L.kcap = k;
            L.warps_per_block = o.warps_per_block;
            L.smem_bytes = sgm_extend_smem_bytes(k, o.warps_per_block, false) +
                           (o.steal_mode == 1 && o.split_min > 0 ? sizeof(BlockMail) : 0);
            int bps = sgm_extend_max_blocks_per_sm(kmode, false, L.gather != 0, o.warps_per_block, L.smem_bytes);
            if (bps < 1) return fail(SGM_E_CUDA, "extension kernel does not fit on an SM (smem %zu)", L.smem_bytes);
            if (o.blocks_per_sm > 0) bps = std::min(bps, o.blocks_per_sm);
            blocks = bps * e->sms;
            L.blocks = blocks;
            QueueTask* queue = nullptr;
            int32_t qcap = 0;
            if (o.split_min > 0) {
                qcap = 4096;
                SGM_TRY(buf_ensure(e->queue, sizeof(QueueTask) * qcap));
                SGM_CUDA_TRY(cudaMemsetAsync(e->queue.p, 0, sizeof(QueueTask) * qcap, s));
                queue = (QueueTask*)e->queue.p;
            }
            const uint64_t cap_ns = o.time_cap_s > 0 ? (uint64_t)(o.time_cap_s * 1e9) : 0;
            pa.one_parent = o.exec_model == SGM_EXEC_FINE_NAIVE ? 1 : 0;
            pa.block_mail = (o.steal_mode == 1 && o.split_min > 0) ? 1 : 0;
            DevGraph Gs = G;
            if (cg) {
                // the G' edge of every (backward level i, level j) of the order
                std::vector<CgEdge>& tab = e->h_cgtab;  // (outlives the asynchronous copy)
                tab.assign(32 * 32, CgEdge{});
                for (int j = 1; j < k; ++j)
                    for (int i = 0; i < j; ++i) {
                        const int ui = q->order[i], uj = q->order[j];
                        const int idx = cg->edge_of[ui][uj];
                        if (idx < 0) continue;
                        CgEdge& t = tab[i * 32 + j];
                        t.ptr = (const int64_t*)cg->ptr.p + cg->ptr_off[idx];
                        t.adj = (const int32_t*)cg->adj.p + cg->adj_off[idx];
                        t.rank = (const int32_t*)cg->rank.p + (size_t)ui * (G.words + 1);
                        t.bits = (const uint32_t*)cg->bits.p + (size_t)ui * G.words;
                    }
                SGM_TRY(buf_ensure(e->cgtab, sizeof(CgEdge) * tab.size()));
                SGM_CUDA_TRY(cudaMemcpyAsync(e->cgtab.p, tab.data(), sizeof(CgEdge) * tab.size(),
                                             cudaMemcpyHostToDevice, s));
                Gs.cg = (const CgEdge*)e->cgtab.p;
            }
            if (coarse) {
                // a stack of k x unroll x d_max int32 per warp, within 16 GiB
                const int32_t warps = sgm_coarse_warps(e->sms, k, o.unroll, g->dmax, (int64_t)16 << 30);
                const size_t bytes = (size_t)warps * k * o.unroll * (size_t)std::max(g->dmax, 1) * sizeof(int32_t);
                SGM_TRY(buf_ensure(e->coarse, bytes));
                SGM_CUDA_TRY(sgm_launch_coarse(G, dP, pa, st, (int32_t*)e->coarse.p, std::max(g->dmax, 1), o.unroll,
                                               warps, cap_ns, s));
                blocks = warps / 8;
                e->stats.stack_bytes = bytes;
            } else {
                SGM_CUDA_TRY(sgm_launch_extend(L, Gs, dP, pa, st, queue, qcap, out, cap, cap_ns, o.work_cap, nullptr, s));
                e->stats.stack_bytes = (uint64_t)L.blocks * L.smem_bytes;
            }
            ++launches;
        }
    }
    SGM_CUDA_TRY(cudaEventRecord(e->ev[3], s));
    SGM_CUDA_TRY(cudaMemcpyAsync(e->h_state, st, sizeof(RunState), cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    const RunState& hs = *e->h_state;

    float ms = 0;
    cudaEventElapsedTime(&ms, e->ev[0], e->ev[1]);
    e->stats.ms_filter = ms;
    cudaEventElapsedTime(&ms, e->ev[1], e->ev[2]);
    e->stats.ms_init = ms;
    cudaEventElapsedTime(&ms, e->ev[2], e->ev[3]);
    e->stats.ms_search = ms;
    e->stats.init_depth = D;
    e->stats.grid_blocks = blocks;
    e->stats.pool_size = n_cur;
    e->stats.cand_checked = hs.cand_checked;
    e->stats.list_elems = hs.list_elems;
    e->stats.search_probes = hs.search_probes;
    e->stats.bitmap_probes = hs.bitmap_probes;
    e->stats.filter_probes = hs.filter_probes;
    e->stats.launches = launches;
    e->stats.task_groups = hs.task_groups;
    e->stats.steals = hs.steals;
    e->stats.idle_lanes = hs.idle_lanes;
    e->stats.scatter_rounds = hs.scatter_rounds;
    e->stats.alg_bytes = hs.alg_bytes;

    if (hs.status)
        return fail(hs.status, hs.status == SGM_E_TIME_CAP   ? "time cap reached: query unsolved"
                               : hs.status == SGM_E_WORK_CAP ? "work cap reached: query unsolved"
                                                             : "device error %d",
                    hs.status);
    if (hs.overflow) return fail(SGM_E_COUNT_OVERFLOW, "embedding count exceeds 2^64 - 1");
    e->stats.aut_size = (uint64_t)aut_n;
    res.rows = hs.rows;
    res.count = kmode == SGM_KMODE_ENUM ? hs.rows : hs.count;
    if (kmode == SGM_KMODE_COUNT && aut_n > 1 &&
        __builtin_mul_overflow(res.count, (uint64_t)aut_n, &res.count))
        return fail(SGM_E_COUNT_OVERFLOW, "embedding count exceeds 2^64 - 1");
    res.hash = hs.hash;
    if (n_cur > 0)
        for (int l = D; l < k; ++l) res.level[l] = hs.level[l];
    if (D >= k && n_cur > 0) res.level[k - 1] = res.count;
    return SGM_OK;
}

static sgm_status count_common(sgm_engine* e, const sgm_graph* g, const sgm_query* q, const sgm_opts* opts,
                               int64_t lo, int64_t hi, uint64_t* count, uint64_t* hash, uint64_t* level_counts) {
    if (!e || !g || !q || !count) return fail(SGM_E_INVALID_ARG, "sgm_count: NULL argument");
    if (g->e != e || q->e != e) return fail(SGM_E_INVALID_ARG, "graph or query belongs to another engine");
    const int mode = (hash || (opts && opts->mode == SGM_MODE_HASH)) ? SGM_KMODE_HASH : SGM_KMODE_COUNT;
    RunResult r;
    SGM_TRY(run(e, g, const_cast<sgm_query*>(q), opts, mode, lo, hi, nullptr, 0, r));
    *count = r.count;
    if (hash) *hash = r.hash;
    if (level_counts) memcpy(level_counts, r.level, sizeof(uint64_t) * q->k);
    return SGM_OK;
}

extern "C" sgm_status sgm_count(sgm_engine* e, const sgm_graph* g, const sgm_query* q, const sgm_opts* opts,
                                uint64_t* count, uint64_t* hash, uint64_t* level_counts) {
    if (!g) return fail(SGM_E_INVALID_ARG, "sgm_count: graph is NULL");
    return count_common(e, g, q, opts, 0, g->G.n, count, hash, level_counts);
}

extern "C" sgm_status sgm_count_cgraph(sgm_engine* e, const sgm_graph* g, sgm_query* q, const sgm_cgraph* c,
                                       const sgm_opts* opts, int64_t root_lo, int64_t root_hi, uint64_t* count,
                                       uint64_t* hash, uint64_t* level_counts) {
    if (!e || !g || !q || !c || !count) return fail(SGM_E_INVALID_ARG, "sgm_count_cgraph: NULL argument");
    if (root_lo > root_hi) return fail(SGM_E_INVALID_ARG, "root_lo > root_hi");
    if (g->e != e || q->e != e || c->e != e) return fail(SGM_E_INVALID_ARG, "objects of another engine");
    const int mode = (hash || (opts && opts->mode == SGM_MODE_HASH)) ? SGM_KMODE_HASH : SGM_KMODE_COUNT;
    RunResult r;
    SGM_TRY(run(e, g, q, opts, mode, root_lo, root_hi, nullptr, 0, r, c));
    *count = r.count;
    if (hash) *hash = r.hash;
    if (level_counts) memcpy(level_counts, r.level, sizeof(uint64_t) * q->k);
    return SGM_OK;
}

extern "C" sgm_status sgm_count_root_range(sgm_engine* e, const sgm_graph* g, const sgm_query* q,
                                           const sgm_opts* opts, int64_t root_lo, int64_t root_hi, uint64_t* count,
                                           uint64_t* hash, uint64_t* level_counts) {
    if (root_lo > root_hi) return fail(SGM_E_INVALID_ARG, "root_lo > root_hi");
    return count_common(e, g, q, opts, root_lo, root_hi, count, hash, level_counts);
}

extern "C" sgm_status sgm_enumerate(sgm_engine* e, const sgm_graph* g, const sgm_query* q, const sgm_opts* opts,
                                    int32_t* dev_out, uint64_t cap, uint64_t* written, uint64_t* total,
                                    uint64_t* hash) {
    if (!e || !g || !q || !written || !total) return fail(SGM_E_INVALID_ARG, "sgm_enumerate: NULL argument");
    if (cap > 0 && !dev_out) return fail(SGM_E_INVALID_ARG, "sgm_enumerate: dev_out is NULL with cap > 0");
    if (g->e != e || q->e != e) return fail(SGM_E_INVALID_ARG, "graph or query belongs to another engine");
    RunResult r;
    SGM_TRY(run(e, g, const_cast<sgm_query*>(q), opts, SGM_KMODE_ENUM, 0, g->G.n, dev_out, cap, r));
    *total = r.rows;
    *written = std::min<uint64_t>(r.rows, cap);
    if (hash) *hash = r.hash;
    return r.rows > cap ? SGM_W_TRUNCATED : SGM_OK;
}

// ---------------------------------------------------------------------------
// host-only views of the query preprocessing (no engine, no device)
// ---------------------------------------------------------------------------
// Builds a host-only query from an edge list (same checks as registration).
static sgm_status host_query(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels, sgm_query& q) {
    if (k < 1 || k > SGM_KMAX || m < 0 || (m > 0 && !edges)) return fail(SGM_E_INVALID_ARG, "bad k = %d or m = %d", k, m);
    q.e = nullptr;
    q.k = k;
    q.m = m;
    memset(q.adj, 0, sizeof(q.adj));
    for (int32_t i = 0; i < m; ++i) {
        const int32_t a = edges[2 * i], b = edges[2 * i + 1];
        if (a < 0 || b < 0 || a >= k || b >= k || a == b || ((q.adj[a] >> b) & 1u))
            return fail(SGM_E_QUERY_INVALID, "query edge %d = (%d, %d) invalid or repeated", i, a, b);
        q.adj[a] |= 1u << b;
        q.adj[b] |= 1u << a;
    }
    for (int32_t u = 0; u < k; ++u) q.label[u] = labels ? labels[u] : 0;
    enumerate_automorphisms(q);
    return SGM_OK;
}

extern "C" sgm_status sgm_query_automorphisms(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                              int32_t* aut_out, int32_t cap, int32_t* n_out) {
    if (!n_out || (cap > 0 && !aut_out)) return fail(SGM_E_INVALID_ARG, "sgm_query_automorphisms: NULL argument");
    sgm_query q;
    SGM_TRY(host_query(k, m, edges, labels, q));
    *n_out = (int32_t)q.aut.size();  // 0: more than the enumeration cap
    for (int32_t a = 0; a < (int32_t)q.aut.size() && a < cap; ++a)
        for (int32_t u = 0; u < k; ++u) aut_out[a * k + u] = q.aut[a][u];
    return SGM_OK;
}

extern "C" sgm_status sgm_query_symmetry_plan(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                              const int32_t* phi, int32_t count_mode, uint32_t* sb_gt_out,
                                              uint32_t* up_out, int32_t* group_out, int32_t group_cap,
                                              int32_t* group_n, int32_t* arith_out) {
    if (!phi || !sb_gt_out || !group_n) return fail(SGM_E_INVALID_ARG, "sgm_query_symmetry_plan: NULL argument");
    sgm_query q;
    SGM_TRY(host_query(k, m, edges, labels, q));
    SGM_TRY(sgm_check_order(&q, phi));
    memcpy(q.order, phi, sizeof(int32_t) * k);
    q.has_order = true;
    sgm_opts o;
    sgm_opts_default(&o);
    sgm_graph g;  // only G.words is read by the plan builder
    memset(&g.G, 0, sizeof(g.G));
    QueryPlan P;
    std::vector<int8_t> aut_flat;
    int aut_n = 1;
    sgm_build_plan(&g, &q, o, count_mode ? SGM_KMODE_COUNT : SGM_KMODE_HASH, true, nullptr, P, aut_flat, aut_n);
    for (int l = 0; l < k; ++l) {
        sb_gt_out[l] = P.lv[l].sb_gt;
        if (up_out) up_out[l] = P.lv[l].up;
    }
    *group_n = aut_n;
    for (int a = 0; a < aut_n && a < group_cap && group_out; ++a)
        for (int u = 0; u < k; ++u) group_out[a * k + u] = aut_flat[(size_t)a * k + u];
    if (arith_out) *arith_out = P.arith;
    return SGM_OK;
}

extern "C" sgm_status sgm_query_greedy_order_host(int32_t k, int32_t m, const int32_t* edges, const int32_t* labels,
                                                  const unsigned long long* label_count, int32_t num_labels,
                                                  int32_t root, int32_t* phi_out) {
    if (!phi_out || (num_labels > 0 && !label_count) || num_labels < 0 || num_labels > 256)
        return fail(SGM_E_INVALID_ARG, "sgm_query_greedy_order_host: bad argument");
    sgm_query q;
    SGM_TRY(host_query(k, m, edges, labels, q));
    if (root >= k) return fail(SGM_E_INVALID_ARG, "root %d outside [0, %d)", root, k);
    uint32_t seen = 1u, frontier = 1u;
    while (frontier) {
        uint32_t next = 0;
        for (int32_t u = 0; u < k; ++u)
            if ((frontier >> u) & 1u) next |= q.adj[u];
        next &= ~seen;
        seen |= next;
        frontier = next;
    }
    if (seen != (k == 32 ? 0xffffffffu : ((1u << k) - 1u)))
        return fail(SGM_E_QUERY_DISCONNECTED, "query graph is not connected");
    sgm_graph g;  // only the label histogram is read by the order rule
    g.label_hist.assign(label_count, label_count + num_labels);
    sgm_greedy_order(&q, &g, root < 0 ? -1 : root);
    memcpy(phi_out, q.order, sizeof(int32_t) * k);
    return SGM_OK;
}
