// batch.cu - many queries in one captured CUDA graph (an addition of this
// library; the paper runs one query at a time). A batch holds, for every
// query, its plan and candidate bitmaps; the run is one CUDA graph captured
// at creation: clear the run states -> candidate filter of every query (one
// launch) -> breadth-first phase of every query with a narrow root range, one
// launch per level over all of them, into a device-managed arena (Sec. 4.3's
// initialisation phase) -> range and 32-row tasks from the final frontiers ->
// one persistent extension kernel per size class of k, the classes on
// parallel branches of the graph, each with its own queue of stealable
// ranges. Queries with wide root ranges start from chunks of root
// candidates instead of a breadth-first pool.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "objects.h"

struct sgm_batch {
    sgm_engine* e = nullptr;
    const sgm_graph* g = nullptr;
    int32_t nq = 0;
    int32_t kmode = SGM_KMODE_COUNT;
    sgm_opts o;
    std::vector<int32_t> perm;      // batch position i holds the caller's query perm[i] (grouped by class)
    std::vector<int32_t> k;         // per batch position
    std::vector<int32_t> aut_n;     // per batch position: |H| the count is multiplied by
    DevBuf bits, bits_off, specs, plans, qst, gst, bfs, cls, sc, rbase, task_base, arena, chunk_q, chunk_w, queue,
        auts, cnt, lazy_idx;
    size_t cnt_bytes = 0;           // count tables of the arithmetic last levels
    RunState* h_qst = nullptr;      // pinned [nq]
    RunState* h_gst = nullptr;      // pinned [ncls]
    BatchBfs* h_bfs0 = nullptr;     // pinned [nq]: breadth-first states at the start of a run
    BatchBfs* h_bfs = nullptr;      // pinned [nq]: ... and at its end (statistics)
    BatchClass* h_cls0 = nullptr;   // pinned [ncls]
    BatchScalars* h_sc0 = nullptr;  // pinned
    BatchScalars* h_sc = nullptr;   // pinned
    cudaStream_t stream = nullptr;  // private stream: capture needs a non-default stream
    cudaStream_t cstream[SGM_BATCH_MAX_CLASSES] = {};  // one graph branch per size class
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t ev_filter = nullptr;  // recorded inside the graph after the filter ...
    cudaEvent_t ev_tasks = nullptr;   // ... and once the tasks are cut, before the persistent launches
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[SGM_BATCH_MAX_CLASSES] = {};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t ncls = 0;
    int32_t blocks = 0;             // resident blocks of all class launches together
    uint64_t launches = 0;          // kernels in the captured graph
};

static void batch_release(sgm_batch* b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    DevBuf* bufs[] = {&b->bits, &b->bits_off, &b->specs, &b->plans,     &b->qst,     &b->gst,
                      &b->bfs,  &b->cls,      &b->sc,    &b->rbase,     &b->task_base, &b->arena,
                      &b->chunk_q, &b->chunk_w, &b->queue, &b->auts, &b->cnt, &b->lazy_idx};
    for (DevBuf* d : bufs) buf_free(*d);
    void* pinned[] = {b->h_qst, b->h_gst, b->h_bfs0, b->h_bfs, b->h_cls0, b->h_sc0, b->h_sc};
    for (void* p : pinned)
        if (p) cudaFreeHost(p);
    for (cudaEvent_t& ev : b->ev)
        if (ev) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->ev_filter) cudaEventDestroy(b->ev_filter);
    if (b->ev_tasks) cudaEventDestroy(b->ev_tasks);
    for (cudaEvent_t& ev : b->join)
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t& cs : b->cstream)
        if (cs) cudaStreamDestroy(cs);
    if (b->stream) cudaStreamDestroy(b->stream);
}

// Size class of a query with k vertices: its per-warp stack is laid out for
// at most 8, 16, 24 or 32 levels.
static int size_class(int k) { return std::min(3, (std::max(k, 1) - 1) / 8); }

template <class T>
static sgm_status pinned_alloc(T** p, size_t n) {
    SGM_CUDA_TRY(cudaMallocHost((void**)p, sizeof(T) * std::max<size_t>(n, 1)));
    memset(*p, 0, sizeof(T) * std::max<size_t>(n, 1));
    return SGM_OK;
}

static sgm_status batch_build(sgm_batch* b, sgm_query* const* qs_in, const int64_t* ranges_in) {
    sgm_engine* e = b->e;
    const sgm_graph* g = b->g;
    const DevGraph& G = g->G;
    const int nq = b->nq;
    const sgm_opts& o = b->o;
    SGM_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : b->ev) SGM_CUDA_TRY(cudaEventCreate(&ev));
    SGM_CUDA_TRY(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
    SGM_CUDA_TRY(cudaEventCreate(&b->ev_filter));
    SGM_CUDA_TRY(cudaEventCreate(&b->ev_tasks));
    // order the queries by size class (stable), so that a class is a
    // contiguous range of batch positions
    b->perm.resize(nq);
    for (int i = 0; i < nq; ++i) b->perm[i] = i;
    std::stable_sort(b->perm.begin(), b->perm.end(),
                     [&](int x, int y) { return size_class(qs_in[x]->k) < size_class(qs_in[y]->k); });
    std::vector<sgm_query*> qs(nq);
    std::vector<int64_t> root_lo(nq, 0), root_hi(nq, G.n);
    for (int i = 0; i < nq; ++i) {
        qs[i] = qs_in[b->perm[i]];
        if (ranges_in) {
            root_lo[i] = std::max<int64_t>(0, ranges_in[2 * b->perm[i]]);
            root_hi[i] = std::min<int64_t>(G.n, ranges_in[2 * b->perm[i] + 1]);
            if (root_lo[i] > root_hi[i])
                return sgm_fail(SGM_E_INVALID_ARG, "query %d: root range [%lld, %lld)", b->perm[i],
                                (long long)root_lo[i], (long long)root_hi[i]);
        }
    }
    // size classes
    std::vector<BatchClass> cls;
    std::vector<int32_t> cls_of(nq);
    for (int i = 0; i < nq; ++i) {
        const int c = size_class(qs[i]->k);
        if (cls.empty() || size_class(qs[cls.back().q0]->k) != c) {
            BatchClass C;
            memset(&C, 0, sizeof(C));
            C.q0 = i;
            cls.push_back(C);
        }
        cls.back().q1 = i + 1;
        cls.back().kcap = std::max(cls.back().kcap, qs[i]->k);
        cls_of[i] = (int32_t)cls.size() - 1;
    }
    b->ncls = (int32_t)cls.size();
    // bitmaps: query i's k_i bitmaps start at word bits_off[i]
    std::vector<int64_t> off(nq + 1, 0);
    for (int i = 0; i < nq; ++i) off[i + 1] = off[i] + (int64_t)qs[i]->k * G.words;
    SGM_TRY(buf_ensure(b->bits, sizeof(uint32_t) * (size_t)std::max<int64_t>(off[nq], 1)));
    uint32_t* bits = (uint32_t*)b->bits.p;
    // plans, filter specs and automorphism tables
    std::vector<QueryPlan> plans(nq);
    std::vector<FilterSpec> specs(nq);
    std::vector<std::vector<int8_t>> auts(nq);
    size_t aut_bytes = 0;
    b->k.resize(nq);
    b->aut_n.resize(nq);
    std::vector<int32_t> lazy;  // queries with a count table of their own
    for (int i = 0; i < nq; ++i) {
        sgm_query* q = qs[i];
        if (!q->has_order) sgm_greedy_order(q, g, -1);
        SGM_TRY(sgm_check_order(q, q->order));
        SGM_TRY(sgm_build_filter_spec(g, q, o.use_filter, specs[i]));
        int an = 1;
        sgm_build_plan(g, q, o, b->kmode, root_lo[i] == 0 && root_hi[i] == G.n, bits + off[i], plans[i], auts[i],
                       an);
        plans[i].D = 1;
        plans[i].root_lo = (int32_t)root_lo[i];
        plans[i].root_hi = (int32_t)root_hi[i];
        // an arithmetic last level reads the degrees (unlabelled graphs) or
        // a count table of its own, filled on demand during the run
        if (plans[i].arith && !G.labels) plans[i].cnt_last = const_cast<int32_t*>(G.deg);
        if (plans[i].arith && G.labels) {
            plans[i].cnt_lazy = 1;
            lazy.push_back(i);
        }
        b->k[i] = q->k;
        b->aut_n[i] = an;
        aut_bytes += auts[i].size();
    }
    SGM_TRY(buf_ensure(b->auts, std::max<size_t>(aut_bytes, 1)));
    {
        std::vector<int8_t> flat;
        flat.reserve(aut_bytes);
        size_t o8 = 0;
        for (int i = 0; i < nq; ++i) {
            plans[i].aut = (const int8_t*)b->auts.p + o8;
            flat.insert(flat.end(), auts[i].begin(), auts[i].end());
            o8 += auts[i].size();
        }
        if (!flat.empty()) SGM_CUDA_TRY(cudaMemcpy(b->auts.p, flat.data(), flat.size(), cudaMemcpyHostToDevice));
    }
    // count tables of the arithmetic last levels: n int32 per query, -1 until filled
    b->cnt_bytes = sizeof(int32_t) * (size_t)G.n * lazy.size();
    SGM_TRY(buf_ensure(b->cnt, std::max<size_t>(b->cnt_bytes, 4)));
    for (size_t j = 0; j < lazy.size(); ++j) plans[lazy[j]].cnt_last = (int32_t*)b->cnt.p + (size_t)G.n * j;
    SGM_TRY(buf_ensure(b->lazy_idx, sizeof(int32_t) * std::max<size_t>(lazy.size(), 1)));
    if (!lazy.empty())
        SGM_CUDA_TRY(cudaMemcpy(b->lazy_idx.p, lazy.data(), sizeof(int32_t) * lazy.size(), cudaMemcpyHostToDevice));
    SGM_TRY(buf_ensure(b->plans, sizeof(QueryPlan) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->specs, sizeof(FilterSpec) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->bits_off, sizeof(int64_t) * std::max(nq, 1)));
    if (nq) {
        SGM_CUDA_TRY(cudaMemcpy(b->plans.p, plans.data(), sizeof(QueryPlan) * nq, cudaMemcpyHostToDevice));
        SGM_CUDA_TRY(cudaMemcpy(b->specs.p, specs.data(), sizeof(FilterSpec) * nq, cudaMemcpyHostToDevice));
        SGM_CUDA_TRY(cudaMemcpy(b->bits_off.p, off.data(), sizeof(int64_t) * nq, cudaMemcpyHostToDevice));
    }
    // The arena of the breadth-first phase (int32 elements; 4 x
    // opts.pool_cap_bytes, at most max(256 MiB, 16 MiB per query)): the root lists
    // are reserved here, at its start; every later level is handed out on the
    // device. A query expands breadth-first when k >= 2 and its root range
    // has at most 2^20 vertices and fits the first quarter of the arena;
    // the others start from chunks of root candidates.
    const uint64_t arena_elems = std::max<uint64_t>(
        std::min<uint64_t>((uint64_t)o.pool_cap_bytes * 4 / sizeof(int32_t),
                           std::max<uint64_t>((uint64_t)nq << 22, (uint64_t)1 << 26)),
        1u << 20);
    SGM_TRY(pinned_alloc(&b->h_bfs0, nq));
    SGM_TRY(pinned_alloc(&b->h_bfs, nq));
    uint64_t used0 = 0;
    int n_bfs = 0;
    int32_t max_depth = 1;
    int64_t max_range = 1;
    for (int i = 0; i < nq; ++i) {
        const int64_t w = root_hi[i] - root_lo[i];
        if (qs[i]->k >= 2 && w > 0 && w <= ((int64_t)1 << 20) && used0 + (uint64_t)w <= arena_elems / 4) {
            BatchBfs& z = b->h_bfs0[i];
            z.off = z.next_off = (int64_t)used0;
            z.active = 1;
            used0 += (uint64_t)w;
            ++n_bfs;
            max_depth = std::max(max_depth, qs[i]->k - 1);
            max_range = std::max(max_range, w);
        }
        b->h_bfs0[i].cls = cls_of[i];
    }
    const unsigned long long tau_q = (unsigned long long)std::max<int64_t>(256, o.tau / std::max(n_bfs, 1));
    for (int i = 0; i < nq; ++i) b->h_bfs0[i].tau = tau_q;
    SGM_TRY(buf_ensure(b->arena, sizeof(int32_t) * (size_t)arena_elems));
    SGM_TRY(buf_ensure(b->bfs, sizeof(BatchBfs) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->rbase, sizeof(unsigned long long) * (size_t)(nq + 1)));
    SGM_TRY(buf_ensure(b->task_base, sizeof(unsigned long long) * (size_t)(nq + 1)));
    SGM_TRY(buf_ensure(b->sc, sizeof(BatchScalars)));
    SGM_TRY(pinned_alloc(&b->h_sc0, 1));
    SGM_TRY(pinned_alloc(&b->h_sc, 1));
    b->h_sc0->arena_used = used0;
    // root chunks: chunk_words bitmap words of phi[0] candidates each, over
    // the words the query's root range touches, contiguous per class
    std::vector<int32_t> cq;
    std::vector<int64_t> cw;
    std::vector<int64_t> cls_ch(b->ncls + 1, 0);
    for (int c = 0; c < b->ncls; ++c) {
        for (int i = cls[c].q0; i < cls[c].q1; ++i) {
            if (b->h_bfs0[i].active || root_lo[i] >= root_hi[i]) continue;
            const int64_t w0 = root_lo[i] / 32, w1 = (root_hi[i] + 31) / 32;
            for (int64_t w = w0; w < w1; w += o.chunk_words) {
                cq.push_back(i);
                cw.push_back(w);
            }
        }
        cls_ch[c + 1] = (int64_t)cq.size();
    }
    SGM_TRY(buf_ensure(b->chunk_q, sizeof(int32_t) * std::max<size_t>(cq.size(), 1)));
    SGM_TRY(buf_ensure(b->chunk_w, sizeof(int64_t) * std::max<size_t>(cw.size(), 1)));
    if (!cq.empty()) {
        SGM_CUDA_TRY(cudaMemcpy(b->chunk_q.p, cq.data(), sizeof(int32_t) * cq.size(), cudaMemcpyHostToDevice));
        SGM_CUDA_TRY(cudaMemcpy(b->chunk_w.p, cw.data(), sizeof(int64_t) * cw.size(), cudaMemcpyHostToDevice));
    }
    // classes, run states and work queues (one per class)
    SGM_TRY(pinned_alloc(&b->h_cls0, b->ncls));
    for (int c = 0; c < b->ncls; ++c) b->h_cls0[c] = cls[c];
    SGM_TRY(buf_ensure(b->cls, sizeof(BatchClass) * std::max(b->ncls, 1)));
    SGM_TRY(buf_ensure(b->qst, sizeof(RunState) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->gst, sizeof(RunState) * std::max(b->ncls, 1)));
    SGM_TRY(pinned_alloc(&b->h_qst, nq));
    SGM_TRY(pinned_alloc(&b->h_gst, b->ncls));
    const int32_t qcap = o.split_min > 0 ? 4096 : 0;
    if (qcap) SGM_TRY(buf_ensure(b->queue, sizeof(QueueTask) * (size_t)qcap * b->ncls));
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.plans = (const QueryPlan*)b->plans.p;
    B.qst = (RunState*)b->qst.p;
    B.bfs = (BatchBfs*)b->bfs.p;
    B.cls = (BatchClass*)b->cls.p;
    B.sc = (BatchScalars*)b->sc.p;
    B.rbase = (unsigned long long*)b->rbase.p;
    B.task_base = (unsigned long long*)b->task_base.p;
    B.arena = (int32_t*)b->arena.p;
    B.arena_cap = arena_elems;
    B.words = G.words;
    B.chunk_words = o.chunk_words;
    B.nq = nq;
    const uint64_t cap_ns = o.time_cap_s > 0 ? (uint64_t)(o.time_cap_s * 1e9) : 0;
    const int32_t root_blocks = (int32_t)std::max<int64_t>(1, std::min<int64_t>(256, (max_range + 2047) / 2048));
    // capture the whole run once: clear -> filter -> breadth-first phase ->
    // tasks -> one persistent launch per size class on its own branch
    cudaStream_t s = b->stream;
    for (int c = 0; c < b->ncls; ++c) {
        SGM_CUDA_TRY(cudaStreamCreateWithFlags(&b->cstream[c], cudaStreamNonBlocking));
        SGM_CUDA_TRY(cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming));
    }
    std::vector<ExtendLaunch> L(b->ncls);
    b->blocks = 0;
    for (int c = 0; c < b->ncls; ++c) {
        L[c].mode = b->kmode;
        L[c].gather = G.labels ? 1 : 0;
        L[c].kcap = std::max(cls[c].kcap, 1);
        L[c].warps_per_block = o.warps_per_block;
        L[c].smem_bytes = sgm_extend_smem_bytes(L[c].kcap, o.warps_per_block, true);
        int bps = sgm_extend_max_blocks_per_sm(b->kmode, true, L[c].gather != 0, o.warps_per_block,
                                               L[c].smem_bytes);
        if (bps < 1)
            return sgm_fail(SGM_E_CUDA, "batched extension kernel does not fit on an SM (smem %zu)", L[c].smem_bytes);
        if (o.blocks_per_sm > 0) bps = std::min(bps, o.blocks_per_sm);
        L[c].blocks = bps * e->sms;
        b->blocks += L[c].blocks;
    }
    SGM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    uint64_t launches = 0;
    cudaError_t err = cudaMemsetAsync(b->qst.p, 0, sizeof(RunState) * nq, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(b->gst.p, 0, sizeof(RunState) * b->ncls, s);
    if (err == cudaSuccess && qcap) err = cudaMemsetAsync(b->queue.p, 0, sizeof(QueueTask) * qcap * b->ncls, s);
    if (err == cudaSuccess && b->cnt_bytes) err = cudaMemsetAsync(b->cnt.p, 0xff, b->cnt_bytes, s);
    if (err == cudaSuccess && nq)
        err = cudaMemcpyAsync(b->bfs.p, b->h_bfs0, sizeof(BatchBfs) * nq, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && b->ncls)
        err = cudaMemcpyAsync(b->cls.p, b->h_cls0, sizeof(BatchClass) * b->ncls, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(b->sc.p, b->h_sc0, sizeof(BatchScalars), cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess && nq) {
        err = sgm_launch_batch_filter(G, (const FilterSpec*)b->specs.p, (const int64_t*)b->bits_off.p, bits, nq,
                                      e->sms, s, (size_t)off[nq]);
        ++launches;
    }
    if (err == cudaSuccess && !lazy.empty() && G.hubs > 0) {
        // the hub entries of the count tables, by the whole GPU
        err = sgm_launch_cnt_hubs(G, (const QueryPlan*)b->plans.p, (const int32_t*)b->lazy_idx.p,
                                  (int32_t)lazy.size(), e->sms, s);
        ++launches;
    }
    // event nodes of the graph: the run's filter / initialisation / search split
    if (err == cudaSuccess) err = cudaEventRecordWithFlags(b->ev_filter, s, cudaEventRecordExternal);
    if (err == cudaSuccess && n_bfs > 0) err = sgm_launch_batch_bfs(G, B, max_depth, root_blocks, e->sms, s, &launches);
    if (err == cudaSuccess && n_bfs > 0) err = sgm_launch_batch_tasks(G, B, b->ncls, e->sms, s, &launches);
    if (err == cudaSuccess) err = cudaEventRecordWithFlags(b->ev_tasks, s, cudaEventRecordExternal);
    if (err == cudaSuccess) err = cudaEventRecord(b->fork, s);
    for (int c = 0; c < b->ncls && err == cudaSuccess; ++c) {
        cudaStream_t cs = b->cstream[c];
        err = cudaStreamWaitEvent(cs, b->fork, 0);
        BatchArgs Bc = B;
        Bc.cls_id = c;
        Bc.plan_bytes = sgm_batch_plan_bytes(L[c].kcap);
        Bc.chunk_q = (const int32_t*)b->chunk_q.p + cls_ch[c];
        Bc.chunk_w = (const int64_t*)b->chunk_w.p + cls_ch[c];
        Bc.nchunks = cls_ch[c + 1] - cls_ch[c];
        PoolArgs none;
        memset(&none, 0, sizeof(none));
        if (err == cudaSuccess)
            err = sgm_launch_extend(L[c], G, nullptr, none, (RunState*)b->gst.p + c,
                                    qcap ? (QueueTask*)b->queue.p + (size_t)qcap * c : nullptr, qcap, nullptr, 0,
                                    cap_ns, o.work_cap, &Bc, cs);
        ++launches;
        if (err == cudaSuccess) err = cudaEventRecord(b->join[c], cs);
        if (err == cudaSuccess) err = cudaStreamWaitEvent(s, b->join[c], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(s, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return sgm_fail(SGM_E_CUDA, "batch capture: %s", cudaGetErrorString(err != cudaSuccess ? err : end));
    }
    b->graph = graph;
    SGM_CUDA_TRY(cudaGraphInstantiate(&b->exec, graph, 0));
    b->launches = launches;
    return SGM_OK;
}

extern "C" sgm_status sgm_batch_create(sgm_engine* e, const sgm_graph* g, sgm_query* const* qs, int32_t nq,
                                       const int64_t* root_ranges, const sgm_opts* opts, int32_t want_hash,
                                       sgm_batch** out) {
    if (!e || !g || !out || (nq > 0 && !qs) || nq < 0) return sgm_fail(SGM_E_INVALID_ARG, "sgm_batch_create: bad argument");
    if (nq > 65535) return sgm_fail(SGM_E_INVALID_ARG, "a batch holds at most 65535 queries (%d given)", nq);
    *out = nullptr;
    if (g->e != e) return sgm_fail(SGM_E_INVALID_ARG, "graph belongs to another engine");
    for (int i = 0; i < nq; ++i)
        if (!qs[i] || qs[i]->e != e) return sgm_fail(SGM_E_INVALID_ARG, "query %d is NULL or of another engine", i);
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    sgm_batch* b = new (std::nothrow) sgm_batch();
    if (!b) return sgm_fail(SGM_E_OOM, "host allocation failed");
    b->e = e;
    b->g = g;
    b->nq = nq;
    b->kmode = want_hash ? SGM_KMODE_HASH : SGM_KMODE_COUNT;
    sgm_status st = sgm_resolve_opts(opts, b->o);
    if (st == SGM_OK && b->o.refine_rounds != 0)
        st = sgm_fail(SGM_E_INVALID_ARG, "refine_rounds is not supported in batched runs");
    if (st == SGM_OK && (b->o.exec_model != SGM_EXEC_FINE_BATCH || b->o.steal_mode != 0))
        st = sgm_fail(SGM_E_INVALID_ARG, "batched runs use the fine-grained batched model and steal_mode 0 only");
    if (st == SGM_OK) st = batch_build(b, qs, root_ranges);
    if (st < 0) {
        batch_release(b);
        delete b;
        return st;
    }
    *out = b;
    return SGM_OK;
}

extern "C" sgm_status sgm_batch_free(sgm_batch* b) {
    if (!b) return SGM_OK;
    cudaSetDevice(b->e->device);
    batch_release(b);
    delete b;
    return SGM_OK;
}

extern "C" sgm_status sgm_batch_run(sgm_batch* b, uint64_t* counts, uint64_t* hashes, sgm_status* statuses,
                                    double* ms) {
    if (!b || (b->nq > 0 && !counts)) return sgm_fail(SGM_E_INVALID_ARG, "sgm_batch_run: bad argument");
    sgm_engine* e = b->e;
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    // order after the caller's work on the engine stream, run on the private one
    SGM_CUDA_TRY(cudaEventRecord(b->ev[0], e->stream));
    SGM_CUDA_TRY(cudaStreamWaitEvent(b->stream, b->ev[0], 0));
    SGM_CUDA_TRY(cudaEventRecord(b->ev[1], b->stream));
    SGM_CUDA_TRY(cudaGraphLaunch(b->exec, b->stream));
    SGM_CUDA_TRY(cudaEventRecord(b->ev[2], b->stream));
    if (b->nq) {
        SGM_CUDA_TRY(cudaMemcpyAsync(b->h_qst, b->qst.p, sizeof(RunState) * b->nq, cudaMemcpyDeviceToHost, b->stream));
        SGM_CUDA_TRY(cudaMemcpyAsync(b->h_bfs, b->bfs.p, sizeof(BatchBfs) * b->nq, cudaMemcpyDeviceToHost, b->stream));
    }
    if (b->ncls)
        SGM_CUDA_TRY(cudaMemcpyAsync(b->h_gst, b->gst.p, sizeof(RunState) * b->ncls, cudaMemcpyDeviceToHost, b->stream));
    SGM_CUDA_TRY(cudaMemcpyAsync(b->h_sc, b->sc.p, sizeof(BatchScalars), cudaMemcpyDeviceToHost, b->stream));
    // the caller's stream waits for the run (results on the host come with the sync below)
    SGM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    float t = 0.f, tf = 0.f, ti = 0.f, ts = 0.f;
    cudaEventElapsedTime(&t, b->ev[1], b->ev[2]);
    cudaEventElapsedTime(&tf, b->ev[1], b->ev_filter);
    cudaEventElapsedTime(&ti, b->ev_filter, b->ev_tasks);
    cudaEventElapsedTime(&ts, b->ev_tasks, b->ev[2]);
    cudaGetLastError();
    if (ms) *ms = t;
    memset(&e->stats, 0, sizeof(e->stats));
    e->stats.ms_filter = tf;  // clear + candidate filter
    e->stats.ms_init = ti;    // breadth-first phase + tasks
    e->stats.ms_search = ts;  // the persistent launches of every size class
    e->stats.grid_blocks = b->blocks;
    e->stats.launches = b->launches;
    int32_t status = 0;
    for (int c = 0; c < b->ncls; ++c) {
        const RunState& gs = b->h_gst[c];
        if (gs.status && !status) status = gs.status;
        e->stats.cand_checked += gs.cand_checked;
        e->stats.list_elems += gs.list_elems;
        e->stats.search_probes += gs.search_probes;
        e->stats.bitmap_probes += gs.bitmap_probes;
        e->stats.filter_probes += gs.filter_probes;
        e->stats.task_groups += gs.task_groups;
        e->stats.steals += gs.steals;
        e->stats.idle_lanes += gs.idle_lanes;
        e->stats.scatter_rounds += gs.scatter_rounds;
        e->stats.alg_bytes += gs.alg_bytes;
    }
    for (int i = 0; i < b->nq; ++i) {
        e->stats.pool_size += (int64_t)b->h_bfs[i].n;
        e->stats.init_depth = std::max(e->stats.init_depth, b->h_bfs[i].depth);
    }
    sgm_status worst = SGM_OK;
    for (int i = 0; i < b->nq; ++i) {
        const RunState& q = b->h_qst[i];
        const int dst = b->perm[i];
        sgm_status st = status ? status : q.status;  // a stop of the whole run, else the query's own
        uint64_t c = q.count;
        if (!st && q.overflow) st = SGM_E_COUNT_OVERFLOW;
        if (!st && b->kmode == SGM_KMODE_COUNT && b->aut_n[i] > 1 &&
            __builtin_mul_overflow(c, (uint64_t)b->aut_n[i], &c))
            st = SGM_E_COUNT_OVERFLOW;
        counts[dst] = st ? 0 : c;
        if (hashes) hashes[dst] = st ? 0 : q.hash;
        if (statuses) statuses[dst] = st;
        if (st && !worst) worst = st;
    }
    if (worst)
        return sgm_fail(worst, status == SGM_E_TIME_CAP ? "time cap reached: batch unsolved"
                               : worst == SGM_E_WORK_CAP ? "work cap reached by at least one query (unsolved)"
                                                         : "a query of the batch failed (%d)",
                        worst);
    return SGM_OK;
}

extern "C" sgm_status sgm_batch_query_work(const sgm_batch* b, uint64_t* work) {
    if (!b || (b->nq > 0 && !work)) return sgm_fail(SGM_E_INVALID_ARG, "sgm_batch_query_work: bad argument");
    for (int i = 0; i < b->nq; ++i) work[b->perm[i]] = b->h_qst[i].work;
    return SGM_OK;
}

extern "C" sgm_status sgm_count_batch(sgm_engine* e, const sgm_graph* g, sgm_query* const* qs, int32_t nq,
                                      const int64_t* root_ranges, const sgm_opts* opts, uint64_t* counts,
                                      uint64_t* hashes, sgm_status* statuses) {
    sgm_batch* b = nullptr;
    SGM_TRY(sgm_batch_create(e, g, qs, nq, root_ranges, opts, hashes != nullptr, &b));
    const sgm_status st = sgm_batch_run(b, counts, hashes, statuses, nullptr);
    const char* keep = sgm_last_error();
    char msg[512];
    strncpy(msg, keep, sizeof(msg) - 1);
    msg[sizeof(msg) - 1] = 0;
    sgm_batch_free(b);
    if (st < 0) return sgm_fail(st, "%s", msg);
    return st;
}
