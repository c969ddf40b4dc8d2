// batch.cu - many queries in one persistent launch (an addition of this
// library; the paper runs one query at a time). A batch holds, for every
// query, its plan and candidate bitmaps; the run is one CUDA graph captured
// at creation: clear the run states -> candidate filter of every query ->
// breadth-first pools of the queries with narrow root ranges -> one
// persistent extension kernel whose initial tasks are 32-row slices of those
// pools and chunks of the other queries' root candidates, sharing one work
// queue of stealable ranges.
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
    std::vector<int32_t> k;         // per query
    std::vector<int32_t> aut_n;     // per query: |H| the count is multiplied by
    DevBuf bits, plans, qst, gst, chunk_q, chunk_w, queue, auts, bfs, fr0, fr1, task_base;
    RunState* h_qst = nullptr;      // pinned [nq]
    RunState* h_gst = nullptr;      // pinned
    BatchBfs* h_bfs0 = nullptr;     // pinned [nq]: breadth-first states at the start of a run
    cudaStream_t stream = nullptr;  // private stream: capture needs a non-default stream
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t nchunks = 0;
    int32_t blocks = 0;
    int32_t kcap = 0;
    uint64_t launches = 0;          // kernels in the captured graph
};

static void batch_release(sgm_batch* b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    DevBuf* bufs[] = {&b->bits, &b->plans, &b->qst, &b->gst, &b->chunk_q, &b->chunk_w, &b->queue,
                      &b->auts, &b->bfs,  &b->fr0,   &b->fr1, &b->task_base};
    for (DevBuf* d : bufs) buf_free(*d);
    if (b->h_bfs0) cudaFreeHost(b->h_bfs0);
    if (b->h_qst) cudaFreeHost(b->h_qst);
    if (b->h_gst) cudaFreeHost(b->h_gst);
    for (cudaEvent_t& ev : b->ev)
        if (ev) cudaEventDestroy(ev);
    if (b->stream) cudaStreamDestroy(b->stream);
}

static sgm_status batch_build(sgm_batch* b, sgm_query* const* qs, const int64_t* ranges, int32_t want_hash) {
    sgm_engine* e = b->e;
    const sgm_graph* g = b->g;
    const DevGraph& G = g->G;
    const int nq = b->nq;
    const sgm_opts& o = b->o;
    SGM_CUDA_TRY(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    for (cudaEvent_t& ev : b->ev) SGM_CUDA_TRY(cudaEventCreate(&ev));
    // bitmaps: query i's k_i bitmaps start at word offset off[i]
    std::vector<size_t> off(nq + 1, 0);
    for (int i = 0; i < nq; ++i) off[i + 1] = off[i] + (size_t)qs[i]->k * (size_t)G.words;
    SGM_TRY(buf_ensure(b->bits, sizeof(uint32_t) * std::max<size_t>(off[nq], 1)));
    uint32_t* bits = (uint32_t*)b->bits.p;
    // plans and automorphism tables
    std::vector<QueryPlan> plans(nq);
    std::vector<FilterSpec> specs(nq);
    std::vector<std::vector<int8_t>> auts(nq);
    size_t aut_bytes = 0;
    std::vector<int64_t> root_lo(nq), root_hi(nq);
    b->k.resize(nq);
    b->aut_n.resize(nq);
    for (int i = 0; i < nq; ++i) {
        sgm_query* q = qs[i];
        if (!q->has_order) sgm_greedy_order(q, g, -1);
        SGM_TRY(sgm_check_order(q, q->order));
        SGM_TRY(sgm_build_filter_spec(g, q, o.use_filter, specs[i]));
        // batched runs start from root candidates (no initial pool), and count
        // the last level arithmetically only where its counts are the degrees
        // (unlabelled graphs): no per-query count table is built
        sgm_opts oq = o;
        if (G.labels) oq.arith_last = 0;
        int64_t lo = 0, hi = G.n;
        if (ranges) {
            lo = std::max<int64_t>(0, ranges[2 * i]);
            hi = std::min<int64_t>(G.n, ranges[2 * i + 1]);
            if (lo > hi) return sgm_fail(SGM_E_INVALID_ARG, "query %d: root range [%lld, %lld)", i, (long long)lo,
                                         (long long)hi);
        }
        int an = 1;
        sgm_build_plan(g, q, oq, b->kmode, lo == 0 && hi == G.n, bits + off[i], plans[i], auts[i], an);
        plans[i].D = 1;
        // ranges may be offered at every level, with a threshold that doubles
        // per level towards the leaves (tasks of queries without a
        // breadth-first pool start at the root level)
        plans[i].split_depth = SGM_KMAX;
        plans[i].root_lo = (int32_t)lo;
        plans[i].root_hi = (int32_t)hi;
        if (plans[i].arith) plans[i].cnt_last = G.deg;
        root_lo[i] = lo;
        root_hi[i] = hi;
        b->k[i] = q->k;
        b->aut_n[i] = an;
        b->kcap = std::max(b->kcap, q->k);
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
    SGM_TRY(buf_ensure(b->plans, sizeof(QueryPlan) * std::max(nq, 1)));
    if (nq) SGM_CUDA_TRY(cudaMemcpy(b->plans.p, plans.data(), sizeof(QueryPlan) * nq, cudaMemcpyHostToDevice));
    // Breadth-first pools for the queries whose root range fits a frontier
    // region (anchored queries and other narrow ranges): each region holds
    // cap rows of up to k levels; expansion stops at tau rows.
    const int64_t kRowsTotal = (int64_t)1 << 22, kTauTotal = (int64_t)1 << 20;
    std::vector<char> use_bfs(nq, 0);
    int n_bfs = 0;
    int32_t max_depth = 1;
    for (int i = 0; i < nq; ++i)
        if (qs[i]->k >= 2 && root_hi[i] - root_lo[i] <= kRowsTotal / 64) {
            use_bfs[i] = 1;
            ++n_bfs;
        }
    const int64_t cap_rows = std::max<int64_t>(4096, kRowsTotal / std::max(n_bfs, 1));
    const unsigned long long tau = (unsigned long long)std::max<int64_t>(256, kTauTotal / std::max(n_bfs, 1));
    SGM_CUDA_TRY(cudaMallocHost((void**)&b->h_bfs0, sizeof(BatchBfs) * std::max(nq, 1)));
    int64_t fr_elems = 0;
    for (int i = 0; i < nq; ++i) {
        BatchBfs& z = b->h_bfs0[i];
        memset(&z, 0, sizeof(z));
        if (use_bfs[i] && root_hi[i] - root_lo[i] > cap_rows) use_bfs[i] = 0;
        if (!use_bfs[i]) continue;
        z.off = fr_elems;
        z.cap_rows = cap_rows;
        z.tau = tau;
        z.depth = 1;
        fr_elems += cap_rows * qs[i]->k;
        max_depth = std::max(max_depth, qs[i]->k - 1);
    }
    SGM_TRY(buf_ensure(b->bfs, sizeof(BatchBfs) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->fr0, sizeof(int32_t) * (size_t)std::max<int64_t>(fr_elems, 1)));
    SGM_TRY(buf_ensure(b->fr1, sizeof(int32_t) * (size_t)std::max<int64_t>(fr_elems, 1)));
    SGM_TRY(buf_ensure(b->task_base, sizeof(unsigned long long) * (size_t)(nq + 1)));
    // initial tasks of the other queries: chunks of chunk_words bitmap words of
    // each query's phi[0] candidates, over the words its root range touches
    {
        std::vector<int32_t> cq;
        std::vector<int64_t> cw;
        for (int i = 0; i < nq; ++i) {
            if (use_bfs[i] || root_lo[i] >= root_hi[i]) continue;
            const int64_t w0 = root_lo[i] / 32, w1 = (root_hi[i] + 31) / 32;
            for (int64_t w = w0; w < w1; w += o.chunk_words) {
                cq.push_back(i);
                cw.push_back(w);
            }
        }
        b->nchunks = (int64_t)cq.size();
        SGM_TRY(buf_ensure(b->chunk_q, sizeof(int32_t) * std::max<int64_t>(b->nchunks, 1)));
        SGM_TRY(buf_ensure(b->chunk_w, sizeof(int64_t) * std::max<int64_t>(b->nchunks, 1)));
        if (b->nchunks) {
            SGM_CUDA_TRY(cudaMemcpy(b->chunk_q.p, cq.data(), sizeof(int32_t) * b->nchunks, cudaMemcpyHostToDevice));
            SGM_CUDA_TRY(cudaMemcpy(b->chunk_w.p, cw.data(), sizeof(int64_t) * b->nchunks, cudaMemcpyHostToDevice));
        }
    }
    // run states and the work queue
    SGM_TRY(buf_ensure(b->qst, sizeof(RunState) * std::max(nq, 1)));
    SGM_TRY(buf_ensure(b->gst, sizeof(RunState)));
    SGM_CUDA_TRY(cudaMallocHost((void**)&b->h_qst, sizeof(RunState) * std::max(nq, 1)));
    SGM_CUDA_TRY(cudaMallocHost((void**)&b->h_gst, sizeof(RunState)));
    const int32_t qcap = o.split_min > 0 ? 4096 : 0;
    if (qcap) SGM_TRY(buf_ensure(b->queue, sizeof(QueueTask) * qcap));
    // launch shape of the persistent kernel
    ExtendLaunch L;
    L.mode = b->kmode;
    L.kcap = std::max(b->kcap, 1);
    L.warps_per_block = o.warps_per_block;
    L.smem_bytes = sgm_extend_smem_bytes(L.kcap, o.warps_per_block, true);
    int bps = sgm_extend_max_blocks_per_sm(b->kmode, true, o.warps_per_block, L.smem_bytes);
    if (bps < 1) return sgm_fail(SGM_E_CUDA, "batched extension kernel does not fit on an SM (smem %zu)", L.smem_bytes);
    if (o.blocks_per_sm > 0) bps = std::min(bps, o.blocks_per_sm);
    b->blocks = bps * e->sms;
    L.blocks = b->blocks;
    BatchArgs B;
    memset(&B, 0, sizeof(B));
    B.plans = (const QueryPlan*)b->plans.p;
    B.qst = (RunState*)b->qst.p;
    B.chunk_q = (const int32_t*)b->chunk_q.p;
    B.chunk_w = (const int64_t*)b->chunk_w.p;
    B.nchunks = b->nchunks;
    B.words = G.words;
    B.chunk_words = o.chunk_words;
    B.nq = nq;
    B.bfs = (BatchBfs*)b->bfs.p;
    B.fr[0] = (int32_t*)b->fr0.p;
    B.fr[1] = (int32_t*)b->fr1.p;
    B.task_base = (unsigned long long*)b->task_base.p;
    const int32_t bfs_blocks = std::max(2, std::min(128, 8 * e->sms / std::max(n_bfs, 1)));
    const uint64_t cap_ns = o.time_cap_s > 0 ? (uint64_t)(o.time_cap_s * 1e9) : 0;
    (void)want_hash;
    // capture the whole run once
    cudaStream_t s = b->stream;
    SGM_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    cudaError_t err = cudaMemsetAsync(b->qst.p, 0, sizeof(RunState) * nq, s);
    if (err == cudaSuccess) err = cudaMemsetAsync(b->gst.p, 0, sizeof(RunState), s);
    if (err == cudaSuccess && qcap) err = cudaMemsetAsync(b->queue.p, 0, sizeof(QueueTask) * qcap, s);
    if (err == cudaSuccess && nq)
        err = cudaMemcpyAsync(b->bfs.p, b->h_bfs0, sizeof(BatchBfs) * nq, cudaMemcpyHostToDevice, s);
    uint64_t launches = 0;
    for (int i = 0; i < nq && err == cudaSuccess; ++i) {
        err = sgm_launch_filter(G, specs[i], bits + off[i], s);
        ++launches;
    }
    if (err == cudaSuccess && nq) {
        err = sgm_launch_batch_bfs(G, B, nq, max_depth, bfs_blocks, s);
        launches += 3 + 2 * (uint64_t)std::max(0, max_depth - 1);
    }
    if (err == cudaSuccess && (b->nchunks > 0 || n_bfs > 0)) {
        PoolArgs none;
        memset(&none, 0, sizeof(none));
        err = sgm_launch_extend(L, G, nullptr, none, (RunState*)b->gst.p, qcap ? (QueueTask*)b->queue.p : nullptr,
                                qcap, nullptr, 0, cap_ns, o.work_cap, &B, s);
        ++launches;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t end = cudaStreamEndCapture(s, &graph);
    if (err != cudaSuccess || end != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
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
    if (st == SGM_OK) st = batch_build(b, qs, root_ranges, want_hash);
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
    SGM_CUDA_TRY(cudaMemcpyAsync(b->h_qst, b->qst.p, sizeof(RunState) * b->nq, cudaMemcpyDeviceToHost, b->stream));
    SGM_CUDA_TRY(cudaMemcpyAsync(b->h_gst, b->gst.p, sizeof(RunState), cudaMemcpyDeviceToHost, b->stream));
    SGM_CUDA_TRY(cudaStreamSynchronize(b->stream));
    float t = 0.f;
    cudaEventElapsedTime(&t, b->ev[1], b->ev[2]);
    if (ms) *ms = t;
    const RunState& gs = *b->h_gst;
    memset(&e->stats, 0, sizeof(e->stats));
    e->stats.ms_search = t;
    e->stats.grid_blocks = b->blocks;
    e->stats.cand_checked = gs.cand_checked;
    e->stats.list_elems = gs.list_elems;
    e->stats.search_probes = gs.search_probes;
    e->stats.bitmap_probes = gs.bitmap_probes;
    e->stats.filter_probes = gs.filter_probes;
    e->stats.task_groups = gs.task_groups;
    e->stats.steals = gs.steals;
    e->stats.idle_lanes = gs.idle_lanes;
    e->stats.scatter_rounds = gs.scatter_rounds;
    e->stats.launches = b->launches;
    sgm_status worst = SGM_OK;
    for (int i = 0; i < b->nq; ++i) {
        const RunState& q = b->h_qst[i];
        sgm_status st = gs.status ? gs.status : SGM_OK;
        uint64_t c = q.count;
        if (!st && q.overflow) st = SGM_E_COUNT_OVERFLOW;
        if (!st && b->kmode == SGM_KMODE_COUNT && b->aut_n[i] > 1 &&
            __builtin_mul_overflow(c, (uint64_t)b->aut_n[i], &c))
            st = SGM_E_COUNT_OVERFLOW;
        counts[i] = st ? 0 : c;
        if (hashes) hashes[i] = st ? 0 : q.hash;
        if (statuses) statuses[i] = st;
        if (st && !worst) worst = st;
    }
    if (worst)
        return sgm_fail(worst, gs.status == SGM_E_TIME_CAP   ? "time cap reached: batch unsolved"
                               : gs.status == SGM_E_WORK_CAP ? "work cap reached: batch unsolved"
                                                             : "a query of the batch failed (%d)",
                        worst);
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
