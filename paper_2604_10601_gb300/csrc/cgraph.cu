// cgraph.cu - the candidate graph G' on the device (Sec. 6.1, Methods Under
// Study; App. C): the candidate sets C(u) as bitmaps (the filter, then the
// support rule of sgm_refine), a rank table per bitmap (the set bits before
// each word, so that a candidate's row is found in O(1)), and for every query
// edge in both directions (u, u2) the lists N(v) ∩ C(u2) of every v in C(u),
// in a CSR of their own (int64 offsets, int32 entries, rows in vertex order).
// Built in three passes over C(u): count every row, scan the counts into
// offsets, fill the rows; one warp per bitmap word, the lanes streaming each
// neighbour list 32 entries at a time and testing the entries' bits in C(u2).
#include <algorithm>
#include <cstring>

#include "objects.h"
#include "sgm_device.cuh"

namespace {

constexpr int kScan = 1024;
constexpr int kThreads = 256;

// Exclusive scan of one value per thread over a block of kScan threads;
// *total receives the sum.
template <class T>
__device__ T block_excl_scan(T x, T* total) {
    __shared__ T warp_sum[kScan / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    T incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(SGM_FULL, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        T w = warp_sum[lane];
        T wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(SGM_FULL, wi, o);
            if (lane >= o) wi += y;
        }
        warp_sum[lane] = wi - w;  // exclusive
        if (lane == 31) *total = wi;
    }
    __syncthreads();
    const T r = warp_sum[wid] + incl - x;
    __syncthreads();
    return r;
}

// rank[u][w] = set bits of bitmap u in words 0 .. w-1; rank[u][words] = |C(u)|.
// One block per bitmap, each thread a contiguous run of words.
__global__ void __launch_bounds__(kScan) cg_rank_kernel(const uint32_t* __restrict__ bits, int64_t words,
                                                        int32_t* __restrict__ rank) {
    __shared__ int32_t total;
    const uint32_t* b = bits + (int64_t)blockIdx.x * words;
    int32_t* r = rank + (int64_t)blockIdx.x * (words + 1);
    const int64_t chunk = (words + kScan - 1) / kScan;
    const int64_t lo = std::min<int64_t>(words, (int64_t)threadIdx.x * chunk);
    const int64_t hi = std::min<int64_t>(words, lo + chunk);
    int32_t s = 0;
    for (int64_t w = lo; w < hi; ++w) s += __popc(__ldg(b + w));
    int32_t at = block_excl_scan<int32_t>(s, &total);
    for (int64_t w = lo; w < hi; ++w) {
        r[w] = at;
        at += __popc(__ldg(b + w));
    }
    if (threadIdx.x == 0) r[words] = total;
}

// One directed edge (u, u2) as the build kernels see it.
struct CgJob {
    const uint32_t* bu;   // C(u)
    const int32_t* ru;    // rank of C(u)
    const uint32_t* bu2;  // C(u2)
    int64_t* ptr;         // [rows + 1]
    int32_t* adj;         // [entries] (fill pass)
};

// Count pass (FILL = false): ptr[r + 1] = |N(v) ∩ C(u2)| for row r = rank of
// v in C(u). Fill pass: the list itself at adj[ptr[r] ..]. A warp per word
// of C(u) (grid-stride), blockIdx.y = the directed edge.
template <bool FILL>
__global__ void __launch_bounds__(kThreads) cg_rows_kernel(DevGraph G, const CgJob* __restrict__ jobs) {
    const CgJob J = jobs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
    for (int64_t w = warp; w < G.words; w += nwarps) {
        uint32_t m = __ldg(J.bu + w);
        if (!m) continue;
        int32_t r = __ldg(J.ru + w);
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1u;
            const int32_t v = (int32_t)(w * 32 + b);
            const int32_t* nb = G.col + __ldg(G.rowptr + v);
            const int32_t d = __ldg(G.deg + v);
            int64_t at = FILL ? J.ptr[r] : 0;
            for (int32_t j0 = 0; j0 < d; j0 += 32) {
                const int32_t j = j0 + lane;
                int32_t y = 0;
                bool ok = false;
                if (j < d) {
                    y = __ldg(nb + j);
                    ok = sgm_bit(J.bu2, y);
                }
                const unsigned bal = __ballot_sync(SGM_FULL, ok);
                if (FILL && ok) J.adj[at + __popc(bal & sgm_lanemask_lt())] = y;
                at += __popc(bal);
            }
            if (!FILL && lane == 0) J.ptr[r + 1] = at;
            ++r;
        }
    }
}

// ptr[1 .. rows] of every edge: counts -> inclusive prefix sums (ptr[0] = 0).
// One block per edge.
__global__ void __launch_bounds__(kScan) cg_scan_kernel(const CgJob* __restrict__ jobs,
                                                        const int64_t* __restrict__ rows) {
    __shared__ int64_t total;
    int64_t* p = jobs[blockIdx.x].ptr;
    const int64_t n = rows[blockIdx.x];
    const int64_t chunk = (n + kScan - 1) / kScan;
    const int64_t lo = 1 + std::min<int64_t>(n, (int64_t)threadIdx.x * chunk);
    const int64_t hi = 1 + std::min<int64_t>(n, (lo - 1) + chunk);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += p[i];
    int64_t at = block_excl_scan<int64_t>(s, &total);
    for (int64_t i = lo; i < hi; ++i) {
        at += p[i];
        p[i] = at;
    }
    if (threadIdx.x == 0) p[0] = 0;
}

// vs[rank of v] = v for every v in C(u): the vertices of C(u) ascending.
__global__ void cg_expand_kernel(const uint32_t* __restrict__ bu, const int32_t* __restrict__ ru, int64_t words,
                                 int32_t* __restrict__ vs) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words * 32;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t w = i >> 5;
        const uint32_t m = __ldg(bu + w);
        const int b = (int)(i & 31);
        if ((m >> b) & 1u) vs[__ldg(ru + w) + __popc(m & ((1u << b) - 1u))] = (int32_t)i;
    }
}

}  // namespace

static sgm_status cg_check(const sgm_cgraph* c, int32_t u, int32_t u2, int32_t* idx) {
    if (!c || u < 0 || u2 < 0 || u >= c->k || u2 >= c->k || c->edge_of[u][u2] < 0)
        return sgm_fail(SGM_E_INVALID_ARG, "(%d, %d) is not a directed query edge of this candidate graph", u, u2);
    *idx = c->edge_of[u][u2];
    return SGM_OK;
}

static void cg_release(sgm_cgraph* c) {
    DevBuf* bufs[] = {&c->bits, &c->rank, &c->ptr, &c->adj};
    for (DevBuf* b : bufs) buf_free(*b);
}

static sgm_status cg_build(sgm_cgraph* c, int32_t use_filter, int32_t refine_rounds) {
    sgm_engine* e = c->e;
    const sgm_graph* g = c->g;
    const sgm_query* q = c->q;
    const DevGraph& G = g->G;
    cudaStream_t s = e->stream;
    const int k = q->k;
    const int64_t words = G.words;
    // candidate sets
    SGM_TRY(buf_ensure(c->bits, sizeof(uint32_t) * (size_t)std::max<int64_t>(words * k, 1)));
    uint32_t* bits = (uint32_t*)c->bits.p;
    if (refine_rounds > 0) SGM_TRY(sgm_refine(e, g, q, use_filter, refine_rounds, bits, nullptr));
    else SGM_TRY(sgm_filter(e, g, q, use_filter, bits));
    SGM_TRY(buf_ensure(c->rank, sizeof(int32_t) * (size_t)(words + 1) * k));
    int32_t* rank = (int32_t*)c->rank.p;
    cg_rank_kernel<<<k, kScan, 0, s>>>(bits, words, rank);
    SGM_CUDA_TRY(cudaGetLastError());
    // the directed edges and their row counts
    std::vector<int32_t> sizes(k);
    for (int u = 0; u < k; ++u)
        SGM_CUDA_TRY(cudaMemcpyAsync(&sizes[u], rank + (size_t)u * (words + 1) + words, sizeof(int32_t),
                                     cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    for (int u = 0; u < SGM_KMAX; ++u)
        for (int u2 = 0; u2 < SGM_KMAX; ++u2) c->edge_of[u][u2] = -1;
    int64_t ptr_total = 0;
    for (int u = 0; u < k; ++u)
        for (int u2 = 0; u2 < k; ++u2)
            if ((q->adj[u] >> u2) & 1u) {
                c->edge_of[u][u2] = (int32_t)c->eu.size();
                c->eu.push_back(u);
                c->ev.push_back(u2);
                c->rows.push_back(sizes[u]);
                c->ptr_off.push_back(ptr_total);
                ptr_total += sizes[u] + 1;
            }
    const int ne = (int)c->eu.size();
    if (ne == 0) return SGM_OK;
    SGM_TRY(buf_ensure(c->ptr, sizeof(int64_t) * (size_t)ptr_total));
    int64_t* ptr = (int64_t*)c->ptr.p;
    std::vector<CgJob> jobs(ne);
    for (int i = 0; i < ne; ++i) {
        jobs[i].bu = bits + (size_t)c->eu[i] * words;
        jobs[i].ru = rank + (size_t)c->eu[i] * (words + 1);
        jobs[i].bu2 = bits + (size_t)c->ev[i] * words;
        jobs[i].ptr = ptr + c->ptr_off[i];
        jobs[i].adj = nullptr;
    }
    DevBuf djobs, drows;
    struct Free {
        DevBuf* a;
        DevBuf* b;
        ~Free() { buf_free(*a); buf_free(*b); }
    } guard{&djobs, &drows};
    SGM_TRY(buf_ensure(djobs, sizeof(CgJob) * ne));
    SGM_TRY(buf_ensure(drows, sizeof(int64_t) * ne));
    SGM_CUDA_TRY(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(CgJob) * ne, cudaMemcpyHostToDevice, s));
    SGM_CUDA_TRY(cudaMemcpyAsync(drows.p, c->rows.data(), sizeof(int64_t) * ne, cudaMemcpyHostToDevice, s));
    const int64_t gx = std::max<int64_t>(1, std::min<int64_t>((words + kThreads / 32 - 1) / (kThreads / 32),
                                                              (int64_t)e->sms * 8));
    const dim3 grid((unsigned)gx, (unsigned)ne);
    cg_rows_kernel<false><<<grid, kThreads, 0, s>>>(G, (const CgJob*)djobs.p);
    SGM_CUDA_TRY(cudaGetLastError());
    cg_scan_kernel<<<ne, kScan, 0, s>>>((const CgJob*)djobs.p, (const int64_t*)drows.p);
    SGM_CUDA_TRY(cudaGetLastError());
    // list lengths -> the entry array
    c->entries.resize(ne);
    for (int i = 0; i < ne; ++i)
        SGM_CUDA_TRY(cudaMemcpyAsync(&c->entries[i], ptr + c->ptr_off[i] + c->rows[i], sizeof(int64_t),
                                     cudaMemcpyDeviceToHost, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    int64_t adj_total = 0;
    for (int i = 0; i < ne; ++i) {
        c->adj_off.push_back(adj_total);
        adj_total += c->entries[i];
    }
    SGM_TRY(buf_ensure(c->adj, sizeof(int32_t) * (size_t)std::max<int64_t>(adj_total, 1)));
    for (int i = 0; i < ne; ++i) jobs[i].adj = (int32_t*)c->adj.p + c->adj_off[i];
    SGM_CUDA_TRY(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(CgJob) * ne, cudaMemcpyHostToDevice, s));
    cg_rows_kernel<true><<<grid, kThreads, 0, s>>>(G, (const CgJob*)djobs.p);
    SGM_CUDA_TRY(cudaGetLastError());
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    return SGM_OK;
}

extern "C" sgm_status sgm_cgraph_build(sgm_engine* e, const sgm_graph* g, const sgm_query* q, int32_t use_filter,
                                       int32_t refine_rounds, sgm_cgraph** out) {
    if (!e || !g || !q || !out || refine_rounds < 0) return sgm_fail(SGM_E_INVALID_ARG, "sgm_cgraph_build: bad argument");
    if (g->e != e || q->e != e) return sgm_fail(SGM_E_INVALID_ARG, "graph or query belongs to another engine");
    *out = nullptr;
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    sgm_cgraph* c = new (std::nothrow) sgm_cgraph();
    if (!c) return sgm_fail(SGM_E_OOM, "host allocation failed");
    c->e = e;
    c->g = g;
    c->q = q;
    c->k = q->k;
    c->words = g->G.words;
    const sgm_status st = cg_build(c, use_filter, refine_rounds);
    if (st < 0) {
        cg_release(c);
        delete c;
        return st;
    }
    *out = c;
    return SGM_OK;
}

extern "C" sgm_status sgm_cgraph_destroy(sgm_cgraph* c) {
    if (!c) return SGM_OK;
    cudaSetDevice(c->e->device);
    cudaStreamSynchronize(c->e->stream);
    cg_release(c);
    delete c;
    return SGM_OK;
}

extern "C" sgm_status sgm_cgraph_edge_size(const sgm_cgraph* c, int32_t u, int32_t u2, int64_t* rows,
                                           int64_t* entries) {
    int32_t i = 0;
    SGM_TRY(cg_check(c, u, u2, &i));
    if (rows) *rows = c->rows[i];
    if (entries) *entries = c->entries[i];
    return SGM_OK;
}

extern "C" sgm_status sgm_cgraph_edge_copy(const sgm_cgraph* c, int32_t u, int32_t u2, int32_t* vs, int64_t* ptr,
                                           int32_t* adj) {
    int32_t i = 0;
    SGM_TRY(cg_check(c, u, u2, &i));
    SGM_CUDA_TRY(cudaSetDevice(c->e->device));
    cudaStream_t s = c->e->stream;
    const int64_t rows = c->rows[i];
    if (vs && rows > 0) {
        DevBuf tmp;
        sgm_status st = buf_ensure(tmp, sizeof(int32_t) * (size_t)rows);
        if (st < 0) return st;
        const int64_t words = c->words;
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((words * 32 + 255) / 256, 4096));
        cg_expand_kernel<<<(unsigned)blocks, 256, 0, s>>>((const uint32_t*)c->bits.p + (size_t)u * words,
                                                          (const int32_t*)c->rank.p + (size_t)u * (words + 1), words,
                                                          (int32_t*)tmp.p);
        cudaError_t err = cudaGetLastError();
        if (err == cudaSuccess) err = cudaMemcpyAsync(vs, tmp.p, sizeof(int32_t) * rows, cudaMemcpyDefault, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        buf_free(tmp);
        SGM_CUDA_TRY(err);
    }
    if (ptr)
        SGM_CUDA_TRY(cudaMemcpyAsync(ptr, (const int64_t*)c->ptr.p + c->ptr_off[i], sizeof(int64_t) * (rows + 1),
                                     cudaMemcpyDefault, s));
    if (adj && c->entries[i] > 0)
        SGM_CUDA_TRY(cudaMemcpyAsync(adj, (const int32_t*)c->adj.p + c->adj_off[i],
                                     sizeof(int32_t) * c->entries[i], cudaMemcpyDefault, s));
    SGM_CUDA_TRY(cudaStreamSynchronize(s));
    return SGM_OK;
}
