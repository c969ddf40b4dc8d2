// mlp.cu - the cost model of the learned matching order: a 3-layer FP32 MLP
// (F -> H -> H -> 1, ReLU) with its forward pass, the gradient of the mean
// squared error and Adam updates (Kingma and Ba, ICLR 2015), all in SIMT
// kernels on sm_103a. The network is tiny (H = 128: under 0.1 MB of
// weights), so these kernels are latency-bound; the point is that training
// and inference run on the device in the project's own code.
//
// Packed parameter layout: [W1 (F x H, row-major), b1 (H), W2 (H x H,
// row-major), b2 (H), w3 (H), b3 (1)].
//
// Sums run in a fixed order (over inputs inside a thread, over rows inside a
// block, over blocks in the reduction kernel), so results are reproducible.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "objects.h"

namespace {

constexpr int kRows = 32;  // rows of X per block

struct Net {
    int F, H;
    const float* W1;
    const float* b1;
    const float* W2;
    const float* b2;
    const float* w3;
    const float* b3;
};

__host__ __device__ inline int64_t n_params(int F, int H) { return (int64_t)F * H + H + (int64_t)H * H + H + H + 1; }

__host__ __device__ inline Net net_of(const float* p, int F, int H) {
    Net n;
    n.F = F;
    n.H = H;
    n.W1 = p;
    n.b1 = n.W1 + (int64_t)F * H;
    n.W2 = n.b1 + H;
    n.b2 = n.W2 + (int64_t)H * H;
    n.w3 = n.b2 + H;
    n.b3 = n.w3 + H;
    return n;
}

// Forward pass for rows [r0, r0 + kRows): thread j owns hidden unit j. Writes
// y, and the pre-activations Z1, Z2 (row-major, N x H) when they are asked for.
__global__ void mlp_fwd_kernel(const float* __restrict__ params, int F, int H, const float* __restrict__ X, int64_t N,
                               float* __restrict__ y, float* __restrict__ Z1g, float* __restrict__ Z2g) {
    extern __shared__ float sm[];
    float* xs = sm;                   // [kRows][F]
    float* h1 = xs + kRows * F;       // [kRows][H]
    float* red = h1 + kRows * H;      // [kRows][H / 32] warp partials of y
    const Net n = net_of(params, F, H);
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    const int rows = (int)(N - r0 < kRows ? N - r0 : kRows);
    for (int i = threadIdx.x; i < kRows * F; i += blockDim.x) {
        const int r = i / F;
        xs[i] = r < rows ? X[(r0 + r) * F + (i - r * F)] : 0.f;
    }
    __syncthreads();
    const int j = threadIdx.x;
    // layer 1
    for (int r = 0; r < rows; ++r) {
        float z = n.b1[j];
        for (int f = 0; f < F; ++f) z = fmaf(xs[r * F + f], n.W1[(int64_t)f * H + j], z);
        if (Z1g) Z1g[(r0 + r) * H + j] = z;
        h1[r * H + j] = fmaxf(z, 0.f);
    }
    __syncthreads();
    // layer 2 and the output layer
    const int lane = j & 31, warp = j >> 5;
    for (int r = 0; r < rows; ++r) {
        float z = n.b2[j];
        for (int i = 0; i < H; ++i) z = fmaf(h1[r * H + i], n.W2[(int64_t)i * H + j], z);
        if (Z2g) Z2g[(r0 + r) * H + j] = z;
        float c = fmaxf(z, 0.f) * n.w3[j];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) red[r * (H / 32) + warp] = c;
    }
    __syncthreads();
    if (j < rows) {
        float s = n.b3[0];
        for (int w = 0; w < H / 32; ++w) s += red[j * (H / 32) + w];
        y[r0 + j] = s;
    }
}

// Backward pass for rows [r0, r0 + kRows): per-block partial gradients
// (packed layout) of L = (1/N) sum (y - t)^2, from the saved pre-activations.
__global__ void mlp_bwd_kernel(const float* __restrict__ params, int F, int H, const float* __restrict__ X,
                               const float* __restrict__ t, const float* __restrict__ y, const float* __restrict__ Z1g,
                               const float* __restrict__ Z2g, int64_t N, float* __restrict__ partial,
                               float* __restrict__ sq_err) {
    extern __shared__ float sm[];
    float* xs = sm;                   // [kRows][F]
    float* h1 = xs + kRows * F;       // [kRows][H] relu(Z1)
    float* d2 = h1 + kRows * H;       // [kRows][H] dL/dZ2
    float* d1 = d2 + kRows * H;       // [kRows][H] dL/dZ1
    float* dy = d1 + kRows * H;       // [kRows]
    const Net n = net_of(params, F, H);
    const int64_t r0 = (int64_t)blockIdx.x * kRows;
    const int rows = (int)(N - r0 < kRows ? N - r0 : kRows);
    const int j = threadIdx.x;
    for (int i = j; i < kRows * F; i += blockDim.x) {
        const int r = i / F;
        xs[i] = r < rows ? X[(r0 + r) * F + (i - r * F)] : 0.f;
    }
    if (j < kRows) {
        float e = 0.f;
        if (j < rows) e = y[r0 + j] - t[r0 + j];
        dy[j] = 2.f * e / (float)N;
        if (sq_err && j < rows) sq_err[r0 + j] = e * e;
    }
    __syncthreads();
    for (int r = 0; r < kRows; ++r) {
        const bool in = r < rows;
        const float z1 = in ? Z1g[(r0 + r) * H + j] : 0.f;
        const float z2 = in ? Z2g[(r0 + r) * H + j] : 0.f;
        h1[r * H + j] = fmaxf(z1, 0.f);
        d2[r * H + j] = (in && z2 > 0.f) ? dy[r] * n.w3[j] : 0.f;
        d1[r * H + j] = z1;  // pre-activation, replaced by dL/dZ1 below
    }
    __syncthreads();
    // dL/dZ1[r][j] = (sum_i dZ2[r][i] W2[j][i]) * [Z1[r][j] > 0]
    for (int r = 0; r < rows; ++r) {
        float s = 0.f;
        for (int i = 0; i < H; ++i) s = fmaf(d2[r * H + i], n.W2[(int64_t)j * H + i], s);
        d1[r * H + j] = d1[r * H + j] > 0.f ? s : 0.f;
    }
    for (int r = rows; r < kRows; ++r) d1[r * H + j] = 0.f;
    __syncthreads();
    float* g = partial + (int64_t)blockIdx.x * n_params(F, H);
    Net gn = net_of(g, F, H);
    float* gW1 = const_cast<float*>(gn.W1);
    float* gb1 = const_cast<float*>(gn.b1);
    float* gW2 = const_cast<float*>(gn.W2);
    float* gb2 = const_cast<float*>(gn.b2);
    float* gw3 = const_cast<float*>(gn.w3);
    float* gb3 = const_cast<float*>(gn.b3);
    // W1[f][j] = sum_r X[r][f] dZ1[r][j]
    for (int f = 0; f < F; ++f) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s = fmaf(xs[r * F + f], d1[r * H + j], s);
        gW1[(int64_t)f * H + j] = s;
    }
    // W2[i][j] = sum_r H1[r][i] dZ2[r][j]
    for (int i = 0; i < H; ++i) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s = fmaf(h1[r * H + i], d2[r * H + j], s);
        gW2[(int64_t)i * H + j] = s;
    }
    float sb1 = 0.f, sb2 = 0.f, sw3 = 0.f;
    for (int r = 0; r < kRows; ++r) {
        sb1 += d1[r * H + j];
        sb2 += d2[r * H + j];
        const float z2 = r < rows ? Z2g[(r0 + r) * H + j] : 0.f;
        sw3 = fmaf(fmaxf(z2, 0.f), dy[r], sw3);
    }
    gb1[j] = sb1;
    gb2[j] = sb2;
    gw3[j] = sw3;
    if (j == 0) {
        float s = 0.f;
        for (int r = 0; r < kRows; ++r) s += dy[r];
        gb3[0] = s;
    }
}

// grad[i] = sum over blocks b (in order) of partial[b][i]
__global__ void mlp_reduce_kernel(const float* __restrict__ partial, int64_t P, int blocks, float* __restrict__ grad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < blocks; ++b) s += partial[(int64_t)b * P + i];
        grad[i] = s;
    }
}

// Adam (Kingma and Ba, Algorithm 1): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
// theta <- theta - lr * (m / c1) / (sqrt(v / c2) + eps), c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void mlp_adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, int64_t P, float lr, float b1, float b2, float eps, float c1,
                                float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// sum of the squared errors of a full-batch step, written to out[step]
__global__ void mlp_sum_kernel(const float* __restrict__ sq, int64_t N, float* __restrict__ out) {
    __shared__ float red[32];
    float s = 0.f;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += sq[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float tot = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        out[0] = tot / (float)N;
    }
}

size_t fwd_smem(int F, int H) { return sizeof(float) * ((size_t)kRows * F + (size_t)kRows * H + (size_t)kRows * (H / 32)); }
size_t bwd_smem(int F, int H) { return sizeof(float) * ((size_t)kRows * F + 3 * (size_t)kRows * H + kRows); }

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct sgm_model {
    sgm_engine* e = nullptr;
    int device = 0;
    cudaStream_t stream = nullptr;
    int32_t F = 0, H = 0;
    int64_t P = 0;
    int64_t step = 0;               // Adam updates taken
    float* theta = nullptr;         // [P]
    float* grad = nullptr;          // [P]
    float* m = nullptr;             // [P]
    float* v = nullptr;             // [P]
    // per-call scratch, grown on demand
    float* X = nullptr;             // [cap * F]
    float* t = nullptr;             // [cap]
    float* y = nullptr;             // [cap]
    float* Z = nullptr;             // [2 * cap * H]
    float* sq = nullptr;            // [cap]
    float* partial = nullptr;       // [ceil(cap / kRows) * P]
    float* losses = nullptr;        // [loss_cap]
    int64_t cap = 0, loss_cap = 0;
};


static void model_release_scratch(sgm_model* md) {
    float** ps[] = {&md->X, &md->t, &md->y, &md->Z, &md->sq, &md->partial};
    for (float** p : ps) {
        if (*p) cudaFree(*p);
        *p = nullptr;
    }
    md->cap = 0;
}

static sgm_status model_reserve(sgm_model* md, int64_t n) {
    if (n <= md->cap) return SGM_OK;
    model_release_scratch(md);
    const int64_t cap = ((n + kRows - 1) / kRows) * kRows;
    const int64_t blocks = cap / kRows;
    SGM_CUDA_TRY(cudaMalloc(&md->X, sizeof(float) * cap * md->F));
    SGM_CUDA_TRY(cudaMalloc(&md->t, sizeof(float) * cap));
    SGM_CUDA_TRY(cudaMalloc(&md->y, sizeof(float) * cap));
    SGM_CUDA_TRY(cudaMalloc(&md->Z, sizeof(float) * 2 * cap * md->H));
    SGM_CUDA_TRY(cudaMalloc(&md->sq, sizeof(float) * cap));
    SGM_CUDA_TRY(cudaMalloc(&md->partial, sizeof(float) * blocks * md->P));
    md->cap = cap;
    return SGM_OK;
}

static sgm_status set_smem_attrs(int F, int H) {
    SGM_CUDA_TRY(cudaFuncSetAttribute(mlp_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(F, H)));
    SGM_CUDA_TRY(cudaFuncSetAttribute(mlp_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(F, H)));
    return SGM_OK;
}

extern "C" sgm_status sgm_model_create(sgm_engine* e, int32_t in_dim, int32_t hidden, const float* init_params,
                                       sgm_model** out) {
    if (!e || !out || !init_params) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_create: NULL argument");
    *out = nullptr;
    if (in_dim < 1 || in_dim > SGM_MODEL_MAX_IN) return sgm_fail(SGM_E_INVALID_ARG, "in_dim %d outside [1, %d]", in_dim, SGM_MODEL_MAX_IN);
    if (hidden < 32 || hidden > 256 || hidden % 32)
        return sgm_fail(SGM_E_INVALID_ARG, "hidden %d: must be a multiple of 32 in [32, 256]", hidden);
    SGM_CUDA_TRY(cudaSetDevice(e->device));
    SGM_TRY(set_smem_attrs(in_dim, hidden));
    sgm_model* md = new (std::nothrow) sgm_model();
    if (!md) return sgm_fail(SGM_E_OOM, "host allocation failed");
    md->e = e;
    md->device = e->device;
    md->stream = e->stream;
    md->F = in_dim;
    md->H = hidden;
    md->P = n_params(in_dim, hidden);
    cudaError_t err = cudaMalloc(&md->theta, sizeof(float) * md->P * 4);
    if (err != cudaSuccess) {
        delete md;
        return sgm_fail(SGM_E_OOM, "sgm_model_create: %s", cudaGetErrorString(err));
    }
    md->grad = md->theta + md->P;
    md->m = md->grad + md->P;
    md->v = md->m + md->P;
    err = cudaMemcpy(md->theta, init_params, sizeof(float) * md->P, cudaMemcpyHostToDevice);
    if (err == cudaSuccess) err = cudaMemset(md->grad, 0, sizeof(float) * md->P * 3);
    if (err != cudaSuccess) {
        cudaFree(md->theta);
        delete md;
        return sgm_fail(SGM_E_CUDA, "sgm_model_create: %s", cudaGetErrorString(err));
    }
    *out = md;
    return SGM_OK;
}

extern "C" sgm_status sgm_model_free(sgm_model* md) {
    if (!md) return SGM_OK;
    cudaSetDevice(md->device);
    cudaStreamSynchronize(md->stream);
    model_release_scratch(md);
    if (md->losses) cudaFree(md->losses);
    if (md->theta) cudaFree(md->theta);
    delete md;
    return SGM_OK;
}

extern "C" sgm_status sgm_model_info(const sgm_model* md, int32_t* in_dim, int32_t* hidden, int64_t* n_params_out,
                                     int64_t* steps) {
    if (!md) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_info: model is NULL");
    if (in_dim) *in_dim = md->F;
    if (hidden) *hidden = md->H;
    if (n_params_out) *n_params_out = md->P;
    if (steps) *steps = md->step;
    return SGM_OK;
}

extern "C" sgm_status sgm_model_get_params(const sgm_model* md, float* params_out) {
    if (!md || !params_out) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_get_params: NULL argument");
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    SGM_CUDA_TRY(cudaMemcpy(params_out, md->theta, sizeof(float) * md->P, cudaMemcpyDeviceToHost));
    return SGM_OK;
}

extern "C" sgm_status sgm_model_set_params(sgm_model* md, const float* params) {
    if (!md || !params) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_set_params: NULL argument");
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    SGM_CUDA_TRY(cudaMemcpy(md->theta, params, sizeof(float) * md->P, cudaMemcpyHostToDevice));
    SGM_CUDA_TRY(cudaMemset(md->m, 0, sizeof(float) * md->P * 2));
    md->step = 0;
    return SGM_OK;
}

static cudaError_t launch_fwd(sgm_model* md, int64_t n, bool keep) {
    const int blocks = (int)((n + kRows - 1) / kRows);
    mlp_fwd_kernel<<<blocks, md->H, fwd_smem(md->F, md->H), md->stream>>>(
        md->theta, md->F, md->H, md->X, n, md->y, keep ? md->Z : nullptr, keep ? md->Z + md->cap * md->H : nullptr);
    return cudaGetLastError();
}

static cudaError_t launch_grad(sgm_model* md, int64_t n, float* loss_slot) {
    const int blocks = (int)((n + kRows - 1) / kRows);
    cudaError_t err = launch_fwd(md, n, true);
    if (err != cudaSuccess) return err;
    mlp_bwd_kernel<<<blocks, md->H, bwd_smem(md->F, md->H), md->stream>>>(
        md->theta, md->F, md->H, md->X, md->t, md->y, md->Z, md->Z + md->cap * md->H, n, md->partial, md->sq);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    mlp_reduce_kernel<<<(int)std::min<int64_t>((md->P + 255) / 256, 1024), 256, 0, md->stream>>>(md->partial, md->P,
                                                                                               blocks, md->grad);
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    if (loss_slot) {
        mlp_sum_kernel<<<1, 1024, 0, md->stream>>>(md->sq, n, loss_slot);
        err = cudaGetLastError();
    }
    return err;
}

static cudaError_t launch_adam(sgm_model* md, float lr, float b1, float b2, float eps) {
    md->step++;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)md->step));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)md->step));
    mlp_adam_kernel<<<(int)std::min<int64_t>((md->P + 255) / 256, 1024), 256, 0, md->stream>>>(
        md->theta, md->grad, md->m, md->v, md->P, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

static sgm_status upload_rows(sgm_model* md, const float* X, const float* t, int64_t n) {
    SGM_TRY(model_reserve(md, n));
    SGM_CUDA_TRY(cudaMemcpyAsync(md->X, X, sizeof(float) * n * md->F, cudaMemcpyHostToDevice, md->stream));
    if (t) SGM_CUDA_TRY(cudaMemcpyAsync(md->t, t, sizeof(float) * n, cudaMemcpyHostToDevice, md->stream));
    return SGM_OK;
}

extern "C" sgm_status sgm_model_forward(sgm_model* md, const float* X, int64_t n, float* y_out) {
    if (!md || (n > 0 && (!X || !y_out)) || n < 0) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_forward: bad argument");
    if (n == 0) return SGM_OK;
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    md->stream = md->e->stream;
    SGM_TRY(upload_rows(md, X, nullptr, n));
    SGM_CUDA_TRY(launch_fwd(md, n, false));
    SGM_CUDA_TRY(cudaMemcpyAsync(y_out, md->y, sizeof(float) * n, cudaMemcpyDeviceToHost, md->stream));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    return SGM_OK;
}

extern "C" sgm_status sgm_model_gradient(sgm_model* md, const float* X, const float* t, int64_t n, float* grad_out,
                                         float* loss_out) {
    if (!md || !X || !t || n < 1) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_gradient: bad argument");
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    md->stream = md->e->stream;
    SGM_TRY(upload_rows(md, X, t, n));
    if (!md->losses) {
        SGM_CUDA_TRY(cudaMalloc(&md->losses, sizeof(float) * 1024));
        md->loss_cap = 1024;
    }
    SGM_CUDA_TRY(launch_grad(md, n, md->losses));
    if (grad_out) SGM_CUDA_TRY(cudaMemcpyAsync(grad_out, md->grad, sizeof(float) * md->P, cudaMemcpyDeviceToHost, md->stream));
    float l = 0.f;
    SGM_CUDA_TRY(cudaMemcpyAsync(&l, md->losses, sizeof(float), cudaMemcpyDeviceToHost, md->stream));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    if (loss_out) *loss_out = l;
    return SGM_OK;
}

extern "C" sgm_status sgm_model_adam_step(sgm_model* md, float lr, float beta1, float beta2, float eps) {
    if (!md) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_adam_step: model is NULL");
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    md->stream = md->e->stream;
    SGM_CUDA_TRY(launch_adam(md, lr, beta1, beta2, eps));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    return SGM_OK;
}

extern "C" sgm_status sgm_model_train(sgm_model* md, const float* X, const float* t, int64_t n, int32_t steps,
                                      float lr, float* losses_out) {
    if (!md || !X || !t || n < 1 || steps < 0) return sgm_fail(SGM_E_INVALID_ARG, "sgm_model_train: bad argument");
    SGM_CUDA_TRY(cudaSetDevice(md->device));
    md->stream = md->e->stream;
    SGM_TRY(upload_rows(md, X, t, n));
    if (md->loss_cap < steps + 1) {
        if (md->losses) cudaFree(md->losses);
        md->losses = nullptr;
        SGM_CUDA_TRY(cudaMalloc(&md->losses, sizeof(float) * (steps + 1)));
        md->loss_cap = steps + 1;
    }
    for (int32_t s = 0; s < steps; ++s) {
        SGM_CUDA_TRY(launch_grad(md, n, md->losses + s));
        SGM_CUDA_TRY(launch_adam(md, lr, 0.9f, 0.999f, 1e-8f));
    }
    if (losses_out && steps > 0)
        SGM_CUDA_TRY(cudaMemcpyAsync(losses_out, md->losses, sizeof(float) * steps, cudaMemcpyDeviceToHost, md->stream));
    SGM_CUDA_TRY(cudaStreamSynchronize(md->stream));
    return SGM_OK;
}
