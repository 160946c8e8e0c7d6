// mlp.cu -- the plan-cost model: a 3-layer perceptron F -> H -> H -> 1 with
// exact GELU, trained on measured plan timings (log run time, MSE loss, Adam)
// entirely by the kernels below.  No counterpart in the paper, which leaves
// the choice of decomposition to the user; the model ranks candidate plans
// for shapes it has not timed, and exhaustive autotuning stays the fallback.
//
// Parameters are one flat float array: W1 (H x F), b1 (H), W2 (H x H), b2 (H),
// W3 (1 x H), b3 (1), row-major.  Activations are row-major (samples x units).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <random>
#include <vector>

#include "capi_internal.h"

namespace fft3 {

struct MlpLayout {
    int F, H;
    int w1, b1, w2, b2, w3, b3, total;
    explicit MlpLayout(int f = 0, int h = 0) : F(f), H(h)
    {
        w1 = 0;
        b1 = w1 + H * F;
        w2 = b1 + H;
        b2 = w2 + H * H;
        w3 = b2 + H;
        b3 = w3 + H;
        total = b3 + 1;
    }
};

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float x)
{
    const float Phi = 0.5f * (1.f + erff(x * 0.70710678118654752f));
    const float phi = 0.39894228040143268f * expf(-0.5f * x * x);
    return Phi + x * phi;
}

// Z[b, n] = sum_k A[b, k] W[n, k] + bias[n];  H = act ? gelu(Z) : Z.
__global__ void k_mlp_linear(const float *A, const float *W, const float *bias, float *Z, float *Hout, int B, int K,
                             int N, int act)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * N)
        return;
    const int b = i / N, n = i - b * N;
    float s = bias[n];
    for (int k = 0; k < K; ++k)
        s = fmaf(A[b * K + k], W[n * K + k], s);
    Z[i] = s;
    if (Hout)
        Hout[i] = act ? gelu_f(s) : s;
}

// g[b] = (2/B) (pred[b] - y[b]); loss += sum (pred - y)^2 / B.
__global__ void k_mlp_mse(const float *pred, const float *y, int B, float *g, float *loss)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f;
    if (i < B) {
        d = pred[i] - y[i];
        g[i] = 2.f * d / (float)B;
    }
    float v = d * d / (float)B;
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && loss)
        atomicAdd(loss, v);
}

// dW[n, k] = sum_b dZ[b, n] A[b, k]; db[n] = sum_b dZ[b, n] (k == 0 threads).
__global__ void k_mlp_wgrad(const float *dZ, const float *A, int B, int K, int N, float *dW, float *db)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N * (K + 1))
        return;
    const int n = i / (K + 1), k = i - n * (K + 1);
    float s = 0.f;
    if (k < K) {
        for (int b = 0; b < B; ++b)
            s = fmaf(dZ[b * N + n], A[b * K + k], s);
        dW[n * K + k] = s;
    } else {
        for (int b = 0; b < B; ++b)
            s += dZ[b * N + n];
        db[n] = s;
    }
}

// dZprev[b, k] = (sum_n dZ[b, n] W[n, k]) * gelu'(Zprev[b, k]).
__global__ void k_mlp_backprop(const float *dZ, const float *W, const float *Zprev, int B, int K, int N, float *dZprev)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * K)
        return;
    const int b = i / K, k = i - b * K;
    float s = 0.f;
    for (int n = 0; n < N; ++n)
        s = fmaf(dZ[b * N + n], W[n * K + k], s);
    dZprev[i] = s * gelu_grad_f(Zprev[i]);
}

// Adam (Kingma & Ba) with bias correction; t is the 1-based step.
__global__ void k_mlp_adam(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                           float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_mlp_gather(const float *X, const float *y, const int *idx, int B, int F, float *Xb, float *yb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * (F + 1))
        return;
    const int b = i / (F + 1), f = i - b * (F + 1);
    const int s = idx[b];
    if (f < F)
        Xb[b * F + f] = X[s * F + f];
    else
        yb[b] = y[s];
}

} // namespace fft3

using namespace fft3;

struct fft3_mlp_s {
    MlpLayout L;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
    // activations for up to cap samples
    int cap = 0;
    float *z1 = nullptr, *h1 = nullptr, *z2 = nullptr, *h2 = nullptr, *z3 = nullptr, *g3 = nullptr, *g2 = nullptr,
          *g1 = nullptr, *loss = nullptr;
    int step = 0;
};

static void mlp_free_acts(fft3_mlp_s *m)
{
    float *ptrs[] = {m->z1, m->h1, m->z2, m->h2, m->z3, m->g3, m->g2, m->g1};
    for (float *p : ptrs)
        cudaFree(p);
    m->z1 = m->h1 = m->z2 = m->h2 = m->z3 = m->g3 = m->g2 = m->g1 = nullptr;
    m->cap = 0;
}

static int mlp_reserve(fft3_mlp_s *m, int B)
{
    if (B <= m->cap)
        return FFT3_OK;
    mlp_free_acts(m);
    const int H = m->L.H;
    size_t bh = (size_t)B * H * sizeof(float), b1 = (size_t)B * sizeof(float);
    if (cudaMalloc(&m->z1, bh) || cudaMalloc(&m->h1, bh) || cudaMalloc(&m->z2, bh) || cudaMalloc(&m->h2, bh) ||
        cudaMalloc(&m->z3, b1) || cudaMalloc(&m->g3, b1) || cudaMalloc(&m->g2, bh) || cudaMalloc(&m->g1, bh)) {
        cudaGetLastError();
        mlp_free_acts(m);
        return fail(FFT3_ERR_OOM, "MLP activation allocation failed");
    }
    m->cap = B;
    return FFT3_OK;
}

static inline int nblk(int n) { return std::max(1, (n + 255) / 256); }

static int mlp_fwd(fft3_mlp_s *m, const float *X, int B, cudaStream_t st)
{
    const MlpLayout &L = m->L;
    const float *p = m->d_p;
    k_mlp_linear<<<nblk(B * L.H), 256, 0, st>>>(X, p + L.w1, p + L.b1, m->z1, m->h1, B, L.F, L.H, 1);
    k_mlp_linear<<<nblk(B * L.H), 256, 0, st>>>(m->h1, p + L.w2, p + L.b2, m->z2, m->h2, B, L.H, L.H, 1);
    k_mlp_linear<<<nblk(B), 256, 0, st>>>(m->h2, p + L.w3, p + L.b3, m->z3, nullptr, B, L.H, 1, 0);
    CUDA_TRY(cudaGetLastError());
    return FFT3_OK;
}

// Loss and gradient of the MSE over B samples into m->d_g (and m->loss).
static int mlp_bwd(fft3_mlp_s *m, const float *X, const float *y, int B, cudaStream_t st)
{
    const MlpLayout &L = m->L;
    const float *p = m->d_p;
    float *g = m->d_g;
    CUDA_TRY(cudaMemsetAsync(m->loss, 0, sizeof(float), st));
    k_mlp_mse<<<nblk(B), 256, 0, st>>>(m->z3, y, B, m->g3, m->loss);
    k_mlp_wgrad<<<nblk(1 * (L.H + 1)), 256, 0, st>>>(m->g3, m->h2, B, L.H, 1, g + L.w3, g + L.b3);
    k_mlp_backprop<<<nblk(B * L.H), 256, 0, st>>>(m->g3, p + L.w3, m->z2, B, L.H, 1, m->g2);
    k_mlp_wgrad<<<nblk(L.H * (L.H + 1)), 256, 0, st>>>(m->g2, m->h1, B, L.H, L.H, g + L.w2, g + L.b2);
    k_mlp_backprop<<<nblk(B * L.H), 256, 0, st>>>(m->g2, p + L.w2, m->z1, B, L.H, L.H, m->g1);
    k_mlp_wgrad<<<nblk(L.H * (L.F + 1)), 256, 0, st>>>(m->g1, X, B, L.F, L.H, g + L.w1, g + L.b1);
    CUDA_TRY(cudaGetLastError());
    return FFT3_OK;
}

extern "C" {

int fft3_mlp_create(fft3_mlp *out, int n_features, int hidden, unsigned long long seed)
{
    if (!out || n_features < 1 || hidden < 1 || n_features > 4096 || hidden > 4096)
        return fail(FFT3_ERR_INVALID_ARG, "bad MLP shape");
    *out = nullptr;
    int dev = 0;
    int rc = check_device(&dev);
    if (rc)
        return rc;
    auto *m = new (std::nothrow) fft3_mlp_s();
    if (!m)
        return fail(FFT3_ERR_OOM, "host allocation failed");
    m->L = MlpLayout(n_features, hidden);
    const size_t bytes = (size_t)m->L.total * sizeof(float);
    if (cudaMalloc(&m->d_p, bytes) || cudaMalloc(&m->d_g, bytes) || cudaMalloc(&m->d_m, bytes) ||
        cudaMalloc(&m->d_v, bytes) || cudaMalloc(&m->loss, sizeof(float))) {
        cudaGetLastError();
        fft3_mlp_destroy(m);
        return fail(FFT3_ERR_OOM, "MLP allocation failed");
    }
    // He-style initialisation from a seeded generator on the host
    std::mt19937_64 rng(seed);
    std::vector<float> p(m->L.total, 0.f);
    auto fill = [&](int off, int rows, int cols) {
        std::normal_distribution<double> nd(0.0, std::sqrt(2.0 / cols));
        for (int i = 0; i < rows * cols; ++i)
            p[off + i] = (float)nd(rng);
    };
    fill(m->L.w1, hidden, n_features);
    fill(m->L.w2, hidden, hidden);
    fill(m->L.w3, 1, hidden);
    cudaMemcpy(m->d_p, p.data(), bytes, cudaMemcpyHostToDevice);
    cudaMemset(m->d_m, 0, bytes);
    cudaMemset(m->d_v, 0, bytes);
    cudaMemset(m->d_g, 0, bytes);
    *out = m;
    return FFT3_OK;
}

int fft3_mlp_destroy(fft3_mlp m)
{
    if (!m)
        return fail(FFT3_ERR_INVALID_ARG, "null model");
    mlp_free_acts(m);
    cudaFree(m->d_p);
    cudaFree(m->d_g);
    cudaFree(m->d_m);
    cudaFree(m->d_v);
    cudaFree(m->loss);
    delete m;
    return FFT3_OK;
}

int fft3_mlp_num_params(fft3_mlp m) { return m ? m->L.total : fail(FFT3_ERR_INVALID_ARG, "null model"); }

int fft3_mlp_set_params(fft3_mlp m, const float *h_params)
{
    if (!m || !h_params)
        return fail(FFT3_ERR_INVALID_ARG, "null argument");
    CUDA_TRY(cudaMemcpy(m->d_p, h_params, (size_t)m->L.total * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(m->d_m, 0, (size_t)m->L.total * 4));
    CUDA_TRY(cudaMemset(m->d_v, 0, (size_t)m->L.total * 4));
    m->step = 0;
    return FFT3_OK;
}

int fft3_mlp_get_params(fft3_mlp m, float *h_params)
{
    if (!m || !h_params)
        return fail(FFT3_ERR_INVALID_ARG, "null argument");
    CUDA_TRY(cudaMemcpy(h_params, m->d_p, (size_t)m->L.total * 4, cudaMemcpyDeviceToHost));
    return FFT3_OK;
}

int fft3_mlp_forward(fft3_mlp m, const float *d_X, int B, float *d_pred, void *stream)
{
    if (!m || !d_X || !d_pred || B < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_mlp_forward");
    int rc = mlp_reserve(m, B);
    if (!rc)
        rc = mlp_fwd(m, d_X, B, (cudaStream_t)stream);
    if (rc)
        return rc;
    CUDA_TRY(cudaMemcpyAsync(d_pred, m->z3, (size_t)B * 4, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return FFT3_OK;
}

int fft3_mlp_grad(fft3_mlp m, const float *d_X, const float *d_y, int B, float *d_grad, float *d_loss, void *stream)
{
    if (!m || !d_X || !d_y || B < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_mlp_grad");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = mlp_reserve(m, B);
    if (!rc)
        rc = mlp_fwd(m, d_X, B, st);
    if (!rc)
        rc = mlp_bwd(m, d_X, d_y, B, st);
    if (rc)
        return rc;
    if (d_grad)
        CUDA_TRY(cudaMemcpyAsync(d_grad, m->d_g, (size_t)m->L.total * 4, cudaMemcpyDeviceToDevice, st));
    if (d_loss)
        CUDA_TRY(cudaMemcpyAsync(d_loss, m->loss, 4, cudaMemcpyDeviceToDevice, st));
    return FFT3_OK;
}

int fft3_mlp_adam_step(fft3_mlp m, const float *d_grad, float lr, void *stream)
{
    if (!m || lr <= 0.f)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_mlp_adam_step");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    m->step += 1;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_mlp_adam<<<nblk(m->L.total), 256, 0, (cudaStream_t)stream>>>(m->d_p, d_grad ? d_grad : m->d_g, m->d_m,
                                                                     m->d_v, m->L.total, lr, b1, b2, eps, c1, c2);
    CUDA_TRY(cudaGetLastError());
    return FFT3_OK;
}

int fft3_mlp_train(fft3_mlp m, const float *h_X, const float *h_y, int n, int epochs, int batch, float lr,
                   unsigned long long seed, float *h_loss_curve)
{
    if (!m || !h_X || !h_y || n < 1 || epochs < 1 || batch < 1 || lr <= 0.f)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_mlp_train");
    const int F = m->L.F;
    batch = std::min(batch, n);
    float *dX = nullptr, *dy = nullptr, *dXb = nullptr, *dyb = nullptr;
    int *didx = nullptr;
    auto cleanup = [&]() {
        cudaFree(dX);
        cudaFree(dy);
        cudaFree(dXb);
        cudaFree(dyb);
        cudaFree(didx);
    };
    if (cudaMalloc(&dX, (size_t)n * F * 4) || cudaMalloc(&dy, (size_t)n * 4) ||
        cudaMalloc(&dXb, (size_t)batch * F * 4) || cudaMalloc(&dyb, (size_t)batch * 4) ||
        cudaMalloc(&didx, (size_t)n * 4)) {
        cudaGetLastError();
        cleanup();
        return fail(FFT3_ERR_OOM, "training buffers");
    }
    cudaMemcpy(dX, h_X, (size_t)n * F * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(dy, h_y, (size_t)n * 4, cudaMemcpyHostToDevice);
    int rc = mlp_reserve(m, std::max(batch, n));
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i)
        perm[i] = i;
    std::mt19937_64 rng(seed);
    for (int ep = 0; ep < epochs && !rc; ++ep) {
        std::shuffle(perm.begin(), perm.end(), rng);
        cudaMemcpy(didx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice);
        for (int s = 0; s < n && !rc; s += batch) {
            const int b = std::min(batch, n - s);
            k_mlp_gather<<<nblk(b * (F + 1)), 256>>>(dX, dy, didx + s, b, F, dXb, dyb);
            rc = mlp_fwd(m, dXb, b, nullptr);
            if (!rc)
                rc = mlp_bwd(m, dXb, dyb, b, nullptr);
            if (!rc)
                rc = fft3_mlp_adam_step(m, nullptr, lr, nullptr);
        }
        if (!rc && h_loss_curve) {
            // full-data loss after the epoch
            rc = mlp_fwd(m, dX, n, nullptr);
            if (!rc)
                rc = mlp_bwd(m, dX, dy, n, nullptr);
            float l = 0.f;
            if (!rc && cudaMemcpy(&l, m->loss, 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = fail(FFT3_ERR_CUDA, "loss readback");
            h_loss_curve[ep] = l;
        }
    }
    if (!rc && cudaDeviceSynchronize() != cudaSuccess)
        rc = fail(FFT3_ERR_CUDA, "training failed");
    cleanup();
    return rc;
}

int fft3_mlp_predict(fft3_mlp m, const float *h_X, int n, float *h_pred)
{
    if (!m || !h_X || !h_pred || n < 1)
        return fail(FFT3_ERR_INVALID_ARG, "bad argument to fft3_mlp_predict");
    float *dX = nullptr;
    if (cudaMalloc(&dX, (size_t)n * m->L.F * 4)) {
        cudaGetLastError();
        return fail(FFT3_ERR_OOM, "predict buffer");
    }
    cudaMemcpy(dX, h_X, (size_t)n * m->L.F * 4, cudaMemcpyHostToDevice);
    int rc = mlp_reserve(m, n);
    if (!rc)
        rc = mlp_fwd(m, dX, n, nullptr);
    if (!rc && cudaMemcpy(h_pred, m->z3, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = fail(FFT3_ERR_CUDA, "predict readback");
    cudaFree(dX);
    return rc;
}

} // extern "C"
