// apo_surrogate.cu -- the surrogate network object (apo_mlp_*) and the
// surrogate-assisted APO run (apo_run_surrogate).
//
// Surrogate-assisted form: every protozoon draws k candidates per iteration
// (candidate c uses its own Philox slots, c = 0 being the plain candidate),
// the MLP ranks them, only the best-ranked one is evaluated exactly and goes
// through the greedy replacement of Algorithm 1.  Every exact evaluation is
// appended to an archive (ring buffer of the last 50 000); the network is
// retrained on it every `retrain_every` iterations.  The plain method (k = 1)
// runs until the first retrain and whenever the surrogate's Spearman rank
// correlation on the last screened batch falls below 0.3.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.h"
#include "apo_mlp.h"

using namespace apo;

namespace {

constexpr int kH = 256;   // hidden width of both layers

#define SUR_CUDA(expr)                                                                    \
    do {                                                                                  \
        const cudaError_t e_ = (expr);                                                    \
        if (e_ != cudaSuccess) {                                                          \
            char m_[256];                                                                 \
            snprintf(m_, sizeof(m_), "%s failed: %s", #expr, cudaGetErrorString(e_));    \
            apo::set_last_error(m_);                                                      \
            return e_ == cudaErrorMemoryAllocation ? APO_ERR_OOM : APO_ERR_CUDA;          \
        }                                                                                 \
    } while (0)

// x (fp32 [n][D]) -> bf16 [n][Kp], zero padded.
__global__ void to_bf16_kernel(int n, int D, int Kp, const float* __restrict__ x, __nv_bfloat16* __restrict__ xb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)n * Kp; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / Kp), c = (int)(i - (size_t)r * Kp);
        xb[i] = __float2bfloat16(c < D ? x[(size_t)r * D + c] : 0.f);
    }
}

// idx[i] = uniform index in [0, n) from Philox (seed, step, i); the whole
// set in order when the batch covers it (B >= n).
__global__ void rand_idx_kernel(int B, int n, uint32_t seed, uint32_t step, int* __restrict__ idx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B && B >= n) {
        idx[i] = i < n ? i : n - 1;
    } else if (i < B) {
        const uint4 w = philox(step, (uint32_t)i, 0xFFFFFFFFu, 0x100u, seed, 0x7FFFFFFFu);
        idx[i] = (int)idx_draw(w.x, (uint32_t)n);
    }
}

}  // namespace

struct apo_mlp {
    int D, Kp, cap;   // input width, padded width, workspace rows
    int step;         // Adam steps taken
    // fp32 master parameters, Adam moments, gradients; bf16 copies
    float *W1, *b1, *W2, *b2, *w3, *b3;
    float *mW1, *mb1, *mW2, *mb2, *mw3, *mb3, *vW1, *vb1, *vW2, *vb2, *vw3, *vb3;
    float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3;
    __nv_bfloat16 *W1b, *W2b, *w3b;
    // per-row workspace
    __nv_bfloat16 *Xb, *H1b, *H2b, *dZ2b, *dZ1b;
    float *Z1, *Z2, *dZ2, *dZ1, *y, *t, *dy, *loss;
    int* idx;
    void* mem;
};

namespace {

apo_status mlp_alloc(apo_mlp* M, int cap)
{
    const int D = M->D, Kp = M->Kp;
    (void)D;
    const size_t nW1 = (size_t)Kp * kH, nW2 = (size_t)kH * kH;
    size_t off = 0;
    std::vector<std::pair<void**, size_t>> items;
    auto add = [&](void** p, size_t bytes) { items.emplace_back(p, bytes); };
    float** f32s[] = {&M->W1, &M->mW1, &M->vW1, &M->gW1};
    for (float** p : f32s) add((void**)p, nW1 * 4);
    float** f32h[] = {&M->b1, &M->mb1, &M->vb1, &M->gb1, &M->b2, &M->mb2, &M->vb2, &M->gb2,
                      &M->w3, &M->mw3, &M->vw3, &M->gw3};
    for (float** p : f32h) add((void**)p, kH * 4);
    float** f32w2[] = {&M->W2, &M->mW2, &M->vW2, &M->gW2};
    for (float** p : f32w2) add((void**)p, nW2 * 4);
    float** f32s1[] = {&M->b3, &M->mb3, &M->vb3, &M->gb3, &M->loss};
    for (float** p : f32s1) add((void**)p, 16);
    add((void**)&M->W1b, nW1 * 2);
    add((void**)&M->W2b, nW2 * 2);
    add((void**)&M->w3b, kH * 2);
    add((void**)&M->Xb, (size_t)cap * Kp * 2);
    __nv_bfloat16** bh[] = {&M->H1b, &M->H2b, &M->dZ2b, &M->dZ1b};
    for (auto p : bh) add((void**)p, (size_t)cap * kH * 2);
    float** fh[] = {&M->Z1, &M->Z2, &M->dZ2, &M->dZ1};
    for (auto p : fh) add((void**)p, (size_t)cap * kH * 4);
    float** fr[] = {&M->y, &M->t, &M->dy};
    for (auto p : fr) add((void**)p, (size_t)cap * 4);
    add((void**)&M->idx, (size_t)cap * 4);
    for (auto& it : items) off = (off + 255) / 256 * 256 + it.second;
    SUR_CUDA(cudaMalloc(&M->mem, off));
    SUR_CUDA(cudaMemset(M->mem, 0, off));
    unsigned char* base = static_cast<unsigned char*>(M->mem);
    off = 0;
    for (auto& it : items) {
        off = (off + 255) / 256 * 256;
        *it.first = base + off;
        off += it.second;
    }
    M->cap = cap;
    return APO_OK;
}

__global__ void f32_to_bf16_kernel(int n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) b[i] = __float2bfloat16(a[i]);
}

apo_status refresh_bf16(apo_mlp* M, cudaStream_t st)
{
    f32_to_bf16_kernel<<<256, 256, 0, st>>>(M->Kp * kH, M->W1, M->W1b);
    f32_to_bf16_kernel<<<256, 256, 0, st>>>(kH * kH, M->W2, M->W2b);
    f32_to_bf16_kernel<<<1, 256, 0, st>>>(kH, M->w3, M->w3b);
    SUR_CUDA(cudaGetLastError());
    return APO_OK;
}

// Forward pass of n rows of M->Xb (bf16 [n][Kp]); keeps Z1, H1, Z2, H2, y.
apo_status mlp_forward_rows(apo_mlp* M, int n, cudaStream_t st)
{
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    g.M = n; g.N = kH; g.K = M->Kp; g.A = M->Xb; g.lda = M->Kp; g.B = M->W1b; g.ldb = kH;
    g.bias = M->b1; g.relu = 1; g.Cf = M->Z1; g.ldc = kH; g.Cb = M->H1b; g.ldcb = kH;
    SUR_CUDA(gemm_bf16(g, false, false, st));
    g.K = kH; g.A = M->H1b; g.lda = kH; g.B = M->W2b; g.bias = M->b2; g.Cf = M->Z2; g.Cb = M->H2b;
    SUR_CUDA(gemm_bf16(g, false, false, st));
    SUR_CUDA(launch_out_layer(n, kH, M->H2b, M->w3b, M->b3, M->y, st));
    return APO_OK;
}

// Gradients of mean((y - t)^2) over n rows (after mlp_forward_rows).
apo_status mlp_backward_rows(apo_mlp* M, int n, cudaStream_t st)
{
    SUR_CUDA(cudaMemsetAsync(M->loss, 0, 4, st));
    SUR_CUDA(launch_out_backward(n, kH, M->y, M->t, M->w3b, M->Z2, M->dZ2, M->dZ2b, M->loss, st));
    SUR_CUDA(launch_dy(n, M->y, M->t, M->dy, st));
    SUR_CUDA(launch_colsum(n, kH, nullptr, M->H2b, M->dy, M->gw3, st));   // dw3 = H2^T dy
    SUR_CUDA(launch_colsum(n, 1, M->dy, nullptr, nullptr, M->gb3, st));   // db3 = sum dy
    SUR_CUDA(launch_colsum(n, kH, M->dZ2, nullptr, nullptr, M->gb2, st)); // db2
    GemmArgs g;
    std::memset(&g, 0, sizeof(g));
    // dW2 = H1^T dZ2
    g.M = kH; g.N = kH; g.K = n; g.A = M->H1b; g.lda = kH; g.B = M->dZ2b; g.ldb = kH; g.Cf = M->gW2; g.ldc = kH;
    SUR_CUDA(gemm_bf16(g, true, false, st));
    // dZ1 = (dZ2 W2^T) masked by Z1 > 0
    std::memset(&g, 0, sizeof(g));
    g.M = n; g.N = kH; g.K = kH; g.A = M->dZ2b; g.lda = kH; g.B = M->W2b; g.ldb = kH;
    g.mask = M->Z1; g.ldm = kH; g.Cf = M->dZ1; g.ldc = kH; g.Cb = M->dZ1b; g.ldcb = kH;
    SUR_CUDA(gemm_bf16(g, false, true, st));
    SUR_CUDA(launch_colsum(n, kH, M->dZ1, nullptr, nullptr, M->gb1, st)); // db1
    // dW1 = X^T dZ1
    std::memset(&g, 0, sizeof(g));
    g.M = M->Kp; g.N = kH; g.K = n; g.A = M->Xb; g.lda = M->Kp; g.B = M->dZ1b; g.ldb = kH; g.Cf = M->gW1; g.ldc = kH;
    SUR_CUDA(gemm_bf16(g, true, false, st));
    return APO_OK;
}

apo_status mlp_adam(apo_mlp* M, float lr, cudaStream_t st)
{
    M->step += 1;
    const int s = M->step;
    SUR_CUDA(launch_adam(M->Kp * kH, M->W1, M->gW1, M->mW1, M->vW1, M->W1b, lr, s, st));
    SUR_CUDA(launch_adam(kH, M->b1, M->gb1, M->mb1, M->vb1, nullptr, lr, s, st));
    SUR_CUDA(launch_adam(kH * kH, M->W2, M->gW2, M->mW2, M->vW2, M->W2b, lr, s, st));
    SUR_CUDA(launch_adam(kH, M->b2, M->gb2, M->mb2, M->vb2, nullptr, lr, s, st));
    SUR_CUDA(launch_adam(kH, M->w3, M->gw3, M->mw3, M->vw3, M->w3b, lr, s, st));
    SUR_CUDA(launch_adam(1, M->b3, M->gb3, M->mb3, M->vb3, nullptr, lr, s, st));
    return APO_OK;
}

apo_status load_inputs(apo_mlp* M, const float* d_X, int n, cudaStream_t st)
{
    to_bf16_kernel<<<(int)std::min<size_t>(((size_t)n * M->Kp + 255) / 256, 4096), 256, 0, st>>>(n, M->D, M->Kp, d_X,
                                                                                                M->Xb);
    SUR_CUDA(cudaGetLastError());
    return APO_OK;
}

}  // namespace

extern "C" apo_status apo_mlp_create(int D, uint32_t seed, apo_mlp** out)
{
    if (!out || D < 1 || D > 4096) { apo::set_last_error("apo_mlp_create: D must be 1..4096"); return APO_ERR_INVALID_ARG; }
    *out = nullptr;
    apo_mlp* M = new apo_mlp();
    std::memset(M, 0, sizeof(*M));
    M->D = D;
    M->Kp = (D + 7) & ~7;
    apo_status rc = mlp_alloc(M, 2048);
    if (rc != APO_OK) { delete M; return rc; }
    // He-uniform initialisation (seeded, host side); padded input rows stay 0
    std::mt19937_64 g(seed);
    std::vector<float> W1((size_t)M->Kp * kH, 0.f), W2((size_t)kH * kH), w3(kH);
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    const double l1 = std::sqrt(6.0 / D), l2 = std::sqrt(6.0 / kH);
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < kH; ++j) W1[(size_t)i * kH + j] = (float)(l1 * u(g));
    for (auto& w : W2) w = (float)(l2 * u(g));
    for (auto& w : w3) w = (float)(l2 * u(g));
    cudaError_t e = cudaMemcpy(M->W1, W1.data(), W1.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(M->W2, W2.data(), W2.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(M->w3, w3.data(), w3.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && refresh_bf16(M, 0) == APO_OK) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(M->mem);
        delete M;
        apo::set_last_error("apo_mlp_create: upload failed");
        return APO_ERR_CUDA;
    }
    *out = M;
    return APO_OK;
}

extern "C" void apo_mlp_destroy(apo_mlp* M)
{
    if (!M) return;
    cudaDeviceSynchronize();
    cudaFree(M->mem);
    delete M;
}

extern "C" apo_status apo_mlp_set_params(apo_mlp* M, const float* W1, const float* b1, const float* W2, const float* b2,
                                         const float* w3, float b3)
{
    if (!M || !W1 || !b1 || !W2 || !b2 || !w3) { apo::set_last_error("apo_mlp_set_params: NULL argument"); return APO_ERR_INVALID_ARG; }
    std::vector<float> w1p((size_t)M->Kp * kH, 0.f);
    std::memcpy(w1p.data(), W1, sizeof(float) * (size_t)M->D * kH);
    SUR_CUDA(cudaMemcpy(M->W1, w1p.data(), w1p.size() * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemcpy(M->b1, b1, kH * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemcpy(M->W2, W2, (size_t)kH * kH * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemcpy(M->b2, b2, kH * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemcpy(M->w3, w3, kH * 4, cudaMemcpyHostToDevice));
    SUR_CUDA(cudaMemcpy(M->b3, &b3, 4, cudaMemcpyHostToDevice));
    apo_status rc = refresh_bf16(M, 0);
    if (rc != APO_OK) return rc;
    SUR_CUDA(cudaDeviceSynchronize());
    return APO_OK;
}

extern "C" apo_status apo_mlp_forward(apo_mlp* M, const float* d_X, int n, float* d_y, void* stream)
{
    if (!M || n < 0 || (n > 0 && (!d_X || !d_y))) { apo::set_last_error("apo_mlp_forward: bad arguments"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    for (int r0 = 0; r0 < n; r0 += M->cap) {
        const int rows = std::min(M->cap, n - r0);
        apo_status rc = load_inputs(M, d_X + (size_t)r0 * M->D, rows, st);
        if (rc == APO_OK) rc = mlp_forward_rows(M, rows, st);
        if (rc != APO_OK) return rc;
        SUR_CUDA(cudaMemcpyAsync(d_y + r0, M->y, sizeof(float) * rows, cudaMemcpyDeviceToDevice, st));
    }
    return APO_OK;
}

extern "C" apo_status apo_mlp_gradients(apo_mlp* M, const float* d_X, const float* d_t, int n, float* gW1, float* gb1,
                                        float* gW2, float* gb2, float* gw3, float* gb3, float* loss)
{
    if (!M || n < 1 || n > M->cap || !d_X || !d_t) { apo::set_last_error("apo_mlp_gradients: bad arguments"); return APO_ERR_INVALID_ARG; }
    apo_status rc = load_inputs(M, d_X, n, 0);
    if (rc != APO_OK) return rc;
    SUR_CUDA(cudaMemcpy(M->t, d_t, sizeof(float) * n, cudaMemcpyDeviceToDevice));
    rc = mlp_forward_rows(M, n, 0);
    if (rc == APO_OK) rc = mlp_backward_rows(M, n, 0);
    if (rc != APO_OK) return rc;
    SUR_CUDA(cudaDeviceSynchronize());
    std::vector<float> tmp((size_t)M->Kp * kH);
    if (gW1) {
        SUR_CUDA(cudaMemcpy(tmp.data(), M->gW1, tmp.size() * 4, cudaMemcpyDeviceToHost));
        std::memcpy(gW1, tmp.data(), sizeof(float) * (size_t)M->D * kH);
    }
    if (gb1) SUR_CUDA(cudaMemcpy(gb1, M->gb1, kH * 4, cudaMemcpyDeviceToHost));
    if (gW2) SUR_CUDA(cudaMemcpy(gW2, M->gW2, (size_t)kH * kH * 4, cudaMemcpyDeviceToHost));
    if (gb2) SUR_CUDA(cudaMemcpy(gb2, M->gb2, kH * 4, cudaMemcpyDeviceToHost));
    if (gw3) SUR_CUDA(cudaMemcpy(gw3, M->gw3, kH * 4, cudaMemcpyDeviceToHost));
    if (gb3) SUR_CUDA(cudaMemcpy(gb3, M->gb3, 4, cudaMemcpyDeviceToHost));
    if (loss) SUR_CUDA(cudaMemcpy(loss, M->loss, 4, cudaMemcpyDeviceToHost));
    return APO_OK;
}

namespace {

// `steps` Adam steps on batches of `batch` rows drawn uniformly from the
// first n rows of (Xa bf16 [.][Kp], ta).
apo_status mlp_train_rows(apo_mlp* M, const __nv_bfloat16* Xa, const float* ta, int n, int steps, int batch, float lr,
                          uint32_t seed, cudaStream_t st)
{
    batch = std::min(batch, M->cap);
    if (batch >= n) batch = n;   // full batch, rows in order
    for (int s = 0; s < steps; ++s) {
        rand_idx_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, n, seed, (uint32_t)(M->step + 1), M->idx);
        SUR_CUDA(cudaGetLastError());
        SUR_CUDA(launch_gather_rows(batch, M->Kp, M->idx, Xa, ta, M->Xb, M->t, st));
        apo_status rc = mlp_forward_rows(M, batch, st);
        if (rc == APO_OK) rc = mlp_backward_rows(M, batch, st);
        if (rc == APO_OK) rc = mlp_adam(M, lr, st);
        if (rc != APO_OK) return rc;
    }
    return APO_OK;
}

}  // namespace

extern "C" apo_status apo_mlp_train(apo_mlp* M, const float* d_X, const float* d_t, int n, int steps, int batch, float lr,
                                    uint32_t seed, void* stream)
{
    if (!M || n < 1 || steps < 0 || batch < 1 || !d_X || !d_t) { apo::set_last_error("apo_mlp_train: bad arguments"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    __nv_bfloat16* Xa = nullptr;
    SUR_CUDA(cudaMallocAsync(&Xa, (size_t)n * M->Kp * 2, st));
    to_bf16_kernel<<<(int)std::min<size_t>(((size_t)n * M->Kp + 255) / 256, 4096), 256, 0, st>>>(n, M->D, M->Kp, d_X, Xa);
    apo_status rc = mlp_train_rows(M, Xa, d_t, n, steps, batch, lr, seed, st);
    cudaFreeAsync(Xa, st);
    return rc;
}

extern "C" apo_status apo_mlp_get_params(const apo_mlp* M, float* W1, float* b1, float* W2, float* b2, float* w3, float* b3)
{
    if (!M) { apo::set_last_error("apo_mlp_get_params: NULL"); return APO_ERR_INVALID_ARG; }
    SUR_CUDA(cudaDeviceSynchronize());
    std::vector<float> tmp((size_t)M->Kp * kH);
    if (W1) {
        SUR_CUDA(cudaMemcpy(tmp.data(), M->W1, tmp.size() * 4, cudaMemcpyDeviceToHost));
        std::memcpy(W1, tmp.data(), sizeof(float) * (size_t)M->D * kH);
    }
    if (b1) SUR_CUDA(cudaMemcpy(b1, M->b1, kH * 4, cudaMemcpyDeviceToHost));
    if (W2) SUR_CUDA(cudaMemcpy(W2, M->W2, (size_t)kH * kH * 4, cudaMemcpyDeviceToHost));
    if (b2) SUR_CUDA(cudaMemcpy(b2, M->b2, kH * 4, cudaMemcpyDeviceToHost));
    if (w3) SUR_CUDA(cudaMemcpy(w3, M->w3, kH * 4, cudaMemcpyDeviceToHost));
    if (b3) SUR_CUDA(cudaMemcpy(b3, M->b3, 4, cudaMemcpyDeviceToHost));
    return APO_OK;
}
