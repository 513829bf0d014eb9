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
// Rows are taken from the window [start, start + n) of a ring buffer of cap rows.
__global__ void rand_idx_kernel(int B, int n, uint32_t seed, uint32_t step, int* __restrict__ idx, long long start,
                                int cap)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = 0;
    if (i < B && B >= n) {
        j = i < n ? i : n - 1;
    } else if (i < B) {
        const uint4 w = philox(step, (uint32_t)i, 0xFFFFFFFFu, 0x100u, seed, 0x7FFFFFFFu);
        j = (int)idx_draw(w.x, (uint32_t)n);
    }
    if (i < B) idx[i] = (int)((start + j) % cap);
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
    float* ws;        // split-K workspace of the GEMMs (kSplitWsElems floats)
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
    add((void**)&M->ws, kSplitWsElems * 4);
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
    g.ws = M->ws;
    g.ws_elems = kSplitWsElems;
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
    g.ws = M->ws;
    g.ws_elems = kSplitWsElems;
    // dW2 = H1^T dZ2
    g.M = kH; g.N = kH; g.K = n; g.A = M->H1b; g.lda = kH; g.B = M->dZ2b; g.ldb = kH; g.Cf = M->gW2; g.ldc = kH;
    SUR_CUDA(gemm_bf16(g, true, false, st));
    // dZ1 = (dZ2 W2^T) masked by Z1 > 0
    std::memset(&g, 0, sizeof(g));
    g.ws = M->ws;
    g.ws_elems = kSplitWsElems;
    g.M = n; g.N = kH; g.K = kH; g.A = M->dZ2b; g.lda = kH; g.B = M->W2b; g.ldb = kH;
    g.mask = M->Z1; g.ldm = kH; g.Cf = M->dZ1; g.ldc = kH; g.Cb = M->dZ1b; g.ldcb = kH;
    SUR_CUDA(gemm_bf16(g, false, true, st));
    SUR_CUDA(launch_colsum(n, kH, M->dZ1, nullptr, nullptr, M->gb1, st)); // db1
    // dW1 = X^T dZ1
    std::memset(&g, 0, sizeof(g));
    g.ws = M->ws;
    g.ws_elems = kSplitWsElems;
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
    if (int* status = device_status_word()) {   // a GEMM wait that ran out
        int h = 0;
        SUR_CUDA(cudaMemcpy(&h, status, 4, cudaMemcpyDeviceToHost));
        if (h != 0) {
            cudaMemset(status, 0, 4);
            apo::set_last_error("a device-side wait exceeded its limit");
            return (apo_status)h;
        }
    }
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
                          uint32_t seed, cudaStream_t st, long long start = 0, int cap = 0)
{
    if (cap <= 0) cap = n;
    batch = std::min(batch, M->cap);
    if (batch >= n) batch = n;   // full batch, rows in order
    for (int s = 0; s < steps; ++s) {
        rand_idx_kernel<<<(batch + 255) / 256, 256, 0, st>>>(batch, n, seed, (uint32_t)(M->step + 1), M->idx, start, cap);
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

// ===================================================== surrogate-assisted APO
#include "apo_path.cuh"

namespace {

constexpr int kSurThreads = 256;

// Stable sort of the population by (F, previous rank): perm_out[rank] = slot;
// curve[t - 1] = the smallest fitness.  One CTA, keys in shared memory.
__global__ void __launch_bounds__(1024) surr_sort_kernel(int ps, int ps_pad, const float* __restrict__ F,
                                                         const uint32_t* __restrict__ perm_prev,
                                                         uint32_t* __restrict__ perm_out, float* curve, int t)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    using KO = KeyOf<float>;
    KO::T* keys = reinterpret_cast<KO::T*>(dyn);
    for (int r = threadIdx.x; r < ps_pad; r += blockDim.x)
        keys[r] = r < ps ? KO::make(F[perm_prev[r]], (uint32_t)r) : KO::pad();
    __syncthreads();
    bitonic_sort<KO>(keys, ps_pad);
    for (int r = threadIdx.x; r < ps; r += blockDim.x) perm_out[r] = perm_prev[KO::idx(keys[r])];
    if (threadIdx.x == 0 && curve) curve[t - 1] = F[perm_prev[KO::idx(keys[0])]];
}

template <int QPL>
__device__ void surr_setup(const ApoRun* run, ApoRun& R, unsigned char* smem, Smem<float>& S,
                           const uint32_t* __restrict__ perm, bool copy_perm)
{
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(run);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(&R);
    for (int i = threadIdx.x; i < (int)(sizeof(ApoRun) / 8); i += blockDim.x) d[i] = s[i];
    __syncthreads();
    S = carve<float>(smem, R.plan);
    load_constants<float>(R, S);
    if (copy_perm)
        for (int r = threadIdx.x; r < R.ps; r += blockDim.x) S.perm[0][r] = perm[r];
    __syncthreads();
}

// Initial population (Algorithm 1): X_p = Xmin + U (Xmax - Xmin), F = f(X).
template <int QPL>
__global__ void __launch_bounds__(kSurThreads) surr_init_kernel(const ApoRun* __restrict__ run, float* X, float* F)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    Smem<float> S;
    surr_setup<QPL>(run, R, smem, S, nullptr, false);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int Dp = R.prob.Dp, CH = R.plan.chunk;
    for (int c0 = blockIdx.x * CH; c0 < R.ps; c0 += gridDim.x * CH) {
        const int rows = min(CH, R.ps - c0);
        for (int row = warp; row < rows; row += nw) gen_init_row<float, QPL>(R, S, c0 + row, row);
        __syncthreads();
        eval_chunk<float>(R, S, rows);
        for (int row = warp; row < rows; row += nw) {
            for (int d = lane; d < Dp; d += 32) X[(size_t)(c0 + row) * Dp + d] = S.Xc[(size_t)row * Dp + d];
            if (lane == 0) F[c0 + row] = S.rowF[row];
        }
        __syncthreads();
    }
}

// k candidates per protozoon (rank r, candidate c = q mod k): the rows of
// Xcand [ps k][Dp] and the network inputs Xin [ps k][Kp] (bf16, scaled to
// [-1, 1] by the bounds).
template <int QPL>
__global__ void __launch_bounds__(kSurThreads) surr_gen_kernel(const ApoRun* __restrict__ run, int k, int t,
                                                              const uint32_t* __restrict__ perm,
                                                              const float* __restrict__ X, const float* __restrict__ F,
                                                              float* __restrict__ Xcand, __nv_bfloat16* __restrict__ Xin,
                                                              int Kp)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    Smem<float> S;
    surr_setup<QPL>(run, R, smem, S, perm, true);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int D = R.prob.D, Dp = R.prob.Dp, CH = R.plan.chunk;
    const int nrow = R.ps * k;
    const IterScal is = iter_scal(R, t, magic64((uint32_t)R.ps));
    for (int c0 = blockIdx.x * CH; c0 < nrow; c0 += gridDim.x * CH) {
        const int rows = min(CH, nrow - c0);
        for (int row = warp; row < rows; row += nw) {
            const int q = c0 + row, r = q / k, c = q - r * k;
            gen_step_row<float, QPL>(R, S, X, nullptr, F, S.perm[0], false, false, t, is, r, dr_state(R, t, r), row, c);
            __syncwarp();
            for (int d = lane; d < Dp; d += 32) Xcand[(size_t)q * Dp + d] = S.Xc[(size_t)row * Dp + d];
            if (Xin)
                for (int d = lane; d < Kp; d += 32) {
                    float v = 0.f;
                    if (d < D) v = 2.f * (S.Xc[(size_t)row * Dp + d] - S.lb[d]) / (S.ub[d] - S.lb[d]) - 1.f;
                    Xin[(size_t)q * Kp + d] = __float2bfloat16(v);
                }
        }
        __syncthreads();
    }
}

// For every rank: the best-scored candidate (candidate 0 when kk == 1) is
// evaluated exactly and replaces the protozoon iff it improves it (Algorithm
// 1); the evaluation is appended to the archive.
template <int QPL>
__global__ void __launch_bounds__(kSurThreads) surr_select_kernel(
    const ApoRun* __restrict__ run, int k, int kk, const uint32_t* __restrict__ perm, const float* __restrict__ X,
    const float* __restrict__ F, const float* __restrict__ Xcand, const float* __restrict__ score,
    float* __restrict__ Xn, float* __restrict__ Fn, __nv_bfloat16* __restrict__ Xa, float* __restrict__ Fa, int Kp,
    long long arch_pos, int arch_cap, float* __restrict__ pred, float* __restrict__ truth)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    __shared__ int s_c[64];
    Smem<float> S;
    surr_setup<QPL>(run, R, smem, S, nullptr, false);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int D = R.prob.D, Dp = R.prob.Dp, CH = R.plan.chunk, ps = R.ps;
    for (int c0 = blockIdx.x * CH; c0 < ps; c0 += gridDim.x * CH) {
        const int rows = min(CH, ps - c0);
        for (int row = warp; row < rows; row += nw) {
            const int r = c0 + row;
            int best = 0;
            if (kk > 1) {
                float bv = INFINITY;
                for (int c = 0; c < kk; ++c) {
                    const float v = score[(size_t)r * k + c];
                    if (v < bv) { bv = v; best = c; }
                }
            }
            if (lane == 0) {
                s_c[row] = best;
                S.rowF[CH + row] = F[perm[r]];
            }
            for (int d = lane; d < Dp; d += 32) S.Xc[(size_t)row * Dp + d] = Xcand[((size_t)r * k + best) * Dp + d];
        }
        __syncthreads();
        eval_chunk<float>(R, S, rows);
        for (int row = warp; row < rows; row += nw) {
            const int r = c0 + row, slot = (int)perm[r];
            const float fo = S.rowF[CH + row], fn = S.rowF[row];
            const bool acc = fn < fo;
            for (int d = lane; d < Dp; d += 32)
                Xn[(size_t)slot * Dp + d] = acc ? S.Xc[(size_t)row * Dp + d] : X[(size_t)slot * Dp + d];
            const long long pos = (arch_pos + r) % arch_cap;
            for (int d = lane; d < Kp; d += 32) {
                float v = 0.f;
                if (d < D) v = 2.f * (S.Xc[(size_t)row * Dp + d] - S.lb[d]) / (S.ub[d] - S.lb[d]) - 1.f;
                Xa[(size_t)pos * Kp + d] = __float2bfloat16(v);
            }
            if (lane == 0) {
                Fn[slot] = acc ? fn : fo;
                Fa[pos] = fn;
                pred[r] = kk > 1 ? score[(size_t)r * k + s_c[row]] : NAN;
                truth[r] = fn;
            }
        }
        __syncthreads();
    }
}

// Training targets: standardised log1p(F - min F) over the archive.
__global__ void __launch_bounds__(1024) surr_targets_kernel(int n, const float* __restrict__ Fa_ring,
                                                            float* __restrict__ tgt_ring, long long start, int cap)
{
    // rows i of the window live at (start + i) mod cap
#define Fa(i) Fa_ring[(start + (i)) % cap]
#define TG(i) tgt_ring[(start + (i)) % cap]
    __shared__ double red[1024];
    __shared__ double s_min, s_mean, s_std;
    double mn = INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mn = fmin(mn, (double)Fa(i));
    red[threadIdx.x] = mn;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) s_min = red[0];
    __syncthreads();
    double s = 0.0, s2 = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double v = log1p((double)Fa(i) - s_min);
        s += v;
        s2 += v * v;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_mean = red[0] / n;
    __syncthreads();
    red[threadIdx.x] = s2;
    __syncthreads();
    for (int o = blockDim.x / 2; o; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) s_std = sqrt(fmax(red[0] / n - s_mean * s_mean, 1e-12));
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        TG(i) = (float)((log1p((double)Fa(i) - s_min) - s_mean) / s_std);
#undef Fa
#undef TG
}

double spearman(const std::vector<float>& a, const std::vector<float>& b)
{
    const size_t n = a.size();
    auto ranks = [](const std::vector<float>& v) {
        std::vector<size_t> idx(v.size());
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](size_t i, size_t j) { return v[i] < v[j]; });
        std::vector<double> r(v.size());
        for (size_t i = 0; i < idx.size(); ++i) r[idx[i]] = (double)i;
        return r;
    };
    const std::vector<double> ra = ranks(a), rb = ranks(b);
    double ma = 0, mb = 0;
    for (size_t i = 0; i < n; ++i) { ma += ra[i]; mb += rb[i]; }
    ma /= n; mb /= n;
    double sab = 0, saa = 0, sbb = 0;
    for (size_t i = 0; i < n; ++i) {
        sab += (ra[i] - ma) * (rb[i] - mb);
        saa += (ra[i] - ma) * (ra[i] - ma);
        sbb += (rb[i] - mb) * (rb[i] - mb);
    }
    return (saa > 0 && sbb > 0) ? sab / std::sqrt(saa * sbb) : 0.0;
}

}  // namespace

namespace {

template <int QPL>
cudaError_t launch_surr(int which, dim3 grid, size_t smem, cudaStream_t st, const ApoRun* run, int k, int kk, int t,
                        const uint32_t* perm, const float* X, const float* F, float* Xcand, __nv_bfloat16* Xin,
                        int Kp, const float* score, float* Xn, float* Fn, __nv_bfloat16* Xa, float* Fa,
                        long long arch_pos, int arch_cap, float* pred, float* truth)
{
    if (which == 0) {
        cudaError_t e = cudaFuncSetAttribute(surr_init_kernel<QPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        surr_init_kernel<QPL><<<grid, kSurThreads, smem, st>>>(run, Xn, Fn);
    } else if (which == 1) {
        cudaError_t e = cudaFuncSetAttribute(surr_gen_kernel<QPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        surr_gen_kernel<QPL><<<grid, kSurThreads, smem, st>>>(run, k, t, perm, X, F, Xcand, Xin, Kp);
    } else {
        cudaError_t e = cudaFuncSetAttribute(surr_select_kernel<QPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        surr_select_kernel<QPL><<<grid, kSurThreads, smem, st>>>(run, k, kk, perm, X, F, Xcand, score, Xn, Fn, Xa, Fa,
                                                                 Kp, arch_pos, arch_cap, pred, truth);
    }
    return cudaGetLastError();
}

cudaError_t launch_surr_q(int qpl, int which, dim3 grid, size_t smem, cudaStream_t st, const ApoRun* run, int k, int kk,
                          int t, const uint32_t* perm, const float* X, const float* F, float* Xcand,
                          __nv_bfloat16* Xin, int Kp, const float* score, float* Xn, float* Fn, __nv_bfloat16* Xa,
                          float* Fa, long long arch_pos, int arch_cap, float* pred, float* truth)
{
    switch (qpl) {
    case 1: return launch_surr<1>(which, grid, smem, st, run, k, kk, t, perm, X, F, Xcand, Xin, Kp, score, Xn, Fn, Xa, Fa, arch_pos, arch_cap, pred, truth);
    case 2: return launch_surr<2>(which, grid, smem, st, run, k, kk, t, perm, X, F, Xcand, Xin, Kp, score, Xn, Fn, Xa, Fa, arch_pos, arch_cap, pred, truth);
    default: return launch_surr<4>(which, grid, smem, st, run, k, kk, t, perm, X, F, Xcand, Xin, Kp, score, Xn, Fn, Xa, Fa, arch_pos, arch_cap, pred, truth);
    }
}

}  // namespace

#include "apo_plan.h"

// Test hook: the k candidates of every protozoon at iteration `iter` from a
// given population, generated by the surrogate path's own sort and
// candidate kernels (candidate c draws from the plain slots | (c << 8)).
extern "C" apo_status apo_surrogate_candidates(const apo_problem* P, const apo_params* p_in, int iter, int k,
                                               void* stream, const float* d_X, const float* d_F, float* d_Xcand)
{
    if (!P || !p_in || !d_X || !d_F || !d_Xcand) { apo::set_last_error("apo_surrogate_candidates: NULL argument"); return APO_ERR_INVALID_ARG; }
    if (P->kind == APO_OBJ_OTSU) { apo::set_last_error("apo_surrogate_candidates: float objectives only"); return APO_ERR_UNSUPPORTED; }
    if (P->D > kSmallMaxDim) { apo::set_last_error("apo_surrogate_candidates: D <= 256 only"); return APO_ERR_UNSUPPORTED; }
    apo_params q;
    if (const char* why = normalize_params(p_in, &q)) { apo::set_last_error(why); return APO_ERR_INVALID_ARG; }
    const apo_params* p = &q;
    if (iter < 1 || iter > p->max_iter || k < 1 || k > 32) {
        apo::set_last_error("apo_surrogate_candidates: arguments out of range");
        return APO_ERR_INVALID_ARG;
    }
    if (p->ps > 4096) { apo::set_last_error("apo_surrogate_candidates: ps above 4096"); return APO_ERR_UNSUPPORTED; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ps = p->ps, T = p->max_iter, D = P->D, Dp = P->Dp;
    const int ps_pad = plan_pow2(ps);
    const int qpl = D <= 64 ? 1 : (D <= 128 ? 2 : 4);
    const SmemPlan plan = choose_plan(P, ps, false, false, 232448 - 2048, kChunk);   // one CTA per chunk
    const int W = (ps + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (off + 255) / 256 * 256; const size_t at = off; off += bytes; return at; };
    const size_t o_run = take(sizeof(ApoRun)), o_offs = take(8), o_dr = take((size_t)(T + 1) * W * 4);
    const size_t o_x = take((size_t)ps * Dp * 4), o_f = take((size_t)ps * 4);
    const size_t o_p0 = take((size_t)ps * 4), o_p1 = take((size_t)ps * 4), o_xc = take((size_t)ps * k * Dp * 4);
    void* ws = nullptr;
    if (cudaMalloc(&ws, off) != cudaSuccess) { apo::set_last_error("apo_surrogate_candidates: workspace allocation failed"); return APO_ERR_OOM; }
    unsigned char* b = static_cast<unsigned char*>(ws);
    ApoRun R;
    std::memset(&R, 0, sizeof(R));
    R.prob = P->dev;
    R.plan = plan;
    R.ps = ps; R.np = p->np; R.T = T; R.pdr_form = p->pdr_form; R.pf_max = p->pf_max;
    R.pair_policy = p->pair_policy;
    R.seed = p->seed; R.run = p->run; R.t_begin = iter; R.t_end = iter; R.flags = 0; R.g = 1;
    apo_status rc = sched_tables(ps, p->pdr_form, T, &R.thr_dr, &R.thr_ah, &R.fsc, &R.nsc);
    R.drmask = reinterpret_cast<const uint32_t*>(b + o_dr);
    const int offs[2] = {0, 1};
    std::vector<uint32_t> ident(ps);
    std::iota(ident.begin(), ident.end(), 0u);
    const ApoRun* d_run = reinterpret_cast<const ApoRun*>(b + o_run);
    float* Xp = reinterpret_cast<float*>(b + o_x);
    float* Fp = reinterpret_cast<float*>(b + o_f);
    uint32_t* p0 = reinterpret_cast<uint32_t*>(b + o_p0);
    uint32_t* p1 = reinterpret_cast<uint32_t*>(b + o_p1);
    float* Xc = reinterpret_cast<float*>(b + o_xc);
    cudaError_t e = rc == APO_OK ? cudaSuccess : cudaErrorUnknown;
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_run, &R, sizeof(R), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_offs, offs, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p0, ident.data(), (size_t)ps * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(Xp, 0, (size_t)ps * Dp * 4, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Xp, (size_t)Dp * 4, d_X, (size_t)D * 4, (size_t)D * 4, ps, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Fp, d_F, (size_t)ps * 4, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = launch_dr(d_run, reinterpret_cast<const int*>(b + o_offs), 1, 1, ps_pad, st);
    if (e == cudaSuccess) {
        const size_t sort_smem = (size_t)ps_pad * 8;
        if (sort_smem > 48 * 1024)
            cudaFuncSetAttribute(surr_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);
        surr_sort_kernel<<<1, 1024, sort_smem, st>>>(ps, ps_pad, Fp, p0, p1, nullptr, iter);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = launch_surr_q(qpl, 1, dim3(std::max(1, std::min(1024, (ps * k + plan.chunk - 1) / plan.chunk))), plan.total,
                          st, d_run, k, k, iter, p1, Xp, Fp, Xc, nullptr, 0, nullptr, nullptr, nullptr, nullptr,
                          nullptr, 0, 0, nullptr, nullptr);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(d_Xcand, (size_t)D * 4, Xc, (size_t)Dp * 4, (size_t)D * 4, (size_t)ps * k,
                              cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(ws);
    if (e != cudaSuccess) {
        char m[200];
        snprintf(m, sizeof(m), "apo_surrogate_candidates: %s", cudaGetErrorString(e));
        apo::set_last_error(m);
        return APO_ERR_CUDA;
    }
    return APO_OK;
}

extern "C" apo_status apo_run_surrogate(const apo_problem* P, const apo_params* p_in, const apo_surrogate_params* sp,
                                        void* stream, float* best_x, double* best_f, float* curve,
                                        apo_surrogate_stats* stats)
{
    if (!P || !p_in || !sp || !best_x || !best_f) { apo::set_last_error("apo_run_surrogate: NULL argument"); return APO_ERR_INVALID_ARG; }
    if (P->kind == APO_OBJ_OTSU) { apo::set_last_error("apo_run_surrogate: float objectives only"); return APO_ERR_UNSUPPORTED; }
    if (P->D > kSmallMaxDim) { apo::set_last_error("apo_run_surrogate: D <= 256 only"); return APO_ERR_UNSUPPORTED; }
    apo_params q;
    if (const char* why = normalize_params(p_in, &q)) { apo::set_last_error(why); return APO_ERR_INVALID_ARG; }
    const apo_params* p = &q;
    if (p->ps > 4096) { apo::set_last_error("apo_run_surrogate: ps above 4096"); return APO_ERR_UNSUPPORTED; }
    const int k = sp->k, R_every = sp->retrain_every;
    if (k < 1 || k > 32 || R_every < 1 || sp->archive_cap < p->ps || sp->train_steps < 0 || sp->batch < 1) {
        apo::set_last_error("apo_run_surrogate: surrogate params out of range (1 <= k <= 32, retrain_every >= 1, "
                            "archive_cap >= ps, batch >= 1)");
        return APO_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int ps = p->ps, T = p->max_iter, D = P->D, Dp = P->Dp;
    const int ps_pad = plan_pow2(ps);
    const int qpl = D <= 64 ? 1 : (D <= 128 ? 2 : 4);
    int* status = device_status_word();
    if (!status) { apo::set_last_error("status word allocation failed"); return APO_ERR_OOM; }

    apo_mlp* M = nullptr;
    apo_status rc = apo_mlp_create(D, sp->net_seed, &M);
    if (rc != APO_OK) return rc;
    if (M->cap < ps * k) {
        cudaFree(M->mem);
        rc = mlp_alloc(M, ps * k);
        if (rc != APO_OK) { delete M; return rc; }
        // re-initialise the parameters of the larger allocation
        apo_mlp* tmp = nullptr;
        rc = apo_mlp_create(D, sp->net_seed, &tmp);
        if (rc != APO_OK) { apo_mlp_destroy(M); return rc; }
        cudaMemcpy(M->W1, tmp->W1, (size_t)M->Kp * kH * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(M->W2, tmp->W2, (size_t)kH * kH * 4, cudaMemcpyDeviceToDevice);
        cudaMemcpy(M->w3, tmp->w3, kH * 4, cudaMemcpyDeviceToDevice);
        apo_mlp_destroy(tmp);
        refresh_bf16(M, 0);
    }
    const int Kp = M->Kp;
    const SmemPlan plan = choose_plan(P, ps, false, false, 232448 - 2048, kChunk);   // one CTA per chunk

    // workspace
    const int W = (ps + 31) / 32;
    const int acap = sp->archive_cap;
    size_t off = 0;
    auto take = [&](size_t bytes) { off = (off + 255) / 256 * 256; const size_t at = off; off += bytes; return at; };
    const size_t o_run = take(sizeof(ApoRun)), o_offs = take(8), o_dr = take((size_t)(T + 1) * W * 4);
    const size_t o_x0 = take((size_t)ps * Dp * 4), o_x1 = take((size_t)ps * Dp * 4);
    const size_t o_f0 = take((size_t)ps * 4), o_f1 = take((size_t)ps * 4);
    const size_t o_p0 = take((size_t)ps * 4), o_p1 = take((size_t)ps * 4);
    const size_t o_xc = take((size_t)ps * k * Dp * 4), o_xa = take((size_t)acap * Kp * 2);
    const size_t o_fa = take((size_t)acap * 4), o_tg = take((size_t)acap * 4);
    const size_t o_pr = take((size_t)ps * 4), o_tr = take((size_t)ps * 4), o_cv = take((size_t)(T + 1) * 4);
    void* ws = nullptr;
    cudaError_t e = cudaMalloc(&ws, off);
    if (e != cudaSuccess) { apo_mlp_destroy(M); apo::set_last_error("apo_run_surrogate: workspace allocation failed"); return APO_ERR_OOM; }
    unsigned char* b = static_cast<unsigned char*>(ws);
    auto fail = [&](apo_status s, const char* msg) {
        if (msg) apo::set_last_error(msg);
        cudaStreamSynchronize(st);
        cudaFree(ws);
        apo_mlp_destroy(M);
        return s;
    };

    ApoRun R;
    std::memset(&R, 0, sizeof(R));
    R.prob = P->dev;
    R.plan = plan;
    R.ps = ps; R.np = p->np; R.T = T; R.pdr_form = p->pdr_form; R.pf_max = p->pf_max;
    R.pair_policy = p->pair_policy;
    R.seed = p->seed; R.run = p->run; R.t_begin = 1; R.t_end = T; R.flags = kFlagInit; R.g = 1;
    if (sched_tables(ps, p->pdr_form, T, &R.thr_dr, &R.thr_ah, &R.fsc, &R.nsc) != APO_OK)
        return fail(APO_ERR_CUDA, nullptr);
    R.drmask = reinterpret_cast<const uint32_t*>(b + o_dr);
    const int offs[2] = {0, T};
    std::vector<uint32_t> ident(ps);
    std::iota(ident.begin(), ident.end(), 0u);
    e = cudaMemcpyAsync(b + o_run, &R, sizeof(R), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_offs, offs, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_p0, ident.data(), (size_t)ps * 4, cudaMemcpyHostToDevice, st);
    const ApoRun* d_run = reinterpret_cast<const ApoRun*>(b + o_run);
    if (e == cudaSuccess) e = launch_dr(d_run, reinterpret_cast<const int*>(b + o_offs), 1, T, ps_pad, st);
    if (e != cudaSuccess) return fail(APO_ERR_CUDA, "apo_run_surrogate: set-up failed");

    float* X[2] = {reinterpret_cast<float*>(b + o_x0), reinterpret_cast<float*>(b + o_x1)};
    float* F[2] = {reinterpret_cast<float*>(b + o_f0), reinterpret_cast<float*>(b + o_f1)};
    uint32_t* pm[2] = {reinterpret_cast<uint32_t*>(b + o_p0), reinterpret_cast<uint32_t*>(b + o_p1)};
    float* Xcand = reinterpret_cast<float*>(b + o_xc);
    __nv_bfloat16* Xa = reinterpret_cast<__nv_bfloat16*>(b + o_xa);
    float* Fa = reinterpret_cast<float*>(b + o_fa);
    float* tgt = reinterpret_cast<float*>(b + o_tg);
    float* pred = reinterpret_cast<float*>(b + o_pr);
    float* truth = reinterpret_cast<float*>(b + o_tr);
    float* d_curve = reinterpret_cast<float*>(b + o_cv);
    const size_t smem = plan.total;
    const int grid_rows = (ps + plan.chunk - 1) / plan.chunk;
    const size_t sort_smem = (size_t)ps_pad * 8;
    if (sort_smem > 48 * 1024) cudaFuncSetAttribute(surr_sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem);

    cudaEvent_t t_all0, t_all1, tr0, tr1;
    cudaEventCreate(&t_all0); cudaEventCreate(&t_all1); cudaEventCreate(&tr0); cudaEventCreate(&tr1);
    cudaEventRecord(t_all0, st);
    // initial population, evaluated and archived
    e = launch_surr_q(qpl, 0, dim3(grid_rows), smem, st, d_run, 1, 1, 0, pm[0], nullptr, nullptr, nullptr, nullptr, Kp,
                      nullptr, X[0], F[0], nullptr, nullptr, 0, acap, nullptr, nullptr);
    if (e != cudaSuccess) return fail(APO_ERR_CUDA, "apo_run_surrogate: init launch failed");
    long long arch_count = 0;   // the initial population is not archived (no candidate image)
    int cur = 0, pc = 0;
    bool screening = false;
    apo_surrogate_stats S = {};
    S.true_evals = ps;
    double train_ms = 0.0;
    for (int t = 1; t <= T; ++t) {
        surr_sort_kernel<<<1, 1024, sort_smem, st>>>(ps, ps_pad, F[cur], pm[pc], pm[pc ^ 1], d_curve, t);
        pc ^= 1;
        const int kk = screening ? k : 1;
        e = launch_surr_q(qpl, 1, dim3(std::max(1, std::min(1024, (ps * kk + plan.chunk - 1) / plan.chunk))), smem, st,
                          d_run, kk, kk, t, pm[pc], X[cur], F[cur], Xcand, kk > 1 ? M->Xb : nullptr, Kp, nullptr,
                          nullptr, nullptr, nullptr, nullptr, 0, acap, nullptr, nullptr);
        if (e != cudaSuccess) return fail(APO_ERR_CUDA, "apo_run_surrogate: candidate launch failed");
        if (kk > 1) {
            rc = mlp_forward_rows(M, ps * kk, st);
            if (rc != APO_OK) return fail(rc, nullptr);
        }
        e = launch_surr_q(qpl, 2, dim3(grid_rows), smem, st, d_run, kk, kk, t, pm[pc], X[cur], F[cur], Xcand, nullptr,
                          Kp, M->y, X[cur ^ 1], F[cur ^ 1], Xa, Fa, arch_count, acap, pred, truth);
        if (e != cudaSuccess) return fail(APO_ERR_CUDA, "apo_run_surrogate: select launch failed");
        arch_count += ps;
        cur ^= 1;
        S.true_evals += ps;
        S.screened += (long long)ps * kk;
        if (kk > 1) ++S.screening_iters;
        if (t % R_every == 0 && t < T) {
            // error monitor of the last screened batch, then retrain
            if (screening) {
                std::vector<float> hp(ps), ht(ps);
                cudaMemcpyAsync(hp.data(), pred, (size_t)ps * 4, cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(ht.data(), truth, (size_t)ps * 4, cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                S.last_rank_corr = spearman(hp, ht);
            }
            // the training window: the most recent rows of the archive
            const long long avail = std::min<long long>(arch_count, acap);
            const int n = (int)std::min<long long>(avail, sp->train_window > 0 ? sp->train_window : avail);
            const long long start = ((arch_count - n) % acap + acap) % acap;
            surr_targets_kernel<<<1, 1024, 0, st>>>(n, Fa, tgt, start, acap);
            cudaEventRecord(tr0, st);
            rc = mlp_train_rows(M, Xa, tgt, n, sp->train_steps, sp->batch, sp->lr, sp->net_seed + (uint32_t)t, st,
                                start, acap);
            cudaEventRecord(tr1, st);
            if (rc != APO_OK) return fail(rc, nullptr);
            ++S.retrains;
            const bool was = screening;
            screening = !was || S.last_rank_corr >= sp->min_rank_corr;
            cudaEventSynchronize(tr1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, tr0, tr1);
            train_ms += ms;
        }
        if (kk == 1 && t > R_every) ++S.fallback_iters;
    }
    // the best of the final population
    surr_sort_kernel<<<1, 1024, sort_smem, st>>>(ps, ps_pad, F[cur], pm[pc], pm[pc ^ 1], d_curve, T + 1);
    pc ^= 1;
    uint32_t bslot = 0;
    e = cudaMemcpyAsync(&bslot, pm[pc], 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<float> xb(Dp);
    float fb = 0.f;
    if (e == cudaSuccess) e = cudaMemcpy(xb.data(), X[cur] + (size_t)bslot * Dp, (size_t)Dp * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&fb, F[cur] + bslot, 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && curve) e = cudaMemcpy(curve, d_curve, (size_t)(T + 1) * 4, cudaMemcpyDeviceToHost);
    cudaEventRecord(t_all1, st);
    cudaEventSynchronize(t_all1);
    float all_ms = 0.f;
    cudaEventElapsedTime(&all_ms, t_all0, t_all1);
    cudaEventDestroy(t_all0); cudaEventDestroy(t_all1); cudaEventDestroy(tr0); cudaEventDestroy(tr1);
    if (e != cudaSuccess) return fail(APO_ERR_CUDA, "apo_run_surrogate: result copy failed");
    std::memcpy(best_x, xb.data(), sizeof(float) * D);
    *best_f = fb;
    S.train_ms = train_ms;
    S.total_ms = all_ms;
    if (stats) *stats = S;
    cudaFree(ws);
    apo_mlp_destroy(M);
    int h = 0;
    cudaMemcpy(&h, status, 4, cudaMemcpyDeviceToHost);
    if (h != 0) {
        cudaMemset(status, 0, 4);
        apo::set_last_error("a device-side wait exceeded its limit");
        return (apo_status)h;
    }
    return APO_OK;
}
