// apo_mlp.h -- surrogate-network kernels (apo_mlp.cu) used by the
// surrogate-assisted APO driver.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

namespace apo {

// Arguments of the bf16 tensor-core GEMM (see gemm_bf16_kernel).
struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    int lda;
    const __nv_bfloat16* B;
    int ldb;
    const float* bias;   // [N] or nullptr
    const float* mask;   // [M][ldm] fp32, keep where > 0 (ReLU derivative), or nullptr
    int ldm;
    int relu;
    float* Cf;           // fp32 output or nullptr
    int ldc;
    __nv_bfloat16* Cb;   // bf16 output or nullptr
    int ldcb;
    float* ws;           // split-K workspace owned by the caller, or nullptr (no split)
    size_t ws_elems;     // its size in floats; kSplitWsElems covers every shape
};

// Split K runs only with fewer than 128 output tiles of 128 x 64, and then
// ksplit M N <= 128 (128 x 64): one workspace of this many floats serves
// every GEMM shape.
constexpr size_t kSplitWsElems = (size_t)128 * 128 * 64;

cudaError_t gemm_bf16(const GemmArgs& g, bool ta, bool tb, cudaStream_t st);
cudaError_t launch_out_layer(int M, int K, const __nv_bfloat16* H, const __nv_bfloat16* w, const float* b, float* y,
                             cudaStream_t st);
cudaError_t launch_out_backward(int M, int K, const float* y, const float* t, const __nv_bfloat16* w3,
                                const float* Z2, float* dZ2, __nv_bfloat16* dZ2b, float* loss, cudaStream_t st);
cudaError_t launch_colsum(int M, int K, const float* A, const __nv_bfloat16* Ab, const float* rowscale, float* out,
                          cudaStream_t st);
cudaError_t launch_dy(int M, const float* y, const float* t, float* dy, cudaStream_t st);
cudaError_t launch_adam(int n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, int step,
                        cudaStream_t st);
cudaError_t launch_gather_rows(int B, int Kp, const int* idx, const __nv_bfloat16* Xa, const float* ta,
                               __nv_bfloat16* Xb, float* tb, cudaStream_t st);

}  // namespace apo
