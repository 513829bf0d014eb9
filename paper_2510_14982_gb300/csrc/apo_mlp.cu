// apo_mlp.cu -- the surrogate network of the surrogate-assisted APO form: an
// MLP D -> 256 -> 256 -> 1 (ReLU) with bfloat16 weights and activations and
// float32 accumulation, trained online with mean squared error and Adam.
//
// Kernels: a bfloat16 tensor-core GEMM (mma.sync m16n8k16, fp32 accumulate)
// with fused epilogues (bias, ReLU, ReLU-derivative mask, fp32 and bf16
// outputs), the 256 -> 1 output layer and its gradients, column sums for the
// bias gradients, the loss gradient, Adam, and the gather of a training batch
// from the archive.
#include <cuda_bf16.h>

#include "apo_mlp.h"

namespace apo {

constexpr int kGT = 64;        // GEMM tile (rows and columns) per CTA
constexpr int kGK = 32;        // K step
constexpr int kGPad = 8;       // shared-memory row padding (bf16 elements)

__device__ __forceinline__ uint32_t pack_bf16(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n]; then v = acc + bias[n],
// v *= (mask[m ldm + n] > 0) when mask, v = max(v, 0) when relu; stored to
// Cf (fp32) and / or Cb (bf16).  128 threads: 2 x 2 warps of 32 x 32.
template <bool TA, bool TB>
__global__ void __launch_bounds__(128) gemm_bf16_kernel(GemmArgs g)
{
    __shared__ __align__(16) __nv_bfloat16 As[kGT][kGK + kGPad];
    __shared__ __align__(16) __nv_bfloat16 Bs[kGT][kGK + kGPad];   // Bs[n][k]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = 0; k0 < g.K; k0 += kGK) {
        for (int i = tid; i < kGT * kGK; i += 128) {
            const int r = i / kGK, kk = i - r * kGK;
            const int m = m0 + r, k = k0 + kk;
            As[r][kk] = (m < g.M && k < g.K) ? (TA ? g.A[(size_t)k * g.lda + m] : g.A[(size_t)m * g.lda + k]) : zero;
            const int n = n0 + r;
            Bs[r][kk] = (n < g.N && k < g.K) ? (TB ? g.B[(size_t)n * g.ldb + k] : g.B[(size_t)k * g.ldb + n]) : zero;
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kGK; ks += 16) {
            uint32_t af[2][4], bfr[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + gq;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][ks + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + 8 * j + gq;
                bfr[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tq]);
                bfr[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[c][ks + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + gq + (e >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tq + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                float v = acc[i][j][e];
                if (g.bias) v += g.bias[n];
                if (g.mask) v = g.mask[(size_t)m * g.ldm + n] > 0.f ? v : 0.f;
                if (g.relu) v = fmaxf(v, 0.f);
                if (g.Cf) g.Cf[(size_t)m * g.ldc + n] = v;
                if (g.Cb) g.Cb[(size_t)m * g.ldcb + n] = __float2bfloat16(v);
            }
}

cudaError_t gemm_bf16(const GemmArgs& g, bool ta, bool tb, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    dim3 grid((g.N + kGT - 1) / kGT, (g.M + kGT - 1) / kGT);
    if (!ta && !tb) gemm_bf16_kernel<false, false><<<grid, 128, 0, st>>>(g);
    else if (ta && !tb) gemm_bf16_kernel<true, false><<<grid, 128, 0, st>>>(g);
    else if (!ta && tb) gemm_bf16_kernel<false, true><<<grid, 128, 0, st>>>(g);
    else gemm_bf16_kernel<true, true><<<grid, 128, 0, st>>>(g);
    return cudaGetLastError();
}

// y[m] = sum_k H[m][k] w[k] + b (warp per row, fp32 accumulation).
__global__ void out_layer_kernel(int M, int K, const __nv_bfloat16* __restrict__ H, const __nv_bfloat16* __restrict__ w,
                                 const float* __restrict__ b, float* __restrict__ y)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= M) return;
    float s = 0.f;
    for (int k = lane; k < K; k += 32)
        s = fmaf(__bfloat162float(H[(size_t)m * K + k]), __bfloat162float(w[k]), s);
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[m] = s + b[0];
}

// Loss gradient dy = 2 (y - t) / M, the output-layer weight and bias
// gradients, and dZ2 = dy w3^T masked by Z2 > 0 (fp32 and bf16).
__global__ void out_backward_kernel(int M, int K, const float* __restrict__ y, const float* __restrict__ t,
                                    const __nv_bfloat16* __restrict__ w3, const float* __restrict__ Z2,
                                    float* __restrict__ dZ2, __nv_bfloat16* __restrict__ dZ2b, float* __restrict__ loss)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)M * K; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / K), k = (int)(i - (size_t)m * K);
        const float dy = 2.f * (y[m] - t[m]) / (float)M;
        const float v = Z2[i] > 0.f ? dy * __bfloat162float(w3[k]) : 0.f;
        dZ2[i] = v;
        dZ2b[i] = __float2bfloat16(v);
        if (k == 0) atomicAdd(loss, (y[m] - t[m]) * (y[m] - t[m]) / (float)M);
    }
}

// out[k] = sum_m A[m][k] * (scale ? scale[m] : 1) * sscale  (column sums; one thread per column,
// rows split over blockIdx.y and summed with atomics)
__global__ void colsum_kernel(int M, int K, const float* __restrict__ A, const __nv_bfloat16* __restrict__ Ab,
                              const float* __restrict__ rowscale, float* __restrict__ out)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int per = (M + gridDim.y - 1) / gridDim.y;
    const int mb = blockIdx.y * per, me = min(M, mb + per);
    float s = 0.f;
    for (int m = mb; m < me; ++m) {
        const float a = A ? A[(size_t)m * K + k] : __bfloat162float(Ab[(size_t)m * K + k]);
        s = fmaf(a, rowscale ? rowscale[m] : 1.f, s);
    }
    atomicAdd(&out[k], s);
}

// dy[m] = 2 (y[m] - t[m]) / M
__global__ void dy_kernel(int M, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ dy)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < M) dy[m] = 2.f * (y[m] - t[m]) / (float)M;
}

// Adam (Kingma and Ba) with bias correction on fp32 master weights; writes the
// bf16 copy used by the GEMMs.
__global__ void adam_kernel(int n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, float lr, float b1, float b2,
                            float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float w = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = w;
        if (pb) pb[i] = __float2bfloat16(w);
    }
}

// Training batch: rows idx[i] of the archive (bf16 inputs and fp32 targets).
__global__ void gather_rows_kernel(int B, int Kp, const int* __restrict__ idx, const __nv_bfloat16* __restrict__ Xa,
                                   const float* __restrict__ ta, __nv_bfloat16* __restrict__ Xb, float* __restrict__ tb)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * Kp; i += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(i / Kp), c = (int)(i - (size_t)r * Kp);
        const int s = idx[r];
        Xb[i] = Xa[(size_t)s * Kp + c];
        if (c == 0) tb[r] = ta[s];
    }
}

cudaError_t launch_out_layer(int M, int K, const __nv_bfloat16* H, const __nv_bfloat16* w, const float* b, float* y,
                             cudaStream_t st)
{
    if (M <= 0) return cudaSuccess;
    out_layer_kernel<<<(M + 7) / 8, 256, 0, st>>>(M, K, H, w, b, y);
    return cudaGetLastError();
}

cudaError_t launch_out_backward(int M, int K, const float* y, const float* t, const __nv_bfloat16* w3, const float* Z2,
                                float* dZ2, __nv_bfloat16* dZ2b, float* loss, cudaStream_t st)
{
    const size_t n = (size_t)M * K;
    const int grid = (int)std::min<size_t>((n + 255) / 256, 4096);
    out_backward_kernel<<<grid, 256, 0, st>>>(M, K, y, t, w3, Z2, dZ2, dZ2b, loss);
    return cudaGetLastError();
}

cudaError_t launch_colsum(int M, int K, const float* A, const __nv_bfloat16* Ab, const float* rowscale, float* out,
                          cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(float) * K, st);
    if (e != cudaSuccess) return e;
    dim3 grid((K + 127) / 128, std::max(1, std::min(64, M / 16)));
    colsum_kernel<<<grid, 128, 0, st>>>(M, K, A, Ab, rowscale, out);
    return cudaGetLastError();
}

cudaError_t launch_dy(int M, const float* y, const float* t, float* dy, cudaStream_t st)
{
    dy_kernel<<<(M + 255) / 256, 256, 0, st>>>(M, y, t, dy);
    return cudaGetLastError();
}

cudaError_t launch_adam(int n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, int step,
                        cudaStream_t st)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<std::min(1024, (n + 255) / 256), 256, 0, st>>>(n, p, g, m, v, pb, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(int B, int Kp, const int* idx, const __nv_bfloat16* Xa, const float* ta,
                               __nv_bfloat16* Xb, float* tb, cudaStream_t st)
{
    const size_t n = (size_t)B * Kp;
    gather_rows_kernel<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(B, Kp, idx, Xa, ta, Xb, tb);
    return cudaGetLastError();
}

}  // namespace apo
