// apo_peaks.cu -- microbenchmarks of the pipes that bound the fused APO
// kernels (FP32 FFMA, integer IMAD, and the plain-ALU issue rate), so that
// their roofline fractions are taken against throughputs measured on the
// device rather than derived from unit counts.  Each kernel runs many
// independent dependency chains per thread (enough to hide the pipe
// latency), on every SM, and the rate is ops / elapsed time (CUDA events).
#include <cstdio>

#include "../../include/apo.h"
#include "apo_internal.h"

namespace apo {
namespace {

constexpr int kChains = 8;

// 2 * kChains * iters FP32 flop per thread (fused multiply-adds).
__global__ void __launch_bounds__(256) ffma_kernel(int iters, float a, float b, float* out)
{
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 1234.5f) out[0] = s;   // keeps the chains live
}

// kChains * iters 32-bit integer multiply-adds per thread.
__global__ void __launch_bounds__(256) imad_kernel(int iters, unsigned a, unsigned b, unsigned* out)
{
    unsigned v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = v[c] * a + b;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= v[c];
    if (s == 0x12345u) out[0] = s;
}

// kChains * iters plain ALU operations (xor-add) per thread: the issue rate
// of simple integer instructions.
__global__ void __launch_bounds__(256) alu_kernel(int iters, unsigned a, unsigned* out)
{
    unsigned v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = threadIdx.x * 7u + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) v[c] = (v[c] ^ a) + (unsigned)c;
    }
    unsigned s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += v[c];
    if (s == 0x12345u) out[0] = s;
}

template <typename F>
double time_ms(F launch, cudaStream_t st)
{
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    launch();   // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace
}  // namespace apo

extern "C" apo_status apo_measure_peaks(void* stream, double* ffma_tflops, double* imad_tops, double* alu_tops)
{
    using namespace apo;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("apo_measure_peaks: no device");
        return APO_ERR_CUDA;
    }
    void* sink = nullptr;
    if (cudaMalloc(&sink, 64) != cudaSuccess) { set_last_error("apo_measure_peaks: allocation failed"); return APO_ERR_OOM; }
    const int blocks = sms * 8, threads = 256, iters = 1 << 14;
    const double per_thread = (double)kChains * iters, n_threads = (double)blocks * threads;
    const double t_ffma = time_ms([&] { ffma_kernel<<<blocks, threads, 0, st>>>(iters, 1.0000001f, 1e-7f, (float*)sink); }, st);
    const double t_imad = time_ms([&] { imad_kernel<<<blocks, threads, 0, st>>>(iters, 1664525u, 1013904223u, (unsigned*)sink); }, st);
    const double t_alu = time_ms([&] { alu_kernel<<<blocks, threads, 0, st>>>(iters, 0x9E3779B9u, (unsigned*)sink); }, st);
    const cudaError_t e = cudaGetLastError();
    cudaFree(sink);
    if (e != cudaSuccess) { set_last_error("apo_measure_peaks: launch failed"); return APO_ERR_CUDA; }
    if (ffma_tflops) *ffma_tflops = 2.0 * per_thread * n_threads / (t_ffma * 1e-3) / 1e12;
    if (imad_tops) *imad_tops = per_thread * n_threads / (t_imad * 1e-3) / 1e12;
    // the xor-add is two operations
    if (alu_tops) *alu_tops = 2.0 * per_thread * n_threads / (t_alu * 1e-3) / 1e12;
    return APO_OK;
}
