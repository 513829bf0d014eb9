// apo_hist.cu -- 256-bin histograms of 8-bit images and the Otsu prefix
// tables (the thresholding application of the cuAPO paper, Sec. 5.2).
//
// The histogram is HBM-bound: every pixel byte is read once with 16-byte
// vector loads and counted into per-warp shared-memory sub-histograms, which
// are merged into the image's global int32 bins with one atomic per bin and
// CTA.  Integer counting makes the result independent of the order of
// accumulation (bit-exact).
#include "apo_internal.h"

namespace apo {

constexpr int kHistThreads = 256;
constexpr int kHistWarps = kHistThreads / 32;
constexpr int kHistCopies = 4;                 // sub-histograms per warp (lane & 3)
constexpr int kHistStride = 257;               // one pad word: copies sit on shifted banks

__global__ void __launch_bounds__(kHistThreads) histogram_u8_kernel(const uint8_t* __restrict__ px,
                                                                    long long n_per_image,
                                                                    long long chunk, int32_t* hist)
{
    // Equal pixel values within a warp serialise shared-memory atomics; four
    // copies per warp (lanes split by lane & 3) cut those collisions.
    __shared__ unsigned sub[kHistWarps * kHistCopies * kHistStride];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kHistWarps * kHistCopies * kHistStride; i += kHistThreads) sub[i] = 0;
    __syncthreads();

    const int image = blockIdx.y;
    const long long begin = (long long)blockIdx.x * chunk;
    long long end = begin + chunk;
    if (end > n_per_image) end = n_per_image;
    const uint8_t* base = px + (size_t)image * (size_t)n_per_image;
    unsigned* h = sub + (warp * kHistCopies + (lane & (kHistCopies - 1))) * kHistStride;

    // bytes before the first 16-byte boundary and after the last one
    const uintptr_t addr = reinterpret_cast<uintptr_t>(base + begin);
    long long head = (long long)((16 - (addr & 15)) & 15);
    if (head > end - begin) head = end - begin;
    for (long long i = begin + tid; i < begin + head; i += kHistThreads) atomicAdd(&h[base[i]], 1u);
    const long long vbeg = begin + head;
    const long long nvec = (end - vbeg) >> 4;
    const uint4* v = reinterpret_cast<const uint4*>(base + vbeg);
    long long i = tid;
    for (; i + kHistThreads < nvec; i += 2 * kHistThreads) {   // two 16-byte loads in flight
        const uint4 w0 = __ldcs(v + i);
        const uint4 w1 = __ldcs(v + i + kHistThreads);
        const uint32_t words[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            atomicAdd(&h[words[k] & 255u], 1u);
            atomicAdd(&h[(words[k] >> 8) & 255u], 1u);
            atomicAdd(&h[(words[k] >> 16) & 255u], 1u);
            atomicAdd(&h[words[k] >> 24], 1u);
        }
    }
    for (; i < nvec; i += kHistThreads) {
        const uint4 w = __ldcs(v + i);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            atomicAdd(&h[words[k] & 255u], 1u);
            atomicAdd(&h[(words[k] >> 8) & 255u], 1u);
            atomicAdd(&h[(words[k] >> 16) & 255u], 1u);
            atomicAdd(&h[words[k] >> 24], 1u);
        }
    }
    for (long long j = vbeg + (nvec << 4) + tid; j < end; j += kHistThreads) atomicAdd(&h[base[j]], 1u);
    __syncthreads();
    for (int b = tid; b < 256; b += kHistThreads) {
        unsigned s = 0;
#pragma unroll
        for (int c = 0; c < kHistWarps * kHistCopies; ++c) s += sub[c * kHistStride + b];
        if (s) atomicAdd(reinterpret_cast<unsigned*>(hist + (size_t)image * 256 + b), s);
    }
}

cudaError_t launch_histogram_u8(const uint8_t* d_px, int64_t n_per_image, int n_images, int32_t* d_hist,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * 256 * (size_t)n_images, st);
    if (e != cudaSuccess || n_per_image == 0 || n_images == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about eight CTAs per SM over the whole batch, each a 16-byte multiple
    long long total = n_per_image * (long long)n_images;
    long long chunk = total / ((long long)sms * 8);
    if (chunk < 65536) chunk = 65536;
    chunk = (chunk + 15) & ~15ll;
    long long per_image = (n_per_image + chunk - 1) / chunk;
    dim3 grid((unsigned)per_image, (unsigned)n_images);
    histogram_u8_kernel<<<grid, kHistThreads, 0, st>>>(d_px, n_per_image, chunk, d_hist);
    return cudaGetLastError();
}

// P0[v] = sum_{i<=v} h[i], P1[v] = sum_{i<=v} i h[i] (int64, exact).
__global__ void otsu_prefix_kernel(const int32_t* __restrict__ h, long long* P0, long long* P1)
{
    if (threadIdx.x == 0) {
        long long a = 0, b = 0;
        for (int v = 0; v < 256; ++v) {
            a += (long long)h[v];
            b += (long long)v * (long long)h[v];
            P0[v] = a;
            P1[v] = b;
        }
    }
}

cudaError_t launch_otsu_prefix(const int32_t* d_hist, long long* d_P0, long long* d_P1, cudaStream_t st)
{
    otsu_prefix_kernel<<<1, 32, 0, st>>>(d_hist, d_P0, d_P1);
    return cudaGetLastError();
}

// The between-class term omega_c (mu_c - mu_T)^2 of the class covering bins
// [a, b], for every range: omega = n / N, mu = s / n, computed with explicit
// round-to-nearest float64 operations in the order ((omega * dm) * dm); 0 for
// an empty range.  Summing these terms in class order reproduces the
// sigma_B^2 of Sec. 5.2's Otsu objective bit for bit.
__global__ void otsu_table_kernel(const long long* __restrict__ P0, const long long* __restrict__ P1,
                                  double* __restrict__ tab)
{
    const long long N = P0[255], S = P1[255];
    const double muT = __ddiv_rn((double)S, (double)N);
    for (int a = blockIdx.x; a < 256; a += gridDim.x) {
        for (int b = a + threadIdx.x; b < 256; b += blockDim.x) {
            const long long nc = P0[b] - (a > 0 ? P0[a - 1] : 0ll);
            const long long sc = P1[b] - (a > 0 ? P1[a - 1] : 0ll);
            double term = 0.0;
            if (nc > 0) {
                const double omega = __ddiv_rn((double)nc, (double)N);
                const double mu = __ddiv_rn((double)sc, (double)nc);
                const double dm = __dsub_rn(mu, muT);
                term = __dmul_rn(__dmul_rn(omega, dm), dm);
            }
            tab[otsu_tab_index(a, b)] = term;
        }
    }
}

cudaError_t launch_otsu_table(const long long* d_P0, const long long* d_P1, double* d_tab, cudaStream_t st)
{
    otsu_table_kernel<<<256, 256, 0, st>>>(d_P0, d_P1, d_tab);
    return cudaGetLastError();
}

}  // namespace apo
