// apo_hist.cu -- 256-bin histograms of 8-bit images and the Otsu prefix
// tables (the thresholding application of the cuAPO paper, Sec. 5.2).
//
// The histogram is HBM-bound in principle: every pixel byte is read once.
// Shared-memory atomics (even with per-warp copies) cap it near a third of
// the HBM rate on images whose intensities concentrate, so the counting is
// atomic-free: every thread owns one 8-bit counter per bin, incremented with
// a plain shared-memory byte load, add and store.  The counters are laid out
// [bin][64 words], thread (warp w, lane l) owning byte w mod 4 of word l + 32
// (w / 4) of every bin, so the 32 lanes of a warp always touch 32 different
// banks whatever their pixel values.  Before any counter can overflow (at most
// 240 pixels per thread between flushes) the CTA flushes: thread b sums the
// 256 counters of bin b into its own 32-bit register total and clears them.
// The totals go to the image's global int32 bins with one atomic per bin and
// CTA.  Integer counting makes the result independent of the order (bit-exact).
#include "apo_internal.h"

namespace apo {

constexpr int kHistThreads = 256;
constexpr int kHistWords = 64;          // counter words per bin (256 threads x 1 byte)
constexpr int kHistRound = 15;          // 16-byte loads per thread between flushes (240 pixels < 256)
constexpr int kHistBatch = 5;           // loads in flight per thread

// byte offset of thread (warp, lane)'s counter of bin 0; bin b adds 256 b
__device__ __forceinline__ int hist_slot(int warp, int lane)
{
    return 4 * (lane + 32 * (warp >> 2)) + (warp & 3);
}

// adds the 256 counters of bin `bin` (thread = bin) to total and clears them;
// word i of the bin is read at step (i + bin) mod 64, so a warp's lanes read
// 32 different banks
__device__ __forceinline__ void hist_flush(unsigned char* cnt, int bin, unsigned& total)
{
    uint32_t* w = reinterpret_cast<uint32_t*>(cnt) + bin * kHistWords;
    uint32_t lo = 0, hi = 0;   // four 16-bit lanes: at most 64 x 255 < 2^16 each
#pragma unroll 8
    for (int i = 0; i < kHistWords; ++i) {
        const int k = (i + bin) & (kHistWords - 1);
        const uint32_t v = w[k];
        w[k] = 0u;
        lo += v & 0x00FF00FFu;
        hi += (v >> 8) & 0x00FF00FFu;
    }
    total += (lo & 0xFFFFu) + (lo >> 16) + (hi & 0xFFFFu) + (hi >> 16);
}

__global__ void __launch_bounds__(kHistThreads) histogram_u8_kernel(const uint8_t* __restrict__ px,
                                                                    long long n_per_image,
                                                                    long long chunk, int32_t* hist)
{
    extern __shared__ __align__(16) unsigned char cnt[];   // 256 * kHistWords * 4 = 64 KB
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < 256 * kHistWords; i += kHistThreads) reinterpret_cast<uint32_t*>(cnt)[i] = 0u;
    __syncthreads();
    unsigned char* my = cnt + hist_slot(warp, lane);
    unsigned total = 0;   // this thread's bin (tid) over the flushes

    const int image = blockIdx.y;
    const long long begin = (long long)blockIdx.x * chunk;
    long long end = begin + chunk;
    if (end > n_per_image) end = n_per_image;
    const uint8_t* base = px + (size_t)image * (size_t)n_per_image;
    auto count = [&](uint32_t word) {
        my[256 * (word & 255u)] += 1;
        my[256 * ((word >> 8) & 255u)] += 1;
        my[256 * ((word >> 16) & 255u)] += 1;
        my[256 * (word >> 24)] += 1;
    };

    // bytes before the first 16-byte boundary and after the last one (fewer
    // than 16 + 15 per CTA: one per thread at most)
    const uintptr_t addr = reinterpret_cast<uintptr_t>(base + begin);
    long long head = (long long)((16 - (addr & 15)) & 15);
    if (head > end - begin) head = end - begin;
    const long long vbeg = begin + head;
    const long long nvec = (end - vbeg) >> 4;
    const long long tail0 = vbeg + (nvec << 4);
    if (tid < head) my[256 * base[begin + tid]] += 1;
    if (tid < end - tail0) my[256 * base[tail0 + tid]] += 1;

    const uint4* v = reinterpret_cast<const uint4*>(base + vbeg);
    const long long per_round = (long long)kHistRound * kHistThreads;
    for (long long r0 = 0; r0 < nvec; r0 += per_round) {
        // one round: at most kHistRound loads (4 kHistRound + 2 bytes) per thread
#pragma unroll 1
        for (int b0 = 0; b0 < kHistRound; b0 += kHistBatch) {
            uint4 w[kHistBatch];
#pragma unroll
            for (int k = 0; k < kHistBatch; ++k) {
                const long long i = r0 + (long long)(b0 + k) * kHistThreads + tid;
                w[k] = i < nvec ? __ldcs(v + i) : make_uint4(0u, 0u, 0u, 0u);
            }
#pragma unroll
            for (int k = 0; k < kHistBatch; ++k) {
                const long long i = r0 + (long long)(b0 + k) * kHistThreads + tid;
                if (i < nvec) {
                    count(w[k].x);
                    count(w[k].y);
                    count(w[k].z);
                    count(w[k].w);
                }
            }
        }
        __syncthreads();
        hist_flush(cnt, tid, total);
        __syncthreads();
    }
    if (nvec == 0) {   // the head / tail bytes only
        __syncthreads();
        hist_flush(cnt, tid, total);
    }
    if (total) atomicAdd(reinterpret_cast<unsigned*>(hist + (size_t)image * 256 + tid), total);
}

cudaError_t launch_histogram_u8(const uint8_t* d_px, int64_t n_per_image, int n_images, int32_t* d_hist,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(d_hist, 0, sizeof(int32_t) * 256 * (size_t)n_images, st);
    if (e != cudaSuccess || n_per_image == 0 || n_images == 0) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // about three CTAs per SM at a time (64 KB of counters each), a few waves
    // over the whole batch, each chunk a 16-byte multiple
    long long total = n_per_image * (long long)n_images;
    long long chunk = total / ((long long)sms * 12);
    if (chunk < 65536) chunk = 65536;
    chunk = (chunk + 15) & ~15ll;
    long long per_image = (n_per_image + chunk - 1) / chunk;
    dim3 grid((unsigned)per_image, (unsigned)n_images);
    const int smem = 256 * kHistWords * 4;
    e = cudaFuncSetAttribute(histogram_u8_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    histogram_u8_kernel<<<grid, kHistThreads, smem, st>>>(d_px, n_per_image, chunk, d_hist);
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
