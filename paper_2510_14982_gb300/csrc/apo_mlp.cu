// apo_mlp.cu -- the surrogate network of the surrogate-assisted APO form: an
// MLP D -> 256 -> 256 -> 1 (ReLU) with bfloat16 weights and activations and
// float32 accumulation, trained online with mean squared error and Adam.
//
// Kernels: a bfloat16 GEMM on the Blackwell tensor cores (tcgen05.mma with
// the accumulator in tensor memory) with fused epilogues (bias, ReLU, ReLU-derivative mask, fp32 and bf16
// outputs), the 256 -> 1 output layer and its gradients, column sums for the
// bias gradients, the loss gradient, Adam, and the gather of a training batch
// from the archive.
#include <cuda_bf16.h>

#include <algorithm>

#include "apo_internal.h"
#include "apo_mlp.h"

namespace apo {

// ------------------------------------------------- tcgen05 GEMM (Blackwell)
// C = A B on the fifth-generation tensor cores: one CTA of 128 threads owns a
// 128 x 64 tile of C, accumulated in tensor memory (TMEM, 64 fp32 columns)
// by tcgen05.mma kind::f16 (bf16 inputs) issued by a single thread.  A and B
// are staged in shared memory per 64-wide K chunk (double buffered, the next
// chunk's global loads in flight while the current chunk's MMAs run) in the
// canonical K-major layout without swizzle: 8-row x 16-byte core matrices,
// K-adjacent core matrices kLBO bytes apart, 8-row groups kSBO bytes apart.
// The MMAs of a chunk are committed to an mbarrier; a buffer is refilled
// only after the MMAs that read it have completed, and every wait gives up
// after one second (error flag, no hang).  The epilogue reads the
// accumulator with tcgen05.ld (thread = row) into a shared-memory tile and
// writes it out row-contiguously with bias, the ReLU derivative mask and
// ReLU applied.
constexpr int kTM = 128;                   // tile rows (UMMA M)
constexpr int kTN = 64;                    // tile columns (UMMA N)
constexpr int kTK = 64;                    // K chunk: 4 UMMA steps of K = 16
constexpr int kTThreads = 128;
constexpr uint32_t kTileA = kTM * kTK * 2; // bytes per A buffer
constexpr uint32_t kTileB = kTN * kTK * 2; // bytes per B buffer
constexpr uint32_t kLBO = 128;             // K-adjacent core matrices
constexpr uint32_t kSBO = 1024;            // 8-row groups (8 core matrices of K)
constexpr size_t kTcSmem = 2 * (size_t)kTileA + 2 * (size_t)kTileB;   // 48 KB
// instruction descriptor: fp32 accumulate, bf16 A and B, both K-major, N, M
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTN >> 3) << 17) |
                            ((uint32_t)(kTM >> 4) << 24);

// byte offset of element (row, k) of a K-major tile
__device__ __forceinline__ uint32_t kmaj_off(int row, int k)
{
    return (uint32_t)((((row >> 3) * (kTK / 8) + (k >> 3)) * 128) + ((row & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kLBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((kSBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of tcgen05; base offset 0, no swizzle
    return d;
}

__device__ __forceinline__ unsigned long long tc_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase of the given parity of an mbarrier; false after 1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    const unsigned long long t0 = tc_ns();
    for (unsigned n = 0;; ++n) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if ((n & 255u) == 255u && tc_ns() - t0 > 1000000000ull) return false;
    }
}

// Loads K chunk k0 of A (rows m0..m0+127) and B (columns n0..n0+63) into
// registers, 8 consecutive elements per group, zero outside M, N, K:
// A(m, k) = TA ? A[k lda + m] : A[m lda + k]; B(k, n) = TB ? B[n ldb + k] :
// B[k ldb + n].  A group is one 16-byte load when in range and aligned.  All
// of a thread's loads are issued before any is used, so they overlap each
// other (and the MMAs of the previous chunk).
constexpr int kGA = kTM * kTK / 8 / kTThreads;   // A groups per thread (8)
constexpr int kGB = kTN * kTK / 8 / kTThreads;   // B groups per thread (4)

// Group q of a K-contiguous tile: row (q & 7) + 8 (q >> 6), k group (q >> 3) & 7.
// A warp's 32 groups then cover 8 rows x 4 k groups: 4 whole core matrices,
// so its 16-byte shared stores fall on distinct banks.
__device__ __forceinline__ int kc_row(int q) { return (q & 7) + 8 * (q >> 6); }
__device__ __forceinline__ int kc_kg(int q) { return (q >> 3) & 7; }

// Group q of an M- or N-contiguous source (a group is 8 rows of the tile at
// one k): k = (q & 7) + 8 ((q >> 5) & 7), row group (q >> 3) & 3 + 4 (q >> 8).
// Its 8 elements go to 8 rows of one core matrix, element by element; lane
// offset mc_rot rotates the order so that the 32 lanes of a store
// instruction write 32 distinct banks.
__device__ __forceinline__ int mc_k(int q) { return (q & 7) + 8 * ((q >> 5) & 7); }
__device__ __forceinline__ int mc_g(int q) { return ((q >> 3) & 3) + 4 * (q >> 8); }
__device__ __forceinline__ int mc_rot(int q) { return (q & 7) + 2 * ((q >> 3) & 3); }

// element i (0..7) of 8 packed bf16, selected in registers
__device__ __forceinline__ uint16_t pick_half(const uint4& v, int i)
{
    const uint32_t w = (i & 4) ? ((i & 2) ? v.w : v.z) : ((i & 2) ? v.y : v.x);
    return (uint16_t)((i & 1) ? (w >> 16) : (w & 0xFFFFu));
}

__device__ __forceinline__ uint4 ld_group(const __nv_bfloat16* src, bool vec, int avail)
{
    if (vec && avail >= 8) return __ldg(reinterpret_cast<const uint4*>(src));
    __nv_bfloat16 e[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) e[i] = i < avail ? src[i] : __float2bfloat16(0.f);
    return *reinterpret_cast<const uint4*>(e);
}

template <bool TA, bool TB>
__device__ __forceinline__ void tc_load(const GemmArgs& g, int m0, int n0, int k0, bool va, bool vb,
                                        uint4 (&ra)[kGA], uint4 (&rb)[kGB])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < kGA; ++i) {
        const int q = tid + i * kTThreads;
        ra[i] = make_uint4(0u, 0u, 0u, 0u);
        if (!TA) {   // group (m, 8 k); the 8 rows of a core matrix in consecutive lanes
            const int gm = m0 + kc_row(q), gk = k0 + 8 * kc_kg(q);
            if (gm < g.M && gk < g.K) ra[i] = ld_group(g.A + (size_t)gm * g.lda + gk, va, g.K - gk);
        } else {     // group (k, 8 m)
            const int gk = k0 + mc_k(q), gm = m0 + 8 * mc_g(q);
            if (gk < g.K && gm < g.M) ra[i] = ld_group(g.A + (size_t)gk * g.lda + gm, va, g.M - gm);
        }
    }
#pragma unroll
    for (int i = 0; i < kGB; ++i) {
        const int q = tid + i * kTThreads;
        rb[i] = make_uint4(0u, 0u, 0u, 0u);
        if (TB) {    // group (n, 8 k); the 8 rows of a core matrix in consecutive lanes
            const int gn = n0 + kc_row(q), gk = k0 + 8 * kc_kg(q);
            if (gn < g.N && gk < g.K) rb[i] = ld_group(g.B + (size_t)gn * g.ldb + gk, vb, g.K - gk);
        } else {     // group (k, 8 n)
            const int gk = k0 + mc_k(q), gn = n0 + 8 * mc_g(q);
            if (gk < g.K && gn < g.N) rb[i] = ld_group(g.B + (size_t)gk * g.ldb + gn, vb, g.N - gn);
        }
    }
}

// Writes the loaded groups into the K-major tiles (a K-contiguous group as
// one 16-byte store, an M- or N-contiguous group element by element).
template <bool TA, bool TB>
__device__ __forceinline__ void tc_store(unsigned char* As, unsigned char* Bs, const uint4 (&ra)[kGA],
                                         const uint4 (&rb)[kGB])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int i = 0; i < kGA; ++i) {
        const int q = tid + i * kTThreads;
        if (!TA) {
            *reinterpret_cast<uint4*>(As + kmaj_off(kc_row(q), 8 * kc_kg(q))) = ra[i];
        } else {
            const int k = mc_k(q), g8 = 8 * mc_g(q), rot = mc_rot(q);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ri = (j + rot) & 7;
                *reinterpret_cast<uint16_t*>(As + kmaj_off(g8 + ri, k)) = pick_half(ra[i], ri);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < kGB; ++i) {
        const int q = tid + i * kTThreads;
        if (TB) {
            *reinterpret_cast<uint4*>(Bs + kmaj_off(kc_row(q), 8 * kc_kg(q))) = rb[i];
        } else {
            const int k = mc_k(q), g8 = 8 * mc_g(q), rot = mc_rot(q);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int ri = (j + rot) & 7;
                *reinterpret_cast<uint16_t*>(Bs + kmaj_off(g8 + ri, k)) = pick_half(rb[i], ri);
            }
        }
    }
}

// With ws (split K), CTA z of the grid's z dimension accumulates only the K
// chunks [z cps, (z + 1) cps) and writes its raw fp32 tile to ws[z][M][N];
// splitk_epilogue_kernel then sums the slices in order and applies the
// epilogue.  Without ws, cps covers all of K and the epilogue is fused.
template <bool TA, bool TB>
__global__ void __launch_bounds__(kTThreads) gemm_bf16_tc_kernel(GemmArgs g, bool va, bool vb, int cps, float* ws,
                                                                 int* err)
{
    extern __shared__ __align__(128) unsigned char gsm[];
    __shared__ __align__(8) unsigned long long mbar[2];
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    unsigned char* As[2] = {gsm, gsm + kTileA};
    unsigned char* Bs[2] = {gsm + 2 * kTileA, gsm + 2 * kTileA + kTileB};
    const uint32_t mb[2] = {(uint32_t)__cvta_generic_to_shared(&mbar[0]),
                            (uint32_t)__cvta_generic_to_shared(&mbar[1])};
    if (warp == 0) {
        const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&tmem_slot);
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" : : "r"(slot), "r"(kTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" : : : "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(mb[0]) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(mb[1]) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
    const uint32_t tmem = tmem_slot;
    // this CTA's K chunks: c0 .. c0 + nch - 1 (K bounded to their end)
    const int c0 = blockIdx.z * cps;
    const int nch = max(0, min((g.K + kTK - 1) / kTK - c0, cps));
    GemmArgs gk = g;
    gk.K = min(g.K, (c0 + nch) * kTK);
    bool ok = true;
    uint4 ra[kGA], rb[kGB];
    if (nch > 0) {
        tc_load<TA, TB>(gk, m0, n0, c0 * kTK, va, vb, ra, rb);
        tc_store<TA, TB>(As[0], Bs[0], ra, rb);
        asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
        __syncthreads();
    }
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(As[b]);
            const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(Bs[b]);
#pragma unroll
            for (int s = 0; s < kTK / 16; ++s) {
                const uint64_t ad = umma_desc(a0 + 2u * kLBO * s), bd = umma_desc(b0 + 2u * kLBO * s);
                const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    :
                    : "r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" : : "r"(mb[b])
                         : "memory");
        }
        if (c + 1 < nch) {
            const int nb = (c + 1) & 1;
            tc_load<TA, TB>(gk, m0, n0, (c0 + c + 1) * kTK, va, vb, ra, rb);   // in flight during the MMAs
            // the MMAs of chunk c - 1 read buffer nb
            if (c >= 1 && !mbar_wait(mb[nb], (uint32_t)((c - 1) >> 1) & 1u)) ok = false;
            tc_store<TA, TB>(As[nb], Bs[nb], ra, rb);
            asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
            __syncthreads();
        }
    }
    // the last commit covers every MMA of the tile
    if (nch > 0 && !mbar_wait(mb[(nch - 1) & 1], (uint32_t)((nch - 1) >> 1) & 1u)) ok = false;
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");

    // epilogue: row r of the tile = TMEM lane r, read 16 columns per load
    // into a padded fp32 tile in the (now idle) operand buffers, then written
    // out row-contiguously across the lanes (coalesced bias, mask and C)
    constexpr int kTS = kTN + 1;   // tile row stride in floats
    float* tile = reinterpret_cast<float*>(gsm);
    const int rl = 32 * warp + lane;
#pragma unroll
    for (int cg = 0; cg < kTN / 16; ++cg) {
        uint32_t r[16];
        if (nch > 0) {
            const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(16 * cg);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" : : : "memory");
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) r[j] = 0u;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) tile[rl * kTS + 16 * cg + j] = __uint_as_float(r[j]);
    }
    __syncthreads();
    // split K: the raw tile goes to this CTA's slice of the workspace
    GemmArgs ge = g;
    if (ws) {
        ge.bias = nullptr;
        ge.mask = nullptr;
        ge.relu = 0;
        ge.Cb = nullptr;
        ge.Cf = ws + (size_t)blockIdx.z * g.M * g.N;
        ge.ldc = g.N;
    }
    if (ok) {
        // 8 elements per thread at a time: their bias and mask loads are all
        // issued before any result is stored (the outputs could alias them)
        constexpr int kU = 8;
        for (int i0 = tid; i0 < kTM * kTN; i0 += kU * kTThreads) {
            float bv[kU], mv[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * kTThreads;
                const int rr = i / kTN, cc = i - rr * kTN;
                const int m = m0 + rr, n = n0 + cc;
                const bool in = i < kTM * kTN && m < g.M && n < g.N;
                bv[u] = (in && ge.bias) ? __ldg(ge.bias + n) : 0.f;
                mv[u] = (in && ge.mask) ? __ldg(ge.mask + (size_t)m * ge.ldm + n) : 1.f;
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int i = i0 + u * kTThreads;
                const int rr = i / kTN, cc = i - rr * kTN;
                const int m = m0 + rr, n = n0 + cc;
                if (i >= kTM * kTN || m >= g.M || n >= g.N) continue;
                float v = tile[rr * kTS + cc] + bv[u];
                if (ge.mask) v = mv[u] > 0.f ? v : 0.f;
                if (ge.relu) v = fmaxf(v, 0.f);
                if (ge.Cf) ge.Cf[(size_t)m * ge.ldc + n] = v;
                if (ge.Cb) ge.Cb[(size_t)m * ge.ldcb + n] = __float2bfloat16(v);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(tmem), "r"(kTN) : "memory");
    if (!ok && tid == 0) atomicCAS(err, 0, 4 /* APO_ERR_TIMEOUT */);
}

// Sum of the ksplit slices of ws (in slice order) and the epilogue of
// gemm_bf16_tc_kernel: bias, ReLU-derivative mask, ReLU, fp32 / bf16 outputs.
__global__ void splitk_epilogue_kernel(GemmArgs g, const float* __restrict__ ws, int ksplit)
{
    const size_t MN = (size_t)g.M * g.N;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < MN; i += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(i / g.N), n = (int)(i - (size_t)m * g.N);
        float v = 0.f;
        for (int z = 0; z < ksplit; ++z) v += ws[(size_t)z * MN + i];
        v += g.bias ? g.bias[n] : 0.f;
        if (g.mask) v = g.mask[(size_t)m * g.ldm + n] > 0.f ? v : 0.f;
        if (g.relu) v = fmaxf(v, 0.f);
        if (g.Cf) g.Cf[(size_t)m * g.ldc + n] = v;
        if (g.Cb) g.Cb[(size_t)m * g.ldcb + n] = __float2bfloat16(v);
    }
}

// C(m, n) = sum_k A(m, k) B(k, n), A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n]; then v = acc + bias[n],
// v *= (mask[m ldm + n] > 0) when mask, v = max(v, 0) when relu; stored to
// Cf (fp32) and / or Cb (bf16).  A wait that runs out records
// APO_ERR_TIMEOUT in the device status word.
cudaError_t gemm_bf16(const GemmArgs& g, bool ta, bool tb, cudaStream_t st)
{
    if (g.M <= 0 || g.N <= 0) return cudaSuccess;
    int* err = device_status_word();
    if (!err) return cudaErrorMemoryAllocation;
    // 16-byte loads need 16-byte aligned rows
    const bool va = (reinterpret_cast<uintptr_t>(g.A) & 15u) == 0 && (g.lda & 7) == 0;
    const bool vb = (reinterpret_cast<uintptr_t>(g.B) & 15u) == 0 && (g.ldb & 7) == 0;
    static bool attr_set = false;   // 48 KB of dynamic shared memory next to the static words
    if (!attr_set) {
        cudaFuncSetAttribute(gemm_bf16_tc_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        cudaFuncSetAttribute(gemm_bf16_tc_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        cudaFuncSetAttribute(gemm_bf16_tc_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        cudaFuncSetAttribute(gemm_bf16_tc_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        attr_set = true;
    }
    // Few output tiles (the network's layers make 8 to 16) leave most SMs
    // idle while each CTA walks K chunk by chunk, so K is split until about
    // kSplitTarget CTAs run; the slices are summed in a fixed order by the
    // epilogue kernel (deterministic).  The slices go to the caller's
    // workspace (g.ws); without one, or when it is too small, K is not split.
    constexpr int kSplitTarget = 128;
    const int tiles = ((g.N + kTN - 1) / kTN) * ((g.M + kTM - 1) / kTM);
    const int nch = (g.K + kTK - 1) / kTK;
    int cps = nch > 0 ? nch : 1, ksplit = 1;
    if (nch > 1 && tiles < kSplitTarget) {
        const int want = std::min(nch, std::max(1, kSplitTarget / tiles));
        cps = (nch + want - 1) / want;
        ksplit = (nch + cps - 1) / cps;
    }
    if (ksplit > 1 && (!g.ws || (size_t)ksplit * g.M * g.N > g.ws_elems)) {
        ksplit = 1;
        cps = nch > 0 ? nch : 1;
    }
    float* ws = ksplit > 1 ? g.ws : nullptr;
    dim3 grid((g.N + kTN - 1) / kTN, (g.M + kTM - 1) / kTM, ksplit);
    if (!ta && !tb) gemm_bf16_tc_kernel<false, false><<<grid, kTThreads, kTcSmem, st>>>(g, va, vb, cps, ws, err);
    else if (ta && !tb) gemm_bf16_tc_kernel<true, false><<<grid, kTThreads, kTcSmem, st>>>(g, va, vb, cps, ws, err);
    else if (!ta && tb) gemm_bf16_tc_kernel<false, true><<<grid, kTThreads, kTcSmem, st>>>(g, va, vb, cps, ws, err);
    else gemm_bf16_tc_kernel<true, true><<<grid, kTThreads, kTcSmem, st>>>(g, va, vb, cps, ws, err);
    if (ksplit > 1) {
        const size_t MN = (size_t)g.M * g.N;
        const int blocks = (int)std::min<size_t>((MN + 255) / 256, 1024);
        splitk_epilogue_kernel<<<blocks, 256, 0, st>>>(g, ws, ksplit);
    }
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
