// apo_umma.cuh -- the rotation z = M (x - o) of the cooperative grid kernel
// on the fifth-generation tensor cores (tcgen05, accumulator in tensor
// memory), for a single rotated component with D <= kTcM.
//
// A chunk of kTcN candidate rows is one MMA tile with the rotation as the M
// side (kTcM rows n) and the candidates as the N side:
//   acc[n][row] = sum_k B[n][k] y[row][k],   y = ysc (x - o),  B = msc M,
// so TMEM lane n, column row holds z[row][n] / zsc.  Both operands are fp16
// hi + lo parts in shared memory in the canonical K-major layout (umma_off):
// the rotation's (TA) loaded once per launch, the candidates' (TY) split from
// the chunk per chunk.  One thread issues three MMAs per K = 16 step,
// y_lo B_hi, y_hi B_lo, y_hi B_hi, in that order, accumulating in fp32 (the
// dropped y_lo B_lo is below 2^-22 of a product), and commits them to an
// mbarrier that every thread waits on with a time limit.  The accumulator is
// then read with tcgen05.ld into the row-major Z tile, scaled by zsc, for
// the objective epilogue.  The operand values and the MMA sequence are those
// of the mma.sync rotation (tile_gemm_f16x3).
#pragma once

#include "apo_path.cuh"

namespace apo {

// instruction descriptor: fp32 accumulator, f16 A and B, both K-major,
// N = kTcN, M = kTcM
constexpr uint32_t kRotIdesc = (1u << 4) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
constexpr unsigned long long kMmaTimeoutNs = 1000000000ull;   // 1 s per wait

struct TcState {
    uint32_t tmem;    // accumulator: kTcN of kTcCols columns x kTcM lanes
    uint32_t mbar;    // shared address of the completion mbarrier
    uint32_t phase;   // commits waited for so far
};

// Shared-memory descriptor of a K-major operand with Kt columns at saddr.
__device__ __forceinline__ uint64_t umma_kdesc(uint32_t saddr, int Kt)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;                                 // K-adjacent core matrices
    d |= (uint64_t)((((uint32_t)Kt * 16u) >> 4) & 0x3FFFu) << 32;     // 8-row groups
    d |= (uint64_t)1 << 46;                                           // tcgen05 version; no swizzle
    return d;
}

// Allocates the accumulator and initialises the mbarrier.  Whole CTA.
__device__ __forceinline__ void tc_setup(TcState& st, uint32_t* tmem_slot, unsigned long long* mbar)
{
    st.mbar = (uint32_t)__cvta_generic_to_shared(mbar);
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"((uint32_t)__cvta_generic_to_shared(tmem_slot)), "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" : : : "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" : : "r"(st.mbar) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
    st.tmem = *tmem_slot;
    st.phase = 0;
}

// Frees the accumulator.  Whole CTA, after its last tcgen05 operation.
__device__ __forceinline__ void tc_teardown(const TcState& st)
{
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(st.tmem), "r"(kTcCols)
                     : "memory");
}

// Waits for the completion of the given parity of the mbarrier; false after
// the time limit.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    const unsigned long long t0 = global_ns();
    for (unsigned n = 0;; ++n) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (done) return true;
        if ((n & 255u) == 255u && global_ns() - t0 > kMmaTimeoutNs) return false;
    }
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :
        : "r"(tmem), "l"(ad), "l"(bd), "r"(kRotIdesc), "r"(accumulate)
        : "memory");
}

// Evaluates the candidate rows Xc[0, rows) (rows <= kTcN) of the single
// rotated component into rowF.  Whole CTA of at least 4 warps (a multiple of
// 4); ends synchronised.  Returns false, for every thread, when the MMAs did
// not complete within the time limit (rowF is then not written).
template <typename FitT>
__device__ bool eval_chunk_tc(const ApoRun& R, const Smem<FitT>& S, int rows, TcState& st)
{
    const DevProblem& P = R.prob;
    const DevComp& C = P.comp[0];
    const int D = P.D, Dp = P.Dp, Np = P.Np;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;

    // TY: y = ysc (x - o) of the chunk rows as fp16 hi and lo parts, zero for
    // rows >= rows and k >= D.  Task i covers 8 k of one row; 8 consecutive
    // tasks are the 8 rows of one core matrix, so a quarter-warp's 16-byte
    // stores fill 128 contiguous bytes, and (rows Dp floats apart, Dp a
    // multiple of 4) its 16-byte loads of x fall on distinct banks when Dp is
    // 4 mod 8.  The last 16-byte group of a row may read past Dp (into the
    // next row, or the region after the candidates, or past o): those k are
    // >= D and masked.
    const int nkb = Np >> 3;
    const float ysc = C.ysc;
    unsigned char* yh = S.TY;
    unsigned char* yl = S.TY + (size_t)kTcN * Np * 2;
    const uint32_t gm = div_magic((uint32_t)(8 * nkb));
    for (int i = tid; i < kTcN * nkb; i += blockDim.x) {
        const int grp = (int)div_small((uint32_t)i, gm);   // 8-row group
        const int r = (i & 7) + 8 * grp;
        const int kb = (i >> 3) - grp * nkb;
        const float4* xr = reinterpret_cast<const float4*>(S.Xc + (size_t)r * Dp + 8 * kb);
        const float4* orow = reinterpret_cast<const float4*>(S.o + 8 * kb);
        const float4 x0 = xr[0], x1 = xr[1], o0 = orow[0], o1 = orow[1];
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float ov[8] = {o0.x, o0.y, o0.z, o0.w, o1.x, o1.y, o1.z, o1.w};
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int k = 8 * kb + 2 * e;
            const float y0 = (r < rows && k < D) ? (xv[2 * e] - ov[2 * e]) * ysc : 0.f;
            const float y1 = (r < rows && k + 1 < D) ? (xv[2 * e + 1] - ov[2 * e + 1]) * ysc : 0.f;
            split_f16x2(y0, y1, h[e], l[e]);
        }
        const uint32_t off = umma_off(r, 8 * kb, Np);
        *reinterpret_cast<uint4*>(yh + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(yl + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
    // the generic-proxy writes of TY (and of TA, at load time) become
    // visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" : : : "memory");
    __syncthreads();
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
        const uint32_t ah = (uint32_t)__cvta_generic_to_shared(S.TA);
        const uint32_t al = ah + (uint32_t)(Np * Np * 2);
        // a K step advances every operand by two core matrices (256 bytes),
        // i.e. 16 in the descriptor's address field (which cannot carry:
        // shared addresses stay below 2^18)
        uint64_t dah = umma_kdesc(ah, Np), dal = umma_kdesc(al, Np);
        uint64_t dbh = umma_kdesc((uint32_t)__cvta_generic_to_shared(yh), Np);
        uint64_t dbl = umma_kdesc((uint32_t)__cvta_generic_to_shared(yl), Np);
        for (int s = 0; s < (Np >> 4); ++s) {
            umma_f16(st.tmem, dah, dbl, s > 0 ? 1u : 0u);
            umma_f16(st.tmem, dal, dbh, 1u);
            umma_f16(st.tmem, dah, dbh, 1u);
            dah += 16u; dal += 16u; dbh += 16u; dbl += 16u;
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     :
                     : "r"(st.mbar)
                     : "memory");
    }
    const bool done = tc_wait(st.mbar, st.phase & 1u);
    ++st.phase;
    if (!__syncthreads_and(done)) return false;
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");

    // accumulator -> Z tile: warp w reads TMEM lanes 32 (w & 3) .. + 31
    // (n = lane) and 16 columns (candidate rows) per load
    const float zsc = C.zsc;
    const int n = 32 * (warp & 3) + lane;
    for (int cg = warp >> 2; cg < kTcN / 16; cg += nw >> 2) {
        uint32_t v[16];
        const uint32_t taddr = st.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(16 * cg);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" : : : "memory");
        if (n < Np) {
#pragma unroll
            for (int j = 0; j < 16; ++j) S.Zc[(size_t)(16 * cg + j) * Np + n] = __uint_as_float(v[j]) * zsc;
        }
    }
    // the next chunk's MMAs overwrite the accumulator only after every read
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    zrows_to_f<FitT>(S, C, D, Np, rows);
    __syncthreads();
    return true;
}

}  // namespace apo
