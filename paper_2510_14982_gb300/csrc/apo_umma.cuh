// apo_umma.cuh -- the rotation z = M (x - o) of the cooperative grid kernel
// on the fifth-generation tensor cores (tcgen05, accumulator in tensor
// memory), for a single rotated component with D <= kTcM, and the objective
// read straight from the accumulator.
//
// A chunk of kTcN candidate rows is one MMA tile with the candidates as the
// M side (kTcM rows read, the rows past kTcN unused) and the output
// dimensions as the N side (Np):
//   acc[row][n] = sum_k y[row][k] B[n][k],   y = ysc (x - o),  B = msc M,
// so TMEM lane row, column n holds z[row][n] / zsc.  Both operands are fp16
// hi + lo parts in shared memory in the canonical K-major layout (umma_off):
// the rotation's (TA) loaded once per launch, the candidates' (TY) split from
// the chunk per chunk.  One thread issues three MMAs per K = 16 step,
// y_lo B_hi, y_hi B_lo, y_hi B_hi, in that order, accumulating in fp32 (the
// dropped y_lo B_lo is below 2^-22 of a product), and commits them to an
// mbarrier that every thread waits on with a time limit.  Each thread then
// reads one candidate's z over a quarter of the output dimensions with
// tcgen05.ld, scaled by zsc, and sums its objective terms; the quarters are
// combined in column order through shared memory.
#pragma once

#include "apo_path.cuh"

namespace apo {

// instruction descriptor: fp32 accumulator, f16 A and B, both K-major,
// M = kTcM candidate rows, N = Np output dimensions (a multiple of 16)
__device__ __forceinline__ uint32_t rot_idesc(int Np)
{
    return (1u << 4) | ((uint32_t)(Np >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}
constexpr unsigned long long kMmaTimeoutNs = 1000000000ull;   // 1 s per wait

struct TcState {
    uint32_t tmem;    // accumulator: Np of kTcCols columns x kTcM lanes
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

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        :
        : "r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

// One accumulator column of the calling thread's TMEM lane (warp w reads
// lanes 32 (w mod 4) .. + 31), without waiting.
__device__ __forceinline__ void tmem_ld1(uint32_t taddr, uint32_t& a)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(a) : "r"(taddr));
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
    for (int i = tid; i < kTcN * nkb; i += blockDim.x) {
        const int r = (i & 7) + 8 * (i / (8 * nkb));
        const int kb = (i >> 3) % nkb;
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
        const uint32_t bh = (uint32_t)__cvta_generic_to_shared(S.TA);
        const uint32_t bl = bh + (uint32_t)(Np * Np * 2);
        // A K step advances every operand by two core matrices (256 bytes),
        // i.e. 16 in the descriptor's address field (which cannot carry:
        // shared addresses stay below 2^18).  The A side reads kTcM candidate
        // rows: rows past kTcN of the hi part fall into the lo part, those of
        // the lo part into the tables after TY; their accumulator rows are
        // never read.
        uint64_t dyh = umma_kdesc((uint32_t)__cvta_generic_to_shared(yh), Np);
        uint64_t dyl = umma_kdesc((uint32_t)__cvta_generic_to_shared(yl), Np);
        uint64_t dbh = umma_kdesc(bh, Np), dbl = umma_kdesc(bl, Np);
        const uint32_t idesc = rot_idesc(Np);
        for (int s = 0; s < (Np >> 4); ++s) {
            umma_f16(st.tmem, dyl, dbh, idesc, s > 0 ? 1u : 0u);
            umma_f16(st.tmem, dyh, dbl, idesc, 1u);
            umma_f16(st.tmem, dyh, dbh, idesc, 1u);
            dyh += 16u; dyl += 16u; dbh += 16u; dbl += 16u;
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

    // Objective from the accumulator, in exactly the arithmetic of seg_value
    // (the evaluation of the other kernels), so that every kernel gives the
    // same fitness bit for bit: there lane l of a warp accumulates the output
    // dimensions d = l, l + 32, ... in order, and the 32 lane sums are added
    // by the xor butterfly (16, 8, 4, 2, 1).  Here warp w takes the candidate
    // rows 32 (w mod 4) + lane (its TMEM lanes) and plays the lanes
    // l = l0 + 8 m (m = 0..3) for l0 = 2 q, 2 q + 1 (q = w / 4), reading one
    // accumulator column per load; the butterfly's first two levels (xor 16,
    // xor 8) stay within the thread, and its last three combine the eight
    // level-2 values of a row through shared memory (the TY region, free once
    // the MMAs have completed).
    const float zsc = C.zsc;
    const int form = C.form;
    const bool f2 = form == kHGBat || form == kGriewank;
    float* w1 = reinterpret_cast<float*>(S.TY);   // [8][kTcN] level-2 values of the (first) sum
    float* w2 = w1 + 8 * kTcN;                    // [8][kTcN] of the second sum (HGBat, Griewank)
    const int row = 32 * (warp & 3) + lane;
    const uint32_t tl = st.tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    for (int q = warp >> 2; q < 4; q += nw >> 2) {
        float a[8], c[8];   // lane l = 2 q + (i & 1) + 8 (i >> 1)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            a[i] = 0.f;
            c[i] = form == kGriewank ? 1.f : 0.f;
        }
        for (int j = 0; 32 * j < D; ++j) {
            // columns d0 = 32 j + 8 m + 2 q, d0 + 1, and d0 + 2 (z[d + 1] of
            // the Rosenbrock chain at d = d0 + 1); the column conditions are
            // uniform over the warp, and every column read lies below Np
            uint32_t v[12];
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const int d0 = 32 * j + 8 * m + 2 * q;
                v[3 * m] = v[3 * m + 1] = v[3 * m + 2] = 0u;
                if (d0 < Np) {
                    tmem_ld1(tl + (uint32_t)d0, v[3 * m]);
                    tmem_ld1(tl + (uint32_t)(d0 + 1), v[3 * m + 1]);
                }
                if (d0 + 2 < Np) tmem_ld1(tl + (uint32_t)(d0 + 2), v[3 * m + 2]);
            }
            asm volatile("tcgen05.wait::ld.sync.aligned;" : : : "memory");
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int i = 2 * m + e, d = 32 * j + 8 * m + 2 * q + e;
                    if (d >= D) continue;
                    const float z = __uint_as_float(v[3 * m + e]) * zsc;
                    if (form == kHGBat) {
                        const float u = z * 0.05f;
                        a[i] = fmaf(u, u, a[i] - u);
                        c[i] = fmaf(u, u, c[i]);
                    } else if (form == kGriewank) {
                        const float y = 6.f * z;
                        a[i] = fmaf(y, y, a[i]);
                        c[i] *= cospif(y * S.ew[d]);
                    } else if (d < C.s1) {
                        a[i] = fmaf(S.ew[d] * z, z, a[i]);
                    } else if (d < C.s2) {
                        if (d + 1 < C.s2) a[i] += rosen_term(z, __uint_as_float(v[3 * m + e + 1]) * zsc);
                    } else {
                        a[i] += rast_term(z);
                    }
                }
        }
        if (row < kTcN) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                // levels xor 16 and xor 8: (s_l0 + s_l0+16) + (s_l0+8 + s_l0+24)
                w1[(2 * q + e) * kTcN + row] = (a[e] + a[4 + e]) + (a[2 + e] + a[6 + e]);
                if (f2)
                    w2[(2 * q + e) * kTcN + row] = form == kGriewank ? (c[e] * c[4 + e]) * (c[2 + e] * c[6 + e])
                                                                      : (c[e] + c[4 + e]) + (c[2 + e] + c[6 + e]);
            }
        }
    }
    // the next chunk's MMAs overwrite the accumulator only after every read
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    // levels xor 4, xor 2, xor 1 as lane 0 adds them
    auto tree = [&](const float* w, int r, bool prod) {
        float x[8];
#pragma unroll
        for (int l0 = 0; l0 < 8; ++l0) x[l0] = w[l0 * kTcN + r];
        if (prod) return ((x[0] * x[4]) * (x[2] * x[6])) * ((x[1] * x[5]) * (x[3] * x[7]));
        return ((x[0] + x[4]) + (x[2] + x[6])) + ((x[1] + x[5]) + (x[3] + x[7]));
    };
    for (int r = tid; r < rows; r += blockDim.x) {
        float f;
        if (form == kHGBat) f = hgbat_from_sums(tree(w1, r, false), tree(w2, r, false), D);
        else if (form == kGriewank) f = fmaf(tree(w1, r, false), 1.f / 4000.f, 1.f - tree(w2, r, true));
        else f = tree(w1, r, false);
        S.rowF[r] = (FitT)f;
    }
    __syncthreads();
    return true;
}

}  // namespace apo
