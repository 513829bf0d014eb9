// apo_kernels.cu -- the APO population update on the GPU (cuAPO paper,
// Sec. 3 Eq. 1-13 and Algorithm 1).
//
// One CTA (resident mode) or a group of g cooperating CTAs (grid mode) runs
// the whole device-side iteration loop of one optimisation run:
//   sort (F, previous rank) -> [Dr_index, precomputed by dr_kernel]
//   -> candidate generation, one warp per protozoon (Eq. 1-10, 12-13)
//   -> bound clamp -> evaluation (z = M (x - o) as a shared-memory tile GEMM,
//      then the objective epilogue) -> greedy replacement -> barrier.
// In resident mode the population, its fitness and the rotation live in
// shared memory; in grid mode the population lives in global memory (L2) and
// is double buffered so that every candidate reads the start-of-iteration
// snapshot, as the synchronous "parallel for" of Algorithm 1 requires.
#include <cstdio>

#include "apo_device.cuh"
#include "apo_internal.h"

namespace apo {

constexpr float kEps = 2.220446049250313e-16f;  // eps of Eq. 7 and Eq. 10 (2^-52)

// ------------------------------------------------------------- Dr_index
// Eq. 11 and Algorithm 1: pf = pf_max * rand, m = ceil(ps * pf) (float64),
// Dr_index = the m smallest (Philox key, rank) pairs.  One CTA per (run, t);
// an exact radix select over 8-bit digits of the 32-bit keys.
__global__ void __launch_bounds__(kThreads) dr_kernel(const ApoRun* __restrict__ runs,
                                                      const int* __restrict__ offs, int n_runs,
                                                      int n_work)
{
    extern __shared__ __align__(16) unsigned char dyn[];
    uint32_t* keys = reinterpret_cast<uint32_t*>(dyn);
    __shared__ unsigned hist[256];
    __shared__ unsigned s_prefix, s_need, s_eq;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int w = blockIdx.x; w < n_work; w += gridDim.x) {
        int lo = 0, hi = n_runs - 1;  // run k with offs[k] <= w < offs[k+1]
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (offs[mid] <= w) lo = mid; else hi = mid - 1;
        }
        const ApoRun& R = runs[lo];
        const int t = R.t_begin + (w - offs[lo]);
        const int ps = R.ps;
        const int W = (ps + 31) >> 5;
        uint32_t* out = const_cast<uint32_t*>(R.drmask) + (size_t)t * W;

        const uint4 pw = philox((uint32_t)t, kAll, kAll, kSlotPF, R.seed, R.run);
        const double u = (double)m24p1(pw.x) * 5.9604644775390625e-8;
        const double pf = R.pf_max * u;
        const int m = (int)ceil((double)ps * pf);

        for (int q = tid; q < ((ps + 3) >> 2); q += blockDim.x) {
            const uint4 k4 = philox((uint32_t)t, (uint32_t)q, kAll, kSlotDR, R.seed, R.run);
            const uint32_t kv[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
            for (int e = 0; e < 4; ++e)
                if (4 * q + e < ps) keys[4 * q + e] = kv[e];
        }
        __syncthreads();

        uint32_t K = 0;
        unsigned need = (unsigned)m, eq = 0;
        if (m > 0 && m < ps) {
            uint32_t prefix = 0, pmask = 0;
            for (int pass = 0; pass < 4; ++pass) {
                const int shift = 24 - 8 * pass;
                for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
                __syncthreads();
                for (int r = tid; r < ps; r += blockDim.x) {
                    const uint32_t k = keys[r];
                    if ((k & pmask) == prefix) atomicAdd(&hist[(k >> shift) & 255u], 1u);
                }
                __syncthreads();
                if (warp == 0) {
                    unsigned s = 0;
#pragma unroll
                    for (int i = 0; i < 8; ++i) s += hist[8 * lane + i];
                    unsigned incl = s;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned v = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= o) incl += v;
                    }
                    const unsigned ballot = __ballot_sync(0xffffffffu, incl >= need);
                    const int L = __ffs(ballot) - 1;
                    if (lane == L) {
                        unsigned cum = incl - s;
                        int digit = 8 * lane;
                        for (int i = 0; i < 8; ++i) {
                            if (cum + hist[8 * lane + i] >= need) { digit = 8 * lane + i; break; }
                            cum += hist[8 * lane + i];
                        }
                        s_prefix = prefix | ((uint32_t)digit << shift);
                        s_need = need - cum;
                        s_eq = hist[digit];
                    }
                }
                __syncthreads();
                prefix = s_prefix;
                pmask |= 255u << shift;
                need = s_need;
                eq = s_eq;
                __syncthreads();
            }
            K = prefix;
        }
        for (int base = warp * 32; base < W * 32; base += blockDim.x) {
            const int r = base + lane;
            bool sel = false;
            if (r < ps) {
                if (m >= ps) sel = true;
                else if (m > 0) {
                    const uint32_t k = keys[r];
                    if (k < K) sel = true;
                    else if (k == K) {
                        if (need >= eq) sel = true;
                        else {  // exact key ties: the lowest ranks first
                            unsigned before = 0;
                            for (int r2 = 0; r2 < r; ++r2) before += (keys[r2] == K);
                            sel = before < need;
                        }
                    }
                }
            }
            const unsigned b = __ballot_sync(0xffffffffu, sel);
            if (lane == 0) out[base >> 5] = b;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- shared layout
template <typename FitT>
struct Smem {
    float* X[2];
    FitT* F[2];
    uint32_t* perm[2];
    void* keys;
    float* MT;
    float *o, *lb, *ub, *ew;
    float *Xc, *Xo, *Yc, *Zc;
    FitT* rowF;
    float *compG, *compA;
    long long *P0, *P1;
    int* otsu;
    void* red;
    int* seg;
};

template <typename FitT>
__device__ __forceinline__ Smem<FitT> carve(unsigned char* base, const SmemPlan& L)
{
    Smem<FitT> S;
    S.X[0] = reinterpret_cast<float*>(base + L.X0);
    S.X[1] = reinterpret_cast<float*>(base + L.X1);
    S.F[0] = reinterpret_cast<FitT*>(base + L.F0);
    S.F[1] = reinterpret_cast<FitT*>(base + L.F1);
    S.perm[0] = reinterpret_cast<uint32_t*>(base + L.perm0);
    S.perm[1] = reinterpret_cast<uint32_t*>(base + L.perm1);
    S.keys = base + L.keys;
    S.MT = reinterpret_cast<float*>(base + L.MT);
    S.o = reinterpret_cast<float*>(base + L.o);
    S.lb = reinterpret_cast<float*>(base + L.lb);
    S.ub = reinterpret_cast<float*>(base + L.ub);
    S.ew = reinterpret_cast<float*>(base + L.ew);
    S.Xc = reinterpret_cast<float*>(base + L.Xc);
    S.Xo = reinterpret_cast<float*>(base + L.Xo);
    S.Yc = reinterpret_cast<float*>(base + L.Yc);
    S.Zc = reinterpret_cast<float*>(base + L.Zc);
    S.rowF = reinterpret_cast<FitT*>(base + L.rowF);
    S.compG = reinterpret_cast<float*>(base + L.compG);
    S.compA = reinterpret_cast<float*>(base + L.compA);
    S.P0 = reinterpret_cast<long long*>(base + L.P0);
    S.P1 = reinterpret_cast<long long*>(base + L.P1);
    S.otsu = reinterpret_cast<int*>(base + L.otsu);
    S.red = base + L.red;
    S.seg = reinterpret_cast<int*>(base + L.seg);
    return S;
}

// Loads the run's constant vectors (and the rotation of a single-component
// objective when it fits) into shared memory.
template <typename FitT>
__device__ __forceinline__ void load_constants(const ApoRun& R, const Smem<FitT>& S)
{
    const DevProblem& P = R.prob;
    const int Dp = P.Dp;
    const DevComp& C = P.comp[0];
    for (int i = threadIdx.x; i < Dp; i += blockDim.x) {
        S.lb[i] = P.lb[i];
        S.ub[i] = P.ub[i];
        S.o[i] = C.o ? C.o[i] : 0.f;
        S.ew[i] = C.ew ? C.ew[i] : 1.f;
    }
    if (R.plan.mt_smem && C.MT) {
        const float4* src = reinterpret_cast<const float4*>(C.MT);
        float4* dst = reinterpret_cast<float4*>(S.MT);
        for (int i = threadIdx.x; i < Dp * P.Np / 4; i += blockDim.x) dst[i] = src[i];
    }
    if (P.kind == kOtsu) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) {
            S.P0[i] = P.P0[i];
            S.P1[i] = P.P1[i];
        }
    }
}

// ------------------------------------------------------------ evaluation
// 16-byte shared-memory load through an explicit shared-window address.
__device__ __forceinline__ float4 lds4(uint32_t addr)
{
    float4 v;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// Z[rows][Np] = Y[rows][Dp] * MT[Dp][Np] with Y stored transposed (YT[k][row],
// row stride CH) and both operands zero padded beyond D.  FP32 FMA.  A warp
// computes an 8-row x 128-column tile, lane L the columns 4L..4L+3 of the 8
// rows: per k the 8 row values are two broadcast 16-byte loads shared by the
// whole warp and the columns one 16-byte load per lane.  MT_SHARED selects a
// rotation held in shared memory (explicit ld.shared) or read through L1.
template <bool MT_SHARED, int TR>
__device__ __forceinline__ void tile_gemm_t(const float* __restrict__ YT, const float* __restrict__ MT,
                                            float* __restrict__ Z, int rows, int Dp, int Np, int CH)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rt = (rows + TR - 1) / TR, ct = (Np + 127) >> 7;
    const uint32_t yt_s = (uint32_t)__cvta_generic_to_shared(YT);
    const uint32_t mt_s = MT_SHARED ? (uint32_t)__cvta_generic_to_shared(MT) : 0u;
    for (int tile = warp; tile < rt * ct; tile += nw) {
        const int tr = tile / ct, tc = tile - tr * ct;
        const int rb = TR * tr, c = 128 * tc + 4 * lane;
        const bool col_ok = c < Np;
        float acc[TR][4];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
#pragma unroll 2
        for (int k = 0; k < Dp; ++k) {
            const uint32_t ya = yt_s + 4u * (uint32_t)(k * CH + rb);
            const float4 a0 = lds4(ya);
            const float4 a1 = TR == 8 ? lds4(ya + 16u) : make_float4(0.f, 0.f, 0.f, 0.f);
            float4 b = make_float4(0.f, 0.f, 0.f, 0.f);
            if (col_ok) {
                if (MT_SHARED) b = lds4(mt_s + 4u * (uint32_t)(k * Np + c));
                else b = __ldg(reinterpret_cast<const float4*>(MT + (size_t)k * Np + c));
            }
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                acc[i][0] = fmaf(av[i], b.x, acc[i][0]);
                acc[i][1] = fmaf(av[i], b.y, acc[i][1]);
                acc[i][2] = fmaf(av[i], b.z, acc[i][2]);
                acc[i][3] = fmaf(av[i], b.w, acc[i][3]);
            }
        }
        if (col_ok) {
#pragma unroll
            for (int i = 0; i < TR; ++i)
                if (rb + i < rows)
                    *reinterpret_cast<float4*>(Z + (size_t)(rb + i) * Np + c) =
                        make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        }
    }
}

// 8-row tiles when they keep every warp busy, 4-row tiles otherwise.
template <bool MT_SHARED>
__device__ __forceinline__ void tile_gemm(const float* __restrict__ YT, const float* __restrict__ MT,
                                          float* __restrict__ Z, int rows, int Dp, int Np, int CH)
{
    const int nw = blockDim.x >> 5, ct = (Np + 127) >> 7;
    if (((rows + 7) >> 3) * ct >= nw) tile_gemm_t<MT_SHARED, 8>(YT, MT, Z, rows, Dp, Np, CH);
    else tile_gemm_t<MT_SHARED, 4>(YT, MT, Z, rows, Dp, Np, CH);
}

// Segmented objective of one row by one warp (z[d * zs]): [0, s1) high-conditioned
// elliptic, [s1, s2) chained Rosenbrock, [s2, D) Rastrigin cosine sum.
__device__ __forceinline__ float seg_value(const float* z, int zs, const DevComp& C, const float* ew, int D)
{
    const int lane = threadIdx.x & 31;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float v = z[(size_t)d * zs];
        if (d < C.s1) {
            s = fmaf(ew[d] * v, v, s);
        } else if (d < C.s2) {
            if (d + 1 < C.s2) {
                const float a = z[(size_t)(d + 1) * zs] - v * v;
                const float b = v - 1.f;
                s += 100.f * a * a + b * b;
            }
        } else {
            s += v * v - 10.f * cospif(2.f * v) + 10.f;
        }
    }
    return warp_sum(s);
}

// Otsu between-class variance of one row by one warp (thresholds in lanes
// 0..T-1), negated.  The float64 operations follow a fixed order with
// explicit round-to-nearest intrinsics (no contraction) so that the value is
// reproducible bit for bit.
__device__ __forceinline__ double otsu_row(const float* x, int T, const long long* P0, const long long* P1,
                           int* scratch)
{
    const int lane = threadIdx.x & 31;
    int tv = 0;
    if (lane < T) {
        float f = floorf(x[lane]);
        f = fminf(fmaxf(f, 0.f), 255.f);
        tv = (int)f;
    }
    int rank = 0;
    for (int i = 0; i < T; ++i) {
        const int ti = __shfl_sync(0xffffffffu, tv, i);
        if (ti < tv || (ti == tv && i < lane)) ++rank;
    }
    __syncwarp();
    if (lane < T) scratch[rank] = tv;
    __syncwarp();
    double sigma = 0.0;
    if (lane == 0) {
        const long long N = P0[255], Ssum = P1[255];
        const double muT = __ddiv_rn((double)Ssum, (double)N);
        int prev = -1;
        for (int c = 0; c <= T; ++c) {
            const int hi = (c < T) ? scratch[c] : 255;
            long long nc = 0, sc = 0;
            if (hi > prev) {
                nc = P0[hi] - (prev >= 0 ? P0[prev] : 0ll);
                sc = P1[hi] - (prev >= 0 ? P1[prev] : 0ll);
                prev = hi;
            }
            if (nc > 0) {
                const double omega = __ddiv_rn((double)nc, (double)N);
                const double mu = __ddiv_rn((double)sc, (double)nc);
                const double dm = __dsub_rn(mu, muT);
                double term = __dmul_rn(omega, dm);
                term = __dmul_rn(term, dm);
                sigma = __dadd_rn(sigma, term);
            }
        }
    }
    sigma = __shfl_sync(0xffffffffu, sigma, 0);
    __syncwarp();
    return -sigma;
}

// Evaluates the candidate rows Xc[0, rows) into rowF.  Called by the whole
// CTA; ends synchronised.
template <typename FitT>
__device__ __forceinline__ void eval_chunk(const ApoRun& R, const Smem<FitT>& S, int rows)
{
    const DevProblem& P = R.prob;
    const int D = P.D, Dp = P.Dp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (P.kind == kOtsu) {
        for (int row = warp; row < rows; row += nw) {
            const double f = otsu_row(S.Xc + (size_t)row * Dp, D, S.P0, S.P1, S.otsu + warp * 32);
            if (lane == 0) S.rowF[row] = (FitT)f;
        }
        __syncthreads();
        return;
    }
    const int CH = R.plan.chunk, Np = P.Np;
    for (int c = 0; c < P.ncomp; ++c) {
        const DevComp& C = P.comp[c];
        const float* o = (c == 0) ? S.o : C.o;
        // YT[d][row] = x - o (zero beyond D)
        for (int i = threadIdx.x; i < CH * Dp; i += blockDim.x) {
            const int d = i / CH, row = i - d * CH;
            S.Yc[i] = (d < D && row < rows) ? S.Xc[(size_t)row * Dp + d] - o[d] : 0.f;
        }
        __syncthreads();
        if (C.MT) {
            if (c == 0 && R.plan.mt_smem) tile_gemm<true>(S.Yc, S.MT, S.Zc, rows, Dp, Np, CH);
            else tile_gemm<false>(S.Yc, C.MT, S.Zc, rows, Dp, Np, CH);
            __syncthreads();
        }
        const float* ew = (c == 0) ? S.ew : C.ew;
        for (int row = warp; row < rows; row += nw) {
            const float v = C.MT ? seg_value(S.Zc + (size_t)row * Np, 1, C, ew, D)
                                 : seg_value(S.Yc + row, CH, C, ew, D);
            if (P.ncomp == 1) {
                if (lane == 0) S.rowF[row] = (FitT)v;
            } else {
                float d2 = 0.f;
                for (int d = lane; d < D; d += 32) {
                    const float y = S.Yc[(size_t)d * CH + row];
                    d2 = fmaf(y, y, d2);
                }
                d2 = warp_sum(d2);
                if (lane == 0) {
                    S.compG[row * kMaxComp + c] = v;
                    S.compA[row * kMaxComp + c] = -d2 * C.inv_2Dsig2;
                }
            }
        }
        __syncthreads();
    }
    if (P.ncomp > 1) {
        // f = sum_k w_k (g_k + bias_k) / sum_k w_k, w_k = exp(a_k - max a).
        for (int row = warp; row < rows; row += nw) {
            const bool on = lane < P.ncomp;
            const float a = on ? S.compA[row * kMaxComp + lane] : -INFINITY;
            const float amax = warp_max(a);
            const float w = on ? expf(a - amax) : 0.f;
            const float gv = on ? S.compG[row * kMaxComp + lane] + P.comp[lane < kMaxComp ? lane : 0].bias : 0.f;
            const float num = warp_sum(w * gv);
            const float den = warp_sum(w);
            if (lane == 0) S.rowF[row] = (FitT)(num / den);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------- state access
template <typename T>
__device__ __forceinline__ T ldst(const T* p, bool resident)
{
    return resident ? *p : __ldcg(p);
}

// ------------------------------------------------- candidate generation
// Population initialisation (Algorithm 1): X_p = Xmin + U (Xmax - Xmin).
template <typename FitT, int QPL>
__device__ __forceinline__ void gen_init_row(const ApoRun& R, const Smem<FitT>& S, int p, int row)
{
    const int lane = threadIdx.x & 31;
    const int D = R.prob.D, Dp = R.prob.Dp;
    float* xc = S.Xc + (size_t)row * Dp;
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = lane + 32 * j;
        const int d0 = 2 * q;
        if (d0 < D) {
            const uint4 w = philox(0u, (uint32_t)p, (uint32_t)q, kSlotInit, R.seed, R.run);
            xc[d0] = fmaf(u01(w.x), S.ub[d0] - S.lb[d0], S.lb[d0]);
            if (d0 + 1 < D) xc[d0 + 1] = fmaf(u01(w.z), S.ub[d0 + 1] - S.lb[d0 + 1], S.lb[d0 + 1]);
            else if (d0 + 1 < Dp) xc[d0 + 1] = 0.f;
        } else if (d0 < Dp) {
            xc[d0] = 0.f;
            xc[d0 + 1] = 0.f;
        }
    }
}

// One candidate (rank r, 0-based) by one warp: mode selection (Eq. 12-13,
// Algorithm 1), masks (Eq. 3, Eq. 5), dormancy (Eq. 1), reproduction
// (Eq. 2), autotrophic (Eq. 6-7) or heterotrophic (Eq. 8-10) foraging, then
// the bound clamp.  Writes row `row` of Xc (candidate) and of Xo (the old
// position, kept for the greedy replacement).  The per-protozoon draws are
// computed once per warp, one Philox call per lane; the gathered rows are
// requested before the per-dimension draws and the mask selection so that
// their latency overlaps that arithmetic.
template <typename FitT, int QPL>
__device__ __forceinline__ void gen_step_row(const ApoRun& R, const Smem<FitT>& S, const float* __restrict__ X,
                             const FitT* __restrict__ F, const uint32_t* perm, bool res, int t,
                             int r, int row)
{
    const int lane = threadIdx.x & 31;
    const int D = R.prob.D, Dp = R.prob.Dp, ps = R.ps, np = R.np;
    const uint32_t seed = R.seed, run = R.run;
    // lane 0: SCAL, lane 1: SCAL2, lane 2 + k: PAIR k
    uint32_t jslot = kSlotPair, jd = (uint32_t)(lane - 2);
    if (lane == 0) { jslot = kSlotScal; jd = kAll; }
    if (lane == 1) { jslot = kSlotScal2; jd = kAll; }
    const uint4 jw = philox((uint32_t)t, (uint32_t)r, jd, jslot, seed, run);
    uint4 sc, sc2;
    sc.x = __shfl_sync(0xffffffffu, jw.x, 0); sc.y = __shfl_sync(0xffffffffu, jw.y, 0);
    sc.z = __shfl_sync(0xffffffffu, jw.z, 0); sc.w = __shfl_sync(0xffffffffu, jw.w, 0);
    sc2.x = __shfl_sync(0xffffffffu, jw.x, 1); sc2.y = __shfl_sync(0xffffffffu, jw.y, 1);
    const int W = (ps + 31) >> 5;
    const bool in_dr = (R.drmask[(size_t)t * W + (r >> 5)] >> (r & 31)) & 1u;
    const uint32_t mm = m24p1(sc.x);
    int mode;
    if (in_dr) mode = (mm < R.thr_dr[r]) ? kDormancy : kReproduction;
    else mode = (mm < R.thr_ah[t]) ? kAutotrophic : kHeterotrophic;
    const bool forage = mode == kAutotrophic || mode == kHeterotrophic;

    // rows from the snapshot: X_i, X_j (autotrophic) and the first pair
    const int si = (int)perm[r];
    int sj = si, sa = si, sb = si;
    if (mode == kAutotrophic) {
        sj = (int)perm[idx_draw(sc2.y, (uint32_t)ps)];
        const uint32_t p0 = __shfl_sync(0xffffffffu, jw.x, 2), p1 = __shfl_sync(0xffffffffu, jw.y, 2);
        sa = (int)perm[idx_draw(p0, (uint32_t)ps)];
        sb = (int)perm[idx_draw(p1, (uint32_t)ps)];
    } else if (mode == kHeterotrophic) {
        sa = (int)perm[r - 1 < 0 ? 0 : r - 1];
        sb = (int)perm[r + 1 > ps - 1 ? ps - 1 : r + 1];
    }
    float xi[2 * QPL], xj[2 * QPL], xa[2 * QPL], xb[2 * QPL];
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = lane + 32 * j;
        float2 vi = make_float2(0.f, 0.f), vj = vi, va = vi, vb = vi;
        if (2 * q < D) {
            vi = ldst(reinterpret_cast<const float2*>(X + (size_t)si * Dp) + q, res);
            if (mode == kAutotrophic) vj = ldst(reinterpret_cast<const float2*>(X + (size_t)sj * Dp) + q, res);
            if (forage) {
                va = ldst(reinterpret_cast<const float2*>(X + (size_t)sa * Dp) + q, res);
                vb = ldst(reinterpret_cast<const float2*>(X + (size_t)sb * Dp) + q, res);
            }
        }
        xi[2 * j] = vi.x; xi[2 * j + 1] = vi.y;
        xj[2 * j] = vj.x; xj[2 * j + 1] = vj.y;
        xa[2 * j] = va.x; xa[2 * j + 1] = va.y;
        xb[2 * j] = vb.x; xb[2 * j + 1] = vb.y;
    }
    float fa = 0.f, fb = 1.f;
    if (forage) {
        fa = (float)ldst(F + sa, res);
        fb = (float)ldst(F + sb, res);
    }
    if (lane == 0) S.rowF[R.plan.chunk + row] = ldst(F + si, res);   // old fitness for the greedy step

    // per-dimension draws and the mask (independent of the gathered rows)
    uint32_t A[2 * QPL], B[2 * QPL];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = lane + 32 * j;
        if (2 * q < D) {
            const uint4 w = philox((uint32_t)t, (uint32_t)r, (uint32_t)q, kSlotDim, seed, run);
            A[2 * j] = w.x; B[2 * j] = w.y; A[2 * j + 1] = w.z; B[2 * j + 1] = w.w;
            valid |= 1u << (2 * j);
            if (2 * q + 1 < D) valid |= 1u << (2 * j + 1);
        } else {
            A[2 * j] = B[2 * j] = A[2 * j + 1] = B[2 * j + 1] = 0u;
        }
    }
    uint32_t mask = 0;
    if (mode == kReproduction) {
        const int k = (int)(((unsigned long long)D * m24p1(sc2.x) + 0xFFFFFFull) >> 24);
        mask = warp_kselect<QPL>(B, valid, k);
    } else if (forage) {
        const int k = (D * (r + 1) + ps - 1) / ps;
        mask = warp_kselect<QPL>(B, valid, k);
    }

    // Eq. 7 / Eq. 10 weights and the pair sums
    float acc[2 * QPL];
    if (forage) {
        const float w = expf(-fabsf(fa / (fb + kEps)));
#pragma unroll
        for (int e = 0; e < 2 * QPL; ++e) acc[e] = w * (xa[e] - xb[e]);
        for (int k = 2; k <= np; ++k) {
            if (mode == kAutotrophic) {
                uint32_t p0, p1;
                if (k + 1 < 32) {
                    p0 = __shfl_sync(0xffffffffu, jw.x, k + 1);
                    p1 = __shfl_sync(0xffffffffu, jw.y, k + 1);
                } else {
                    const uint4 pr = philox((uint32_t)t, (uint32_t)r, (uint32_t)(k - 1), kSlotPair, seed, run);
                    p0 = pr.x;
                    p1 = pr.y;
                }
                sa = (int)perm[idx_draw(p0, (uint32_t)ps)];
                sb = (int)perm[idx_draw(p1, (uint32_t)ps)];
            } else {
                sa = (int)perm[r - k < 0 ? 0 : r - k];
                sb = (int)perm[r + k > ps - 1 ? ps - 1 : r + k];
            }
            const float w2 = expf(-fabsf((float)ldst(F + sa, res) / ((float)ldst(F + sb, res) + kEps)));
#pragma unroll
            for (int j = 0; j < QPL; ++j) {
                const int q = lane + 32 * j;
                if (2 * q < D) {
                    const float2 va = ldst(reinterpret_cast<const float2*>(X + (size_t)sa * Dp) + q, res);
                    const float2 vb = ldst(reinterpret_cast<const float2*>(X + (size_t)sb * Dp) + q, res);
                    acc[2 * j] = fmaf(w2, va.x - vb.x, acc[2 * j]);
                    acc[2 * j + 1] = fmaf(w2, va.y - vb.y, acc[2 * j + 1]);
                }
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < 2 * QPL; ++e) acc[e] = 0.f;
    }
    const float inv_np = 1.f / (float)np;
    const float ff = forage ? u01(sc.y) * R.fsc[t] : 0.f;
    const float s = sign_draw(sc.z);
    const float rho = u01(sc.w);
    const float nsc = R.nsc[t];

    float* xc = S.Xc + (size_t)row * Dp;
    float* xo = S.Xo + (size_t)row * Dp;
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = lane + 32 * j;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int d = 2 * q + e;
            const int sl = 2 * j + e;
            if (d < D) {
                const float lb = S.lb[d], ub = S.ub[d];
                const bool mk = (mask >> sl) & 1u;
                const float x0 = xi[sl];
                float x = x0;
                if (mode == kDormancy) {
                    x = fmaf(u01(A[sl]), ub - lb, lb);                          // Eq. 1
                } else if (mk) {
                    if (mode == kReproduction) {
                        x = x0 + s * rho * fmaf(u01(A[sl]), ub - lb, lb);       // Eq. 2
                    } else if (mode == kAutotrophic) {
                        x = x0 + ff * (xj[sl] - x0 + acc[sl] * inv_np);         // Eq. 6
                    } else {
                        const float xnear = (1.f + s * u01(A[sl]) * nsc) * x0;  // Eq. 9
                        x = x0 + ff * (xnear - x0 + acc[sl] * inv_np);          // Eq. 8
                    }
                }
                xc[d] = fminf(fmaxf(x, lb), ub);
                xo[d] = x0;
            } else if (d < Dp) {
                xc[d] = 0.f;
                xo[d] = 0.f;
            }
        }
    }
}

// -------------------------------------------------------------- the run
template <typename FitT>
__device__ __forceinline__ void find_best(const Smem<FitT>& S, const FitT* F, const uint32_t* perm, int ps,
                          bool res, typename KeyOf<FitT>::T* red, int* out_rank)
{
    using KO = KeyOf<FitT>;
    typename KO::T best = KO::pad();
    for (int r = threadIdx.x; r < ps; r += blockDim.x) {
        const typename KO::T k = KO::make(ldst(F + perm[r], res), (uint32_t)r);
        if (KO::less(k, best)) best = k;
    }
    red[threadIdx.x] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        typename KO::T b = red[0];
        for (int i = 1; i < (int)blockDim.x; ++i)
            if (KO::less(red[i], b)) b = red[i];
        *out_rank = (int)KO::idx(b);
    }
    __syncthreads();
}

template <typename FitT, int QPL>
__device__ __forceinline__ void run_one(const ApoRun& R, int local, unsigned char* smem, int* status, int* s_flag,
                        int* s_int)
{
    using KO = KeyOf<FitT>;
    using KT = typename KO::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const DevProblem& P = R.prob;
    const int D = P.D, Dp = P.Dp, ps = R.ps, g = R.g;
    const SmemPlan& L = R.plan;
    const int CH = L.chunk;
    const Smem<FitT> S = carve<FitT>(smem, L);
    const bool res = L.resident != 0;
    unsigned bgen = 0;

    load_constants<FitT>(R, S);
    for (int r = tid; r < ps; r += blockDim.x) S.perm[0][r] = (uint32_t)r;
    float* Xs[2];
    FitT* Fs[2];
    if (res) {
        Xs[0] = S.X[0]; Xs[1] = S.X[1]; Fs[0] = S.F[0]; Fs[1] = S.F[1];
    } else {
        Xs[0] = R.X[0]; Xs[1] = R.X[1];
        Fs[0] = static_cast<FitT*>(R.F[0]); Fs[1] = static_cast<FitT*>(R.F[1]);
    }
    const int r0 = (int)((long long)ps * local / g);
    const int r1 = (int)((long long)ps * (local + 1) / g);
    __syncthreads();

    if (R.flags & kFlagInit) {
        for (int c0 = r0; c0 < r1; c0 += CH) {
            const int rows = min(CH, r1 - c0);
            for (int row = warp; row < rows; row += nw) gen_init_row<FitT, QPL>(R, S, c0 + row, row);
            __syncthreads();
            eval_chunk<FitT>(R, S, rows);
            for (int row = warp; row < rows; row += nw) {
                float* dst = Xs[0] + (size_t)(c0 + row) * Dp;
                for (int d = lane; d < Dp; d += 32) dst[d] = S.Xc[(size_t)row * Dp + d];
                if (lane == 0) Fs[0][c0 + row] = S.rowF[row];
            }
            __syncthreads();
        }
    } else if (res) {
        const float* gx = R.X[0];
        const FitT* gf = static_cast<const FitT*>(R.F[0]);
        for (int i = tid; i < ps * Dp; i += blockDim.x) Xs[0][i] = gx[i];
        for (int i = tid; i < ps; i += blockDim.x) Fs[0][i] = gf[i];
        __syncthreads();
    }
    if (!run_barrier(R.bar, g, bgen, status, s_flag)) return;

    int cur = 0, pc = 0;
    KT* keys = static_cast<KT*>(S.keys);
    for (int t = R.t_begin; t <= R.t_end; ++t) {
        // Algorithm 1: sort by fitness; ties keep the previous order.
        const uint32_t* perm = S.perm[pc];
        uint32_t* pnew = S.perm[pc ^ 1];
        for (int r = tid; r < L.ps_pad; r += blockDim.x)
            keys[r] = r < ps ? KO::make(ldst(Fs[cur] + perm[r], res), (uint32_t)r) : KO::pad();
        __syncthreads();
        bitonic_sort<KO>(keys, L.ps_pad);
        for (int r = tid; r < ps; r += blockDim.x) pnew[r] = perm[KO::idx(keys[r])];
        __syncthreads();
        pc ^= 1;
        perm = pnew;
        if (local == 0 && tid == 0 && R.curve) R.curve[t - 1] = (float)ldst(Fs[cur] + perm[0], res);

        for (int c0 = r0; c0 < r1; c0 += CH) {
            const int rows = min(CH, r1 - c0);
            for (int row = warp; row < rows; row += nw)
                gen_step_row<FitT, QPL>(R, S, Xs[cur], Fs[cur], perm, res, t, c0 + row, row);
            __syncthreads();
            eval_chunk<FitT>(R, S, rows);
            // Greedy replacement (Algorithm 1): keep X_new iff f(X_new) < f(X_i).
            for (int row = warp; row < rows; row += nw) {
                const int slot = (int)perm[c0 + row];
                const FitT fo = S.rowF[CH + row];
                const FitT fn = S.rowF[row];
                const bool acc = fn < fo;
                const float4* src = reinterpret_cast<const float4*>((acc ? S.Xc : S.Xo) + (size_t)row * Dp);
                float4* dst = reinterpret_cast<float4*>(Xs[cur ^ 1] + (size_t)slot * Dp);
                for (int v = lane; v < (Dp >> 2); v += 32) dst[v] = src[v];
                if (lane == 0) Fs[cur ^ 1][slot] = acc ? fn : fo;
            }
            __syncthreads();
        }
        if (!run_barrier(R.bar, g, bgen, status, s_flag)) return;
        cur ^= 1;
    }

    const uint32_t* perm = S.perm[pc];
    if (R.flags & kFlagStepOut) {
        float* xo = R.X_out;
        FitT* fo = static_cast<FitT*>(R.F_out);
        for (int r = r0 + warp; r < r1; r += nw) {
            const int slot = (int)perm[r];
            for (int d = lane; d < D; d += 32) xo[(size_t)r * D + d] = ldst(Xs[cur] + (size_t)slot * Dp + d, res);
            if (lane == 0) fo[r] = ldst(Fs[cur] + slot, res);
        }
    } else if (local == 0) {
        find_best<FitT>(S, Fs[cur], perm, ps, res, static_cast<KT*>(S.red), s_int);
        const int slot = (int)perm[*s_int];
        const FitT fb = ldst(Fs[cur] + slot, res);
        if (tid == 0) {
            if (R.curve) R.curve[R.t_end] = (float)fb;
            if (R.best_f) *R.best_f = (double)fb;
        }
        if (R.best_x)
            for (int d = tid; d < D; d += blockDim.x) R.best_x[d] = ldst(Xs[cur] + (size_t)slot * Dp + d, res);
    }
    __syncthreads();
}

__device__ __forceinline__ void copy_run(ApoRun* dst, const ApoRun* src)
{
    static_assert(sizeof(ApoRun) % 8 == 0, "ApoRun must be 8-byte sized");
    const unsigned long long* s = reinterpret_cast<const unsigned long long*>(src);
    unsigned long long* d = reinterpret_cast<unsigned long long*>(dst);
    for (int i = threadIdx.x; i < (int)(sizeof(ApoRun) / 8); i += blockDim.x) d[i] = s[i];
}

template <typename FitT, int QPL>
__global__ void __launch_bounds__(kThreads, 2) run_kernel(const ApoRun* __restrict__ runs, int n_runs,
                                                       int* queue, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    __shared__ int s_run, s_flag, s_int;
    for (;;) {
        if (threadIdx.x == 0) s_run = atomicAdd(queue, 1);
        __syncthreads();
        const int run = s_run;
        if (run >= n_runs) return;
        copy_run(&R, runs + run);
        __syncthreads();
        run_one<FitT, QPL>(R, 0, smem, status, &s_flag, &s_int);
        __syncthreads();
    }
}

// ------------------------------------------------------------ grid mode
// g CTAs run one optimisation run; CTA `local` owns the rank positions
// [r0, r1) of every iteration and keeps a full copy of the rank -> slot
// permutation in shared memory.  Per iteration:
//   R1  sort the keys (F, previous rank) of the own rank range and publish
//       them as a sorted segment of keys_g;                       barrier A
//   R2  the new rank of each own key = its position in its own segment plus
//       its lower bound in every other segment (the stable sort of
//       Algorithm 1, distributed); scatter perm_g[rank] = slot;    barrier B
//   R3  copy perm_g, then generate, evaluate and replace the own rank range;
//       candidates read the double-buffered snapshot of the iteration.
__device__ __forceinline__ unsigned long long lds_key(uint32_t a, unsigned long long*)
{
    unsigned long long v;
    asm("ld.shared.u64 %0, [%1];" : "=l"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ ulonglong2 lds_key(uint32_t a, ulonglong2*)
{
    ulonglong2 v;
    asm("ld.shared.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(a));
    return v;
}

// Number of keys of the sorted shared-memory segment seg[0, len) below k.
template <typename FitT>
__device__ __forceinline__ int lower_bound_key(const typename KeyOf<FitT>::T* seg, int len,
                                               typename KeyOf<FitT>::T k)
{
    using KT = typename KeyOf<FitT>::T;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(seg);
    int lo = 0, hi = len;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (KeyOf<FitT>::less(lds_key(base + (uint32_t)(mid * sizeof(KT)), (KT*)nullptr), k)) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ unsigned long long shfl_xor_key(unsigned long long v, int m)
{
    return __shfl_xor_sync(0xffffffffu, v, m);
}
__device__ __forceinline__ ulonglong2 shfl_xor_key(ulonglong2 v, int m)
{
    return make_ulonglong2(__shfl_xor_sync(0xffffffffu, v.x, m), __shfl_xor_sync(0xffffffffu, v.y, m));
}

// Copies n elements from global (L2, bypassing L1) to shared memory with
// eight independent loads in flight per thread.
template <typename T>
__device__ __forceinline__ void copy_cg(T* dst, const T* __restrict__ src, int n)
{
    for (int base = threadIdx.x; base < n; base += 8 * blockDim.x) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * blockDim.x;
            if (i < n) v[u] = __ldcg(src + i);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = base + u * blockDim.x;
            if (i < n) dst[i] = v[u];
        }
    }
}

template <typename FitT, int QPL>
__device__ __forceinline__ void run_grid(const ApoRun& R, int local, unsigned char* smem, int* status, int* s_flag)
{
    using KO = KeyOf<FitT>;
    using KT = typename KO::T;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int NT = blockDim.x;
    const DevProblem& P = R.prob;
    const int D = P.D, Dp = P.Dp, ps = R.ps, g = R.g;
    const SmemPlan& L = R.plan;
    const int CH = L.chunk;
    const Smem<FitT> S = carve<FitT>(smem, L);
    unsigned bgen = 0;

    load_constants<FitT>(R, S);
    float* Xs[2] = {R.X[0], R.X[1]};
    FitT* Fs[2] = {static_cast<FitT*>(R.F[0]), static_cast<FitT*>(R.F[1])};
    uint32_t* perm = S.perm[0];
    KT* keys = static_cast<KT*>(S.keys);
    KT* keys_g = static_cast<KT*>(R.keys_g);
    int* seg = S.seg;   // seg[c] = first rank position of CTA c; seg[g] = ps
    for (int c = tid; c <= g; c += NT) seg[c] = (int)((long long)ps * c / g);
    const int r0 = (int)((long long)ps * local / g);
    const int r1 = (int)((long long)ps * (local + 1) / g);
    const int nown = r1 - r0;
    int npad = 1;
    while (npad < nown) npad <<= 1;
    for (int r = tid; r < ps; r += NT) perm[r] = (uint32_t)r;
    __syncthreads();

    if (R.flags & kFlagInit) {
        for (int c0 = r0; c0 < r1; c0 += CH) {
            const int rows = min(CH, r1 - c0);
            for (int row = warp; row < rows; row += nw) gen_init_row<FitT, QPL>(R, S, c0 + row, row);
            __syncthreads();
            eval_chunk<FitT>(R, S, rows);
            for (int row = warp; row < rows; row += nw) {
                float* dst = Xs[0] + (size_t)(c0 + row) * Dp;
                for (int d = lane; d < Dp; d += 32) dst[d] = S.Xc[(size_t)row * Dp + d];
                if (lane == 0) Fs[0][c0 + row] = S.rowF[row];
            }
            __syncthreads();
        }
    }

    int cur = 0;
    bool keys_ready = false;   // the greedy step already wrote the own keys
    const bool step_out = (R.flags & kFlagStepOut) != 0;
    for (int t = R.t_begin;; ++t) {
        // R1: own keys (F, rank in the current order), sorted and published
        if (!keys_ready)
            for (int i = tid; i < nown; i += NT)
                keys[i] = KO::make(ldst(Fs[cur] + perm[r0 + i], false), (uint32_t)(r0 + i));
        __syncthreads();
        if (nown <= 2 * NT) {
            // rank by counting among the own keys (all distinct)
            for (int i = tid; i < nown; i += NT) {
                const KT k = keys[i];
                int rk = 0;
                for (int j = 0; j < nown; ++j) rk += KO::less(keys[j], k) ? 1 : 0;
                keys_g[r0 + rk] = k;
            }
        } else {
            for (int i = tid; i < npad; i += NT)
                if (i >= nown) keys[i] = KO::pad();
            __syncthreads();
            bitonic_sort<KO>(keys, npad);
            for (int i = tid; i < nown; i += NT) keys_g[r0 + i] = keys[i];
        }
        if (!run_barrier(R.bar, g, bgen, status, s_flag)) return;

        // the best of the population after iteration t - 1: the smallest head
        if (local == 0) {
            if (warp == 0) {
                KT best = KO::pad();
                for (int c = lane; c < g; c += 32) {
                    if (seg[c + 1] > seg[c]) {
                        const KT h = __ldcg(keys_g + seg[c]);
                        if (KO::less(h, best)) best = h;
                    }
                }
#pragma unroll
                for (int m = 16; m; m >>= 1) {
                    const KT o = shfl_xor_key(best, m);
                    if (KO::less(o, best)) best = o;
                }
                if (lane == 0) *reinterpret_cast<int*>(S.red) = (int)perm[KO::idx(best)];
            }
            __syncthreads();
            const int bslot = *reinterpret_cast<int*>(S.red);
            const FitT fb = ldst(Fs[cur] + bslot, false);
            if (tid == 0 && R.curve) R.curve[t - 1] = (float)fb;
            if (t > R.t_end && !step_out) {
                if (tid == 0 && R.best_f) *R.best_f = (double)fb;
                if (R.best_x)
                    for (int d = tid; d < D; d += NT) R.best_x[d] = ldst(Xs[cur] + (size_t)bslot * Dp + d, false);
            }
        }
        if (t > R.t_end) break;

        // R2: distributed ranking -- new rank = position in the own segment +
        // lower bound in every other segment (one warp per key, lanes over segments)
        copy_cg(keys, keys_g, ps);
        __syncthreads();
        for (int i = warp; i < nown; i += nw) {
            const KT k = keys[r0 + i];
            int cnt = 0;
            for (int c = lane; c < g; c += 32)
                if (c != local) cnt += lower_bound_key<FitT>(keys + seg[c], seg[c + 1] - seg[c], k);
            cnt = __reduce_add_sync(0xffffffffu, cnt) + i;
            if (lane == 0) R.perm_g[cnt] = perm[KO::idx(k)];
        }
        if (!run_barrier(R.bar, g, bgen, status, s_flag)) return;

        // R3: the new permutation, then the own rank range
        copy_cg(perm, R.perm_g, ps);
        __syncthreads();
        for (int c0 = r0; c0 < r1; c0 += CH) {
            const int rows = min(CH, r1 - c0);
            for (int row = warp; row < rows; row += nw)
                gen_step_row<FitT, QPL>(R, S, Xs[cur], Fs[cur], perm, false, t, c0 + row, row);
            __syncthreads();
            eval_chunk<FitT>(R, S, rows);
            // Greedy replacement (Algorithm 1): keep X_new iff f(X_new) < f(X_i);
            // the kept fitness also forms the own sort key of the next iteration.
            for (int row = warp; row < rows; row += nw) {
                const int slot = (int)perm[c0 + row];
                const FitT fo = S.rowF[CH + row];
                const FitT fn = S.rowF[row];
                const bool acc = fn < fo;
                const float4* src = reinterpret_cast<const float4*>((acc ? S.Xc : S.Xo) + (size_t)row * Dp);
                float4* dst = reinterpret_cast<float4*>(Xs[cur ^ 1] + (size_t)slot * Dp);
                for (int v = lane; v < (Dp >> 2); v += 32) dst[v] = src[v];
                if (lane == 0) {
                    Fs[cur ^ 1][slot] = acc ? fn : fo;
                    keys[c0 + row - r0] = KO::make(acc ? fn : fo, (uint32_t)(c0 + row));
                }
            }
            __syncthreads();
        }
        keys_ready = true;
        cur ^= 1;
        if (step_out && t == R.t_end) {
            float* xo = R.X_out;
            FitT* fo = static_cast<FitT*>(R.F_out);
            for (int r = r0 + warp; r < r1; r += nw) {
                const int slot = (int)perm[r];
                for (int d = lane; d < D; d += 32) xo[(size_t)r * D + d] = ldst(Xs[cur] + (size_t)slot * Dp + d, false);
                if (lane == 0) fo[r] = ldst(Fs[cur] + slot, false);
            }
            break;
        }
    }
    __syncthreads();
}

template <typename FitT, int QPL>
__global__ void __launch_bounds__(kGridThreads, 1) grid_kernel(const ApoRun* __restrict__ runs, int n_runs,
                                                                int grid_g, int* status)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    __shared__ int s_flag;
    const int run = blockIdx.x / grid_g, local = blockIdx.x % grid_g;
    if (run >= n_runs) return;
    copy_run(&R, runs + run);
    __syncthreads();
    run_grid<FitT, QPL>(R, local, smem, status, &s_flag);
}

// ------------------------------------------------------- evaluation hook
template <typename FitT, int QPL>
__global__ void __launch_bounds__(kThreads) eval_kernel(const ApoRun* __restrict__ run, int n,
                                                        const float* __restrict__ X, FitT* F,
                                                        int select, float* Xsel, FitT* Fsel)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ApoRun R;
    copy_run(&R, run);
    __syncthreads();
    const Smem<FitT> S = carve<FitT>(smem, R.plan);
    load_constants<FitT>(R, S);
    __syncthreads();
    const int D = R.prob.D, Dp = R.prob.Dp, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int c0 = blockIdx.x * R.plan.chunk; c0 < n; c0 += gridDim.x * R.plan.chunk) {
        const int rows = min(R.plan.chunk, n - c0);
        for (int row = warp; row < rows; row += (int)(blockDim.x >> 5)) {
            for (int d = lane; d < Dp; d += 32) {
                float x = d < D ? X[(size_t)(c0 + row) * D + d] : 0.f;
                if (select && d < D) x = fminf(fmaxf(x, S.lb[d]), S.ub[d]);
                S.Xc[(size_t)row * Dp + d] = x;
            }
        }
        __syncthreads();
        eval_chunk<FitT>(R, S, rows);
        for (int row = warp; row < rows; row += (int)(blockDim.x >> 5)) {
            const int i = c0 + row;
            const FitT fn = S.rowF[row];
            if (!select) {
                if (lane == 0) F[i] = fn;
                continue;
            }
            float* xnew = const_cast<float*>(X) + (size_t)i * D;
            for (int d = lane; d < D; d += 32) xnew[d] = S.Xc[(size_t)row * Dp + d];
            const bool acc = fn < Fsel[i];
            if (acc)
                for (int d = lane; d < D; d += 32) Xsel[(size_t)i * D + d] = S.Xc[(size_t)row * Dp + d];
            __syncwarp();
            if (lane == 0) {
                F[i] = fn;
                if (acc) Fsel[i] = fn;
            }
        }
        __syncthreads();
    }
}

__global__ void philox_kernel(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int n,
                              uint32_t* __restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint4 w = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
        out[4 * i] = w.x;
        out[4 * i + 1] = w.y;
        out[4 * i + 2] = w.z;
        out[4 * i + 3] = w.w;
    }
}

// ------------------------------------------------------- host launchers
cudaError_t launch_dr(const ApoRun* d_runs, const int* d_offs, int n_runs, int n_work,
                      int max_ps_pad, cudaStream_t st)
{
    if (n_work <= 0) return cudaSuccess;
    const size_t smem = (size_t)max_ps_pad * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(dr_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = n_work < sms * 8 ? n_work : sms * 8;
    dr_kernel<<<grid, kThreads, smem, st>>>(d_runs, d_offs, n_runs, n_work);
    return cudaGetLastError();
}

template <typename FitT, int QPL>
static cudaError_t launch_run_t(const ApoRun* d_runs, int n_runs, int grid_g, int n_ctas, int* d_queue,
                                int* d_status, size_t smem, cudaStream_t st)
{
    if (grid_g > 0) {
        auto fn = grid_kernel<FitT, QPL>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        void* args[] = {(void*)&d_runs, (void*)&n_runs, (void*)&grid_g, (void*)&d_status};
        return cudaLaunchCooperativeKernel((const void*)fn, dim3(n_runs * grid_g), dim3(kGridThreads), args,
                                           smem, st);
    }
    auto fn = run_kernel<FitT, QPL>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<n_ctas, kThreads, smem, st>>>(d_runs, n_runs, d_queue, d_status);
    return cudaGetLastError();
}

cudaError_t launch_run(const ApoRun* d_runs, int n_runs, int grid_g, int n_ctas, int* d_queue, int* d_status,
                       size_t smem, bool fit64, int qpl, cudaStream_t st)
{
    if (fit64) {
        if (qpl == 1) return launch_run_t<double, 1>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, st);
        return cudaErrorInvalidValue;
    }
    switch (qpl) {
    case 1: return launch_run_t<float, 1>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, st);
    case 2: return launch_run_t<float, 2>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, st);
    case 4: return launch_run_t<float, 4>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

template <typename FitT, int QPL>
static int capacity_t(size_t smem, bool grid)
{
    int per_sm = 0, dev = 0, sms = 0;
    if (grid) {
        auto fn = grid_kernel<FitT, QPL>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGridThreads, smem) != cudaSuccess) return 0;
    } else {
        auto fn = run_kernel<FitT, QPL>;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess) return 0;
    }
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

int run_kernel_capacity(bool fit64, int qpl, size_t smem, bool grid)
{
    if (fit64) return qpl == 1 ? capacity_t<double, 1>(smem, grid) : 0;
    switch (qpl) {
    case 1: return capacity_t<float, 1>(smem, grid);
    case 2: return capacity_t<float, 2>(smem, grid);
    case 4: return capacity_t<float, 4>(smem, grid);
    default: return 0;
    }
}

template <typename FitT, int QPL>
static cudaError_t launch_eval_t(const ApoRun* d_run, int n, const float* d_X, void* d_F, int select,
                                 float* d_Xsel, void* d_Fsel, size_t smem, cudaStream_t st)
{
    auto fn = eval_kernel<FitT, QPL>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (n + kChunk - 1) / kChunk;
    fn<<<grid, kThreads, smem, st>>>(d_run, n, d_X, static_cast<FitT*>(d_F), select, d_Xsel,
                                     static_cast<FitT*>(d_Fsel));
    return cudaGetLastError();
}

cudaError_t launch_eval(const ApoRun* d_run, int n, const float* d_X, void* d_F, int select, float* d_Xsel,
                        void* d_Fsel, size_t smem, bool fit64, int qpl, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    if (fit64) return launch_eval_t<double, 1>(d_run, n, d_X, d_F, select, d_Xsel, d_Fsel, smem, st);
    return launch_eval_t<float, 1>(d_run, n, d_X, d_F, select, d_Xsel, d_Fsel, smem, st);
}

cudaError_t launch_philox(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, int n, uint32_t* d_out,
                          cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const int grid = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    philox_kernel<<<grid, 256, 0, st>>>(d_ctr, k0, k1, n, d_out);
    return cudaGetLastError();
}

}  // namespace apo
