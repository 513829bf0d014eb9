// apo_path.cuh -- per-CTA building blocks of the APO update shared by the
// fused iteration-loop kernels and the surrogate-assisted form: the shared
// memory carve-up, constant loading, candidate generation (Eq. 1-13), the
// rotation GEMM, the objective epilogues and the evaluation of a chunk.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "apo_device.cuh"

namespace apo {

constexpr float kEps = 2.220446049250313e-16f;  // eps of Eq. 7 and Eq. 10 (2^-52)

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
    uint8_t* nloc;
    unsigned char *TA, *TY;   // tcgen05 rotation operands (plan.tc)
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
    S.nloc = reinterpret_cast<uint8_t*>(base + L.nloc);
    S.Yc = reinterpret_cast<float*>(base + L.Yc);
    S.Zc = reinterpret_cast<float*>(base + L.Zc);
    S.rowF = reinterpret_cast<FitT*>(base + L.rowF);
    S.compG = reinterpret_cast<float*>(base + L.compG);
    S.compA = reinterpret_cast<float*>(base + L.compA);
    S.P0 = reinterpret_cast<long long*>(base + L.P0);
    S.P1 = reinterpret_cast<long long*>(base + L.P1);
    S.otsu = reinterpret_cast<int*>(base + L.otsu);
    S.red = base + L.red;
    S.TA = base + L.TA;
    S.TY = base + L.TY;
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
    if (R.plan.mt_smem && C.Bh) {
        // split rotation: Bh then Bl, Np * bws words each (multiples of 4)
        const int n4 = P.Np * P.bws / 4;
        const uint4* sh = reinterpret_cast<const uint4*>(C.Bh);
        const uint4* sl = reinterpret_cast<const uint4*>(C.Bl);
        uint4* dst = reinterpret_cast<uint4*>(S.MT);
        for (int i = threadIdx.x; i < n4; i += blockDim.x) {
            dst[i] = sh[i];
            dst[n4 + i] = sl[i];
        }
    }
    if (R.plan.tc) {
        // canonical-layout rotation parts: Th then Tl, Np * Np halves each
        const int n16 = P.Np * P.Np / 8;
        uint4* dst = reinterpret_cast<uint4*>(S.TA);
        for (int i = threadIdx.x; i < n16; i += blockDim.x) {
            dst[i] = C.Th[i];
            dst[n16 + i] = C.Tl[i];
        }
    }
    if (P.kind == kOtsu) {
        for (int i = threadIdx.x; i < 256; i += blockDim.x) {
            S.P0[i] = P.P0[i];
            S.P1[i] = P.P1[i];
        }
    }
}

// ------------------------------------------------------------ evaluation
// ------------------------------------------------ tensor-core rotation
// (a, b) -> fp16 pairs hi = round(a, b), lo = round((a, b) - hi); hi + lo
// carries 22 significant bits.  The lower half holds a.
__device__ __forceinline__ void split_f16x2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    const __half2 h = __floats2half2_rn(a, b);
    const float2 f = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// c += a b for one m16n8k16 tile (fp16 inputs, fp32 accumulation).
__device__ __forceinline__ void mma_f16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

template <bool SHARED>
__device__ __forceinline__ uint2 ldb2(const uint32_t* p)
{
    return SHARED ? *reinterpret_cast<const uint2*>(p) : __ldg(reinterpret_cast<const uint2*>(p));
}

// y = ysc (x - o) for the k pair (x0, x1) of one candidate row, split into
// the fp16 hi and lo words of the tensor-core A operand.
__device__ __forceinline__ void split_y(float x0, float x1, float o0, float o1, float ysc, uint32_t& hi,
                                        uint32_t& lo)
{
    split_f16x2((x0 - o0) * ysc, (x1 - o1) * ysc, hi, lo);
}

// Z[rows][Np] = (Xc - o)[rows][D] * MT[D][Np] on the tensor cores with a
// three-term fp16 split: with y = ysc (x - o) = y_hi + y_lo and
// B = msc MT = B_hi + B_lo (each part an fp16 value, hi + lo exact to 22
// bits), Z = zsc (y_lo B_hi + y_hi B_lo + y_hi B_hi) accumulated in fp32.
// The dropped y_lo B_lo is below 2^-22 of a product; the power-of-two
// scales keep every part inside the fp16 range and are undone exactly.
// A warp takes a 16-row x 32-column tile (four n8 tiles of mma.m16n8k16);
// its A fragments are split here from the row-major candidate rows (Dp apart,
// zero beyond D), its B fragments (one 64-bit load each, pair_word order)
// come from the pre-split rotation (shared memory or, when it does not fit,
// global memory: the same arithmetic).  Rows at or beyond `rows` are computed
// from row rows-1 and discarded.
template <bool B_SHARED>
__device__ __forceinline__ void tile_gemm_f16x3(const float* __restrict__ Xc, int Dp, const float* __restrict__ o,
                                                const uint32_t* __restrict__ Bh, const uint32_t* __restrict__ Bl,
                                                int bws, float ysc, float zsc, float* __restrict__ Z, int Np,
                                                int rows, int D)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    const int mtiles = (rows + 15) >> 4, ngroups = (Np + 31) >> 5, ksteps = (D + 15) >> 4;
    for (int item = warp; item < mtiles * ngroups; item += nw) {
        const int mt = item % mtiles, ng = item / mtiles;
        const int r0 = 16 * mt + g, r1 = r0 + 8;
        const int nb = 32 * ng;
        const int ntn = min(4, (Np - nb) >> 3);
        const float* x0 = Xc + (size_t)min(r0, rows - 1) * Dp;
        const float* x1 = Xc + (size_t)min(r1, rows - 1) * Dp;
        const uint32_t* bh = Bh + (size_t)(nb + g) * bws + 2 * t;
        const uint32_t* bl = Bl + (size_t)(nb + g) * bws + 2 * t;
        float acc[4][4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
        for (int ks = 0; ks < ksteps; ++ks) {
            const int p = 8 * ks;
            // A elements (r, k0), (r, k0 + 1) and (r, k0 + 8), (r, k0 + 9);
            // Dp is a multiple of 4, so a pair is either inside the row or past it
            const int k0 = 16 * ks + 2 * t, k1 = k0 + 8;
            float2 u0 = make_float2(0.f, 0.f), v0 = u0, u1 = u0, v1 = u0, o0 = u0, o1 = u0;
            if (k0 < Dp) {
                o0 = *reinterpret_cast<const float2*>(o + k0);
                u0 = *reinterpret_cast<const float2*>(x0 + k0);
                v0 = *reinterpret_cast<const float2*>(x1 + k0);
            }
            if (k1 < Dp) {
                o1 = *reinterpret_cast<const float2*>(o + k1);
                u1 = *reinterpret_cast<const float2*>(x0 + k1);
                v1 = *reinterpret_cast<const float2*>(x1 + k1);
            }
            uint32_t ah[4], al[4];
            split_y(u0.x, u0.y, o0.x, o0.y, ysc, ah[0], al[0]);
            split_y(v0.x, v0.y, o0.x, o0.y, ysc, ah[1], al[1]);
            split_y(u1.x, u1.y, o1.x, o1.y, ysc, ah[2], al[2]);
            split_y(v1.x, v1.y, o1.x, o1.y, ysc, ah[3], al[3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j < ntn) {
                    const size_t cj = (size_t)(8 * j) * bws + p;
                    const uint2 hb = ldb2<B_SHARED>(bh + cj);
                    const uint2 lb = ldb2<B_SHARED>(bl + cj);
                    mma_f16(acc[j], al, hb.x, hb.y);
                    mma_f16(acc[j], ah, lb.x, lb.y);
                    mma_f16(acc[j], ah, hb.x, hb.y);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (j < ntn) {
                const int c = nb + 8 * j + 2 * t;
                if (r0 < rows)
                    *reinterpret_cast<float2*>(Z + (size_t)r0 * Np + c) = make_float2(acc[j][0] * zsc, acc[j][1] * zsc);
                if (r1 < rows)
                    *reinterpret_cast<float2*>(Z + (size_t)r1 * Np + c) = make_float2(acc[j][2] * zsc, acc[j][3] * zsc);
            }
        }
    }
}

// HGBat of Sec. 5.1 from its per-row sums, with u = z / 20 (y = u - 1):
// (sum y^2)^2 - (sum y)^2 = (sum y^2 + sum y)(sum y^2 - sum y) = a b with
// a = sum u (u - 1) and b = sum (u - 1)(u - 2) = 3 a - 2 c + 2 D, c = sum u^2,
// and (sum y^2 / 2 + sum y) / D + 1/2 = c / (2 D).  The same value as the
// definition, without its cancellation near the optimum.
__device__ __forceinline__ float hgbat_from_sums(float a, float c, int D)
{
    const float b = fmaf(3.f, a, fmaf(-2.f, c, 2.f * (float)D));
    return sqrtf(fabsf(a * b)) + c / (2.f * (float)D);
}

// HGBat or Griewank (the forms that are not sums of per-coordinate terms) of
// one row by one warp (z[d * zs]); Griewank uses y = 6 z and ew[d] = 1 / (pi
// sqrt(d + 1)), so that cos(y / sqrt(d + 1)) = cospi(y ew[d]).
__device__ __forceinline__ float form2_value(const float* z, int zs, const DevComp& C, const float* ew, int D)
{
    const int lane = threadIdx.x & 31;
    if (C.form == kHGBat) {
        float a = 0.f, c = 0.f;
        for (int d = lane; d < D; d += 32) {
            const float u = z[(size_t)d * zs] * 0.05f;
            a = fmaf(u, u, a - u);
            c = fmaf(u, u, c);
        }
        return hgbat_from_sums(warp_sum(a), warp_sum(c), D);
    }
    float s = 0.f, p = 1.f;
    for (int d = lane; d < D; d += 32) {
        const float y = 6.f * z[(size_t)d * zs];
        s = fmaf(y, y, s);
        p *= cospif(y * ew[d]);
    }
    return fmaf(warp_sum(s), 1.f / 4000.f, 1.f - warp_prod(p));
}

// Segmented objective of one row by one warp (z[d * zs]): [0, s1) high-conditioned
// elliptic, [s1, s2) chained Rosenbrock, [s2, D) Rastrigin cosine sum.
__device__ __forceinline__ float seg_value(const float* z, int zs, const DevComp& C, const float* ew, int D)
{
    if (C.form == kHGBat || C.form == kGriewank) return form2_value(z, zs, C, ew, D);
    const int lane = threadIdx.x & 31;
    float s = 0.f;
    for (int d = lane; d < D; d += 32) {
        const float v = z[(size_t)d * zs];
        if (d < C.s1) {
            s = fmaf(ew[d] * v, v, s);
        } else if (d < C.s2) {
            if (d + 1 < C.s2) {
                s += rosen_term(v, z[(size_t)(d + 1) * zs]);
            }
        } else {
            s += rast_term(v);
        }
    }
    return warp_sum(s);
}

// seg_value of NR rows at once (elements contiguous): the same per-lane
// accumulation order and warp sum per row as seg_value, with the rows'
// element work and reductions interleaved.
template <int NR>
__device__ __forceinline__ void seg_values(const float* const (&z)[NR], const DevComp& C, const float* ew, int D,
                                           float (&out)[NR])
{
    if (C.form == kHGBat || C.form == kGriewank) {
#pragma unroll 1
        for (int i = 0; i < NR; ++i) out[i] = form2_value(z[i], 1, C, ew, D);
        return;
    }
    const int lane = threadIdx.x & 31;
    float s[NR];
#pragma unroll
    for (int i = 0; i < NR; ++i) s[i] = 0.f;
    for (int d = lane; d < D; d += 32) {
        if (d < C.s1) {
            const float w = ew[d];
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                const float v = z[i][d];
                s[i] = fmaf(w * v, v, s[i]);
            }
        } else if (d < C.s2) {
            if (d + 1 < C.s2) {
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    s[i] += rosen_term(z[i][d], z[i][d + 1]);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                s[i] += rast_term(z[i][d]);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
#pragma unroll
        for (int i = 0; i < NR; ++i) s[i] += __shfl_xor_sync(0xffffffffu, s[i], off);
#pragma unroll
    for (int i = 0; i < NR; ++i) out[i] = s[i];
}

// Objective of the rows [0, rows) of the Z tile (rows Np apart) into rowF:
// warp w takes rows w, w + nw, ..., w + 7 nw together (one pass for up to
// 8 nw rows).
template <typename FitT>
__device__ __forceinline__ void zrows_to_f(const Smem<FitT>& S, const DevComp& C, int D, int Np, int rows)
{
    constexpr int NR = 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r0 = warp; r0 < rows; r0 += NR * nw) {
        // rows past the last one repeat it (computed, not stored)
        const float* z[NR];
#pragma unroll
        for (int i = 0; i < NR; ++i) z[i] = S.Zc + (size_t)min(r0 + i * nw, rows - 1) * Np;
        float f[NR];
        seg_values<NR>(z, C, S.ew, D, f);
        if (lane == 0)
#pragma unroll
            for (int i = 0; i < NR; ++i)
                if (r0 + i * nw < rows) S.rowF[r0 + i * nw] = (FitT)f[i];
    }
}

// Otsu between-class variance of one row by one warp (thresholds in lanes
// 0..T-1), negated.  The thresholds are sorted by rank counting; lane c then
// fetches the precomputed float64 term of class c (the bin range between
// consecutive distinct thresholds), and lane 0 adds the terms in class order
// with round-to-nearest adds, reproducing the class-by-class sum exactly.
__device__ __forceinline__ double otsu_row(const float* x, int T, const double* __restrict__ tab, int* scratch)
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
    // class c covers (t_{c-1}, t_c] with t_{-1} = -1, t_T = 255; a repeated
    // threshold gives no class
    double term = 0.0;
    bool has = false;
    if (lane <= T) {
        const int hi = lane < T ? scratch[lane] : 255;
        const int prev = lane > 0 ? scratch[lane - 1] : -1;
        if (hi > prev) {
            has = true;
            term = tab[otsu_tab_index(prev + 1, hi)];
        }
    }
    double sigma = 0.0;
    for (int c = 0; c <= T; ++c) {
        const double v = __shfl_sync(0xffffffffu, term, c);
        const bool h = __shfl_sync(0xffffffffu, has, c);
        if (h) sigma = __dadd_rn(sigma, v);
    }
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
            const double f = otsu_row(S.Xc + (size_t)row * Dp, D, P.otsu_tab, S.otsu + warp * 32);
            if (lane == 0) S.rowF[row] = (FitT)f;
        }
        __syncthreads();
        return;
    }
    const int CH = R.plan.chunk, Np = P.Np;
    if (P.ncomp == 1 && P.comp[0].Bh) {
        // one rotated component: tensor-core rotation
        const DevComp& C = P.comp[0];
        if (R.plan.mt_smem) {
            const uint32_t* sb = reinterpret_cast<const uint32_t*>(S.MT);
            tile_gemm_f16x3<true>(S.Xc, Dp, S.o, sb, sb + (size_t)Np * P.bws, P.bws, C.ysc, C.zsc, S.Zc, Np, rows, D);
        } else {
            tile_gemm_f16x3<false>(S.Xc, Dp, S.o, C.Bh, C.Bl, P.bws, C.ysc, C.zsc, S.Zc, Np, rows, D);
        }
        __syncthreads();
        zrows_to_f<FitT>(S, P.comp[0], D, Np, rows);
        __syncthreads();
        return;
    }
    for (int c = 0; c < P.ncomp; ++c) {
        const DevComp& C = P.comp[c];
        const float* o = (c == 0) ? S.o : C.o;
        if (C.Bh) {
            // a rotated component of the composition: tensor-core rotation,
            // its split rotation read from global memory
            tile_gemm_f16x3<false>(S.Xc, Dp, o, C.Bh, C.Bl, P.bws, C.ysc, C.zsc, S.Zc, Np, rows, D);
        } else {
            // no rotation: YT[d][row] = x - o (zero beyond D)
            const uint32_t chm = div_magic((uint32_t)CH);
            for (int i = threadIdx.x; i < CH * Dp; i += blockDim.x) {
                const int d = (int)div_small((uint32_t)i, chm), row = i - d * CH;
                S.Yc[i] = (d < D && row < rows) ? S.Xc[(size_t)row * Dp + d] - o[d] : 0.f;
            }
        }
        __syncthreads();
        const float* ew = (c == 0) ? S.ew : C.ew;
        for (int row = warp; row < rows; row += nw) {
            const float v = C.Bh ? seg_value(S.Zc + (size_t)row * Np, 1, C, ew, D)
                                 : seg_value(S.Yc + row, CH, C, ew, D);
            if (P.ncomp == 1) {
                if (lane == 0) S.rowF[row] = (FitT)v;
            } else {
                float d2 = 0.f;
                for (int d = lane; d < D; d += 32) {
                    const float y = S.Xc[(size_t)row * Dp + d] - o[d];
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
// Dormancy/reproduction input of rank position r at iteration t: bit 31 set
// when r is in Dr_index (Algorithm 1); the low bits hold its p_dr threshold
// ceil(p_dr 2^24) (Eq. 4, below 2^25).  Both loads are unconditional, so
// neither waits behind the other.
__device__ __forceinline__ uint32_t dr_state(const ApoRun& R, int t, int r)
{
    const int W = (R.ps + 31) >> 5;
    const uint32_t word = R.drmask[(size_t)t * W + (r >> 5)];
    const uint32_t thr = R.thr_dr[r];
    return ((word >> (r & 31)) & 1u) ? (0x80000000u | thr) : 0u;
}

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

// The iteration's scalars of Eq. 7, Eq. 9 and Eq. 11-13 (p_ah threshold, the
// foraging factor's scale, the neighbourhood scale and 1 / np), loaded once
// per iteration by the caller rather than once per candidate row.
// psm: the run's reciprocal of ps for the mask sizes of Eq. 5 (magic64),
// computed once per launch (0 where the caller divides).
struct IterScal {
    uint32_t thr_ah;
    float fsc, nsc, inv_np;
    unsigned long long psm;
};
__device__ __forceinline__ IterScal iter_scal(const ApoRun& R, int t, unsigned long long psm)
{
    return IterScal{R.thr_ah[t], R.fsc[t], R.nsc[t], 1.f / (float)R.np, psm};
}

// One candidate (rank r, 0-based) by one warp: mode selection (Eq. 12-13,
// Algorithm 1), masks (Eq. 3, Eq. 5), dormancy (Eq. 1), reproduction
// (Eq. 2), autotrophic (Eq. 6-7) or heterotrophic (Eq. 8-10) foraging, then
// the bound clamp.  Writes row `row` of Xc (candidate) and of Xo (the old
// position, kept for the greedy replacement, when keep_old).  Population rows
// are addressed through perm entries: slot | buffer bit (kLocBit), the bit
// choosing X1 over X where X1 is given (grid mode keeps each slot's current
// row in one of two buffers).  The per-protozoon draws are
// computed once per warp, one Philox call per lane; the gathered rows are
// requested before the per-dimension draws and the mask selection so that
// their latency overlaps that arithmetic.
template <typename FitT, int QPL, bool kMagicK = true, int kAdjust = 2>
__device__ __forceinline__ void gen_step_row(const ApoRun& R, const Smem<FitT>& S, const float* __restrict__ X,
                             const float* __restrict__ X1, const FitT* __restrict__ F, const uint32_t* perm,
                             bool res, bool keep_old, int t, const IterScal& is, int r, uint32_t drs, int row,
                             int cand = 0)
{
    // candidate c of the surrogate-assisted form draws from slots | (c << 8);
    // c = 0 is the plain candidate
    const uint32_t cs = (uint32_t)cand << 8;
    const int lane = threadIdx.x & 31;
    const int D = R.prob.D, Dp = R.prob.Dp, ps = R.ps, np = R.np;
    const uint32_t seed = R.seed, run = R.run;
    const uint32_t thr_ah = is.thr_ah;
    const float fsc = is.fsc, nsc = is.nsc;
    const float inv_np = is.inv_np;
    // Per-protozoon draws, from lanes jb + u: u = 0 SCAL, u = 1 SCAL2,
    // u = 2 + k PAIR k.  The last per-dimension call of a lane covers pairs
    // q = lane + 32 (QPL - 1), of which only q < ceil(D / 2) exist; when at
    // least three lanes are left over there (jb <= 29) the per-protozoon
    // draws take those lanes and the call does both jobs, else they get a
    // call of their own (jb = 0).  Every draw keeps its own counter, so the
    // values do not depend on this placement.
    const int jb_free = max(0, ((D + 1) >> 1) - 32 * (QPL - 1));   // in [0, 32]
    const bool merged = jb_free <= 29;
    const int jb = merged ? jb_free : 0;
    const int u = lane - jb;
    uint32_t jslot = kSlotPair | cs, jd = (uint32_t)(u - 2);
    if (u == 0) { jslot = kSlotScal | cs; jd = kAll; }
    if (u == 1) { jslot = kSlotScal2 | cs; jd = kAll; }
    if (u < 0) { jslot = kSlotDim | cs; jd = (uint32_t)(lane + 32 * (QPL - 1)); }
    const uint4 jw = philox((uint32_t)t, (uint32_t)r, jd, jslot, seed, run);
    uint4 sc, sc2;
    sc.x = __shfl_sync(0xffffffffu, jw.x, jb); sc.y = __shfl_sync(0xffffffffu, jw.y, jb);
    sc.z = __shfl_sync(0xffffffffu, jw.z, jb); sc.w = __shfl_sync(0xffffffffu, jw.w, jb);
    sc2.x = __shfl_sync(0xffffffffu, jw.x, jb + 1); sc2.y = __shfl_sync(0xffffffffu, jw.y, jb + 1);
    const bool in_dr = (drs >> 31) != 0u;
    const uint32_t mm = m24p1(sc.x);
    int mode;
    if (in_dr) mode = (mm < (drs & 0x7FFFFFFFu)) ? kDormancy : kReproduction;
    else mode = (mm < thr_ah) ? kAutotrophic : kHeterotrophic;
    const bool forage = mode == kAutotrophic || mode == kHeterotrophic;

    // rows from the snapshot: X_i, X_j (autotrophic) and the first pair
    auto row_of = [&](uint32_t e) -> const float2* {
        const float* base = (X1 != nullptr && (e & kLocBit)) ? X1 : X;
        return reinterpret_cast<const float2*>(base + (size_t)(e & kSlotMask) * Dp);
    };
    // the candidate rows of both foraging modes are looked up together and
    // selected by the mode (no branch to wait at)
    const uint32_t ei = perm[r];
    const uint32_t p0 = __shfl_sync(0xffffffffu, jw.x, jb + 2), p1 = __shfl_sync(0xffffffffu, jw.y, jb + 2);
    const uint32_t aj = perm[idx_draw(sc2.y, (uint32_t)ps)];
    // the pair ranks of Eq. 6-7: uniform over all ranks (pair policy 0), or
    // k- among the ranks 0..r and k+ among r..ps-1 (pair policy 1)
    const bool pol = R.pair_policy != 0;
    const uint32_t na = pol ? (uint32_t)(r + 1) : (uint32_t)ps, nb = pol ? (uint32_t)(ps - r) : (uint32_t)ps;
    const uint32_t ob = pol ? (uint32_t)r : 0u;
    const uint32_t aa = perm[idx_draw(p0, na)], ab = perm[ob + idx_draw(p1, nb)];
    const uint32_t ha = perm[r - 1 < 0 ? 0 : r - 1], hb = perm[r + 1 > ps - 1 ? ps - 1 : r + 1];
    const bool autot = mode == kAutotrophic, het = mode == kHeterotrophic;
    const uint32_t ej = autot ? aj : ei;
    uint32_t ea = autot ? aa : (het ? ha : ei);   // reassigned per pair when np > 1
    uint32_t eb = autot ? ab : (het ? hb : ei);
    const int si = (int)(ei & kSlotMask), sa = (int)(ea & kSlotMask), sb = (int)(eb & kSlotMask);
    const float2 *pi = row_of(ei), *pj = row_of(ej), *pa = row_of(ea), *pb = row_of(eb);
    // Every lane loads an in-bounds pair of all four rows unconditionally
    // (rows the mode does not use alias X_i, lanes past D repeat the last
    // pair), so no load sits behind a branch whose join would wait for it:
    // the loads stay in flight through the draws and the mask selection
    // below.  Values the mode or the lane does not use are never read.
    const int qmax = ((D + 1) >> 1) - 1;
    float xi[2 * QPL], xj[2 * QPL], xa[2 * QPL], xb[2 * QPL];
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = min(lane + 32 * j, qmax);
        const float2 vi = ldst(pi + q, res), vj = ldst(pj + q, res);
        const float2 va = ldst(pa + q, res), vb = ldst(pb + q, res);
        xi[2 * j] = vi.x; xi[2 * j + 1] = vi.y;
        xj[2 * j] = vj.x; xj[2 * j + 1] = vj.y;
        xa[2 * j] = va.x; xa[2 * j + 1] = va.y;
        xb[2 * j] = vb.x; xb[2 * j + 1] = vb.y;
    }
    const float fa = (float)ldst(F + sa, res), fb = (float)ldst(F + sb, res);
    // old fitness for the greedy step, stored at the end of the row
    const FitT fold = ldst(F + si, res);

    // per-dimension draws and the mask (independent of the gathered rows,
    // overlapping their latency)
    // branch-free, so that the QPL independent Philox chains of a lane
    // interleave (a lane past D computes a draw it then discards)
    uint32_t A[2 * QPL], B[2 * QPL];
    uint32_t valid = 0;
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const int q = lane + 32 * j;
        uint4 w;
        if (j == QPL - 1 && merged) w = jw;   // lanes >= jb hold no pair here (2 q >= D)
        else w = philox((uint32_t)t, (uint32_t)r, (uint32_t)q, kSlotDim | cs, seed, run);
        const bool v0 = 2 * q < D, v1 = 2 * q + 1 < D;
        // slots past D get the key 2^32 - 1, which no threshold counts
        A[2 * j] = v0 ? w.x : 0u; B[2 * j] = v0 ? w.y : 0xFFFFFFFFu;
        A[2 * j + 1] = v0 ? w.z : 0u; B[2 * j + 1] = v1 ? w.w : 0xFFFFFFFFu;
        valid |= (v0 ? 1u : 0u) << (2 * j);
        valid |= (v1 ? 1u : 0u) << (2 * j + 1);
    }
    uint32_t mask = 0;
    if (mode == kReproduction) {
        const int k = (int)(((unsigned long long)D * m24p1(sc2.x) + 0xFFFFFFull) >> 24);
        mask = warp_kselect_interp<QPL, kAdjust>(B, valid, k, D);
    } else if (forage) {
        // ceil(D (r + 1) / ps): by the run's reciprocal, or (kMagicK false:
        // the grid kernel, measured 0.6% faster so) by a division
        const int k = kMagicK ? (int)div_magic64((uint32_t)(D * (r + 1) + ps - 1), is.psm)
                              : (D * (r + 1) + ps - 1) / ps;
        mask = warp_kselect_interp<QPL, kAdjust>(B, valid, k, D);
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
                if (jb + k + 1 < 32) {
                    p0 = __shfl_sync(0xffffffffu, jw.x, jb + k + 1);
                    p1 = __shfl_sync(0xffffffffu, jw.y, jb + k + 1);
                } else {
                    const uint4 pr = philox((uint32_t)t, (uint32_t)r, (uint32_t)(k - 1), kSlotPair | cs, seed, run);
                    p0 = pr.x;
                    p1 = pr.y;
                }
                ea = perm[idx_draw(p0, na)];
                eb = perm[ob + idx_draw(p1, nb)];
            } else {
                ea = perm[r - k < 0 ? 0 : r - k];
                eb = perm[r + k > ps - 1 ? ps - 1 : r + k];
            }
            const float w2 = expf(-fabsf((float)ldst(F + (ea & kSlotMask), res) /
                                         ((float)ldst(F + (eb & kSlotMask), res) + kEps)));
            const float2 *qa = row_of(ea), *qb = row_of(eb);
#pragma unroll
            for (int j = 0; j < QPL; ++j) {
                const int q = lane + 32 * j;
                if (2 * q < D) {
                    const float2 va = ldst(qa + q, res);
                    const float2 vb = ldst(qb + q, res);
                    acc[2 * j] = fmaf(w2, va.x - vb.x, acc[2 * j]);
                    acc[2 * j + 1] = fmaf(w2, va.y - vb.y, acc[2 * j + 1]);
                }
            }
        }
    } else {
#pragma unroll
        for (int e = 0; e < 2 * QPL; ++e) acc[e] = 0.f;
    }
    const float ff = forage ? u01(sc.y) * fsc : 0.f;
    const float s = sign_draw(sc.z);
    const float rho = u01(sc.w);

    float2* xc = reinterpret_cast<float2*>(S.Xc + (size_t)row * Dp);
    float2* xo = reinterpret_cast<float2*>(S.Xo + (size_t)row * Dp);
    // The candidate, one loop per mode (uniform over the warp): the mask bit
    // of a lane is a select, and lanes past D read the bounds of dimension
    // D - 1 and write zeros, so the loop body has no divergent branch.
    auto emit = [&](auto mode_c) {
        constexpr int M = decltype(mode_c)::value;
#pragma unroll
        for (int j = 0; j < QPL; ++j) {
            const int q = lane + 32 * j;
            float out[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int d = 2 * q + e;
                const int sl = 2 * j + e;
                const int dc = d < D ? d : D - 1;
                const float lb = S.lb[dc], ub = S.ub[dc];
                const float x0 = xi[sl];
                float x;
                if constexpr (M == kDormancy) {
                    x = fmaf(u01(A[sl]), ub - lb, lb);                          // Eq. 1
                } else {
                    if constexpr (M == kReproduction) {
                        x = x0 + s * rho * fmaf(u01(A[sl]), ub - lb, lb);       // Eq. 2
                    } else if constexpr (M == kAutotrophic) {
                        x = x0 + ff * (xj[sl] - x0 + acc[sl] * inv_np);         // Eq. 6
                    } else {
                        const float xnear = (1.f + s * u01(A[sl]) * nsc) * x0;  // Eq. 9
                        x = x0 + ff * (xnear - x0 + acc[sl] * inv_np);          // Eq. 8
                    }
                    x = ((mask >> sl) & 1u) ? x : x0;                           // Eq. 3, 5
                }
                out[e] = d < D ? fminf(fmaxf(x, lb), ub) : 0.f;
            }
            // Dp is a multiple of 4, so a pair starting below Dp lies inside
            // the row; the padding past D is written as zeros
            if (2 * q < Dp) {
                xc[q] = make_float2(out[0], out[1]);
                if (keep_old)
                    xo[q] = make_float2(2 * q < D ? xi[2 * j] : 0.f, 2 * q + 1 < D ? xi[2 * j + 1] : 0.f);
            }
        }
    };
    switch (mode) {
    case kDormancy: emit(std::integral_constant<int, kDormancy>{}); break;
    case kReproduction: emit(std::integral_constant<int, kReproduction>{}); break;
    case kAutotrophic: emit(std::integral_constant<int, kAutotrophic>{}); break;
    default: emit(std::integral_constant<int, kHeterotrophic>{}); break;
    }
    if (lane == 0) S.rowF[R.plan.chunk + row] = fold;
}


}  // namespace apo
