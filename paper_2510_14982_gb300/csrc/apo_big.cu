// apo_big.cu -- the APO population update (cuAPO paper, Sec. 3 Eq. 1-13,
// Algorithm 1) for large dimensions, kSmallMaxDim < D <= kBigMaxDim: the
// shapes of the paper's Table 2 (D = 1000, ps 1000 to 10000).
//
// A row no longer fits one warp's registers, and the rotation z = M (x - o)
// of a whole population is a real GEMM (ps x D x D), so every iteration is a
// short sequence of kernels, each shaped for its own work:
//   1. big_sort_kernel    keys (F, previous rank) of 1024-key chunks sorted
//                         in shared memory (bitonic);
//   2. big_rank_kernel    the stable rank of every key: its position in its
//                         own chunk plus the number of smaller keys in every
//                         other chunk (binary searches in shared memory);
//                         the new rank -> slot permutation, the curve;
//   3. big_gen_kernel     one warp per candidate (Eq. 1-10, 12-13, clamp):
//                         the gathered rows staged in shared memory by bulk
//                         copies, a row's mask keys in registers and its
//                         Rand_d words in shared memory, the mask by
//                         k-selection over the warp, the foraging pair sums in
//                         one pass, then the candidate pair by pair; the fp32
//                         row goes to the slot's other population buffer,
//                         y = ysc (x - o) as fp16 hi + lo parts to the GEMM
//                         operand;
//   4. big_gemm_kernel    Z = Y B^T on the tensor cores, persistent (one CTA
//                         per SM over 128 x 128 tiles): the operands staged
//                         by TMA (cp.async.bulk.tensor, 128-byte swizzle) in a
//                         multi-stage mbarrier pipeline, three tcgen05.mma per
//                         K step (y_lo B_hi, y_hi B_lo, y_hi B_hi) into TMEM
//                         accumulators, and the objective's per-row partial
//                         sums computed from TMEM in the epilogue, overlapping
//                         the next tile's MMAs (z never goes to memory);
//   5. big_finalize_kernel  the partial sums combined per row in tile order,
//                         the greedy replacement of Algorithm 1 (a slot's
//                         buffer bit flips when its candidate wins).
// Dormancy / Dr_index (Eq. 11) come from the shared dr_kernel, precomputed for
// every iteration.  The population lives in HBM (ps x D x 4 bytes x 2
// buffers, 80 MB at ps 10000, D 1000); every candidate reads the
// start-of-iteration snapshot, since candidates are written to the other
// buffer and the buffer bits flip only in step 5.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <type_traits>
#include <mutex>
#include <vector>

#include "apo_big.h"
#include "apo_path.cuh"
#include "apo_tma.cuh"

namespace apo {

// ----------------------------------------------------------- constants
constexpr int kBigQPL = kBigMaxDim / 64;   // dimension pairs per lane
// rows per CTA of the row kernels (one warp per row); the generation
// kernel's 166 registers and 4 staged rows per warp then allow three CTAs
// (12 warps) per SM
constexpr int kGenWarps = 4;
constexpr int kGenThreads = 32 * kGenWarps;
constexpr int kBM = 128;                    // GEMM tile rows (candidates)
constexpr int kGemmBN = 128;                // GEMM tile columns (output dimensions)
constexpr int kBK = 64;                     // GEMM K block: 64 fp16 = 128 bytes
constexpr int kSortChunk = 1024;            // keys per sorted chunk
// The GEMM is persistent: one CTA per SM walks its share of the tiles.  Warp
// kEpiWarps (lane 0) issues the TMA loads, warp kEpiWarps + 1 (lane 0) the
// MMAs, and warps 0 .. kEpiWarps - 1 run the epilogue: warp w reads TMEM
// lanes 32 (w mod 4) .. + 31 (its candidate rows) and the column quarter w / 4
// of the tile.  The epilogue hands the accumulator back as soon as it has read
// it, so a tile's objective terms are computed while the next tile's MMAs run.
constexpr int kEpiWarps = 16;
constexpr int kGemmThreads = 32 * (kEpiWarps + 2);
constexpr int kGemmSmem = 192 * 1024;       // operand stages
constexpr int kTileA = kBM * kBK * 2;       // bytes of one A part tile

// ------------------------------------------------------------ kernels
__device__ __forceinline__ const float* big_row(const BigRun& R, uint32_t slot)
{
    return R.X[R.loc[slot]] + (size_t)slot * R.Dp;
}

// Population initialisation (Algorithm 1): X_p = Xmin + U (Xmax - Xmin) from
// the INIT draws, into buffer 0, with its GEMM operand rows (row p).  The
// permutation starts as the identity and every slot's buffer bit as 0.
__global__ void __launch_bounds__(256) big_init_kernel(const BigRun* __restrict__ runs)
{
    const BigRun& R = runs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * kGenWarps + (threadIdx.x >> 5);
    if (p >= R.ps) return;
    const int D = R.D;
    float* x = R.X[0] + (size_t)p * R.Dp;
    uint32_t* yh = reinterpret_cast<uint32_t*>(R.Yh + (size_t)p * R.Kp);
    uint32_t* yl = reinterpret_cast<uint32_t*>(R.Yl + (size_t)p * R.Kp);
    for (int q = lane; 2 * q < D; q += 32) {
        const uint4 w = philox(0u, (uint32_t)p, (uint32_t)q, kSlotInit, R.seed, R.run);
        const int d0 = 2 * q, d1 = min(d0 + 1, D - 1);
        const float lb0 = R.lb[d0], ub0 = R.ub[d0], lb1 = R.lb[d1], ub1 = R.ub[d1];
        const float x0 = fmaf(u01(w.x), ub0 - lb0, lb0);
        const float x1 = d0 + 1 < D ? fmaf(u01(w.z), ub1 - lb1, lb1) : 0.f;
        x[d0] = x0;
        if (d0 + 1 < D) x[d0 + 1] = x1;
        uint32_t h, l;
        split_y(x0, d0 + 1 < D ? x1 : R.o[d1], R.o[d0], R.o[d1], R.ysc, h, l);
        yh[q] = h;
        yl[q] = l;
    }
    if (lane == 0) {
        R.loc[p] = 0;
        R.perm[0][p] = (uint32_t)p;
    }
}

// State given by the caller (row p of X_in / F_in is slot p): buffer bits 0,
// identity permutation at the parity of iteration t_begin - 1, the GEMM
// operand unused until the first candidate.
__global__ void big_state_in_kernel(const BigRun* __restrict__ runs, int t_prev)
{
    const BigRun& R = runs[blockIdx.y];
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < R.ps; p += gridDim.x * blockDim.x) {
        R.loc[p] = 0;
        R.perm[t_prev & 1][p] = (uint32_t)p;
    }
}

// 1. Keys (ord(F), previous rank) of chunk blockIdx.x sorted in shared memory.
__global__ void __launch_bounds__(512) big_sort_kernel(const BigRun* __restrict__ runs, int t)
{
    const BigRun& R = runs[blockIdx.y];
    if ((int)blockIdx.x >= R.nchunk) return;
    __shared__ unsigned long long k[kSortChunk];
    const uint32_t* cur = R.perm[(t + 1) & 1];
    const int base = blockIdx.x * kSortChunk;
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) {
        const int r = base + i;
        k[i] = r < R.ps ? KeyOf<float>::make(R.F[cur[r]], (uint32_t)r) : KeyOf<float>::pad();
    }
    __syncthreads();
    bitonic_sort<KeyOf<float>>(k, kSortChunk);
    for (int i = threadIdx.x; i < kSortChunk; i += blockDim.x) R.keys[base + i] = k[i];
}

// 2. Global rank of each key of chunk blockIdx.x: its position in the chunk
// plus the number of smaller keys in each other chunk (keys are distinct);
// the rank -> slot permutation of iteration t, and the best of iteration
// t - 1 (rank 0) for the curve.
__global__ void __launch_bounds__(1024) big_rank_kernel(const BigRun* __restrict__ runs, int t)
{
    const BigRun& R = runs[blockIdx.y];
    if ((int)blockIdx.x >= R.nchunk) return;
    extern __shared__ __align__(16) unsigned char dyn[];
    unsigned long long* s = reinterpret_cast<unsigned long long*>(dyn);
    const int nk = R.nchunk * kSortChunk;
    for (int i = threadIdx.x; i < nk; i += blockDim.x) s[i] = __ldcg(R.keys + i);
    __syncthreads();
    const int c = blockIdx.x, i = threadIdx.x;
    const unsigned long long key = s[c * kSortChunk + i];
    if (key == KeyOf<float>::pad()) return;
    int rank = i;
    for (int c2 = 0; c2 < R.nchunk; ++c2) {
        if (c2 == c) continue;
        const unsigned long long* seg = s + c2 * kSortChunk;
        int lo = 0;   // number of keys of seg below key
#pragma unroll
        for (int step = kSortChunk / 2; step > 0; step >>= 1)
            if (seg[lo + step - 1] < key) lo += step;
        if (seg[lo] < key) ++lo;   // lo <= kSortChunk - 1 here: the last element
        rank += lo;
    }
    const uint32_t* cur = R.perm[(t + 1) & 1];
    uint32_t* nw = R.perm[t & 1];
    const uint32_t slot = cur[KeyOf<float>::idx(key)];
    nw[rank] = slot;
    if (rank == 0 && R.curve) R.curve[t - 1] = R.F[slot];
}

// 3. One candidate (rank r) per warp: mode (Eq. 12-13), masks (Eq. 3, 5),
// dormancy (Eq. 1), reproduction (Eq. 2), autotrophic (Eq. 6-7) or
// heterotrophic (Eq. 8-10) foraging, the clamp; the same draw contract as the
// fused kernels (counter (t, r, d, slot)).
// The rows a candidate reads (X_i, and X_j and the pair for foraging) are
// staged in the warp's slice of shared memory by bulk copies
// (cp.async.bulk, the TMA's untiled mode) issued before the draws, so that
// up to 16 KB per warp are in flight while the Philox draws and the mask
// selection run (the populations at ps 10000 do not fit L2, and row gathers
// from HBM are latency-bound otherwise).
__global__ void __launch_bounds__(kGenThreads, 3) big_gen_kernel(const BigRun* __restrict__ runs, int t)
{
    extern __shared__ __align__(16) unsigned char gen_dyn[];
    __shared__ __align__(8) unsigned long long row_bar[kGenWarps];
    const BigRun& R = runs[blockIdx.y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r = blockIdx.x * kGenWarps + warp;
    if (r >= R.ps) return;   // warp-uniform; the barrier below is the warp's own
    const uint32_t bar = smem_u32(&row_bar[warp]);
    float* rows_s = reinterpret_cast<float*>(gen_dyn) + (size_t)warp * 4 * R.Dp;   // X_i, X_a, X_b, X_j
    if (lane == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
    }
    __syncwarp();
    const int D = R.D, ps = R.ps, np = R.np;
    const uint32_t seed = R.seed, run = R.run;
    const uint32_t* perm = R.perm[t & 1];
    const uint32_t thr_ah = R.thr_ah[t];
    const float fsc = R.fsc[t], nsc = R.nsc[t];
    const float inv_np = 1.f / (float)np;
    // Dormancy / reproduction input (Dr_index bit and the p_dr threshold, Eq. 11, 13)
    const int W = (ps + 31) >> 5;
    const bool in_dr = ((R.drmask[(size_t)t * W + (r >> 5)] >> (r & 31)) & 1u) != 0u;
    const uint32_t thr_dr = R.thr_dr[r];

    // per-protozoon draws: lane 0 SCAL, lane 1 SCAL2, lane 2 + k PAIR k
    uint32_t jslot = kSlotPair, jd = (uint32_t)(lane - 2);
    if (lane == 0) { jslot = kSlotScal; jd = kAll; }
    if (lane == 1) { jslot = kSlotScal2; jd = kAll; }
    const uint4 jw = philox((uint32_t)t, (uint32_t)r, jd, jslot, seed, run);
    uint4 sc;
    sc.x = __shfl_sync(0xffffffffu, jw.x, 0); sc.y = __shfl_sync(0xffffffffu, jw.y, 0);
    sc.z = __shfl_sync(0xffffffffu, jw.z, 0); sc.w = __shfl_sync(0xffffffffu, jw.w, 0);
    const uint32_t s2x = __shfl_sync(0xffffffffu, jw.x, 1), s2y = __shfl_sync(0xffffffffu, jw.y, 1);
    const uint32_t mm = m24p1(sc.x);
    int mode;
    if (in_dr) mode = mm < thr_dr ? kDormancy : kReproduction;
    else mode = mm < thr_ah ? kAutotrophic : kHeterotrophic;
    const bool forage = mode >= kAutotrophic;

    // rows of the snapshot: X_i, X_j and the first pair
    const bool pol = R.pair_policy != 0;
    const uint32_t na = pol ? (uint32_t)(r + 1) : (uint32_t)ps, nb = pol ? (uint32_t)(ps - r) : (uint32_t)ps;
    const uint32_t ob = pol ? (uint32_t)r : 0u;
    const uint32_t si = perm[r];
    uint32_t sj = si, sa = si, sb = si;
    if (mode == kAutotrophic) {
        sj = perm[idx_draw(s2y, (uint32_t)ps)];
        sa = perm[idx_draw(__shfl_sync(0xffffffffu, jw.x, 2), na)];
        sb = perm[ob + idx_draw(__shfl_sync(0xffffffffu, jw.y, 2), nb)];
    } else if (mode == kHeterotrophic) {
        sa = perm[r - 1 < 0 ? 0 : r - 1];
        sb = perm[r + 1 > ps - 1 ? ps - 1 : r + 1];
    }
    const float w1 = forage ? expf(-fabsf(R.F[sa] / (R.F[sb] + kEps))) : 0.f;
    // the rows the mode reads, by bulk copy into the warp's slice (dormancy reads none)
    const int nrows = mode == kDormancy ? 0 : (mode == kReproduction ? 1 : (mode == kHeterotrophic ? 3 : 4));
    const uint32_t row_bytes = (uint32_t)R.Dp * 4u;
    if (lane == 0 && nrows > 0) {
        const uint32_t slots[4] = {si, sa, sb, sj};
        mbar_expect_tx(bar, row_bytes * (uint32_t)nrows);
        for (int k = 0; k < nrows; ++k)
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                :
                : "r"(smem_u32(rows_s + (size_t)k * R.Dp)), "l"(big_row(R, slots[k])), "r"(row_bytes), "r"(bar)
                : "memory");
    }
    const float2* xi = reinterpret_cast<const float2*>(rows_s);
    const float2* xa = reinterpret_cast<const float2*>(rows_s + R.Dp);
    const float2* xb = reinterpret_cast<const float2*>(rows_s + 2 * R.Dp);
    const float2* xj = reinterpret_cast<const float2*>(rows_s + 3 * R.Dp);

    // per-dimension draws: Rand_d (A) and the mask keys (B) of the whole row
    // The keys stay in registers for the mask selection; Rand_d goes to the
    // warp's fourth row slot (X_j's, which only the autotrophic mode stages,
    // and that mode draws no Rand_d), so that the candidate pass below can
    // be a loop rather than unrolled over the lane's pairs.
    uint32_t B[2 * kBigQPL];
    uint32_t valid = 0;
    uint2* As = reinterpret_cast<uint2*>(rows_s + 3 * R.Dp);
    const bool keep_a = mode != kAutotrophic;
#pragma unroll
    for (int j = 0; j < kBigQPL; ++j) {
        const int q = lane + 32 * j;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (2 * q < D) w = philox((uint32_t)t, (uint32_t)r, (uint32_t)q, kSlotDim, seed, run);
        const bool v0 = 2 * q < D, v1 = 2 * q + 1 < D;
        // slots past D get the key 2^32 - 1, which no threshold counts
        B[2 * j] = v0 ? w.y : 0xFFFFFFFFu;
        B[2 * j + 1] = v1 ? w.w : 0xFFFFFFFFu;
        if (keep_a && v0) As[q] = make_uint2(w.x, w.z);
        valid |= (v0 ? 1u : 0u) << (2 * j);
        valid |= (v1 ? 1u : 0u) << (2 * j + 1);
    }
    // corrections only within one key of k (at 32 keys per lane a correction
    // step costs more than a count: 290 against 297 us per iteration with 2)
    uint32_t mask = 0;
    if (mode == kReproduction) {
        const int k = (int)(((unsigned long long)D * m24p1(s2x) + 0xFFFFFFull) >> 24);
        mask = warp_kselect_interp<kBigQPL, 1>(B, valid, k, D);
    } else if (forage) {
        const int k = (D * (r + 1) + ps - 1) / ps;
        mask = warp_kselect_interp<kBigQPL, 1>(B, valid, k, D);
    }
    const float ff = forage ? u01(sc.y) * fsc : 0.f;
    const float sg = sign_draw(sc.z);
    const float rho = u01(sc.w);
    if (nrows > 0 && !mbar_wait(bar, 0u)) {
        // the copies did not land within the limit: report, and let them land
        // (bounded) before the warp's shared memory is released
        if (lane == 0) set_status(R.status, 4 /* APO_ERR_TIMEOUT */);
        mbar_wait(bar, 0u);
        return;
    }

    float2* xc = reinterpret_cast<float2*>(R.X[R.loc[si] ^ 1u] + (size_t)si * R.Dp);
    uint32_t* yh = reinterpret_cast<uint32_t*>(R.Yh + (size_t)r * R.Kp);
    uint32_t* yl = reinterpret_cast<uint32_t*>(R.Yl + (size_t)r * R.Kp);
    // bounds and shift as pairs (Dp is a multiple of 4; the padding past D is
    // zero, so the operand's padding comes out as ysc (0 - 0) = 0)
    const float2* lb2 = reinterpret_cast<const float2*>(R.lb);
    const float2* ub2 = reinterpret_cast<const float2*>(R.ub);
    const float2* o2 = reinterpret_cast<const float2*>(R.o);
    const float ysc = R.ysc;
    // Eq. 7 / Eq. 10 pair sums of the foraging modes, computed in place of
    // the staged X_b row before the candidate pass: w_1 (X_a - X_b), then
    // the pairs k = 2 .. np (np > 1) added in order, each pair's ranks and
    // weight drawn once per warp.  The candidate pass then reads the sums
    // and stays short (its body is unrolled over the lane's pairs).
    if (forage) {
        float2* acc2 = reinterpret_cast<float2*>(rows_s + 2 * R.Dp);
        for (int q = lane; 2 * q < D; q += 32) {
            const float2 va = xa[q], vb = xb[q];
            acc2[q] = make_float2(w1 * (va.x - vb.x), w1 * (va.y - vb.y));
        }
        for (int k = 2; k <= np; ++k) {
            uint32_t ea, eb;
            if (mode == kAutotrophic) {
                const uint4 pr = philox((uint32_t)t, (uint32_t)r, (uint32_t)(k - 1), kSlotPair, seed, run);
                ea = perm[idx_draw(pr.x, na)];
                eb = perm[ob + idx_draw(pr.y, nb)];
            } else {
                ea = perm[r - k < 0 ? 0 : r - k];
                eb = perm[r + k > ps - 1 ? ps - 1 : r + k];
            }
            const float w2 = expf(-fabsf(R.F[ea] / (R.F[eb] + kEps)));
            const float2* qa = reinterpret_cast<const float2*>(big_row(R, ea));
            const float2* qb = reinterpret_cast<const float2*>(big_row(R, eb));
            for (int q = lane; 2 * q < D; q += 32) {
                const float2 a = __ldcg(qa + q), b = __ldcg(qb + q);
                float2 acc = acc2[q];
                acc.x = fmaf(w2, a.x - b.x, acc.x);
                acc.y = fmaf(w2, a.y - b.y, acc.y);
                acc2[q] = acc;
            }
        }
        __syncwarp();
    }
    // The candidate, one unrolled pass loop per mode (no per-element mode
    // branch); lanes past D skip their pair.
    auto emit = [&](auto mode_c) {
        constexpr int M = decltype(mode_c)::value;
#pragma unroll 1
        for (int j = 0; j < kBigQPL; ++j) {
            const int q = lane + 32 * j;
            if (2 * q >= D) break;
            const float2 lb = __ldg(lb2 + q), ub = __ldg(ub2 + q), o = __ldg(o2 + q);
            const uint2 a = M == kAutotrophic ? make_uint2(0u, 0u) : As[q];
            float2 x;
            if constexpr (M == kDormancy) {
                x.x = fmaf(u01(a.x), ub.x - lb.x, lb.x);                        // Eq. 1
                x.y = fmaf(u01(a.y), ub.y - lb.y, lb.y);
            } else {
                const float2 x0 = xi[q];
                if constexpr (M == kReproduction) {
                    x.x = x0.x + sg * rho * fmaf(u01(a.x), ub.x - lb.x, lb.x);  // Eq. 2
                    x.y = x0.y + sg * rho * fmaf(u01(a.y), ub.y - lb.y, lb.y);
                } else {
                    const float2 acc = xb[q];   // the pair sums
                    if constexpr (M == kAutotrophic) {
                        const float2 vj = xj[q];
                        x.x = x0.x + ff * (vj.x - x0.x + acc.x * inv_np);           // Eq. 6
                        x.y = x0.y + ff * (vj.y - x0.y + acc.y * inv_np);
                    } else {
                        const float nx = (1.f + sg * u01(a.x) * nsc) * x0.x;      // Eq. 9
                        const float ny = (1.f + sg * u01(a.y) * nsc) * x0.y;
                        x.x = x0.x + ff * (nx - x0.x + acc.x * inv_np);              // Eq. 8
                        x.y = x0.y + ff * (ny - x0.y + acc.y * inv_np);
                    }
                }
                x.x = ((mask >> (2 * j)) & 1u) ? x.x : x0.x;                          // Eq. 3, 5
                x.y = ((mask >> (2 * j + 1)) & 1u) ? x.y : x0.y;
            }
            x.x = fminf(fmaxf(x.x, lb.x), ub.x);
            x.y = 2 * q + 1 < D ? fminf(fmaxf(x.y, lb.y), ub.y) : 0.f;
            xc[q] = x;
            uint32_t h, l;
            split_y(x.x, x.y, o.x, o.y, ysc, h, l);
            yh[q] = h;
            yl[q] = l;
        }
    };
    switch (mode) {
    case kDormancy: emit(std::integral_constant<int, kDormancy>{}); break;
    case kReproduction: emit(std::integral_constant<int, kReproduction>{}); break;
    case kAutotrophic: emit(std::integral_constant<int, kAutotrophic>{}); break;
    default: emit(std::integral_constant<int, kHeterotrophic>{}); break;
    }
}

// 4. The rotation GEMM with the objective epilogue.  A tile is candidate
// rows m0 .. m0 + 127 and output dimensions n0 .. n0 + BN - 1 of one run; the
// persistent CTAs walk the tiles (roles and hand-overs below the kernel's
// constants).  The epilogue reads the accumulators back (thread = candidate
// row) and reduces the objective's terms of its columns into per-row partial
// sums.  Every wait has a time limit; on timeout the run's status is set and
// the CTA leaves after its copies landed and its TMEM is freed.
struct BigMaps {
    CUtensorMap yh[kBigMaxRuns], yl[kBigMaxRuns], gh[kBigMaxRuns], gl[kBigMaxRuns];
};

// The tensor cores' fp32 accumulation rounds each MMA's sum relative to the
// accumulator's magnitude, so a long chain of MMAs into one accumulator
// drifts (measured at D 1000: 1.3e-5 relative error in the Rosenbrock form,
// against about 1e-7 for a rounded fp32 sum).  The chain is therefore split:
// the two small correction products (y_lo B_hi, y_hi B_lo) go to their own
// accumulator, and the main products y_hi B_hi to kMainAcc accumulators in
// turn (K block kb to accumulator kb mod kMainAcc); the epilogue adds them in
// fp32.  Each accumulator is BN TMEM columns.
constexpr int kMainAcc = 3;

template <int BN>
struct GemmCfg {
    static constexpr int kTileB = BN * kBK * 2;
    static constexpr int kStage = 2 * kTileA + 2 * kTileB;
    static constexpr int kStages = kGemmSmem / kStage;
    static constexpr uint32_t kIdesc = umma_idesc_f16(kBM, BN);
    static constexpr uint32_t kCols = (uint32_t)(BN * (kMainAcc + 1));   // a power of two (256 or 512)
    static_assert(kStages >= 2, "at least two pipeline stages");
    static_assert((kCols & (kCols - 1)) == 0 && kCols <= 512, "TMEM allocation");
};

// Objective terms of one row's z values z[0..31] at columns n .. n + 31.
// Segment forms: [0, s1) ew z^2, [s1, s2) the Rosenbrock chain (the pair
// (n - 1, n) is added at n, with prev = z_{n-1}), [s2, D) Rastrigin.  HGBat:
// (sum u (u - 1), sum u^2), u = z / 20.  Griewank: (sum y^2, prod cos(y ew)),
// y = 6 z.
struct EpiForm {
    int D, form, s1, s2;
};

template <int W>
__device__ __forceinline__ void epi_terms(const float (&z)[W], int n, const EpiForm& E, const float* __restrict__ ew,
                                          float& s1, float& s2, float& prev, bool& have_prev)
{
#pragma unroll
    for (int i = 0; i < W; ++i) {
        const int c = n + i;
        if (c >= E.D) break;
        const float v = z[i];
        if (E.form == kHGBat) {
            const float u = v * 0.05f;
            s1 = fmaf(u, u, s1 - u);
            s2 = fmaf(u, u, s2);
        } else if (E.form == kGriewank) {
            const float y = 6.f * v;
            s1 = fmaf(y, y, s1);
            s2 *= cospif(y * __ldg(ew + c));   // ew = 1 / (pi sqrt(c + 1))
        } else if (c < E.s1) {
            s1 = fmaf(__ldg(ew + c) * v, v, s1);
        } else if (c < E.s2) {
            if (have_prev && c - 1 >= E.s1) s1 += rosen_term(prev, v);
        } else {
            s1 += rast_term(v);
        }
        prev = v;
        have_prev = true;
    }
}

// Tile t of a launch (N tiles fastest, then M tiles, then runs): run, m0, n0;
// false for tiles outside the run's population or dimension.
struct TileGrid {
    int max_mt, max_nt, BN;
};

__device__ __forceinline__ bool tile_of(int t, const TileGrid& G, const BigRun* runs, int& run, int& m0, int& n0)
{
    const int per_run = G.max_mt * G.max_nt;
    run = t / per_run;
    const int r = t - run * per_run;
    m0 = (r / G.max_nt) * kBM;
    n0 = (r % G.max_nt) * G.BN;
    const BigRun& R = runs[run];
    return m0 < R.ps && n0 < R.D;
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    big_gemm_kernel(const BigRun* __restrict__ runs, const __grid_constant__ BigMaps maps, TileGrid G, int n_tiles)
{
    using Cfg = GemmCfg<BN>;
    extern __shared__ unsigned char gemm_dyn[];
    unsigned char* smem = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(gemm_dyn) + 1023) & ~(uintptr_t)1023);
    __shared__ __align__(8) unsigned long long full_bar[Cfg::kStages], empty_bar[Cfg::kStages];
    __shared__ __align__(8) unsigned long long tfull_bar, tempty_bar, drain_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ float2 s_quart[4][kBM], s_edge[4][kBM];
    __shared__ int s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t sbase = smem_u32(smem);
    auto aborted = [&]() { return *reinterpret_cast<volatile int*>(&s_abort) != 0; };
    auto abort_all = [&](int* status) {
        atomicExch(&s_abort, 1);
        set_status(status, 4 /* APO_ERR_TIMEOUT */);
    };

    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int s = 0; s < Cfg::kStages; ++s) {
            mbar_init(smem_u32(&full_bar[s]), 1);
            mbar_init(smem_u32(&empty_bar[s]), 1);
        }
        mbar_init(smem_u32(&tfull_bar), 1);
        mbar_init(smem_u32(&tempty_bar), kEpiWarps);
        mbar_init(smem_u32(&drain_bar), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" : : : "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :
                     : "r"(smem_u32(&tmem_slot)), "r"(Cfg::kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" : : : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
    const uint32_t tmem = tmem_slot;
    int* status = runs[0].status;

    auto stage_a_hi = [&](int s) { return sbase + (uint32_t)(s * Cfg::kStage); };
    auto stage_a_lo = [&](int s) { return sbase + (uint32_t)(s * Cfg::kStage + kTileA); };
    auto stage_b_hi = [&](int s) { return sbase + (uint32_t)(s * Cfg::kStage + 2 * kTileA); };
    auto stage_b_lo = [&](int s) { return sbase + (uint32_t)(s * Cfg::kStage + 2 * kTileA + Cfg::kTileB); };

    long long issued = 0;   // producer: K blocks whose loads were issued (all tiles)
    if (warp == kEpiWarps) {
        // ---- TMA producer
        if (lane == 0) {
            long long g = 0;
            for (int t = blockIdx.x; t < n_tiles && !aborted(); t += gridDim.x) {
                int run, m0, n0;
                if (!tile_of(t, G, runs, run, m0, n0)) continue;
                const int nk = (runs[run].D + kBK - 1) / kBK;
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % Cfg::kStages);
                    if (g >= Cfg::kStages &&
                        !mbar_wait(smem_u32(&empty_bar[s]), (uint32_t)(((g / Cfg::kStages) - 1) & 1))) {
                        abort_all(status);
                        break;
                    }
                    if (aborted()) break;
                    const uint32_t fb = smem_u32(&full_bar[s]);
                    mbar_expect_tx(fb, (uint32_t)Cfg::kStage);
                    const int k0 = kb * kBK;
                    tma_load_2d(stage_a_hi(s), &maps.yh[run], k0, m0, fb);
                    tma_load_2d(stage_a_lo(s), &maps.yl[run], k0, m0, fb);
                    tma_load_2d(stage_b_hi(s), &maps.gh[run], k0, n0, fb);
                    tma_load_2d(stage_b_lo(s), &maps.gl[run], k0, n0, fb);
                    issued = g + 1;
                }
            }
        }
    } else if (warp == kEpiWarps + 1) {
        // ---- MMA issuer
        if (lane == 0) {
            long long g = 0;
            int it = 0;
            for (int t = blockIdx.x; t < n_tiles && !aborted(); t += gridDim.x) {
                int run, m0, n0;
                if (!tile_of(t, G, runs, run, m0, n0)) continue;
                const int nk = (runs[run].D + kBK - 1) / kBK;
                // the epilogue has read the previous tile's accumulators
                if (it > 0 && !mbar_wait(smem_u32(&tempty_bar), (uint32_t)((it - 1) & 1))) {
                    abort_all(status);
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
                for (int kb = 0; kb < nk; ++kb, ++g) {
                    const int s = (int)(g % Cfg::kStages);
                    if (!mbar_wait(smem_u32(&full_bar[s]), (uint32_t)((g / Cfg::kStages) & 1))) {
                        abort_all(status);
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
                    const uint64_t dah = umma_desc_sw128(stage_a_hi(s)), dal = umma_desc_sw128(stage_a_lo(s));
                    const uint64_t dbh = umma_desc_sw128(stage_b_hi(s)), dbl = umma_desc_sw128(stage_b_lo(s));
                    // accumulators: [0] corrections, [1 + kb mod kMainAcc] main products
                    const uint32_t t_corr = tmem, t_main = tmem + (uint32_t)(BN * (1 + kb % kMainAcc));
                    const bool main_fresh = kb < kMainAcc;
#pragma unroll
                    for (int ks = 0; ks < kBK / 16; ++ks) {
                        // a K step of 16 fp16 = 32 bytes = 2 in the descriptor's address field
                        const uint64_t o = (uint64_t)(2 * ks);
                        umma_f16_ss(t_corr, dal + o, dbh + o, Cfg::kIdesc, (kb > 0 || ks > 0) ? 1u : 0u);
                        umma_f16_ss(t_corr, dah + o, dbl + o, Cfg::kIdesc, 1u);
                        umma_f16_ss(t_main, dah + o, dbh + o, Cfg::kIdesc, (!main_fresh || ks > 0) ? 1u : 0u);
                    }
                    umma_commit(smem_u32(&empty_bar[s]));
                }
                if (aborted()) break;
                umma_commit(smem_u32(&tfull_bar));
                ++it;
            }
            // every MMA issued has completed before the CTA frees TMEM
            umma_commit(smem_u32(&drain_bar));
            mbar_wait(smem_u32(&drain_bar), 0u);
        }
    } else {
        // ---- epilogue: warp w takes candidate rows m0 + 32 (w mod 4) + lane
        // (its TMEM lanes) and the column quarter w / 4 (SW = BN / 4 columns);
        // the quarters of a row are combined in column order through shared
        // memory by the warps of quarter 0
        constexpr int SW = BN / 4;
        const int quarter = warp & 3, split = warp >> 2;
        const int rt = 32 * quarter + lane;
        int it = 0;
        for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
            int run, m0, n0;
            if (!tile_of(t, G, runs, run, m0, n0)) continue;
            const BigRun& R = runs[run];
            const int nk = (R.D + kBK - 1) / kBK;
            // every epilogue warp takes the same decision (a barrier with an
            // AND reduction), so none of them is left waiting at the named
            // barriers below when another gives up
            const bool ok = !aborted() && mbar_wait(smem_u32(&tfull_bar), (uint32_t)(it & 1));
            uint32_t all_ok;
            asm volatile(
                "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.and.pred q, 1, %2, p;\n"
                " selp.u32 %0, 1, 0, q;\n}\n"
                : "=r"(all_ok)
                : "r"(ok ? 1u : 0u), "r"(32 * kEpiWarps)
                : "memory");
            if (!all_ok) {
                if (threadIdx.x == 0) abort_all(status);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" : : : "memory");
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(SW * split);
            const int used = nk < kMainAcc ? nk : kMainAcc;
            // corrections + main accumulators in the order 0, 1, 2 (one
            // buffer in flight at a time keeps the registers within budget)
            uint32_t r0[SW], r1[SW];
            float z[SW];
            tmem_ld_nowait(ta, r0);
            tmem_ld_nowait(ta + (uint32_t)BN, r1);
            tmem_wait(r0, r1);
#pragma unroll
            for (int i = 0; i < SW; ++i) z[i] = __uint_as_float(r0[i]) + __uint_as_float(r1[i]);
            for (int a = 1; a < used; ++a) {
                tmem_ld_nowait(ta + (uint32_t)((a + 1) * BN), r1);
                tmem_wait(r1);
#pragma unroll
                for (int i = 0; i < SW; ++i) z[i] += __uint_as_float(r1[i]);
            }
            // the accumulators are free for the next tile's MMAs
            asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" : : "r"(smem_u32(&tempty_bar)) : "memory");
            ++it;

            const int row = m0 + rt;
            const int c0 = n0 + SW * split;
            const EpiForm E{R.D, R.form, R.s1, R.s2};
            const float zsc = R.zsc;
            float s1 = 0.f, s2 = E.form == kGriewank ? 1.f : 0.f, prev = 0.f;
            bool have_prev = false;
#pragma unroll
            for (int i = 0; i < SW; ++i) z[i] *= zsc;
            const float zfirst = z[0];
            if (c0 < E.D) epi_terms<SW>(z, c0, E, R.ew, s1, s2, prev, have_prev);
            s_quart[split][rt] = make_float2(s1, s2);
            s_edge[split][rt] = make_float2(zfirst, prev);
            asm volatile("bar.sync 1, %0;" : : "r"(32 * kEpiWarps) : "memory");
            if (split == 0 && row < R.ps) {
                // quarters in column order; the Rosenbrock pair (n, n + 1)
                // across a quarter boundary is added here
                float a = s_quart[0][rt].x, b = s_quart[0][rt].y;
                float zl = s_edge[0][rt].y;
                for (int c = 1; c < 4 && n0 + SW * c < E.D; ++c) {
                    const float2 q = s_quart[c][rt];
                    const float2 ed = s_edge[c][rt];
                    a += q.x;
                    if (E.form == kGriewank) b *= q.y;
                    else b += q.y;
                    const int n = n0 + SW * c - 1;
                    if (E.form != kHGBat && E.form != kGriewank && n >= E.s1 && n + 1 < E.s2) a += rosen_term(zl, ed.x);
                    zl = ed.y;
                }
                const size_t o = (size_t)row * R.ntiles + n0 / BN;
                R.part[o] = make_float2(a, b);
                R.zedge[o] = make_float2(s_edge[0][rt].x, zl);   // z at n0 and at the tile's last column
            }
            asm volatile("bar.sync 1, %0;" : : "r"(32 * kEpiWarps) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" : : : "memory");
    __syncthreads();
    // on an abort, the loads already issued must land before the CTA leaves
    if (aborted() && warp == kEpiWarps && lane == 0) {
        for (long long g = issued > Cfg::kStages ? issued - Cfg::kStages : 0; g < issued; ++g)
            mbar_wait(smem_u32(&full_bar[g % Cfg::kStages]), (uint32_t)((g / Cfg::kStages) & 1));
    }
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(tmem), "r"(Cfg::kCols)
                     : "memory");
}

// Objective of row r from its tiles' partial sums, combined in tile order.
__device__ __forceinline__ float big_objective(const BigRun& R, int r)
{
    const float2* P = R.part + (size_t)r * R.ntiles;
    if (R.form == kHGBat) {
        float a = 0.f, c = 0.f;
        for (int i = 0; i < R.ntiles; ++i) { a += P[i].x; c += P[i].y; }
        return hgbat_from_sums(a, c, R.D);
    }
    if (R.form == kGriewank) {
        float s = 0.f, p = 1.f;
        for (int i = 0; i < R.ntiles; ++i) { s += P[i].x; p *= P[i].y; }
        return fmaf(s, 1.f / 4000.f, 1.f - p);
    }
    const float2* Z = R.zedge + (size_t)r * R.ntiles;
    float f = 0.f;
    for (int i = 0; i < R.ntiles; ++i) {
        f += P[i].x;
        // the Rosenbrock pair across the tile boundary (n, n + 1)
        const int n = (i + 1) * R.bn - 1;
        if (i + 1 < R.ntiles && n >= R.s1 && n + 1 < R.s2) f += rosen_term(Z[i].y, Z[i + 1].x);
    }
    return f;
}

// 5. mode 0: initial fitness (row p = slot p); mode 1: the greedy replacement
// of Algorithm 1 for rank r (keep X_new iff f(X_new) < f(X_i)); mode 2:
// evaluation only (F_out[r]).
__global__ void big_finalize_kernel(const BigRun* __restrict__ runs, int t, int mode)
{
    const BigRun& R = runs[blockIdx.y];
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R.ps) return;
    const float f = big_objective(R, r);
    if (mode == 0) {
        R.F[r] = f;
    } else if (mode == 1) {
        const uint32_t slot = R.perm[t & 1][r];
        if (f < R.F[slot]) {
            R.F[slot] = f;
            R.loc[slot] ^= 1u;
        }
    } else {
        R.F_out[r] = f;
    }
}

// The best after the final ranking (rank 0 of the permutation at parity
// t_fin), and the state in the current order of iteration t_state (rank r of
// that permutation to row r).
__global__ void big_out_kernel(const BigRun* __restrict__ runs, int t_fin, int t_state, int best, int state)
{
    const BigRun& R = runs[blockIdx.y];
    const int D = R.D;
    if (best && blockIdx.x == 0) {
        const uint32_t slot = R.perm[t_fin & 1][0];
        if (threadIdx.x == 0 && R.best_f) *R.best_f = (double)R.F[slot];
        if (R.best_x)
            for (int d = threadIdx.x; d < D; d += blockDim.x) R.best_x[d] = big_row(R, slot)[d];
    }
    if (state && R.X_out) {
        const uint32_t* pm = R.perm[t_state & 1];
        for (int r = blockIdx.x; r < R.ps; r += gridDim.x) {
            const uint32_t slot = pm[r];
            const float* src = big_row(R, slot);
            for (int d = threadIdx.x; d < D; d += blockDim.x) R.X_out[(size_t)r * D + d] = src[d];
            if (threadIdx.x == 0) R.F_out[r] = R.F[slot];
        }
    }
}

// Evaluation hook: rows of X_in [ps][D] into the GEMM operand (row r).
__global__ void big_pack_kernel(const BigRun* __restrict__ runs)
{
    const BigRun& R = runs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * kGenWarps + (threadIdx.x >> 5);
    if (r >= R.ps) return;
    const int D = R.D;
    const float* x = R.X_in + (size_t)r * D;
    uint32_t* yh = reinterpret_cast<uint32_t*>(R.Yh + (size_t)r * R.Kp);
    uint32_t* yl = reinterpret_cast<uint32_t*>(R.Yl + (size_t)r * R.Kp);
    for (int q = lane; 2 * q < D; q += 32) {
        const int d0 = 2 * q, d1 = min(d0 + 1, D - 1);
        uint32_t h, l;
        split_y(x[d0], d0 + 1 < D ? x[d1] : R.o[d1], R.o[d0], R.o[d1], R.ysc, h, l);
        yh[q] = h;
        yl[q] = l;
    }
}

// ------------------------------------------------------ host side
namespace {

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encode_fn()
{
    static EncodeFn fn = []() -> EncodeFn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<EncodeFn>(f);
    }();
    return fn;
}

// Tensor map of a row-major fp16 matrix [rows][cols] with row pitch `pitch`
// elements (a multiple of 8), tiles of box_rows x 64 with 128-byte swizzle;
// reads past rows / cols return zeros.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int pitch, int box_rows)
{
    EncodeFn fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_gemm(const BigRun* d_runs, const BigMaps& maps, int n_runs, int max_ps, int max_ntiles,
                        cudaStream_t st)
{
    auto fn = big_gemm_kernel<BN>;
    const int smem = kGemmSmem + 1024;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const TileGrid G{(max_ps + kBM - 1) / kBM, max_ntiles, BN};
    const int n_tiles = G.max_mt * G.max_nt * n_runs;
    // persistent: one CTA per SM (fewer when there are fewer tiles)
    fn<<<std::min(n_tiles, sms), kGemmThreads, smem, st>>>(d_runs, maps, G, n_tiles);
    return cudaGetLastError();
}

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

// Instrumentation: per-stage device time of the large-dimension launches
// (CUDA events around every launch of a stage), when switched on.
std::mutex g_stage_mu;
bool g_stage_on = false;
double g_stage_ms[kBigStages] = {};
long long g_stage_n[kBigStages] = {};

struct StageTimer {
    cudaStream_t st;
    bool on;
    std::vector<cudaEvent_t> ev;
    std::vector<int> stage;
    explicit StageTimer(cudaStream_t s) : st(s)
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        on = g_stage_on;
    }
    // brackets launch() with events when on
    template <typename F>
    cudaError_t run(int k, F launch)
    {
        if (!on) return launch();
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        const cudaError_t e = launch();
        cudaEventRecord(b, st);
        ev.push_back(a);
        ev.push_back(b);
        stage.push_back(k);
        return e;
    }
    ~StageTimer()
    {
        if (!on || ev.empty()) return;
        cudaStreamSynchronize(st);
        std::lock_guard<std::mutex> lk(g_stage_mu);
        for (size_t i = 0; i < stage.size(); ++i) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]) == cudaSuccess) {
                g_stage_ms[stage[i]] += ms;
                g_stage_n[stage[i]] += 1;
            }
        }
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

}  // namespace

void big_stage_timing(int on, double* ms, long long* launches)
{
    std::lock_guard<std::mutex> lk(g_stage_mu);
    for (int k = 0; k < kBigStages; ++k) {
        if (ms) ms[k] = g_stage_ms[k];
        if (launches) launches[k] = g_stage_n[k];
        g_stage_ms[k] = 0.0;
        g_stage_n[k] = 0;
    }
    g_stage_on = on != 0;
}

apo_status big_run_group(const std::vector<BigSpec>& specs, cudaStream_t st, char* err, size_t errlen)
{
    const int n = (int)specs.size();
    if (n == 0) return APO_OK;
    if (n > kBigMaxRuns) { snprintf(err, errlen, "internal: too many runs in one group"); return APO_ERR_INTERNAL; }
    int dev = 0;
    cudaGetDevice(&dev);
    int* status = device_status_word();
    if (!status) { snprintf(err, errlen, "status word allocation failed"); return APO_ERR_OOM; }
    // every run of a group shares t_begin, t_end and flags (the caller groups them)
    const int t_begin = specs[0].t_begin, t_end = specs[0].t_end, flags = specs[0].flags;
    const bool eval_only = (flags & kBigEval) != 0;
    // 128-wide GEMM tiles at every size: the persistent kernel spreads the
    // tiles over the SMs itself, and at N = 64 the MMAs are bound by the
    // operands' shared-memory reads (ps 1000, D 1000: 44 against 54 us)
    constexpr int bn = kGemmBN;
    int max_ps = 1, max_tiles = 1, max_chunk = 1;
    for (const BigSpec& s : specs) max_ps = std::max(max_ps, s.ps);
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) { off = al256(off); const size_t at = off; off += bytes; return at; };
    std::vector<BigRun> runs(n);
    std::vector<ApoRun> drs(n);
    std::vector<int> dr_offs(n + 1, 0);
    struct Offs { size_t x0, x1, loc, F, p0, p1, keys, yh, yl, part, zedge, dr; };
    std::vector<Offs> o(n);
    const size_t o_runs = take(sizeof(BigRun) * n), o_drruns = take(sizeof(ApoRun) * n),
                 o_droffs = take(sizeof(int) * (n + 1));
    for (int k = 0; k < n; ++k) {
        const BigSpec& s = specs[k];
        const int ps = s.ps, D = s.P->D, Dp = s.P->Dp, Kp = s.P->dev.Kp;
        const int rows = (ps + kBM - 1) / kBM * kBM;
        const int ntiles = (D + bn - 1) / bn, nchunk = (ps + kSortChunk - 1) / kSortChunk;
        max_tiles = std::max(max_tiles, ntiles);
        max_chunk = std::max(max_chunk, nchunk);
        const int W = (ps + 31) / 32;
        o[k].x0 = take((size_t)ps * Dp * 4);
        o[k].x1 = eval_only ? 0 : take((size_t)ps * Dp * 4);
        o[k].loc = take((size_t)ps);
        o[k].F = take((size_t)ps * 4);
        o[k].p0 = take((size_t)ps * 4);
        o[k].p1 = take((size_t)ps * 4);
        o[k].keys = take((size_t)nchunk * kSortChunk * 8);
        o[k].yh = take((size_t)rows * Kp * 2);
        o[k].yl = take((size_t)rows * Kp * 2);
        o[k].part = take((size_t)ps * ntiles * 8);
        o[k].zedge = take((size_t)ps * ntiles * 8);
        o[k].dr = take((size_t)(std::max(t_end, 0) + 1) * W * 4);
    }
    void* ws = nullptr;
    if (cudaMallocAsync(&ws, off, st) != cudaSuccess) {
        snprintf(err, errlen, "workspace allocation of %zu bytes failed", off);
        return APO_ERR_OOM;
    }
    unsigned char* b = static_cast<unsigned char*>(ws);
    BigRun* d_runs = reinterpret_cast<BigRun*>(b + o_runs);
    BigMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    apo_status rc = APO_OK;
    int n_work = 0, max_ps_pad = 1;
    for (int k = 0; k < n && rc == APO_OK; ++k) {
        const BigSpec& s = specs[k];
        const DevProblem& P = s.P->dev;
        const DevComp& C = P.comp[0];
        BigRun& R = runs[k];
        std::memset(&R, 0, sizeof(R));
        R.D = P.D; R.Dp = P.Dp; R.Kp = P.Kp; R.form = C.form; R.s1 = C.s1; R.s2 = C.s2;
        R.lb = P.lb; R.ub = P.ub; R.o = C.o; R.ew = C.ew; R.ysc = C.ysc; R.zsc = C.zsc;
        R.ps = s.ps; R.np = s.prm.np; R.pair_policy = s.prm.pair_policy; R.T = s.prm.max_iter;
        R.seed = s.prm.seed; R.run = s.prm.run;
        R.X[0] = reinterpret_cast<float*>(b + o[k].x0);
        R.X[1] = eval_only ? R.X[0] : reinterpret_cast<float*>(b + o[k].x1);
        R.loc = b + o[k].loc;
        R.F = reinterpret_cast<float*>(b + o[k].F);
        R.perm[0] = reinterpret_cast<uint32_t*>(b + o[k].p0);
        R.perm[1] = reinterpret_cast<uint32_t*>(b + o[k].p1);
        R.keys = reinterpret_cast<unsigned long long*>(b + o[k].keys);
        R.nchunk = (s.ps + kSortChunk - 1) / kSortChunk;
        R.Yh = reinterpret_cast<uint16_t*>(b + o[k].yh);
        R.Yl = reinterpret_cast<uint16_t*>(b + o[k].yl);
        R.bn = bn;
        R.ntiles = (P.D + bn - 1) / bn;
        R.part = reinterpret_cast<float2*>(b + o[k].part);
        R.zedge = reinterpret_cast<float2*>(b + o[k].zedge);
        R.drmask = reinterpret_cast<const uint32_t*>(b + o[k].dr);
        R.curve = s.curve; R.best_x = s.best_x; R.best_f = s.best_f;
        R.X_in = s.X_in; R.X_out = s.X_out; R.F_out = s.F_out;
        R.status = status;
        if (!eval_only) {
            rc = sched_tables(s.ps, s.prm.pdr_form, s.prm.max_iter, &R.thr_dr, &R.thr_ah, &R.fsc, &R.nsc);
            ApoRun& A = drs[k];
            std::memset(&A, 0, sizeof(A));
            A.ps = s.ps; A.pf_max = s.prm.pf_max; A.seed = s.prm.seed; A.run = s.prm.run;
            A.t_begin = t_begin; A.t_end = t_end; A.drmask = R.drmask;
            dr_offs[k] = n_work;
            n_work += std::max(0, t_end - t_begin + 1);
            int pp = 1;
            while (pp < s.ps) pp <<= 1;
            max_ps_pad = std::max(max_ps_pad, pp);
        }
        // rows past ps and columns past D read as zeros
        if (!make_map(&maps.yh[k], R.Yh, s.ps, P.D, P.Kp, kBM) || !make_map(&maps.yl[k], R.Yl, s.ps, P.D, P.Kp, kBM) ||
            !make_map(&maps.gh[k], C.Gh, P.D, P.D, P.Kp, bn) || !make_map(&maps.gl[k], C.Gl, P.D, P.D, P.Kp, bn)) {
            snprintf(err, errlen, "cuTensorMapEncodeTiled failed");
            rc = APO_ERR_CUDA;
        }
    }
    dr_offs[n] = n_work;
    cudaError_t e = cudaSuccess;
    if (rc == APO_OK) e = cudaMemcpyAsync(d_runs, runs.data(), sizeof(BigRun) * n, cudaMemcpyHostToDevice, st);
    if (rc == APO_OK && e == cudaSuccess && n_work > 0) {
        e = cudaMemcpyAsync(b + o_drruns, drs.data(), sizeof(ApoRun) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b + o_droffs, dr_offs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = launch_dr(reinterpret_cast<const ApoRun*>(b + o_drruns), reinterpret_cast<const int*>(b + o_droffs),
                          n, n_work, max_ps_pad, st);
    }
    const dim3 g_rows((max_ps + kGenWarps - 1) / kGenWarps, n);
    const dim3 g_fin((max_ps + 255) / 256, n);
    const dim3 g_sort(max_chunk, n);
    const size_t rank_smem = (size_t)max_chunk * kSortChunk * 8;
    if (e == cudaSuccess && rank_smem > 48 * 1024)
        e = cudaFuncSetAttribute(big_rank_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rank_smem);
    // generation: four rows of Dp floats per warp
    int max_dp = 4;
    for (const BigRun& R : runs) max_dp = std::max(max_dp, R.Dp);
    const size_t gen_smem = (size_t)kGenWarps * 4 * max_dp * 4;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(big_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gen_smem);
    StageTimer timer(st);
    auto gemm = [&]() -> cudaError_t {
        return timer.run(kStageGemm, [&] {
            return launch_gemm<kGemmBN>(d_runs, maps, n, max_ps, max_tiles, st);
        });
    };
    auto rank = [&](int t) -> cudaError_t {
        return timer.run(kStageRank, [&] {
            big_sort_kernel<<<g_sort, 512, 0, st>>>(d_runs, t);
            big_rank_kernel<<<g_sort, kSortChunk, rank_smem, st>>>(d_runs, t);
            return cudaGetLastError();
        });
    };
    if (rc == APO_OK && e == cudaSuccess) {
        if (eval_only) {
            big_pack_kernel<<<g_rows, kGenThreads, 0, st>>>(d_runs);
            e = cudaGetLastError();
            if (e == cudaSuccess) e = gemm();
            if (e == cudaSuccess) {
                big_finalize_kernel<<<g_fin, 256, 0, st>>>(d_runs, 0, 2);
                e = cudaGetLastError();
            }
        } else {
            const bool timed = big_timing_before() && big_timing_after() &&
                               !(flags & (kBigStepOut | kBigStateOut)) && (flags & kBigInit);
            if (timed) cudaEventRecord(big_timing_before(), st);
            if (flags & kBigInit) {
                big_init_kernel<<<g_rows, kGenThreads, 0, st>>>(d_runs);
                e = cudaGetLastError();
                if (e == cudaSuccess) e = gemm();
                if (e == cudaSuccess) {
                    big_finalize_kernel<<<g_fin, 256, 0, st>>>(d_runs, 0, 0);
                    e = cudaGetLastError();
                }
            } else {
                // the caller's state: slot p = row p
                for (int k = 0; k < n && e == cudaSuccess; ++k) {
                    const BigSpec& s = specs[k];
                    e = cudaMemcpy2DAsync(runs[k].X[0], (size_t)s.P->Dp * 4, s.X_in, (size_t)s.P->D * 4,
                                          (size_t)s.P->D * 4, s.ps, cudaMemcpyDeviceToDevice, st);
                    if (e == cudaSuccess)
                        e = cudaMemcpyAsync(runs[k].F, s.F_in, (size_t)s.ps * 4, cudaMemcpyDeviceToDevice, st);
                }
                if (e == cudaSuccess) {
                    big_state_in_kernel<<<g_fin, 256, 0, st>>>(d_runs, t_begin - 1);
                    e = cudaGetLastError();
                }
            }
            for (int t = t_begin; t <= t_end && e == cudaSuccess; ++t) {
                e = rank(t);
                if (e == cudaSuccess)
                    e = timer.run(kStageGen, [&] {
                        big_gen_kernel<<<g_rows, kGenThreads, gen_smem, st>>>(d_runs, t);
                        return cudaGetLastError();
                    });
                if (e == cudaSuccess) e = gemm();
                if (e == cudaSuccess)
                    e = timer.run(kStageFinal, [&] {
                        big_finalize_kernel<<<g_fin, 256, 0, st>>>(d_runs, t, 1);
                        return cudaGetLastError();
                    });
            }
            const bool step_out = (flags & kBigStepOut) != 0;
            if (e == cudaSuccess && !step_out) e = rank(t_end + 1);   // the final ranking: curve[t_end], best
            if (e == cudaSuccess) {
                const int state = (flags & (kBigStepOut | kBigStateOut)) != 0;
                big_out_kernel<<<dim3(state ? std::min(max_ps, 1024) : 1, n), 256, 0, st>>>(
                    d_runs, t_end + 1, t_end, step_out ? 0 : 1, state);
                e = cudaGetLastError();
            }
            if (timed) cudaEventRecord(big_timing_after(), st);
        }
    }
    if (e != cudaSuccess && rc == APO_OK) {
        snprintf(err, errlen, "large-dimension launch failed: %s", cudaGetErrorString(e));
        rc = APO_ERR_CUDA;
    }
    cudaFreeAsync(ws, st);
    return rc;
}

}  // namespace apo
