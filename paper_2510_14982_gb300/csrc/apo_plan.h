// apo_plan.h -- shared-memory layout of one run (host side), used by every
// launching path so that the layout always matches the device carve().
#pragma once

#include <cmath>
#include <cstddef>
#include <cstring>

#include "apo_internal.h"

namespace apo {

inline size_t plan_align(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Validates the Algorithm 1 inputs of every entry point and resolves the
// evaluation budget: with max_fes > 0 the run takes T = floor(max_fes / ps)
// - 1 whole iterations (ps evaluations at initialisation, ps per iteration)
// and T replaces max_iter, the iter_max of Eq. 4, 9 and 12.  Returns nullptr
// and writes *out, or returns the reason the params are invalid.
inline const char* normalize_params(const apo_params* p, apo_params* out)
{
    if (!p) return "params must not be NULL";
    if (p->ps < 2) return "ps must be >= 2";
    if (p->np < 1 || 2 * p->np >= p->ps) return "np must satisfy 1 <= np and 2 np < ps";
    if (!(p->pf_max >= 0.0 && p->pf_max <= 1.0)) return "pf_max must be in [0, 1]";
    if (p->pdr_form != 0 && p->pdr_form != 1) return "pdr_form must be 0 or 1";
    if (p->pair_policy != 0 && p->pair_policy != 1) return "pair_policy must be 0 or 1";
    if (p->max_fes < 0) return "max_fes must be >= 0";
    apo_params q = *p;
    if (p->max_fes > 0) {
        const long long T = p->max_fes / p->ps - 1;
        if (T < 1) return "max_fes must allow one iteration (max_fes >= 2 ps)";
        if (T > (1 << 30)) return "max_fes allows more than 2^30 iterations";
        q.max_iter = (int)T;
    }
    if (q.max_iter < 1) return "max_iter must be >= 1";
    *out = q;
    return nullptr;
}

// Host images of the schedule tables: Eq. 13 as a 24-bit threshold per rank
// i = 1..ps (form 0 as printed, form 1 mirrored; rank i goes dormant iff
// ((r >> 8) + 1) < ceil(p_dr(i) 2^24)), and per t = 0..T the Eq. 12
// threshold ceil(p_ah(t) 2^24), the Eq. 4 factor 1 + cos(pi t / T) and the
// Eq. 9 factor 1 - t / T.  Any of the outputs may be nullptr.
inline void fill_sched_tables(int ps, int pdr_form, int T, uint32_t* thr_dr, uint32_t* thr_ah, float* fsc,
                              float* nsc)
{
    if (thr_dr)
        for (int i = 1; i <= ps; ++i) {
            const double cv = cos((1.0 - (double)i / (double)ps) * M_PI);
            const double pr = pdr_form == 0 ? 0.5 * (1.0 - cv) : 0.5 * (1.0 + cv);
            thr_dr[i - 1] = (uint32_t)ceil(pr * 16777216.0);
        }
    for (int t = 0; t <= T && (thr_ah || fsc || nsc); ++t) {
        const double cv = cos(((double)t / (double)T) * M_PI);
        if (thr_ah) thr_ah[t] = (uint32_t)ceil(0.5 * (1.0 + cv) * 16777216.0);
        if (fsc) fsc[t] = (float)(1.0 + cv);
        if (nsc) nsc[t] = (float)(1.0 - (double)t / (double)T);
    }
}
inline int plan_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Layout for a run of population ps (0 for the evaluation hooks).  grid
// selects the cooperative-grid layout (512 threads, 64-row chunks, kTcN rows
// with tc); otherwise the resident / work-queue layout (256 threads, 64-row
// chunks).  An explicit chunk overrides the default.
// tc (grid only) places the tcgen05 rotation operands: TA, the rotation's
// fp16 hi and lo parts (Np x Np each, canonical UMMA layout), then directly
// after it TY, the chunk's split candidates (kTcN x Np each).  The MMAs read
// kTcM rotation rows; rows Np..kTcM-1 of the lo part fall into TY (never
// beyond it, since (kTcM - Np) Np 2 <= 4 kTcN Np) and only produce
// accumulator rows that are not read.  A tc plan takes kTcN-row chunks, and
// the Z tile (kTcN x Np fp32, the same bytes as TY) shares TY's space: it is
// written only after the chunk's MMAs have completed.
static_assert(4 * kTcN >= 2 * kTcM, "the rotation rows read past Np must stay inside TY");
inline SmemPlan make_smem_plan(const apo_problem* P, int ps, bool resident, bool mt_smem, bool grid,
                               int chunk = 0, bool tc = false)
{
    const bool fit64 = P->kind == 6;
    const size_t fsz = fit64 ? 8 : 4;
    const int Dp = P->Dp, Np = P->Np;
    SmemPlan L;
    std::memset(&L, 0, sizeof(L));
    L.ps_pad = ps > 0 ? plan_pow2(ps) : 0;
    L.resident = resident;
    L.mt_smem = mt_smem;
    L.chunk = chunk > 0 ? chunk : (grid ? kGridChunk : kQueueChunk);
    L.threads = grid ? kGridThreads : kThreads;
    // rotated components are evaluated on the tensor cores from the row-major
    // candidates; only an unrotated one needs the transposed copy Yc
    bool any_plain = false;
    for (int c = 0; c < P->ncomp; ++c) any_plain = any_plain || P->dev.comp[c].MT == nullptr;
    const size_t ch = (size_t)L.chunk;
    size_t off = 0;
    auto take = [&](size_t bytes) -> uint32_t {
        off = plan_align(off, 16);
        const uint32_t at = (uint32_t)off;
        off += bytes;
        return at;
    };
    L.X0 = take(resident ? (size_t)ps * Dp * 4 : 0);
    L.X1 = take(resident ? (size_t)ps * Dp * 4 : 0);
    L.F0 = take(resident ? ps * fsz : 0);
    L.F1 = take(resident ? ps * fsz : 0);
    L.perm0 = take((size_t)L.ps_pad * 4);
    L.perm1 = take((size_t)L.ps_pad * 4);
    L.keys = take((size_t)L.ps_pad * (fit64 ? 16 : 8));
    L.MT = take(mt_smem ? (size_t)2 * Np * P->dev.bws * 4 : 0);
    L.tc = tc;
    L.TA = take(tc ? (size_t)4 * Np * Np : 0);
    L.TY = take(tc ? (size_t)4 * kTcN * Np : 0);
    L.o = take(Dp * 4);
    L.lb = take(Dp * 4);
    L.ub = take(Dp * 4);
    L.ew = take(Dp * 4);
    L.Xc = take(ch * Dp * 4);
    L.Xo = take(grid ? 0 : ch * Dp * 4);                // grid mode copies no unchanged rows
    L.Yc = take(any_plain ? ch * Dp * 4 : 0);          // transposed: [Dp][chunk]
    L.Zc = tc ? L.TY : take(P->any_rot ? ch * Np * 4 : 0);   // [chunk][Np]
    L.rowF = take(2 * ch * fsz);   // new fitness | old fitness of the chunk rows
    L.compG = take(P->ncomp > 1 ? ch * kMaxComp * 4 : 0);
    L.compA = take(P->ncomp > 1 ? ch * kMaxComp * 4 : 0);
    L.P0 = take(fit64 ? 256 * 8 : 0);
    L.P1 = take(fit64 ? 256 * 8 : 0);
    L.otsu = take(fit64 ? kMaxWarps * 32 * 4 : 0);
    L.red = take((size_t)L.threads * 16);
    L.nloc = take(grid ? (size_t)L.ps_pad : 0);         // buffer bit of each own slot after the greedy step
    L.total = (uint32_t)plan_align(off, 16);
    return L;
}

// The rotation of a single-component objective stays in shared memory when
// the whole layout still fits.
// chunk0 > 0 replaces the mode's chunk (kernels whose grid is one CTA per
// chunk keep small chunks for parallelism).
inline SmemPlan choose_plan(const apo_problem* P, int ps, bool resident, bool grid, size_t smem_max, int chunk0 = 0)
{
    const bool can = P->ncomp == 1 && P->dev.comp[0].MT;
    if (grid && can && P->dev.comp[0].Th) {
        // the grid kernel's rotation on tcgen05
        SmemPlan L = make_smem_plan(P, ps, resident, false, grid, kTcN, true);
        if (L.total <= smem_max) return L;
    }
    // the mode's chunk (64 rows), else 32-row chunks; the rotation in shared
    // memory when that fits too (results do not depend on the layout)
    const int chunks[2] = {chunk0 > 0 ? chunk0 : (grid ? kGridChunk : kQueueChunk), kChunk};
    SmemPlan L{};
    for (int c : chunks) {
        if (can) {
            L = make_smem_plan(P, ps, resident, true, grid, c);
            if (L.total <= smem_max) return L;
        }
        L = make_smem_plan(P, ps, resident, false, grid, c);
        if (L.total <= smem_max) return L;
    }
    return L;   // does not fit: the caller reports it
}

}  // namespace apo
