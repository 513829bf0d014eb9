// apo_kernels.cu -- the APO population update on the GPU (cuAPO paper,
// Sec. 3 Eq. 1-13 and Algorithm 1).
//
// One CTA (resident mode) or a group of g cooperating CTAs (grid mode) runs
// the whole device-side iteration loop of one optimisation run:
//   sort (F, previous rank) -> [Dr_index, precomputed by dr_kernel]
//   -> candidate generation, one warp per protozoon (Eq. 1-10, 12-13)
//   -> bound clamp -> evaluation (z = M (x - o) as a three-term fp16 tensor
//      core product per chunk, then the objective epilogue) -> greedy
//      replacement -> barrier.
// In resident mode the population, its fitness and the rotation live in
// shared memory; in grid mode the population lives in global memory (L2) and
// is double buffered so that every candidate reads the start-of-iteration
// snapshot, as the synchronous "parallel for" of Algorithm 1 requires.
#include <cstdio>

#include "apo_device.cuh"
#include "apo_internal.h"
#include "apo_path.cuh"
#include "apo_umma.cuh"

namespace apo {

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
    const unsigned long long psm = magic64((uint32_t)ps);
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
        // the curve value is stored after the greedy step, so that no warp
        // waits for its load
        const bool curve_w = local == 0 && tid == 0 && R.curve != nullptr;
        const FitT curve_v = curve_w ? ldst(Fs[cur] + perm[0], res) : (FitT)0;

        const IterScal is = iter_scal(R, t, psm);
        for (int c0 = r0; c0 < r1; c0 += CH) {
            const int rows = min(CH, r1 - c0);
            for (int row = warp; row < rows; row += nw)
                gen_step_row<FitT, QPL, true, 4>(R, S, Xs[cur], nullptr, Fs[cur], perm, res, true, t, is, c0 + row,
                                        dr_state(R, t, c0 + row), row);
            __syncthreads();
            eval_chunk<FitT>(R, S, rows);
            // Greedy replacement (Algorithm 1): keep X_new iff f(X_new) < f(X_i).
            // Every row goes to the other buffer (the candidate if accepted,
            // the old position otherwise): the kept fitness one thread per
            // row, the rows one 16-byte group per thread.
            for (int row = tid; row < rows; row += blockDim.x) {
                const FitT fo = S.rowF[CH + row], fn = S.rowF[row];
                Fs[cur ^ 1][perm[c0 + row]] = fn < fo ? fn : fo;
            }
            const int g4 = Dp >> 2;
            const uint32_t g4m = div_magic((uint32_t)g4);
            for (int i = tid; i < rows * g4; i += blockDim.x) {
                const int row = (int)div_small((uint32_t)i, g4m), v = i - row * g4;
                const bool acc = S.rowF[row] < S.rowF[CH + row];
                const float4* src = reinterpret_cast<const float4*>((acc ? S.Xc : S.Xo) + (size_t)row * Dp);
                float4* dst = reinterpret_cast<float4*>(Xs[cur ^ 1] + (size_t)perm[c0 + row] * Dp);
                dst[v] = src[v];
            }
            __syncthreads();
        }
        if (curve_w) R.curve[t - 1] = (float)curve_v;
        if (!run_barrier(R.bar, g, bgen, status, s_flag)) return;
        cur ^= 1;
    }

    const uint32_t* perm = S.perm[pc];
    if (R.flags & (kFlagStepOut | kFlagStateOut)) {
        // the state in its current order: the rank order of the last
        // iteration's sort (protozoon order when no iteration ran)
        float* xo = R.X_out;
        FitT* fo = static_cast<FitT*>(R.F_out);
        for (int r = r0 + warp; r < r1; r += nw) {
            const int slot = (int)perm[r];
            for (int d = lane; d < D; d += 32) xo[(size_t)r * D + d] = ldst(Xs[cur] + (size_t)slot * Dp + d, res);
            if (lane == 0) fo[r] = ldst(Fs[cur] + slot, res);
        }
    }
    if (!(R.flags & kFlagStepOut) && local == 0) {
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
// local, local + g, local + 2 g, ... of every iteration and keeps a full copy
// of the rank -> slot permutation in shared memory.  Per iteration:
//   R1  sort the keys (F, previous rank) of the own positions and publish
//       them as a sorted segment of keys_g;                       barrier A
//   R2  the new rank of each own key = its position among the own keys plus
//       the number of other segments' keys below it (the stable sort of
//       Algorithm 1, distributed).  Every other key is located among the
//       own sorted keys (eight keys per thread searched in lockstep) and
//       counted there; a prefix sum of the counts gives the ranks; scatter
//       perm_g[rank] = slot.                                      barrier B
//   R3  copy perm_g (its head is the best of the population, the curve
//       value), then generate, evaluate and replace the own positions.
//       Each slot's current row lives in one of two buffers, named by the
//       top bit of its perm entry; an accepted candidate is written to the
//       other buffer, so the iteration's readers keep seeing the snapshot
//       and rejected rows are never copied.  One more R1/R2 after the last
//       iteration ranks the final population for the best.
// Each grid barrier is an arrival and a wait; work no other CTA reads before
// the next barrier (the last chunk's greedy writes, R2's zeroed counts, the
// next iteration's dormancy inputs) goes between the two.
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

// Numbers of keys of the sorted shared-memory segment seg[0, len) below each
// of NK keys: a descent in power-of-two steps
// (p += step while seg[p + step - 1] < k; p is then the number of keys below
// k, since len < 2 P), with the same steps for every key, so that their
// shared-memory loads overlap instead of running one search after another.
template <typename FitT, int NK>
__device__ __forceinline__ void lower_bound_keys(const typename KeyOf<FitT>::T* seg, int len,
                                                 const typename KeyOf<FitT>::T (&k)[NK], int (&p)[NK])
{
    using KT = typename KeyOf<FitT>::T;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(seg);
#pragma unroll
    for (int u = 0; u < NK; ++u) p[u] = 0;
    if (len <= 0) return;
    int P = 1;
    while (2 * P <= len) P <<= 1;
    for (int step = P; step > 0; step >>= 1) {
#pragma unroll
        for (int u = 0; u < NK; ++u) {
            const int q = p[u] + step;
            const KT v = lds_key(base + (uint32_t)((min(q, len) - 1) * (int)sizeof(KT)), (KT*)nullptr);
            if (q <= len && KeyOf<FitT>::less(v, k[u])) p[u] = q;
        }
    }
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

// Inclusive prefix sums of a[0, n) in place, called by all threads of the
// CTA.  Up to 32 x 16 elements are scanned by warp 0 alone: each lane sums a
// contiguous run of at most 16, one shuffle scan over the 32 run totals gives
// each run its offset, and a single CTA barrier publishes the result.
// Longer arrays: each warp scans a contiguous range, offset by the totals of
// the warps before it (wsum: one int per warp).
__device__ __forceinline__ void block_scan_inclusive(int* a, int n, int* wsum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (n <= 32 * 16) {
        if (warp == 0) {
            const int per = (n + 31) >> 5;
            const int b = min(n, lane * per), e = min(n, b + per);
            int tot = 0;
            for (int i = b; i < e; ++i) tot += a[i];
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += u;
            }
            int run = incl - tot;
            for (int i = b; i < e; ++i) {
                run += a[i];
                a[i] = run;
            }
        }
        __syncthreads();
        return;
    }
    const int per = (n + nw - 1) / nw;
    const int b = min(n, warp * per), e = min(n, b + per);
    int carry = 0;
    for (int base = b; base < e; base += 32) {
        const int i = base + lane;
        int v = i < e ? a[i] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        v += carry;
        if (i < e) a[i] = v;
        carry = __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) wsum[warp] = carry;
    __syncthreads();
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wsum[w];
    if (off)
        for (int i = b + lane; i < e; i += 32) a[i] += off;
    __syncthreads();
}

template <typename FitT, int QPL>
__device__ __forceinline__ void run_grid(const ApoRun& R, int local, unsigned char* smem, int* status, int* s_flag,
                                         TcState& tcs)
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
    // chunk evaluation: tcgen05 rotation (plan.tc) or the general path; a
    // tensor-core wait that runs out aborts the run (false for every thread)
    auto evaluate = [&](int rows) -> bool {
        if (!L.tc) {
            eval_chunk<FitT>(R, S, rows);
            return true;
        }
        if (eval_chunk_tc<FitT>(R, S, rows, tcs)) return true;
        if (tid == 0) {
            set_status(status, 4 /* APO_ERR_TIMEOUT */);
            atomicExch(&R.bar[2], 1u);
        }
        return false;
    };

    load_constants<FitT>(R, S);
    float* Xs[2] = {R.X[0], R.X[1]};
    FitT* Fs[2] = {static_cast<FitT*>(R.F[0]), static_cast<FitT*>(R.F[1])};
    uint32_t* perm = S.perm[0];
    KT* keys = static_cast<KT*>(S.keys);      // own keys in the current rank order
    KT* keys_g = static_cast<KT*>(R.keys_g);
    // own rank positions: local, local + g, local + 2 g, ... (interleaved, so
    // that every CTA gets the same mix of ranks and modes); their keys take
    // the segment [kb, kb + nown) of keys_g
    const int nown = (ps - local + g - 1) / g;
    const int kb = local * (ps / g) + min(local, ps % g);
    auto pos_of = [&](int m) { return local + g * m; };
    int npad = 1;
    while (npad < nown) npad <<= 1;
    // own keys sorted: a second array when they are ranked by counting (with
    // g >= 2 two padded own ranges fit the ps_pad keys of the plan), else
    // sorted in place
    const bool count_rank = nown <= 2 * NT && g >= 2;
    KT* skeys = count_rank ? keys + npad : keys;
    int* hist = reinterpret_cast<int*>(S.perm[1]);   // [nown]: other keys per own position
    // [nown]: the own positions' dormancy inputs of the iteration, in the
    // words of hist, which are free from barrier B to the next R2
    uint32_t* drs = S.perm[1];
    for (int r = tid; r < ps; r += NT) perm[r] = (uint32_t)r;
    __syncthreads();

    if (R.flags & kFlagInit) {
        for (int c0 = 0; c0 < nown; c0 += CH) {
            const int rows = min(CH, nown - c0);
            for (int row = warp; row < rows; row += nw) gen_init_row<FitT, QPL>(R, S, pos_of(c0 + row), row);
            __syncthreads();
            if (!evaluate(rows)) return;
            for (int row = warp; row < rows; row += nw) {
                const int p = pos_of(c0 + row);
                float* dst = Xs[0] + (size_t)p * Dp;
                for (int d = lane; d < Dp; d += 32) dst[d] = S.Xc[(size_t)row * Dp + d];
                if (lane == 0) Fs[0][p] = S.rowF[row];
            }
            __syncthreads();
        }
    }

    // Greedy writes of the chunk at c0 (rows rows, fitness and rows in Xc):
    // the kept fitness of each row to Fd, and the accepted rows to their
    // slots' other buffers, a row per warp in 16-byte groups.
    auto write_chunk = [&](int c0, int rows, FitT* Fd) {
        for (int row = tid; row < rows; row += NT) {
            const FitT fo = S.rowF[CH + row], fn = S.rowF[row];
            Fd[perm[pos_of(c0 + row)] & kSlotMask] = fn < fo ? fn : fo;
        }
        const int g4 = Dp >> 2;
        for (int row = warp; row < rows; row += nw) {
            if (!(S.rowF[row] < S.rowF[CH + row])) continue;
            const uint32_t e = perm[pos_of(c0 + row)];
            const float4* src = reinterpret_cast<const float4*>(S.Xc + (size_t)row * Dp);
            float4* dst = reinterpret_cast<float4*>(Xs[(e >> 31) ^ 1u] + (size_t)(e & kSlotMask) * Dp);
            for (int v = lane; v < g4; v += 32) dst[v] = src[v];
        }
    };
    int held_c0 = 0, held_rows = 0;   // greedy writes held for barrier A
    FitT* held_F = nullptr;
    int cur = 0;
    bool keys_ready = false;   // the greedy step already wrote the own keys
    const bool step_out = (R.flags & kFlagStepOut) != 0;
    // the state after t_end is written out (apo_step: and the launch ends there)
    const bool state_out = step_out || (R.flags & kFlagStateOut) != 0;
    uint8_t* nloc = S.nloc;    // [nown]: buffer bit of each own slot after the greedy step
    if (state_out && R.t_end < R.t_begin) {
        // no iteration: the state as initialised or given, in slot order
        float* xo = R.X_out;
        FitT* fo = static_cast<FitT*>(R.F_out);
        for (int m = warp; m < nown; m += nw) {
            const int r = pos_of(m);
            for (int d = lane; d < D; d += 32) xo[(size_t)r * D + d] = ldst(Xs[0] + (size_t)r * Dp + d, false);
            if (lane == 0) fo[r] = ldst(Fs[0] + r, false);
        }
    }
    for (int t = R.t_begin;; ++t) {
        // R1: own keys (F, rank in the current order), sorted and published
        if (!keys_ready)
            for (int i = tid; i < nown; i += NT) {
                const uint32_t e = perm[pos_of(i)];
                keys[i] = KO::make(ldst(Fs[cur] + (e & kSlotMask), false), (uint32_t)pos_of(i));
                nloc[i] = (uint8_t)(e >> 31);
            }
        __syncthreads();
        if (count_rank) {
            // rank by counting among the own keys (all distinct): tpk aligned
            // lanes per key, each counting a strided share, summed by shuffles
            int tpk = 1;
            while (tpk < 32 && 2 * tpk * nown <= NT) tpk <<= 1;
            const int sub = lane & (tpk - 1);
            for (int base = 0; base < nown; base += NT / tpk) {
                const int i = base + tid / tpk;
                const KT k = i < nown ? keys[i] : KO::pad();
                int rk = 0;
#pragma unroll 8
                for (int j = sub; j < nown; j += tpk) rk += KO::less(keys[j], k) ? 1 : 0;
                for (int m = 1; m < tpk; m <<= 1) rk += __shfl_xor_sync(0xffffffffu, rk, m);
                if (sub == 0 && i < nown) {
                    keys_g[kb + rk] = k;
                    skeys[rk] = k;
                }
            }
        } else {
            for (int i = tid; i < npad; i += NT)
                if (i >= nown) keys[i] = KO::pad();
            __syncthreads();
            bitonic_sort<KO>(keys, npad);
            for (int i = tid; i < nown; i += NT) keys_g[kb + i] = keys[i];
        }
        run_barrier_arrive(R.bar, g, bgen);
        if (held_rows > 0) {
            write_chunk(held_c0, held_rows, held_F);
            held_rows = 0;
        }
        for (int i = tid; i < nown; i += NT) hist[i] = 0;   // R2's counts (the wait ends synchronised)
        if (!run_barrier_wait(R.bar, g, bgen, status, s_flag)) return;

        // R2: distributed ranking.  An other key y lies above exactly the
        // p = lower_bound(own sorted keys, y) smallest own keys, so own key i
        // has sum_{p <= i} hist[p] other keys below it (keys are distinct).
        for (int j0 = tid; j0 < ps; j0 += 8 * NT) {
            KT y[8];
            bool ok[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {   // eight loads in flight, none behind a branch
                const int j = j0 + u * NT;
                ok[u] = j < ps && (j < kb || j >= kb + nown);
                y[u] = __ldcg(keys_g + min(j, ps - 1));
            }
            int p[8];
            lower_bound_keys<FitT, 8>(skeys, nown, y, p);   // the eight searches in lockstep
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (ok[u] && p[u] < nown) atomicAdd(&hist[p[u]], 1);
        }
        __syncthreads();
        block_scan_inclusive(hist, nown, reinterpret_cast<int*>(S.red));
        for (int i = tid; i < nown; i += NT) {
            const int pos = (int)KO::idx(skeys[i]);   // previous rank, an own position
            R.perm_g[i + hist[i]] = (perm[pos] & kSlotMask) | ((uint32_t)nloc[(pos - local) / g] << 31);
        }
        // the own positions' dormancy inputs of iteration t are fetched
        // while the barrier completes (all at once, so that no row's mode
        // waits on a global load; hist is free after the arrival's sync)
        run_barrier_arrive(R.bar, g, bgen);
        if (t <= R.t_end)
            for (int m = tid; m < nown; m += NT) drs[m] = dr_state(R, t, pos_of(m));
        if (!run_barrier_wait(R.bar, g, bgen, status, s_flag)) return;

        // R3: the new permutation; its head is the best of iteration t - 1.
        copy_cg(perm, R.perm_g, ps);
        __syncthreads();
        // the curve value is loaded here and stored after the greedy step, so
        // that no warp waits for the load
        FitT curve_v = (FitT)0;
        const bool curve_w = local == 0 && tid == 0 && R.curve != nullptr;
        if (local == 0) {
            const uint32_t eb = perm[0];
            const int bslot = (int)(eb & kSlotMask);
            if (curve_w) curve_v = ldst(Fs[cur] + bslot, false);
            if (t > R.t_end) {
                if (tid == 0 && R.best_f) *R.best_f = (double)ldst(Fs[cur] + bslot, false);
                if (R.best_x) {
                    const float* xb = Xs[eb >> 31] + (size_t)bslot * Dp;
                    for (int d = tid; d < D; d += NT) R.best_x[d] = ldst(xb + d, false);
                }
            }
        }
        if (t > R.t_end) {
            if (curve_w) R.curve[t - 1] = (float)curve_v;
            break;
        }

        // the own positions: generate, evaluate, replace
        const IterScal is = iter_scal(R, t, 0ull);
        for (int c0 = 0; c0 < nown; c0 += CH) {
            const int rows = min(CH, nown - c0);
            for (int row = warp; row < rows; row += nw)
                gen_step_row<FitT, QPL, false>(R, S, Xs[0], Xs[1], Fs[cur], perm, false, false, t, is, pos_of(c0 + row),
                                        drs[c0 + row], row);
            __syncthreads();
            if (!evaluate(rows)) return;
            // Greedy replacement (Algorithm 1): keep X_new iff f(X_new) < f(X_i).
            // An accepted row goes to the slot's other buffer (nobody reads it
            // in this iteration) and flips the slot's buffer bit; a rejected
            // one stays where it is.  The kept fitness also forms the own sort
            // key of the next iteration.  One thread per row decides; the
            // accepted rows are copied by the whole CTA, one 16-byte group
            // per thread.
            // The last chunk's fitness and row writes are held until barrier
            // A's arrival (below), so that its release need not wait for them
            // to drain; nothing reads them before barrier B.  The step output
            // reads them in this iteration, so it takes them here.
            const bool hold = c0 + CH >= nown && !(state_out && t == R.t_end);
            for (int row = tid; row < rows; row += NT) {
                const uint32_t e = perm[pos_of(c0 + row)];
                const uint32_t loc = e >> 31;
                const FitT fo = S.rowF[CH + row];
                const FitT fn = S.rowF[row];
                const bool acc = fn < fo;
                keys[c0 + row] = KO::make(acc ? fn : fo, (uint32_t)pos_of(c0 + row));
                nloc[c0 + row] = (uint8_t)(acc ? (loc ^ 1u) : loc);
            }
            if (hold) {
                held_c0 = c0;
                held_rows = rows;
                held_F = Fs[cur ^ 1];
            } else {
                write_chunk(c0, rows, Fs[cur ^ 1]);
            }
            __syncthreads();
        }
        if (curve_w) R.curve[t - 1] = (float)curve_v;
        keys_ready = true;
        cur ^= 1;
        if (state_out && t == R.t_end) {
            float* xo = R.X_out;
            FitT* fo = static_cast<FitT*>(R.F_out);
            for (int m = warp; m < nown; m += nw) {
                const int r = pos_of(m);
                const int slot = (int)(perm[r] & kSlotMask);
                const float* src = Xs[nloc[m]] + (size_t)slot * Dp;
                for (int d = lane; d < D; d += 32) xo[(size_t)r * D + d] = ldst(src + d, false);
                if (lane == 0) fo[r] = ldst(Fs[cur] + slot, false);
            }
            if (step_out) break;   // apo_step: no best, no curve
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
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(8) unsigned long long tc_mbar;
    TcState tcs{0u, 0u, 0u};
    if (R.plan.tc) tc_setup(tcs, &tmem_slot, &tc_mbar);
    run_grid<FitT, QPL>(R, local, smem, status, &s_flag, tcs);
    if (R.plan.tc) tc_teardown(tcs);
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
                                int* d_status, size_t smem, bool cluster, cudaStream_t st)
{
    if (grid_g > 0 && cluster) {
        // cluster per run: the g CTAs of a run form one thread-block cluster,
        // which the hardware co-schedules, so their barriers always complete;
        // runs need not be co-resident with one another, and clusters are
        // scheduled as SMs free up
        auto fn = grid_kernel<FitT, QPL>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(n_runs * grid_g);
        cfg.blockDim = dim3(kGridThreads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)grid_g;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cudaLaunchKernelEx(&cfg, fn, d_runs, n_runs, grid_g, d_status);
    }
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
                       size_t smem, bool fit64, int qpl, cudaStream_t st, bool cluster)
{
    if (fit64) {
        if (qpl == 1)
            return launch_run_t<double, 1>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, cluster, st);
        return cudaErrorInvalidValue;
    }
    switch (qpl) {
    case 1: return launch_run_t<float, 1>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, cluster, st);
    case 2: return launch_run_t<float, 2>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, cluster, st);
    case 4: return launch_run_t<float, 4>(d_runs, n_runs, grid_g, n_ctas, d_queue, d_status, smem, cluster, st);
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

// Barrier self-test: `launched` CTAs each pass `rounds` grid barriers of a
// run that expects `expected` CTAs.  With launched == expected every barrier
// completes; with fewer, the first wait runs out after its limit, sets
// APO_ERR_TIMEOUT and the run's abort flag, and every CTA returns.
__global__ void barrier_test_kernel(unsigned* bar, int expected, int rounds, int* status)
{
    __shared__ int s_flag;
    unsigned gen = 0;
    for (int i = 0; i < rounds; ++i)
        if (!run_barrier(bar, expected, gen, status, &s_flag)) return;
}

cudaError_t launch_barrier_test(unsigned* d_bar, int launched, int expected, int rounds, int* status, cudaStream_t st)
{
    barrier_test_kernel<<<launched, 64, 0, st>>>(d_bar, expected, rounds, status);
    return cudaGetLastError();
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
