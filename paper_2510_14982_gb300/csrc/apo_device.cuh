// apo_device.cuh -- device-side building blocks of the APO population update
// (cuAPO paper, Sec. 3 Eq. 1-13, Algorithm 1): the counter-based random
// stream, order-preserving fitness keys, shared-memory bitonic sort, warp
// subset selection (randperm), the grid barrier, and the run descriptor that
// the host fills in.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace apo {

constexpr int kThreads = 256;     // threads per CTA of the work-queue (resident) kernels
constexpr int kWarps = kThreads / 32;
constexpr int kGridThreads = 512; // threads per CTA of the cooperative grid kernel
constexpr int kMaxWarps = kGridThreads / 32;
constexpr int kChunk = 32;        // candidate rows evaluated together when larger chunks do not fit
constexpr int kQueueChunk = 64;   // candidate rows evaluated together (work-queue mode)
constexpr int kGridChunk = 64;    // candidate rows evaluated together (grid mode)
constexpr int kMaxComp = 10;      // composition components
constexpr int kMaxGridCtas = 1024; // CTAs cooperating on one run (grid mode)

// Counter slots of the Philox stream: counter = (iter, p, d, slot).
constexpr uint32_t kSlotInit = 1;   // per (p, dim pair): initial population
constexpr uint32_t kSlotPF = 2;     // global: rand of Eq. 11
constexpr uint32_t kSlotDR = 3;     // per 4 ranks: Dr_index keys
constexpr uint32_t kSlotScal = 4;   // per rank: mode rand, f rand, sign, reproduction rand
constexpr uint32_t kSlotScal2 = 5;  // per rank: M_r count rand, index j
constexpr uint32_t kSlotPair = 6;   // per (rank, pair): k-, k+
constexpr uint32_t kSlotDim = 7;    // per (rank, dim pair): Rand_d, mask key
constexpr uint32_t kAll = 0xFFFFFFFFu;

// Rank -> slot permutation entries of the grid kernel carry, in the top bit,
// which of the two population buffers holds the slot's current row.
constexpr uint32_t kLocBit = 0x80000000u;
constexpr uint32_t kSlotMask = 0x7FFFFFFFu;

enum Mode : int { kDormancy = 0, kReproduction = 1, kAutotrophic = 2, kHeterotrophic = 3 };
enum Kind : int { kSphere = 0, kElliptic = 1, kRosenbrock = 2, kRastrigin = 3, kHybrid = 4,
                  kComposition = 5, kOtsu = 6, kBentCigar = 7, kHGBat = 8, kGriewank = 9 };

// Run flags.
constexpr int kFlagInit = 1;      // initialise the population (t = 0)
constexpr int kFlagStepOut = 2;   // write the rank-ordered state to X_out / F_out (no best, no curve)
constexpr int kFlagStateOut = 4;  // also write the state after t_end (current order) to X_out / F_out

// One shifted-rotated component: z = M (x - o), then a segmented form:
// [0, s1) elliptic with weights ew, [s1, s2) Rosenbrock chain, [s2, D) Rastrigin
// (sphere, elliptic, Bent Cigar, Rosenbrock, Rastrigin and hybrid are all of
// this shape), or, by `form`, HGBat or Griewank (ew = 1 / sqrt(i)).
struct DevComp {
    int form;            // objective kind of the component
    const float* o;      // [Dp]
    const float* MT;     // [Dp][Np] transposed rotation, zero padded; nullptr = identity
    // The rotation for the tensor cores: B[k][n] = MT[k][n] * msc split into
    // fp16 high and low parts (hi + lo = B to 22 bits), stored per column n
    // as bws words of k pairs (the lower half holds the even k) in pair_word
    // order, zero padded.
    const uint32_t* Bh;
    const uint32_t* Bl;
    // The same fp16 parts in the canonical K-major UMMA layout (umma_off,
    // Np rows n x Np columns k each), for the tcgen05 rotation of the grid
    // kernel; only for a single component with D <= kTcM, else nullptr.
    const uint4* Th;
    const uint4* Tl;
    float ysc;           // power of two bringing |x - o| over the box below 2^10
    float zsc;           // 1 / (ysc * msc): z = zsc * (ysc (x - o)) . B
    const float* ew;     // [Dp] elliptic weights of the first segment
    int s1, s2;
    float inv_2Dsig2;    // 1 / (2 D sigma^2) (composition)
    float bias;          // composition bias
    // The large-dimension path (D > kSmallMaxDim): the rotation's fp16 hi and
    // lo parts of B = msc M (hybrid: rows permuted), row n = output dimension,
    // K-contiguous [D][Kp], the B operand of the TMA-fed tcgen05 GEMM.
    const uint16_t* Gh;
    const uint16_t* Gl;
};

// Dimensions up to kSmallMaxDim run in the fused kernels (one warp holds a
// whole row in registers); larger ones, up to kBigMaxDim, in the
// large-dimension path.
constexpr int kSmallMaxDim = 256;
constexpr int kBigMaxDim = 1024;

struct DevProblem {
    int D, Dp, Np, kind, ncomp;  // Dp = D rounded up to 4, Np = D rounded up to 16
    int Kp;              // large-dimension path: D rounded up to 64
    int bws;             // words per column of Bh / Bl: split_words(D)
    const float* lb;     // [Dp]
    const float* ub;     // [Dp]
    DevComp comp[kMaxComp];
    const long long* P0; // Otsu: prefix pixel counts [256]
    const long long* P1; // Otsu: prefix first moments [256]
    const double* otsu_tab;  // Otsu: between-class term of every bin range [a, b]
};

// Word of k pair p (k = 2p, 2p + 1) in a row of fp16-pair words laid out for
// the m16n8k16 fragments: the pairs p and p + 4 of a 16-wide k step (the two
// registers a lane loads) are adjacent, so a fragment is one 64-bit load.
__host__ __device__ __forceinline__ int pair_word(int p)
{
    return 8 * (p >> 3) + 2 * (p & 3) + ((p >> 2) & 1);
}

// Words per column of such pairs: Kp / 2 (Kp = D rounded up to 16) raised to
// 8 mod 16, so that the 64-bit fragment loads of 8 columns x 4 lanes fall on
// distinct banks.
__host__ __device__ __forceinline__ int split_words(int D)
{
    const int h = ((D + 15) & ~15) / 2;
    return (h % 16 == 8) ? h : h + 8;
}

// The tcgen05 rotation of the cooperative grid kernel: UMMA M = kTcM output
// dimensions (the rotation rows, D <= kTcM), N = kTcN candidate rows of a
// chunk (the accumulator's TMEM columns; a CTA of 38 per run at ps 4096 owns
// 108 rows, one chunk).  kTcCols TMEM columns are allocated (a power of two).
constexpr int kTcM = 128;
constexpr int kTcN = 112;
constexpr int kTcCols = 128;

// Byte offset of element (r, k) of a K-major operand with Kt columns (a
// multiple of 16) in the canonical UMMA layout without swizzle: core
// matrices of 8 rows x 16 bytes, K-adjacent ones 128 bytes apart, 8-row
// groups Kt * 16 bytes apart.
__host__ __device__ __forceinline__ uint32_t umma_off(int r, int k, int Kt)
{
    return (uint32_t)((r >> 3) * (Kt * 16) + (k >> 3) * 128 + ((r & 7) << 4) + ((k & 7) << 1));
}

// Packed index of the bin range [a, b] (0 <= a <= b <= 255) in the Otsu term table.
__host__ __device__ __forceinline__ int otsu_tab_index(int a, int b)
{
    return 256 * a - (a * (a - 1)) / 2 + (b - a);
}
constexpr int kOtsuTabSize = 32896;   // 256 * 257 / 2

// Shared-memory carve-up of one run (byte offsets into dynamic shared memory).
struct SmemPlan {
    int ps_pad;          // power of two >= ps
    int resident;        // population lives in shared memory
    int mt_smem;         // rotation of component 0 lives in shared memory
    int tc;              // grid kernel rotation on tcgen05 (operands TA, TY)
    int chunk;           // candidate rows evaluated together
    int threads;         // CTA size the plan was made for
    uint32_t X0, X1, F0, F1, perm0, perm1, keys, MT, o, lb, ub, ew, Xc, Xo, Yc, Zc,
        rowF, compG, compA, P0, P1, otsu, red, nloc, TA, TY, total;
};

struct ApoRun {
    DevProblem prob;
    SmemPlan plan;
    int ps, np, T, pdr_form;
    int pair_policy;     // 0: k-, k+ uniform over all ranks; 1: k- in [0, r], k+ in [r, ps)
    int pad_;
    double pf_max;
    uint32_t seed, run;
    int t_begin, t_end;  // iterations executed by this launch
    int flags;
    int g;               // CTAs cooperating on this run (grid mode)
    const uint32_t* thr_dr;  // [ps]    ceil(p_dr(i) 2^24)
    const uint32_t* thr_ah;  // [T+1]   ceil(p_ah(t) 2^24)
    const float* fsc;        // [T+1]   1 + cos(pi t / T)
    const float* nsc;        // [T+1]   1 - t / T
    const uint32_t* drmask;  // [T+1][ceil(ps/32)] Dr_index bitmask per iteration
    float* X[2];             // [ps][Dp] global state buffers (non-resident / step mode)
    void* F[2];              // [ps] FitT
    float* X_out;            // step mode: [ps][D] rank-ordered output
    void* F_out;
    float* best_x;           // [D]
    double* best_f;          // [1]
    float* curve;            // [T+1] or nullptr
    unsigned* bar;           // grid barrier words {count, generation, abort}
    uint32_t* perm_g;        // grid mode: [ps] rank -> slot of the current iteration
    void* keys_g;            // grid mode: [ps] key segments, each CTA's sorted
};

// ---------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): per round two 32x32
// multiplications, the high halves XORed with the other counter words and
// the round key; the key advances by the Weyl increments between rounds.
__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                        uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return make_uint4(c0, c1, c2, c3);
}

// Draw contract: U = ((r >> 8) + 1) 2^-24 in (0, 1] (exact in binary32),
// index = (r n) >> 32, sign = r & 1 ? -1 : +1.
__device__ __forceinline__ float u01(uint32_t r) { return (float)((r >> 8) + 1u) * 5.9604644775390625e-8f; }
__device__ __forceinline__ uint32_t m24p1(uint32_t r) { return (r >> 8) + 1u; }
__device__ __forceinline__ uint32_t idx_draw(uint32_t r, uint32_t n) { return __umulhi(r, n); }
__device__ __forceinline__ float sign_draw(uint32_t r) { return (r & 1u) ? -1.f : 1.f; }

// cos(2 pi v), the Rastrigin term's cosine.  v is reduced exactly to
// r = |v - rint(v)| in [0, 1/2], then to s in [0, 1/4] by
// cos(2 pi r) = -cos(2 pi (1/2 - r)) for r > 1/4; cos(2 pi s) is the Taylor
// series of the cosine through x^12 at x = 2 pi s <= pi / 2 (coefficients
// (-1)^n (2 pi)^(2n) / (2n)!, truncation below (pi/2)^14 / 14! < 7e-9), so
// the result is within about 2e-7 of the exact value, at a third of the
// instructions of a general cosine.
__host__ __device__ __forceinline__ float cos2pi(float v)
{
    const float r = fabsf(v - rintf(v));
    const bool flip = r > 0.25f;
    const float s = flip ? 0.5f - r : r;
    const float x2 = s * s;
    float p = 7.903536371e+00f;
    p = fmaf(p, x2, -2.642625678e+01f);
    p = fmaf(p, x2, 6.024464137e+01f);
    p = fmaf(p, x2, -8.545681721e+01f);
    p = fmaf(p, x2, 6.493939402e+01f);
    p = fmaf(p, x2, -1.973920880e+01f);
    p = fmaf(p, x2, 1.0f);
    return flip ? -p : p;
}

// The per-coordinate terms of the chained Rosenbrock form (the pair (z_d,
// z_{d+1})) and of the Rastrigin form, with every multiply-add written out,
// so that each kernel that evaluates them (whatever the compiler would fuse
// in its context) rounds them the same way.
__host__ __device__ __forceinline__ float rosen_term(float v, float vn)
{
    const float a = fmaf(-v, v, vn);
    const float b = v - 1.f;
    return fmaf(100.f * a, a, b * b);
}
__host__ __device__ __forceinline__ float rast_term(float v)
{
    return fmaf(v, v, fmaf(-10.f, cos2pi(v), 10.f));
}

// floor(i / d) for 0 <= i < 2^16 and 1 <= d < 2^16 by one multiply-high with
// m = div_magic(d) = floor((2^32 - 1) / d) + 1 (m >= 2^32 / d and the error
// i (m - 2^32 / d) / 2^32 < i / 2^32 < 1 / d cannot reach the next integer),
// for the flat index loops whose row length is only known at run time.  (Host
// versions of the multiply-highs serve the host-side checks.)
__host__ __device__ __forceinline__ uint32_t div_magic(uint32_t d) { return d == 1u ? 0u : 0xFFFFFFFFu / d + 1u; }
__host__ __device__ __forceinline__ uint32_t div_small(uint32_t i, uint32_t m)
{
#ifdef __CUDA_ARCH__
    return m == 0u ? i : __umulhi(i, m);
#else
    return m == 0u ? i : (uint32_t)(((unsigned long long)i * m) >> 32);
#endif
}
// The same for any 32-bit i with a 64-bit m = floor((2^64 - 1) / d) + 1
// (error below i / 2^64 < 1 / d): one 64-bit multiply-high.
__host__ __device__ __forceinline__ unsigned long long magic64(uint32_t d) { return d <= 1u ? 0ull : ~0ull / d + 1ull; }
__host__ __device__ __forceinline__ uint32_t div_magic64(uint32_t i, unsigned long long m)
{
#ifdef __CUDA_ARCH__
    return m == 0ull ? i : (uint32_t)__umul64hi((unsigned long long)i, m);
#else
    return m == 0ull ? i : (uint32_t)(((unsigned __int128)i * m) >> 64);
#endif
}

// ------------------------------------------------------- fitness ordering
__device__ __forceinline__ uint32_t ord_key(float f)
{
    if (f == 0.f) f = 0.f;  // -0 sorts with +0
    const uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ unsigned long long ord_key(double f)
{
    if (f == 0.0) f = 0.0;
    const unsigned long long u = (unsigned long long)__double_as_longlong(f);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// Sort keys: (fitness order, previous rank).  float fitness packs into 64 bits.
template <typename FitT> struct KeyOf;
template <> struct KeyOf<float> {
    using T = unsigned long long;
    __device__ static T make(float f, uint32_t r) { return ((T)ord_key(f) << 32) | r; }
    __device__ static T pad() { return ~0ull; }
    __device__ static uint32_t idx(T k) { return (uint32_t)k; }
    __device__ static bool less(T a, T b) { return a < b; }
};
template <> struct KeyOf<double> {
    using T = ulonglong2;
    __device__ static T make(double f, uint32_t r) { return make_ulonglong2(ord_key(f), r); }
    __device__ static T pad() { return make_ulonglong2(~0ull, ~0ull); }
    __device__ static uint32_t idx(T k) { return (uint32_t)k.y; }
    __device__ static bool less(T a, T b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }
};

// Ascending bitonic sort of n (power of two) keys in shared memory by the
// whole CTA.  Ends with a __syncthreads().
template <typename KO>
__device__ void bitonic_sort(typename KO::T* keys, int n)
{
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < (n >> 1); i += blockDim.x) {
                const int lo = ((i & ~(j - 1)) << 1) | (i & (j - 1));
                const int hi = lo + j;
                const bool up = (lo & k) == 0;
                const typename KO::T a = keys[lo], b = keys[hi];
                if (KO::less(b, a) == up) {
                    keys[lo] = b;
                    keys[hi] = a;
                }
            }
            __syncthreads();
        }
    }
}

// ----------------------------------------------------- warp reductions
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_prod(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v *= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// randperm(D, k) of Eq. 3 / Eq. 5: the k smallest (key, dim) pairs over the
// warp.  Lane L holds dims d = 2 (L + 32 j) + e, j < QPL, e in {0, 1}, at
// slot 2 j + e of `key`; `valid` marks dims < D.  Returns the lane's bitmask
// of selected slots.  Bitwise descent on the key from the top bit, counting
// with warp reductions, stops once the remaining candidates are all taken;
// exact key ties fall back to the lowest dims.
template <int QPL>
__device__ uint32_t warp_kselect(const uint32_t (&key)[2 * QPL], uint32_t valid, int k)
{
    const int lane = threadIdx.x & 31;
    uint32_t cand = valid, sel = 0;
    int kk = k;
    if (kk <= 0) return 0;
    int ncand = __reduce_add_sync(0xffffffffu, __popc(cand));
    if (kk >= ncand) return cand;
    for (int b = 31; b >= 0; --b) {
        uint32_t zero = 0;
#pragma unroll
        for (int e = 0; e < 2 * QPL; ++e)
            if (((cand >> e) & 1u) && !((key[e] >> b) & 1u)) zero |= 1u << e;
        const int c0 = __reduce_add_sync(0xffffffffu, __popc(zero));
        if (kk <= c0) {
            cand = zero;
            ncand = c0;
        } else {
            sel |= zero;
            kk -= c0;
            cand &= ~zero;
            ncand -= c0;
        }
        if (ncand == kk) return sel | cand;
    }
    // cand: equal keys; take the kk lowest dims, ordered by (j, lane, e).
    int before = 0;
#pragma unroll
    for (int j = 0; j < QPL; ++j) {
        const uint32_t b0 = __ballot_sync(0xffffffffu, (cand >> (2 * j)) & 1u);
        const uint32_t b1 = __ballot_sync(0xffffffffu, (cand >> (2 * j + 1)) & 1u);
        const uint32_t lt = (1u << lane) - 1u;
        const int mine0 = before + __popc(b0 & lt) + __popc(b1 & lt);
        if (((cand >> (2 * j)) & 1u) && mine0 < kk) sel |= 1u << (2 * j);
        const int mine1 = mine0 + (int)((cand >> (2 * j)) & 1u);
        if (((cand >> (2 * j + 1)) & 1u) && mine1 < kk) sel |= 1u << (2 * j + 1);
        before += __popc(b0) + __popc(b1);
    }
    return sel;
}

// floor((2^32 - 1) / b) for b = 1 .. 2 (kBigMaxDim + 1): fixed-point
// reciprocals of the interpolation denominators b = 2 (chi - clo + 1) <= 2 (n + 1)
// (slot 0 unused)
constexpr int kRecipSize = 2 * (kBigMaxDim + 1) + 1;
struct RecipTable {
    uint32_t v[kRecipSize];
};
constexpr RecipTable make_recip_table()
{
    RecipTable t{};
    for (int b = 1; b < kRecipSize; ++b) t.v[b] = (uint32_t)(0xFFFFFFFFull / (unsigned long long)b);
    return t;
}
static __constant__ RecipTable kRecip = make_recip_table();

// The same subset as warp_kselect, found by interpolation and finished by
// extremes: a threshold T with exactly k valid keys below it selects the k
// smallest (every key below T is smaller than every key at or above it, so
// index tie-breaks cannot arise).  The keys are uniform 32-bit Philox words,
// so interpolating between the bracketing counts lands within a few keys of
// k at the first count (the count is binomial around k).  Once the count c
// at a threshold is within kAdjust of k, the set below it is corrected by c -
// k warp-wide maximum reductions (each drops the largest selected key) or k -
// c minimum reductions (each adds the smallest unselected key), instead of
// further counts; a final count confirms exactly k keys (equal keys at the
// boundary would give another count and take the exact bitwise descent, as
// does no convergence within ten counts).  n = number of valid slots (<= 1024);
// slots outside `valid` must hold the key 2^32 - 1, which no threshold counts.
// kAdjust = 2: a correction step costs about as much as a count, and counts
// close in faster from farther away (measured: 55.4 ms per scale step at 2,
// 55.9 at 4, 57.8 at 8, 59.0 at 16).
template <int QPL, int kAdjust = 2>
__device__ uint32_t warp_kselect_interp(const uint32_t (&key)[2 * QPL], uint32_t valid, int k, int n)
{
    if (k <= 0) return 0;
    if (k >= n) return valid;
    // invariant: clo = #(keys < lo) < k < chi = #(keys <= hm); thresholds are
    // tried in (lo, hm].  Integer arithmetic only (fixed-point fraction), so
    // the dependent chain of a step stays on the integer pipes.
    uint32_t lo = 0u, hm = 0xFFFFFFFFu;
    int clo = 0, chi = n;
#pragma unroll 1
    for (int it = 0; it < 10 && hm > lo; ++it) {
        // the boundary between the (k-clo)-th and (k-clo+1)-th of the chi-clo
        // keys in the bracket sits near the fraction (k - clo + 1/2) / (chi - clo + 1)
        // = a / b, with a < b, so a * floor((2^32 - 1) / b) < 2^32
        const uint32_t a = 2u * (uint32_t)(k - clo) + 1u, b = 2u * (uint32_t)(chi - clo + 1);
        const uint32_t span = hm - lo;
        uint32_t off = __umulhi(span, a * kRecip.v[b]);
        off = off < 1u ? 1u : (off > span ? span : off);
        const uint32_t T = lo + off;
        uint32_t below = 0;
#pragma unroll
        for (int e = 0; e < 2 * QPL; ++e) below |= (key[e] < T ? 1u : 0u) << e;
        const int c = __reduce_add_sync(0xffffffffu, __popc(below));
        if (c == k) return below;
        if (c - k <= kAdjust && k - c <= kAdjust) {
            uint32_t sel = below;
            if (c > k) {
                // drop the c - k largest selected keys
                for (int i = 0; i < c - k; ++i) {
                    uint32_t m = 0u;
#pragma unroll
                    for (int e = 0; e < 2 * QPL; ++e)
                        if ((sel >> e) & 1u) m = max(m, key[e]);
                    m = __reduce_max_sync(0xffffffffu, m);
#pragma unroll
                    for (int e = 0; e < 2 * QPL; ++e)
                        if (((sel >> e) & 1u) && key[e] == m) sel &= ~(1u << e);
                }
            } else {
                // add the k - c smallest unselected keys
                const uint32_t rest = valid & ~below;
                uint32_t cand = rest;
                for (int i = 0; i < k - c; ++i) {
                    uint32_t m = 0xFFFFFFFFu;
#pragma unroll
                    for (int e = 0; e < 2 * QPL; ++e)
                        if ((cand >> e) & 1u) m = min(m, key[e]);
                    m = __reduce_min_sync(0xffffffffu, m);
#pragma unroll
                    for (int e = 0; e < 2 * QPL; ++e)
                        if (((cand >> e) & 1u) && key[e] == m) cand &= ~(1u << e);
                }
                sel = below | (rest & ~cand);
            }
            if (__reduce_add_sync(0xffffffffu, __popc(sel)) == k) return sel;
            break;   // equal keys at the boundary
        }
        if (c < k) { lo = T; clo = c; }
        else { hm = T - 1u; chi = c; }
    }
    return warp_kselect<QPL>(key, valid, k);
}

// ----------------------------------------------------------- barriers
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Records the first error of the process-wide device status word.
__device__ __forceinline__ void set_status(int* status, int code)
{
    atomicCAS(status, 0, code);
}

constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;  // 4 s per wait

__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Barrier over the g CTAs of one run, in two halves.  bar[0] counts arrivals
// and is never reset: the CTA's n-th barrier (n = ++gen) is passed once the
// count reaches n g.  Arrival: after the CTA-wide __syncthreads, thread 0
// arrives with one release reduction (cumulative over the CTA's writes so
// far).  Wait: thread 0 polls with acquire loads, so a barrier costs one trip
// to L2 plus the polling delay; writes a CTA issues between the halves are
// not part of this barrier's release (a later barrier's arrival covers
// them).  bar[2] is the run's abort flag: every 64 polls the waiter checks
// it and the 4 s limit; a wait that runs out sets APO_ERR_TIMEOUT and the
// flag.  The wait returns false (for every thread of the CTA) when the run
// was aborted or the wait timed out; the caller then stops the run.
__device__ __forceinline__ void run_barrier_arrive(unsigned* bar, int g, unsigned& gen)
{
    __syncthreads();
    if (g > 1 && threadIdx.x == 0) {
        ++gen;
        red_release_add(&bar[0], 1u);
    }
}

__device__ __noinline__ static bool run_barrier_wait(unsigned* bar, int g, unsigned gen, int* status, int* s_flag)
{
    if (g > 1) {
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned target = gen * (unsigned)g;
            unsigned long long t0 = 0ull;
            for (unsigned n = 1;; ++n) {
                if ((int)(ld_acquire(&bar[0]) - target) >= 0) break;
                if ((n & 63u) == 0u) {
                    if (ld_acquire(&bar[2]) != 0u) { ok = 0; break; }
                    const unsigned long long now = global_ns();
                    if (t0 == 0ull) {
                        t0 = now;
                    } else if (now - t0 > kBarrierTimeoutNs) {
                        set_status(status, 4 /* APO_ERR_TIMEOUT */);
                        atomicExch(&bar[2], 1u);
                        ok = 0;
                        break;
                    }
                }
            }
            *s_flag = ok;
        }
        __syncthreads();
        return *s_flag != 0;
    }
    __syncthreads();
    return true;
}

__device__ __forceinline__ bool run_barrier(unsigned* bar, int g, unsigned& gen, int* status, int* s_flag)
{
    run_barrier_arrive(bar, g, gen);
    return run_barrier_wait(bar, g, gen, status, s_flag);
}

}  // namespace apo
