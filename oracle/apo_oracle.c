/*
 * apo_oracle.c -- plain, slow, obviously-correct FP64 CPU restatement of the
 * Artificial Protozoa Optimizer (APO) per-iteration population update as the
 * cuAPO paper states it (Sec. 3, Eq. 1-13; Algorithm 1; worked example of
 * Sec. 4.1), together with the objectives the GPU path evaluates and the
 * 256-bin image histogram of the thresholding application (Sec. 5.2).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark load this library.  The GPU product path
 * (libapo.so) never calls it, and the two share no source: this file has its
 * own Philox generator, its own sort, subset selection and objectives.
 *
 * Arithmetic: every quantity is an IEEE double unless stated.  No blocking,
 * fusion or reordering: each step follows the paper's order and notation.
 * Library primitives used as steps: qsort (the fitness sort of Algorithm 1 and
 * the randperm subsets), cos/exp/pow/floor/ceil from libm.
 *
 * Readings of the paper that the text leaves open (each is listed, with its
 * reason, in the design notes at the repository root):
 *   R1  `rand` is one uniform draw per protozoon, `Rand` one per dimension,
 *       `+-` one random sign per protozoon.
 *   R2  j, k-, k+ (autotrophic mode, Eq. 6-7) are independent uniform ranks
 *       over the whole population (the paper prints no draws; pinned by a
 *       statistical test that reads them off unit-vector populations).
 *   R3  X_{i-k}, X_{i+k} (Eq. 8, 10) clamp to ranks 1..ps.
 *   R4  eps (Eq. 7, 10) = 2^-52.
 *   R5  p_dr (Eq. 13) as printed, with the minus sign (pdr_form 0); the
 *       mirrored plus sign is pdr_form 1.
 *   R6  greedy selection (Algorithm 1) keeps X_new iff f(X_new) < f(X_i).
 *   R7  MaxFEs counts iterations: the loop of Algorithm 1 increments FEs once
 *       per pass, so the run is max_iter iterations.
 *   R8  t = 1..T (T = max_iter) in Eq. 4, 9, 12.
 *   R9  the sort of Algorithm 1 is stable: equal fitness keeps the current
 *       order.
 *   R10 randperm(n, k) is the set of the k smallest (Philox key, index) pairs.
 *   R11 out-of-range candidates are clamped to [Xmin, Xmax] (Sec. 4.1 step 6:
 *       13.53 -> 10).
 *   R12 Otsu thresholds are floor() of the position rounded to binary32 (the
 *       precision the GPU state is stored in), clamped to 0..255, sorted.
 *   R23 with an evaluation budget MaxFEs counted in objective evaluations
 *       (the original APO's reading of MaxFEs), the run takes the whole
 *       iterations that fit: ps evaluations at initialisation, ps per
 *       iteration; their number is iter_max.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11), key = (seed, run), counter =
 * (iter, p, d, slot).  The draw contract (which counter and which output word
 * feeds which symbol of the equations) is the one the GPU path implements
 * independently:
 *   U(r)      = ((r >> 8) + 1) / 2^24            uniform in (0, 1]
 *   IDX(r, n) = (r * n) >> 32                    uniform index in [0, n)
 *   SIGN(r)   = (r & 1) ? -1 : +1
 *   per-dimension draws of dim d use counter (t, p, d >> 1, slot) and words
 *   A_d = out[2 (d & 1)], B_d = out[2 (d & 1) + 1].
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- Philox */

/* Philox4x32 round function and key schedule (Salmon et al. 2011, Sec. 4):
 * two 32x32->64 multiplications by the constants M0, M1, the high halves
 * XORed with the other two counter words and the round key, and the key
 * bumped by the Weyl constants W0, W1 between rounds.  Ten rounds. */
#define ORC_PHILOX_M0 0xD2511F53u
#define ORC_PHILOX_M1 0xCD9E8D57u
#define ORC_PHILOX_W0 0x9E3779B9u
#define ORC_PHILOX_W1 0xBB67AE85u

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_W0;
            k1 += ORC_PHILOX_W1;
        }
        uint64_t p0 = (uint64_t)ORC_PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)ORC_PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter slots: which draw a Philox call serves. */
enum {
    ORC_SLOT_INIT = 1,   /* per (p, d): initial population              */
    ORC_SLOT_PF = 2,     /* global: the rand of Eq. 11                  */
    ORC_SLOT_DR = 3,     /* per rank: randperm key of Dr_index          */
    ORC_SLOT_SCAL = 4,   /* per rank: mode rand, f rand, sign, repr rand */
    ORC_SLOT_SCAL2 = 5,  /* per rank: M_r count rand, index j           */
    ORC_SLOT_PAIR = 6,   /* per (rank, k): indices k-, k+               */
    ORC_SLOT_DIM = 7     /* per (rank, d): Rand_d and the mask key      */
};
#define ORC_ALL 0xFFFFFFFFu

static void orc_draw(uint32_t seed, uint32_t run, uint32_t t, uint32_t p,
                     uint32_t d, uint32_t slot, uint32_t out[4])
{
    uint32_t ctr[4] = {t, p, d, slot};
    uint32_t key[2] = {seed, run};
    orc_philox4x32_10(ctr, key, out);
}

static double orc_U(uint32_t r) { return ((double)(r >> 8) + 1.0) / 16777216.0; }
static uint32_t orc_IDX(uint32_t r, uint32_t n)
{
    return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}
static double orc_SIGN(uint32_t r) { return (r & 1u) ? -1.0 : 1.0; }

/* Per-dimension pair (A_d, B_d) of counter (t, p, d >> 1, slot). */
static void orc_dim_words(uint32_t seed, uint32_t run, uint32_t t, uint32_t p,
                          int d, uint32_t slot, uint32_t* A, uint32_t* B)
{
    uint32_t out[4];
    orc_draw(seed, run, t, p, (uint32_t)(d >> 1), slot, out);
    *A = out[2 * (d & 1)];
    *B = out[2 * (d & 1) + 1];
}

/* ------------------------------------------------------------- problem */

enum {
    ORC_OBJ_SPHERE = 0,
    ORC_OBJ_ELLIPTIC = 1,
    ORC_OBJ_ROSENBROCK = 2,
    ORC_OBJ_RASTRIGIN = 3,
    ORC_OBJ_HYBRID = 4,
    ORC_OBJ_COMPOSITION = 5,
    ORC_OBJ_OTSU = 6,
    ORC_OBJ_BENTCIGAR = 7,
    ORC_OBJ_HGBAT = 8,
    ORC_OBJ_GRIEWANK = 9
};

typedef struct {
    int D;
    int kind;
    const double* lb;      /* [D] Xmin */
    const double* ub;      /* [D] Xmax */
    const float* shift;    /* [D] (composition: [n_comp*D]); NULL = 0     */
    const float* rot;      /* [D*D] row-major (composition: [n_comp*D*D]); NULL = I */
    const int32_t* perm;   /* hybrid: [D]; composition: [n_comp*D]        */
    int n_comp;
    const double* comp_sigma; /* [n_comp] */
    const double* comp_bias;  /* [n_comp] */
    const int64_t* hist;   /* Otsu: [256] pixel counts                    */
} orc_problem;

typedef struct {
    int ps;
    int np;
    double pf_max;
    int max_iter;
    uint32_t seed;
    uint32_t run;
    int pdr_form;
    int pair_policy;   /* reading R2 (0) or its alternative (1), see orc_candidate */
    long long max_fes; /* > 0: evaluation budget (orc_apo_run), reading R23  */
} orc_params;

/* Diagnostics of one iteration, all in rank order of that iteration's sort.
 * Every pointer may be NULL. */
typedef struct {
    int32_t* order;      /* [ps] position (before the sort) of rank r      */
    int32_t* m;          /* [1]  |Dr_index| = ceil(ps * pf)                */
    int32_t* in_dr;      /* [ps]                                          */
    int32_t* mode;       /* [ps] 0 dormancy 1 reproduction 2 autotrophic 3 heterotrophic */
    int32_t* mask_count; /* [ps] number of ones in M_r / M_f (0: dormancy) */
    uint8_t* mask;       /* [ps*D]                                        */
    double* xnew_raw;    /* [ps*D] candidate before the bound clamp       */
    double* xnew;        /* [ps*D] candidate after the clamp              */
    double* fnew;        /* [ps]                                          */
    int32_t* accepted;   /* [ps]                                          */
} orc_step_info;

/* ----------------------------------------------------------- objectives */

/* High-conditioned elliptic on a segment of length n:
 * sum_i 10^(6 (i-1)/(n-1)) z_i^2, i = 1..n (weight 1 when n == 1). */
static double orc_elliptic(const double* z, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i) {
        double w = (n > 1) ? pow(10.0, 6.0 * (double)i / (double)(n - 1)) : 1.0;
        s += w * z[i] * z[i];
    }
    return s;
}

/* Chained Rosenbrock: sum_{i<n} 100 (z_{i+1} - z_i^2)^2 + (z_i - 1)^2. */
static double orc_rosenbrock(const double* z, int n)
{
    double s = 0.0;
    for (int i = 0; i + 1 < n; ++i) {
        double a = z[i + 1] - z[i] * z[i];
        double b = z[i] - 1.0;
        s += 100.0 * a * a + b * b;
    }
    return s;
}

/* Rastrigin cosine sum: sum_i z_i^2 - 10 cos(2 pi z_i) + 10. */
static double orc_rastrigin(const double* z, int n)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        s += z[i] * z[i] - 10.0 * cos(2.0 * M_PI * z[i]) + 10.0;
    return s;
}

/* The benchmark forms of Sec. 5.1 (Table 2) that the other forms do not cover,
 * written out from their textbook definitions (the CEC data files are not
 * available; the scalings are the usual ones of those suites):
 * Bent Cigar: z_1^2 + 10^6 sum_{i>=2} z_i^2. */
static double orc_bent_cigar(const double* z, int n)
{
    double s = 0.0;
    for (int i = 1; i < n; ++i) s += z[i] * z[i];
    return z[0] * z[0] + 1e6 * s;
}

/* HGBat on y = z / 20 - 1 (optimum at z = 0):
 * |(sum y^2)^2 - (sum y)^2|^(1/2) + (sum y^2 / 2 + sum y) / n + 1/2. */
static double orc_hgbat(const double* z, int n)
{
    double s2 = 0.0, s1 = 0.0;
    for (int i = 0; i < n; ++i) {
        double y = z[i] * 0.05 - 1.0;
        s2 += y * y;
        s1 += y;
    }
    return sqrt(fabs(s2 * s2 - s1 * s1)) + (0.5 * s2 + s1) / (double)n + 0.5;
}

/* Griewank on y = 6 z: 1 + sum y_i^2 / 4000 - prod cos(y_i / sqrt(i)), i = 1..n. */
static double orc_griewank(const double* z, int n)
{
    double s = 0.0, p = 1.0;
    for (int i = 0; i < n; ++i) {
        double y = 6.0 * z[i];
        s += y * y;
        p *= cos(y / sqrt((double)(i + 1)));
    }
    return 1.0 + s / 4000.0 - p;
}

/* Hybrid: w = z permuted by perm, split ceil(0.3 D) / ceil(0.3 D) / rest
 * across elliptic, Rosenbrock and Rastrigin. */
static void orc_hybrid_sizes(int D, int* n1, int* n2, int* n3)
{
    int a = (3 * D + 9) / 10;           /* ceil(0.3 D) */
    int b = (3 * D + 9) / 10;
    if (a > D) a = D;
    if (b > D - a) b = D - a;
    *n1 = a; *n2 = b; *n3 = D - a - b;
}

static double orc_hybrid(const double* z, const int32_t* perm, int D)
{
    double* w = (double*)malloc(sizeof(double) * (size_t)D);
    for (int k = 0; k < D; ++k) w[k] = z[perm[k]];
    int n1, n2, n3;
    orc_hybrid_sizes(D, &n1, &n2, &n3);
    double f = orc_elliptic(w, n1) + orc_rosenbrock(w + n1, n2) +
               orc_rastrigin(w + n1 + n2, n3);
    free(w);
    return f;
}

/* z = M (x - o) with M row-major D x D (identity when NULL), o = 0 when NULL. */
static void orc_shift_rotate(int D, const float* M, const float* o,
                             const double* x, double* z)
{
    double* y = (double*)malloc(sizeof(double) * (size_t)D);
    for (int j = 0; j < D; ++j) y[j] = x[j] - (o ? (double)o[j] : 0.0);
    for (int i = 0; i < D; ++i) {
        if (!M) { z[i] = y[i]; continue; }
        double s = 0.0;
        for (int j = 0; j < D; ++j) s += (double)M[(size_t)i * D + j] * y[j];
        z[i] = s;
    }
    free(y);
}

/* Basic shifted-rotated form `form` (1..4) at x. */
static double orc_basic_form(int form, int D, const float* M, const float* o,
                             const int32_t* perm, const double* x)
{
    double* z = (double*)malloc(sizeof(double) * (size_t)D);
    orc_shift_rotate(D, M, o, x, z);
    double f = 0.0;
    switch (form) {
    case ORC_OBJ_SPHERE: for (int i = 0; i < D; ++i) f += z[i] * z[i]; break;
    case ORC_OBJ_ELLIPTIC: f = orc_elliptic(z, D); break;
    case ORC_OBJ_ROSENBROCK: f = orc_rosenbrock(z, D); break;
    case ORC_OBJ_RASTRIGIN: f = orc_rastrigin(z, D); break;
    case ORC_OBJ_HYBRID: f = orc_hybrid(z, perm, D); break;
    case ORC_OBJ_BENTCIGAR: f = orc_bent_cigar(z, D); break;
    case ORC_OBJ_HGBAT: f = orc_hgbat(z, D); break;
    case ORC_OBJ_GRIEWANK: f = orc_griewank(z, D); break;
    default: f = NAN;
    }
    free(z);
    return f;
}

/* Composition of n_comp components: component k is basic form
 * 1 + (k mod 4) (elliptic, Rosenbrock, Rastrigin, hybrid) with its own
 * o_k, M_k, perm_k; weights w_k = exp(-||x - o_k||^2 / (2 D sigma_k^2)),
 * f = sum_k w_k (g_k + bias_k) / sum_k w_k.  The weights are evaluated as
 * exp(a_k - max_k a_k), which leaves the ratio unchanged. */
static double orc_composition(const orc_problem* P, const double* x)
{
    const int D = P->D, K = P->n_comp;
    double* a = (double*)malloc(sizeof(double) * (size_t)K);
    double* g = (double*)malloc(sizeof(double) * (size_t)K);
    double amax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        const float* o = P->shift + (size_t)k * D;
        double dist2 = 0.0;
        for (int j = 0; j < D; ++j) {
            double d = x[j] - (double)o[j];
            dist2 += d * d;
        }
        double sg = P->comp_sigma[k];
        a[k] = -dist2 / (2.0 * (double)D * sg * sg);
        if (a[k] > amax) amax = a[k];
        g[k] = orc_basic_form(1 + (k % 4), D, P->rot + (size_t)k * D * D, o,
                              P->perm ? P->perm + (size_t)k * D : NULL, x);
    }
    double num = 0.0, den = 0.0;
    for (int k = 0; k < K; ++k) {
        double w = exp(a[k] - amax);
        num += w * (g[k] + P->comp_bias[k]);
        den += w;
    }
    free(a); free(g);
    return num / den;
}

static int orc_cmp_int(const void* a, const void* b)
{
    int x = *(const int*)a, y = *(const int*)b;
    return (x > y) - (x < y);
}

/* Otsu's between-class variance for thresholds derived from x (reading R12):
 * classes [0, t_1], (t_1, t_2], ..., (t_T, 255]; sigma_B^2 =
 * sum_c omega_c (mu_c - mu_T)^2 with omega_c = n_c / N, mu_c = s_c / n_c,
 * empty classes contributing 0.  Returned negated (APO minimises).  Class
 * counts and first moments are exact int64 sums over the histogram; the FP64
 * operations are evaluated in the order written, without contraction. */
double orc_otsu_sigma_b2(const int64_t* hist, const int* thr_sorted, int T)
{
    int64_t N = 0, S = 0;
    for (int v = 0; v < 256; ++v) { N += hist[v]; S += (int64_t)v * hist[v]; }
    double muT = (double)S / (double)N;
    double sigma = 0.0;
    int lo = 0;                                 /* first bin of the class */
    for (int c = 0; c <= T; ++c) {
        int hi = (c < T) ? thr_sorted[c] : 255; /* last bin of the class  */
        int64_t n_c = 0, s_c = 0;
        for (int v = lo; v <= hi; ++v) { n_c += hist[v]; s_c += (int64_t)v * hist[v]; }
        if (n_c > 0) {
            double omega = (double)n_c / (double)N;
            double mu = (double)s_c / (double)n_c;
            double dm = mu - muT;
            double term = omega * dm;
            term = term * dm;
            sigma = sigma + term;
        }
        if (hi + 1 > lo) lo = hi + 1;
    }
    return sigma;
}

static double orc_otsu(const orc_problem* P, const double* x)
{
    int T = P->D;
    int* t = (int*)malloc(sizeof(int) * (size_t)T);
    for (int j = 0; j < T; ++j) {
        double v = floor((double)(float)x[j]);
        if (v < 0.0) v = 0.0;
        if (v > 255.0) v = 255.0;
        t[j] = (int)v;
    }
    qsort(t, (size_t)T, sizeof(int), orc_cmp_int);
    double s = orc_otsu_sigma_b2(P->hist, t, T);
    free(t);
    return -s;
}

double orc_objective(const orc_problem* P, const double* x)
{
    switch (P->kind) {
    case ORC_OBJ_SPHERE:
    case ORC_OBJ_ELLIPTIC:
    case ORC_OBJ_ROSENBROCK:
    case ORC_OBJ_RASTRIGIN:
    case ORC_OBJ_HYBRID:
    case ORC_OBJ_BENTCIGAR:
    case ORC_OBJ_HGBAT:
    case ORC_OBJ_GRIEWANK:
        return orc_basic_form(P->kind, P->D, P->rot, P->shift, P->perm, x);
    case ORC_OBJ_COMPOSITION: return orc_composition(P, x);
    case ORC_OBJ_OTSU: return orc_otsu(P, x);
    default: return NAN;
    }
}

void orc_objective_batch(const orc_problem* P, int n, const double* X, double* F)
{
    for (int i = 0; i < n; ++i) F[i] = orc_objective(P, X + (size_t)i * P->D);
}

/* --------------------------------------------------------------- sorting */

typedef struct { double f; uint32_t key; int idx; } orc_sort_item;

static int orc_cmp_fitness(const void* a, const void* b)
{
    const orc_sort_item* x = (const orc_sort_item*)a;
    const orc_sort_item* y = (const orc_sort_item*)b;
    if (x->f < y->f) return -1;
    if (x->f > y->f) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

static int orc_cmp_key(const void* a, const void* b)
{
    const orc_sort_item* x = (const orc_sort_item*)a;
    const orc_sort_item* y = (const orc_sort_item*)b;
    if (x->key != y->key) return (x->key > y->key) - (x->key < y->key);
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/* randperm(n, k) (Eq. 3, Eq. 5, Algorithm 1), reading R10: sel[i] = 1 for
 * the k smallest (keys[i], i). */
static void orc_randperm_set(const uint32_t* keys, int n, int k, uint8_t* sel)
{
    if (n <= 0) return;
    orc_sort_item* it = (orc_sort_item*)malloc(sizeof(orc_sort_item) * (size_t)n);
    for (int i = 0; i < n; ++i) { it[i].key = keys[i]; it[i].idx = i; it[i].f = 0.0; }
    qsort(it, (size_t)n, sizeof(orc_sort_item), orc_cmp_key);
    memset(sel, 0, (size_t)n);
    for (int i = 0; i < k && i < n; ++i) sel[it[i].idx] = 1;
    free(it);
}

/* ------------------------------------------------------------ APO steps */

/* Population initialisation (Algorithm 1, "Initialize"): X_p = Xmin +
 * U ⊙ (Xmax - Xmin), then f(X_p). */
int orc_init_population(const orc_problem* P, const orc_params* prm, double* X,
                        double* F)
{
    const int ps = prm->ps, D = P->D;
    for (int p = 0; p < ps; ++p) {
        for (int d = 0; d < D; ++d) {
            uint32_t A, B;
            orc_dim_words(prm->seed, prm->run, 0u, (uint32_t)p, d, ORC_SLOT_INIT, &A, &B);
            X[(size_t)p * D + d] = P->lb[d] + orc_U(A) * (P->ub[d] - P->lb[d]);
        }
        F[p] = orc_objective(P, X + (size_t)p * D);
    }
    return 0;
}

/* Eq. 12 */
static double orc_p_ah(int t, int T)
{
    return 0.5 * (1.0 + cos(((double)t / (double)T) * M_PI));
}

/* Eq. 13 as printed (form 0) and its mirrored sign (form 1); i = 1..ps. */
static double orc_p_dr(int i, int ps, int form)
{
    double c = cos((1.0 - (double)i / (double)ps) * M_PI);
    return form == 0 ? 0.5 * (1.0 - c) : 0.5 * (1.0 + c);
}

/* The candidate of rank r (0-based; i = r + 1) at iteration t from the
 * sorted snapshot (Xs, Fs): mode selection (Eq. 12-13), dormancy (Eq. 1),
 * reproduction (Eq. 2-3) or foraging (Eq. 4-10), then the bound clamp (R11).
 * Every per-protozoon draw uses its slot | slot_off: slot_off = c << 8 gives
 * candidate c of the surrogate-assisted form, 0 the plain method.  in_dr is
 * the iteration's Dr_index set (Eq. 11).  Writes x (clamped) and, if given,
 * xraw (before the clamp), *kmask_out and the mask M[D]; returns the mode
 * (0 dormancy, 1 reproduction, 2 autotrophic, 3 heterotrophic).  Rand[D] and
 * mkey[D] are scratch. */
static int orc_candidate(const orc_problem* P, const orc_params* prm, int t, int r, uint32_t slot_off,
                         const double* Xs, const double* Fs, const uint8_t* in_dr, double* x,
                         double* xraw, int* kmask_out, uint8_t* M, double* Rand, uint32_t* mkey)
{
    const int ps = prm->ps, D = P->D, np = prm->np, T = prm->max_iter;
    const uint32_t seed = prm->seed, run = prm->run;
    const double eps = 2.220446049250313e-16; /* 2^-52, reading R4 */
    /* Eq. 12, Eq. 4 and Eq. 9 schedules. */
    const double p_ah = orc_p_ah(t, T);
    const double fscale = 1.0 + cos(((double)t / (double)T) * M_PI);
    const double nearscale = 1.0 - (double)t / (double)T;
    const int i = r + 1;
    const double* Xi = Xs + (size_t)r * D;
    uint32_t sc[4], sc2[4];
    orc_draw(seed, run, (uint32_t)t, (uint32_t)r, ORC_ALL, ORC_SLOT_SCAL | slot_off, sc);
    orc_draw(seed, run, (uint32_t)t, (uint32_t)r, ORC_ALL, ORC_SLOT_SCAL2 | slot_off, sc2);
    for (int d = 0; d < D; ++d) {
        uint32_t A, B;
        orc_dim_words(seed, run, (uint32_t)t, (uint32_t)r, d, ORC_SLOT_DIM | slot_off, &A, &B);
        Rand[d] = orc_U(A);
        mkey[d] = B;
    }
    const double u_mode = orc_U(sc[0]);
    int mode, kmask = 0;
    if (in_dr[r]) {
        if (orc_p_dr(i, ps, prm->pdr_form) > u_mode) {
            /* Eq. 1: dormancy -- a fresh protozoon replaces X_i. */
            mode = 0;
            for (int d = 0; d < D; ++d)
                x[d] = P->lb[d] + Rand[d] * (P->ub[d] - P->lb[d]);
        } else {
            /* Eq. 2-3: reproduction. */
            mode = 1;
            kmask = (int)ceil((double)D * orc_U(sc2[0]));
            orc_randperm_set(mkey, D, kmask, M);
            const double s = orc_SIGN(sc[2]);
            const double rho = orc_U(sc[3]);
            for (int d = 0; d < D; ++d) {
                if (M[d])
                    x[d] = Xi[d] + s * rho * (P->lb[d] + Rand[d] * (P->ub[d] - P->lb[d]));
                else
                    x[d] = Xi[d];
            }
        }
    } else {
        /* Eq. 4-5: foraging factor f and mask M_f. */
        kmask = (D * i + ps - 1) / ps; /* ceil(D * i / ps) */
        orc_randperm_set(mkey, D, kmask, M);
        const double f = orc_U(sc[1]) * fscale;
        if (p_ah > u_mode) {
            /* Eq. 6-7: autotrophic foraging. */
            mode = 2;
            const int j = (int)orc_IDX(sc2[1], (uint32_t)ps);
            const double* Xj = Xs + (size_t)j * D;
            int* km = (int*)malloc(sizeof(int) * (size_t)np);
            int* kp = (int*)malloc(sizeof(int) * (size_t)np);
            double* wa = (double*)malloc(sizeof(double) * (size_t)np);
            for (int k = 1; k <= np; ++k) {
                uint32_t pr[4];
                orc_draw(seed, run, (uint32_t)t, (uint32_t)r, (uint32_t)(k - 1),
                         ORC_SLOT_PAIR | slot_off, pr);
                if (prm->pair_policy == 0) {
                    /* R2: k-, k+ independent uniform ranks over 1..ps */
                    km[k - 1] = (int)orc_IDX(pr[0], (uint32_t)ps);
                    kp[k - 1] = (int)orc_IDX(pr[1], (uint32_t)ps);
                } else {
                    /* R2 alternative: k- uniform over the ranks 1..i (at
                     * least as good as X_i), k+ uniform over i..ps */
                    km[k - 1] = (int)orc_IDX(pr[0], (uint32_t)i);
                    kp[k - 1] = r + (int)orc_IDX(pr[1], (uint32_t)(ps - r));
                }
                /* Eq. 7 */
                wa[k - 1] = exp(-fabs(Fs[km[k - 1]] / (Fs[kp[k - 1]] + eps)));
            }
            for (int d = 0; d < D; ++d) {
                if (!M[d]) { x[d] = Xi[d]; continue; }
                double acc = 0.0;
                for (int k = 0; k < np; ++k)
                    acc += wa[k] * (Xs[(size_t)km[k] * D + d] - Xs[(size_t)kp[k] * D + d]);
                x[d] = Xi[d] + f * (Xj[d] - Xi[d] + acc / (double)np);
            }
            free(km); free(kp); free(wa);
        } else {
            /* Eq. 8-10: heterotrophic foraging. */
            mode = 3;
            const double s = orc_SIGN(sc[2]);
            for (int d = 0; d < D; ++d) {
                if (!M[d]) { x[d] = Xi[d]; continue; }
                /* Eq. 9 */
                double xnear = (1.0 + s * Rand[d] * nearscale) * Xi[d];
                double acc = 0.0;
                for (int k = 1; k <= np; ++k) {
                    int a = r - k < 0 ? 0 : r - k;          /* R3 */
                    int b = r + k > ps - 1 ? ps - 1 : r + k;
                    /* Eq. 10 */
                    double wh = exp(-fabs(Fs[a] / (Fs[b] + eps)));
                    acc += wh * (Xs[(size_t)a * D + d] - Xs[(size_t)b * D + d]);
                }
                x[d] = Xi[d] + f * (xnear - Xi[d] + acc / (double)np);
            }
        }
    }
    if (xraw) memcpy(xraw, x, sizeof(double) * (size_t)D);
    /* Bound handling (R11). */
    for (int d = 0; d < D; ++d) {
        if (x[d] < P->lb[d]) x[d] = P->lb[d];
        if (x[d] > P->ub[d]) x[d] = P->ub[d];
    }
    if (kmask_out) *kmask_out = kmask;
    return mode;
}

/* One iteration of Algorithm 1 at iteration t (1..max_iter).  X[ps*D], F[ps]
 * are read in their current order and returned in the rank order of this
 * iteration's sort, with the greedy replacement applied. */
int orc_apo_step(const orc_problem* P, const orc_params* prm, int t, double* X,
                 double* F, orc_step_info* info)
{
    const int ps = prm->ps, D = P->D, np = prm->np, T = prm->max_iter;
    const uint32_t seed = prm->seed, run = prm->run;
    if (ps < 1 || D < 1 || np < 1 || T < 1) return -1;

    /* Algorithm 1: sort X_i, i = 1..ps, by fitness (ascending; R9). */
    orc_sort_item* it = (orc_sort_item*)malloc(sizeof(orc_sort_item) * (size_t)ps);
    for (int i = 0; i < ps; ++i) { it[i].f = F[i]; it[i].idx = i; it[i].key = 0; }
    qsort(it, (size_t)ps, sizeof(orc_sort_item), orc_cmp_fitness);
    double* Xs = (double*)malloc(sizeof(double) * (size_t)ps * D);
    double* Fs = (double*)malloc(sizeof(double) * (size_t)ps);
    for (int r = 0; r < ps; ++r) {
        memcpy(Xs + (size_t)r * D, X + (size_t)it[r].idx * D, sizeof(double) * (size_t)D);
        Fs[r] = F[it[r].idx];
        if (info && info->order) info->order[r] = it[r].idx;
    }
    free(it);

    /* Eq. 11: pf = pf_max * rand; Dr_index = randperm(ps, ceil(ps * pf)). */
    uint32_t w[4];
    orc_draw(seed, run, (uint32_t)t, ORC_ALL, ORC_ALL, ORC_SLOT_PF, w);
    double pf = prm->pf_max * orc_U(w[0]);
    int m = (int)ceil((double)ps * pf);
    uint32_t* drkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ps);
    for (int r = 0; r < ps; ++r) {
        orc_draw(seed, run, (uint32_t)t, (uint32_t)(r >> 2), ORC_ALL, ORC_SLOT_DR, w);
        drkey[r] = w[r & 3];
    }
    uint8_t* in_dr = (uint8_t*)malloc((size_t)ps);
    orc_randperm_set(drkey, ps, m, in_dr);
    if (info && info->m) info->m[0] = m;

    double* Xn = (double*)malloc(sizeof(double) * (size_t)ps * D);
    double* Fn = (double*)malloc(sizeof(double) * (size_t)ps);
    double* Rand = (double*)malloc(sizeof(double) * (size_t)D);
    uint32_t* mkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)D);
    uint8_t* M = (uint8_t*)malloc((size_t)D);

    /* Parallel for each i = 1:ps (every candidate reads the sorted snapshot). */
    for (int r = 0; r < ps; ++r) {
        double* x = Xn + (size_t)r * D;
        int kmask = 0;
        const int mode = orc_candidate(P, prm, t, r, 0u, Xs, Fs, in_dr, x,
                                       (info && info->xnew_raw) ? info->xnew_raw + (size_t)r * D : NULL,
                                       &kmask, M, Rand, mkey);
        Fn[r] = orc_objective(P, x);
        if (info) {
            if (info->in_dr) info->in_dr[r] = in_dr[r];
            if (info->mode) info->mode[r] = mode;
            if (info->mask_count) info->mask_count[r] = kmask;
            if (info->mask) {
                for (int d = 0; d < D; ++d)
                    info->mask[(size_t)r * D + d] = (mode == 0) ? 0 : M[d];
            }
            if (info->xnew) memcpy(info->xnew + (size_t)r * D, x, sizeof(double) * (size_t)D);
            if (info->fnew) info->fnew[r] = Fn[r];
        }
    }

    /* Greedy replacement (R6). */
    for (int r = 0; r < ps; ++r) {
        int acc = Fn[r] < Fs[r];
        if (acc) {
            memcpy(Xs + (size_t)r * D, Xn + (size_t)r * D, sizeof(double) * (size_t)D);
            Fs[r] = Fn[r];
        }
        if (info && info->accepted) info->accepted[r] = acc;
    }
    memcpy(X, Xs, sizeof(double) * (size_t)ps * D);
    memcpy(F, Fs, sizeof(double) * (size_t)ps);

    free(Xs); free(Fs); free(drkey); free(in_dr); free(Xn); free(Fn);
    free(Rand); free(mkey); free(M);
    return 0;
}

/* Surrogate-assisted form: the k candidates of every protozoon at iteration
 * t, from X[ps*D], F[ps] in their current order.  The population is sorted
 * and Dr_index drawn as in orc_apo_step; candidate c of rank r draws from the
 * plain slots | (c << 8) (c = 0 is the plain candidate) and is written,
 * clamped, to Xc[(r*k + c)*D ...].  order[r] (optional) = current index of
 * rank r.  Returns 0, or -1 for invalid sizes. */
int orc_candidates(const orc_problem* P, const orc_params* prm, int t, int k, const double* X,
                   const double* F, double* Xc, int32_t* order)
{
    const int ps = prm->ps, D = P->D;
    const uint32_t seed = prm->seed, run = prm->run;
    if (ps < 1 || D < 1 || prm->np < 1 || prm->max_iter < 1 || k < 1 || k > 256) return -1;
    orc_sort_item* it = (orc_sort_item*)malloc(sizeof(orc_sort_item) * (size_t)ps);
    for (int i = 0; i < ps; ++i) { it[i].f = F[i]; it[i].idx = i; it[i].key = 0; }
    qsort(it, (size_t)ps, sizeof(orc_sort_item), orc_cmp_fitness);
    double* Xs = (double*)malloc(sizeof(double) * (size_t)ps * D);
    double* Fs = (double*)malloc(sizeof(double) * (size_t)ps);
    for (int r = 0; r < ps; ++r) {
        memcpy(Xs + (size_t)r * D, X + (size_t)it[r].idx * D, sizeof(double) * (size_t)D);
        Fs[r] = F[it[r].idx];
        if (order) order[r] = it[r].idx;
    }
    free(it);
    /* Eq. 11: the iteration's Dr_index, shared by all candidates. */
    uint32_t w[4];
    orc_draw(seed, run, (uint32_t)t, ORC_ALL, ORC_ALL, ORC_SLOT_PF, w);
    const double pf = prm->pf_max * orc_U(w[0]);
    const int m = (int)ceil((double)ps * pf);
    uint32_t* drkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)ps);
    for (int r = 0; r < ps; ++r) {
        orc_draw(seed, run, (uint32_t)t, (uint32_t)(r >> 2), ORC_ALL, ORC_SLOT_DR, w);
        drkey[r] = w[r & 3];
    }
    uint8_t* in_dr = (uint8_t*)malloc((size_t)ps);
    orc_randperm_set(drkey, ps, m, in_dr);
    double* Rand = (double*)malloc(sizeof(double) * (size_t)D);
    uint32_t* mkey = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)D);
    uint8_t* M = (uint8_t*)malloc((size_t)D);
    for (int r = 0; r < ps; ++r)
        for (int c = 0; c < k; ++c)
            orc_candidate(P, prm, t, r, (uint32_t)c << 8, Xs, Fs, in_dr, Xc + ((size_t)r * k + c) * D, NULL, NULL,
                          M, Rand, mkey);
    free(Xs); free(Fs); free(drkey); free(in_dr); free(Rand); free(mkey); free(M);
    return 0;
}

/* Index of the best protozoon: the first minimum in the current order
 * (rank 0 of a stable sort). */
static int orc_best_index(const double* F, int ps)
{
    int b = 0;
    for (int i = 1; i < ps; ++i)
        if (F[i] < F[b]) b = i;
    return b;
}

/* A whole run: initialisation, max_iter iterations, the best position and
 * fitness, and the convergence curve curve[t] = best fitness after
 * iteration t (curve[0] after initialisation).  curve may be NULL. */
/* The number of iterations a run takes: max_iter, or, with an evaluation
 * budget max_fes > 0 (reading R23: MaxFEs counted in objective evaluations,
 * FEs = ps after the initialisation and += ps per iteration, the loop running
 * while another whole iteration fits), the largest T with ps (T + 1) <=
 * max_fes.  That T is iter_max of Eq. 4, 9 and 12.  -1 when nothing fits. */
int orc_iterations(const orc_params* prm)
{
    if (prm->max_fes <= 0) return prm->max_iter;
    long long fes = prm->ps;   /* the initialisation */
    int T = 0;
    while (fes + prm->ps <= prm->max_fes) {
        fes += prm->ps;
        ++T;
    }
    return T >= 1 ? T : -1;
}

int orc_apo_run(const orc_problem* P, const orc_params* prm_in, double* best_x,
                double* best_f, double* curve)
{
    orc_params prm_v = *prm_in;
    const orc_params* prm = &prm_v;
    prm_v.max_iter = orc_iterations(prm_in);
    if (prm_v.max_iter < 1) return -1;
    const int ps = prm->ps, D = P->D;
    double* X = (double*)malloc(sizeof(double) * (size_t)ps * D);
    double* F = (double*)malloc(sizeof(double) * (size_t)ps);
    orc_init_population(P, prm, X, F);
    if (curve) curve[0] = F[orc_best_index(F, ps)];
    int rc = 0;
    for (int t = 1; t <= prm->max_iter && rc == 0; ++t) {
        rc = orc_apo_step(P, prm, t, X, F, NULL);
        if (curve) curve[t] = F[orc_best_index(F, ps)];
    }
    int b = orc_best_index(F, ps);
    if (best_x) memcpy(best_x, X + (size_t)b * D, sizeof(double) * (size_t)D);
    if (best_f) *best_f = F[b];
    free(X); free(F);
    return rc;
}

/* Many independent runs spread over n_threads host threads (one run per
 * task).  best_x is [n*D_max] with row stride D_max; curves may be NULL. */
typedef struct {
    const orc_problem* const* probs;
    const orc_params* params;
    int n;
    int dstride;
    double* best_x;
    double* best_f;
    int next;
    pthread_mutex_t lock;
} orc_batch_ctx;

static void* orc_batch_worker(void* arg)
{
    orc_batch_ctx* c = (orc_batch_ctx*)arg;
    for (;;) {
        pthread_mutex_lock(&c->lock);
        int k = c->next++;
        pthread_mutex_unlock(&c->lock);
        if (k >= c->n) break;
        orc_apo_run(c->probs[k], &c->params[k],
                    c->best_x ? c->best_x + (size_t)k * c->dstride : NULL,
                    c->best_f ? &c->best_f[k] : NULL, NULL);
    }
    return NULL;
}

int orc_apo_run_many(const orc_problem* const* probs, const orc_params* params,
                     int n, int dstride, int n_threads, double* best_x,
                     double* best_f)
{
    orc_batch_ctx c;
    c.probs = probs; c.params = params; c.n = n; c.dstride = dstride;
    c.best_x = best_x; c.best_f = best_f; c.next = 0;
    pthread_mutex_init(&c.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)n_threads);
    for (int i = 0; i < n_threads; ++i) pthread_create(&th[i], NULL, orc_batch_worker, &c);
    for (int i = 0; i < n_threads; ++i) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&c.lock);
    return 0;
}

/* Sec. 4.1 step 6: clamp each candidate to the bounds, evaluate it, and keep
 * it iff it improves on the old protozoon.  X, F in/out; Xnew in/out
 * (clamped); Fnew out. */
void orc_clamp_eval_select(const orc_problem* P, int n, double* X, double* F,
                           double* Xnew, double* Fnew)
{
    const int D = P->D;
    for (int i = 0; i < n; ++i) {
        double* x = Xnew + (size_t)i * D;
        for (int d = 0; d < D; ++d) {
            if (x[d] < P->lb[d]) x[d] = P->lb[d];
            if (x[d] > P->ub[d]) x[d] = P->ub[d];
        }
        Fnew[i] = orc_objective(P, x);
        if (Fnew[i] < F[i]) {
            memcpy(X + (size_t)i * D, x, sizeof(double) * (size_t)D);
            F[i] = Fnew[i];
        }
    }
}

/* 256-bin histogram of n 8-bit pixels (the thresholding application). */
void orc_histogram_u8(const uint8_t* px, int64_t n, int64_t* hist)
{
    memset(hist, 0, sizeof(int64_t) * 256);
    for (int64_t i = 0; i < n; ++i) hist[px[i]] += 1;
}
