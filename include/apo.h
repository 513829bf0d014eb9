/*
 * apo.h -- C ABI of libapo.so, a GB300 (sm_103a) implementation of the
 * Artificial Protozoa Optimizer (APO) population update described in
 * "cuAPO: A CUDA-based Parallelization of Artificial Protozoa Optimizer"
 * (Soliya and Jain): Sec. 3 (Eq. 1-13), Algorithm 1, and the thresholding
 * application of Sec. 5.2.
 *
 * Conventions shared by every entry point
 *   - Pointers named d_* are CUDA device pointers on the current device;
 *     every other pointer is host memory.  The caller owns every buffer it
 *     passes; the library owns apo_problem objects and its internal
 *     workspace.
 *   - Positions are float32, row-major [n][D] (row stride D, no padding).
 *   - Fitness values are float32, except for APO_OBJ_OTSU, whose fitness
 *     (the negated between-class variance) is float64.  Arguments typed
 *     `void* d_F` follow this rule.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     documented as stream-ordered only enqueue work; calls documented as
 *     synchronous return after their host outputs are written.
 *   - Errors are reported by the return code only; nothing is thrown and
 *     nothing exits.  apo_last_error() returns a static, thread-local detail
 *     string for the last failing call of the calling thread.
 *   - Minimisation: a smaller fitness is better.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed, run),
 * counter = (iteration, protozoon rank, dimension pair, slot).  Identical
 * (seed, run, params, problem) give identical results on a given build.
 */
#ifndef APO_H
#define APO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum apo_status {
    APO_OK = 0,
    APO_ERR_INVALID_ARG = 1, /* an argument is out of its documented range     */
    APO_ERR_CUDA = 2,        /* a CUDA runtime call or a kernel launch failed   */
    APO_ERR_OOM = 3,         /* device or host allocation failed               */
    APO_ERR_TIMEOUT = 4,     /* a device-side wait exceeded its limit           */
    APO_ERR_UNSUPPORTED = 5, /* valid, but outside what the library supports   */
    APO_ERR_INTERNAL = 6
} apo_status;

/* Objective families.  z = M (x - o) with M a D x D rotation (row-major) and
 * o a shift; both are optional (identity / zero when NULL). */
typedef enum apo_objective_kind {
    APO_OBJ_SPHERE = 0,      /* sum z_i^2 (Eq. 14)                                     */
    APO_OBJ_ELLIPTIC = 1,    /* sum 10^(6 (i-1)/(D-1)) z_i^2                          */
    APO_OBJ_ROSENBROCK = 2,  /* sum_{i<D} 100 (z_{i+1} - z_i^2)^2 + (z_i - 1)^2        */
    APO_OBJ_RASTRIGIN = 3,   /* sum z_i^2 - 10 cos(2 pi z_i) + 10                      */
    APO_OBJ_HYBRID = 4,      /* w = z[perm]; ceil(.3D) elliptic, ceil(.3D) Rosenbrock,
                                rest Rastrigin                                        */
    APO_OBJ_COMPOSITION = 5, /* n_comp components, component k = form 1 + (k mod 4)
                                with its own o_k, M_k, perm_k; weights
                                w_k = exp(-||x-o_k||^2 / (2 D sigma_k^2));
                                f = sum w_k (g_k + bias_k) / sum w_k                 */
    APO_OBJ_OTSU = 6,        /* -sigma_B^2 of an image histogram, thresholds
                                t_j = clamp(floor(x_j), 0, 255) sorted (Sec. 5.2)     */
    /* the further benchmark forms of Sec. 5.1 (Table 2), shifted and rotated: */
    APO_OBJ_BENTCIGAR = 7,   /* z_1^2 + 10^6 sum_{i>=2} z_i^2                          */
    APO_OBJ_HGBAT = 8,       /* y = z / 20 - 1: |(sum y^2)^2 - (sum y)^2|^(1/2)
                                + (sum y^2 / 2 + sum y) / D + 1/2                     */
    APO_OBJ_GRIEWANK = 9     /* y = 6 z: 1 + sum y_i^2 / 4000 - prod cos(y_i / sqrt(i)) */
} apo_objective_kind;

#define APO_MAX_COMPONENTS 10
#define APO_MAX_DIM 1024
#define APO_MAX_OTSU_THRESHOLDS 31

typedef struct apo_objective_desc {
    int kind;                  /* apo_objective_kind                              */
    const float* shift;        /* [D] (composition: [n_comp*D]); NULL = 0          */
    const float* rotation;     /* [D*D] row-major (composition: [n_comp*D*D]);
                                  NULL = identity (not allowed for composition)    */
    const int32_t* perm;       /* hybrid: [D] permutation of 0..D-1; composition:
                                  [n_comp*D] (used by its hybrid components)      */
    int n_comp;                /* composition: 1..APO_MAX_COMPONENTS               */
    const double* comp_sigma;  /* composition: [n_comp], > 0                      */
    const double* comp_bias;   /* composition: [n_comp]                           */
    const int32_t* hist;       /* Otsu: [256] pixel counts (host, or device when
                                  hist_on_device != 0); total count > 0            */
    int hist_on_device;
} apo_objective_desc;

/* Algorithm 1 inputs.  Validation: ps >= 2, 1 <= np, 2*np < ps,
 * 0 <= pf_max <= 1, max_iter >= 1 (or max_fes >= 2 ps), pdr_form and
 * pair_policy in {0, 1}, max_fes >= 0. */
typedef struct apo_params {
    int ps;           /* population size                                       */
    int np;           /* neighbour pairs in Eq. 6 and Eq. 8                     */
    double pf_max;    /* maximum proportion fraction (Eq. 11)                   */
    int max_iter;     /* iterations (MaxFEs of Algorithm 1 counts iterations)   */
    uint32_t seed;    /* Philox key word 0                                      */
    uint32_t run;     /* Philox key word 1 (independent stream per run)         */
    int pdr_form;     /* 0: Eq. 13 as printed, p_dr = (1 - cos((1-i/ps) pi))/2;
                         1: the mirrored (1 + cos((1-i/ps) pi))/2               */
    int pair_policy;  /* the pairs (k-, k+) of Eq. 6-7 for rank i (1-based):
                         0: independent uniform ranks over 1..ps;
                         1: k- uniform over the ranks 1..i (at least as good
                            as i), k+ uniform over i..ps (at most as good)     */
    long long max_fes;/* 0: max_iter iterations.  > 0: an evaluation budget
                         (MaxFEs counted in objective evaluations): ps at
                         initialisation and ps per iteration, so the run takes
                         T = floor(max_fes / ps) - 1 whole iterations and T is
                         iter_max of Eq. 4, 9 and 12; max_iter is ignored.
                         apo_effective_iterations() returns T.                  */
} apo_params;

/* The number of iterations a run with these params takes: max_iter, or the
 * iterations that fit the evaluation budget max_fes (see apo_params); -1 when
 * the params are invalid.  Size curves with it (+1 entry). */
int apo_effective_iterations(const apo_params* params);

typedef struct apo_problem apo_problem;

/* Creates a problem: D dimensions (1..APO_MAX_DIM; Otsu: 1..31 thresholds;
 * composition: 1..256),
 * bounds lb < ub per dimension (the Xmin, Xmax of Eq. 1-2), and the
 * objective.  Every array is copied to the device; the caller may free its
 * buffers on return.  Synchronous.  *out is NULL on failure. */
apo_status apo_problem_create(int D, const double* lb, const double* ub,
                              const apo_objective_desc* obj, apo_problem** out);

/* Releases a problem (NULL is a no-op).  Waits for the device to finish work
 * that may still read it. */
void apo_problem_destroy(apo_problem* prob);

int apo_problem_dim(const apo_problem* prob);

/* A whole run of Algorithm 1: initialisation, T = apo_effective_iterations()
 * iterations (max_iter, or what the evaluation budget max_fes allows) of
 * sort, Dr selection (Eq. 11), dormancy / reproduction / autotrophic /
 * heterotrophic candidates (Eq. 1-10, 12-13), bound clamp, evaluation,
 * greedy replacement.  Outputs (host): best_x [D], *best_f, and curve
 * [T + 1] (curve[t] = best fitness after iteration t, curve[0] after
 * initialisation; NULL = not wanted).  Synchronous. */
apo_status apo_run(const apo_problem* prob, const apo_params* params, void* stream,
                   float* best_x, double* best_f, float* curve);

/* Same as apo_run with device outputs: d_best_x [D], d_best_f [1],
 * d_curve [T + 1] or NULL.  Stream-ordered. */
apo_status apo_run_device(const apo_problem* prob, const apo_params* params, void* stream,
                          float* d_best_x, double* d_best_f, float* d_curve);

/* apo_run_device for callers that cannot allocate device memory: callers
 * whose device memory is entirely reserved by their own pool or framework,
 * where a cudaMalloc would fail or take memory the pool accounts for, and
 * callers in latency-critical loops that cannot accept the device-wide
 * synchronisation a cudaFree implies.  The paper has no counterpart; this is
 * a deployment variant of apo_run_device with the same arguments and results.
 * It calls no cudaMalloc, cudaFree or allocating library routine: its
 * workspace is one file-scope device array of 8 MiB that every device loading
 * the library holds until the process exits.  The array's device address is
 * looked up (cudaGetSymbolAddress) by the first call made on each device and
 * context, and again after a cudaDeviceReset; make that first call before any
 * stream capture.  A run whose workspace exceeds 8 MiB is rejected with
 * APO_ERR_UNSUPPORTED and a message naming the size.  The workspace is about
 * 2 KB + ps * 4 + (T + 1) * (12 + 4 * ceil(ps / 32)) bytes, plus, when the run
 * takes the cooperative grid kernel (ps >= 128) or its population does not
 * fit in shared memory, ps * (8 * Dp + 8) bytes for the two population
 * buffers (Dp = D rounded up to 4; Otsu: ps * (8 * Dp + 16)), plus, for the
 * grid kernel, ps * 12 bytes of ranking buffers (Otsu: ps * 20).  Every call
 * shares the array and clears what must start at zero; calls that overlap on
 * the GPU (other host threads or streams) race on it.  Returns after the run
 * has finished (synchronises `stream`). */
apo_status apo_run_device_noalloc(const apo_problem* prob, const apo_params* params, void* stream,
                                  float* d_best_x, double* d_best_f, float* d_curve);

/* n_runs independent runs in as few launches as possible (a persistent
 * work-queue launch for runs whose population fits in shared memory, a
 * cooperative grid launch for the rest).  Run k uses probs[k] and params[k]
 * and writes d_best_x[k*x_stride .. +D), d_best_f[k], and, when d_curves is
 * not NULL, d_curves[k*curve_stride .. + max_iter + 1).  x_stride >= max D,
 * curve_stride >= max (max_iter + 1).  Stream-ordered. */
apo_status apo_run_batch(const apo_problem* const* probs, const apo_params* params, int n_runs,
                         void* stream, float* d_best_x, int x_stride, double* d_best_f,
                         float* d_curves, int curve_stride);

/* A prepared batch: apo_run_batch split into a planning call and a launch
 * call.  apo_batch_create plans the launches, allocates the workspace and
 * uploads the run descriptors (synchronous); apo_batch_launch then only clears
 * control words and launches the kernels (stream-ordered, no allocation, no
 * host copy), so that it can be captured in a CUDA graph and replayed.  Every
 * launch recomputes the runs from their initial populations: same params,
 * same results.  Outputs are the caller's device buffers given at creation
 * (layout as in apo_run_batch).  Launches of one batch must not overlap on
 * the GPU (they share the workspace). */
typedef struct apo_batch apo_batch;

typedef struct apo_batch_options {
    size_t smem_budget;   /* shared memory per work-queue CTA (bytes); 0 = the maximum.
                             Runs whose population fits stay resident in shared memory,
                             the others keep it in global memory.                     */
    int ctas_per_sm;      /* work-queue CTAs per SM; 0 = as many as fit                */
    int cluster_ps;       /* 0: every run of ps <= 1024 takes one work-queue CTA.  > 0:
                             runs with cluster_ps <= ps <= 1024 take one thread-block
                             cluster of cluster_size CTAs each instead (the multi-CTA
                             iteration loop, its CTAs co-scheduled by the hardware)  */
    int cluster_size;     /* 2..8 when cluster_ps > 0                                */
} apo_batch_options;

apo_status apo_batch_create(const apo_problem* const* probs, const apo_params* params, int n_runs,
                            float* d_best_x, int x_stride, double* d_best_f, float* d_curves,
                            int curve_stride, const apo_batch_options* opt, apo_batch** out);
apo_status apo_batch_launch(apo_batch* batch, void* stream);

/* Autotuner: times the batch, truncated to its first `probe_iters`
 * iterations, under candidate configurations -- the work-queue shared-memory
 * budget for 1, 2, 3 and 4 CTAs per SM, each with one CTA per run or with the
 * larger runs on one cluster per run (ps >= 256 on 2 or 4 CTAs, ps >= 384 on
 * 4) -- keeps the fastest and re-plans the batch with it.  Writes the choice
 * to *chosen when not NULL.  Synchronous. */
apo_status apo_batch_autotune(apo_batch* batch, void* stream, int probe_iters, apo_batch_options* chosen);
void apo_batch_destroy(apo_batch* batch);

/* The initial population of a run (Algorithm 1 "Initialize": X_p = Xmin +
 * U (Xmax - Xmin) with the INIT draws of protozoon p, F_p = f(X_p)), written
 * to d_X [ps*D] and d_F [ps] (float64 for Otsu) in protozoon order: the state
 * a run starts from, and the state apo_run_from_state(t_begin = 1) resumes.
 * Stream-ordered. */
apo_status apo_init_state(const apo_problem* prob, const apo_params* params, void* stream, float* d_X,
                          void* d_F);

/* Resume (checkpoint / restart): iterations t_begin..t_end (1 <= t_begin,
 * t_begin - 1 <= t_end <= T, T = apo_effective_iterations(params), the
 * iter_max of the schedules) of the run described by params, starting from
 * the state d_X [ps*D], d_F [ps] that the run had after iteration t_begin - 1
 * (the output of apo_init_state for t_begin = 1, or of a previous
 * apo_run_from_state that ended at t_begin - 1).  On return d_X, d_F hold the
 * state after iteration t_end in its current order (the rank order of
 * iteration t_end's fitness sort, after the greedy replacement), so that runs
 * can be split into segments: the segments give the same results, bit for
 * bit, as one uninterrupted run.  Outputs (device, each may be NULL):
 * d_best_x [D], d_best_f [1] (the best after t_end) and d_curve
 * [t_end - t_begin + 2] with d_curve[j] = best fitness after iteration
 * t_begin - 1 + j.  Stream-ordered. */
apo_status apo_run_from_state(const apo_problem* prob, const apo_params* params, int t_begin, int t_end,
                              void* stream, float* d_X, void* d_F, float* d_best_x, double* d_best_f,
                              float* d_curve);

/* Test hook: iteration `iter` (1..max_iter) of Algorithm 1 applied to a given
 * state.  d_X [ps*D] and d_F [ps] hold the population in its current order;
 * on return they hold it in the rank order of this iteration's fitness sort
 * (ascending, ties kept in current order) after the greedy replacement.
 * Stream-ordered. */
apo_status apo_step(const apo_problem* prob, const apo_params* params, int iter,
                    void* stream, float* d_X, void* d_F);

/* Evaluates the objective at n points d_X [n*D] into d_F [n].  Stream-ordered. */
apo_status apo_evaluate(const apo_problem* prob, void* stream, const float* d_X, int n,
                        void* d_F);

/* Sec. 4.1 step 6 on n protozoa: clamp d_Xnew [n*D] to the bounds (in place),
 * evaluate it into d_Fnew [n], and replace d_X / d_F rows where
 * f(Xnew) < f(X).  Stream-ordered. */
apo_status apo_clamp_eval_select(const apo_problem* prob, void* stream, int n, float* d_X,
                                 void* d_F, float* d_Xnew, void* d_Fnew);

/* 256-bin histograms of n_images 8-bit images stored back to back, the first
 * step of the thresholding application (Sec. 5.2: Otsu's between-class
 * variance is a function of the image histogram only).  Counts are int32
 * (bit-exact; every image has fewer than 2^31 pixels), not the int64 of the
 * Otsu prefix sums, which apo_problem_create forms from them.  Input
 * d_pixels [n_images * n_pixels_per_image], output d_hist [n_images*256]
 * (int32 counts, overwritten; bit-exact).  n_pixels_per_image < 2^31.
 * Stream-ordered. */
apo_status apo_histogram_u8(const uint8_t* d_pixels, int64_t n_pixels_per_image, int n_images,
                            int32_t* d_hist, void* stream);

/* Surrogate network of the surrogate-assisted form: an MLP D -> 256 -> 256 -> 1
 * with ReLU, bfloat16 weights and activations, float32 accumulation on the
 * tensor cores, float32 master weights and Adam (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8) on mean squared error.  Parameters are row-major: W1 [D][256],
 * b1 [256], W2 [256][256], b2 [256], w3 [256], b3.  The paper has no
 * counterpart: the surrogate is an added form of the method. */
typedef struct apo_mlp apo_mlp;

apo_status apo_mlp_create(int D, uint32_t seed, apo_mlp** out);   /* He-uniform init */
void apo_mlp_destroy(apo_mlp* mlp);
apo_status apo_mlp_set_params(apo_mlp* mlp, const float* W1, const float* b1, const float* W2, const float* b2,
                              const float* w3, float b3);   /* host arrays; synchronous */
apo_status apo_mlp_get_params(const apo_mlp* mlp, float* W1, float* b1, float* W2, float* b2, float* w3,
                              float* b3);                   /* host outputs; synchronous */
/* y [n] = f(X [n][D]) for float32 inputs on the device (rounded to bf16). Stream-ordered. */
apo_status apo_mlp_forward(apo_mlp* mlp, const float* d_X, int n, float* d_y, void* stream);
/* Test hook: loss and gradients of mean((f(X) - t)^2) over n <= 2048 rows,
 * written to host arrays (any may be NULL).  Synchronous. */
apo_status apo_mlp_gradients(apo_mlp* mlp, const float* d_X, const float* d_t, int n, float* gW1, float* gb1,
                             float* gW2, float* gb2, float* gw3, float* gb3, float* loss);
/* `steps` Adam steps on batches of `batch` rows drawn uniformly (Philox,
 * seeded) from the n rows of (d_X, d_t).  Stream-ordered. */
apo_status apo_mlp_train(apo_mlp* mlp, const float* d_X, const float* d_t, int n, int steps, int batch, float lr,
                         uint32_t seed, void* stream);

/* Surrogate-assisted APO (an added form; the paper has no counterpart).  Each
 * iteration every protozoon draws k candidates (candidate c >= 1 uses the
 * Philox slots of candidate 0 offset by c << 8, so k = 1 is the plain method
 * draw for draw), the network ranks them, and only the best-ranked one is
 * evaluated exactly and goes through the greedy replacement of Algorithm 1.
 * Exact evaluations fill a ring-buffer archive of archive_cap rows (inputs
 * scaled to [-1, 1] by the bounds, targets the standardised
 * log1p(F - min F) over the training window); every retrain_every
 * iterations the network takes train_steps Adam steps on batches of `batch`
 * rows drawn from the most recent train_window archive rows.  Screening
 * starts after the first retrain and stops, until the next retrain, when the
 * Spearman rank correlation between predicted and true fitness of the last
 * screened batch is below min_rank_corr (the plain method is the fallback).
 * Outputs as in apo_run (host); stats (optional) counts the work.
 * Synchronous.  ps <= 4096; float objectives only. */
typedef struct apo_surrogate_params {
    int k;                /* candidates per protozoon, 1..32            */
    int retrain_every;    /* iterations between retrains                */
    int archive_cap;      /* archive rows (>= ps)                       */
    int train_steps;      /* Adam steps per retrain                     */
    int batch;            /* training batch rows                        */
    float lr;             /* Adam learning rate                         */
    float min_rank_corr;  /* screening threshold on Spearman correlation */
    uint32_t net_seed;    /* network initialisation and batch sampling  */
    int train_window;     /* retrain on the most recent train_window archive rows
                             (targets standardised over them); 0 = the whole archive */
} apo_surrogate_params;

typedef struct apo_surrogate_stats {
    long long true_evals;   /* exact objective evaluations (incl. initial) */
    long long screened;     /* candidates generated                        */
    int retrains;
    int screening_iters;    /* iterations with k > 1                       */
    int fallback_iters;     /* plain iterations after the first retrain    */
    double last_rank_corr;
    double train_ms;        /* device time spent training                  */
    double total_ms;        /* device time of the whole run                */
} apo_surrogate_stats;

apo_status apo_run_surrogate(const apo_problem* prob, const apo_params* params, const apo_surrogate_params* sp,
                             void* stream, float* best_x, double* best_f, float* curve, apo_surrogate_stats* stats);

/* Test hook of the surrogate-assisted form: the k (1..32) candidates of every
 * protozoon at iteration iter (1..max_iter) from the population d_X [ps][D],
 * d_F [ps] (device, float32, current order), as the surrogate path generates
 * them: the population is ranked by the stable (F, index) sort of Algorithm 1
 * and candidate c of rank r draws from the plain method's Philox slots
 * | (c << 8), so c = 0 is the plain candidate (Eq. 1-10, clamped).
 * d_Xcand [ps][k][D] (device) receives candidate c of rank r at row r k + c.
 * ps <= 4096; float objectives only.  Synchronous. */
apo_status apo_surrogate_candidates(const apo_problem* prob, const apo_params* params, int iter, int k,
                                    void* stream, const float* d_X, const float* d_F, float* d_Xcand);

/* Test hook of the grid barrier that the cooperative iteration loop uses
 * between its phases: ctas_launched CTAs (at most one per SM) each pass
 * `rounds` barriers of a run that expects ctas_expected CTAs.  Returns
 * APO_OK when launched == expected; with fewer CTAs the first wait runs out
 * after its limit (4 s), the kernel records APO_ERR_TIMEOUT in the device
 * status word and returns, and the call reports (and clears) that status;
 * the context stays usable.  No counterpart in the paper.  Synchronous. */
apo_status apo_barrier_selftest(int ctas_launched, int ctas_expected, int rounds, void* stream);

/* Test hook: the device Philox4x32-10 on n counters d_ctr [n*4] with key
 * (key0, key1) into d_out [n*4].  Stream-ordered. */
apo_status apo_philox4x32_10(const uint32_t* d_ctr, uint32_t key0, uint32_t key1, int n,
                             uint32_t* d_out, void* stream);

/* Instrumentation: when set (non-NULL cudaEvent_t handles), every later
 * apo_run / apo_run_device / apo_run_batch call records `before` on its
 * stream immediately before its first iteration-loop kernel and `after`
 * immediately after its last, so that a caller can time those kernels with
 * cudaEventElapsedTime.  Process-wide setting; pass NULL, NULL to clear.  The
 * caller keeps ownership of the events. */
apo_status apo_set_timing_events(void* before, void* after);

/* Instrumentation of the large-dimension path (D > 256; no counterpart in
 * the paper): with `on` != 0 every later run on that path brackets each
 * stage launch with CUDA events on its stream and adds the elapsed device
 * time per stage (0 ranking: chunk sort and rank; 1 candidate generation;
 * 2 rotation GEMM with the objective epilogue; 3 greedy replacement), at
 * the cost of a stream synchronisation at the end of each call.  Each call
 * returns the totals since the previous one in ms[4] and launches[4] (either
 * may be NULL), clears them and sets the switch.  Process-wide. */
apo_status apo_large_stage_timing(int on, double* ms, long long* launches);

/* Instrumentation (no counterpart in the paper): microbenchmarks of the
 * pipes that bound the fused kernels, on the current device, every SM busy
 * with independent dependency chains: FP32 fused multiply-add throughput
 * (TFLOP/s, 2 flop per FMA), 32-bit integer multiply-add throughput (Tops/s)
 * and plain integer ALU throughput (xor and add, Tops/s).  Outputs may be
 * NULL.  Synchronous; allocates 64 bytes of device memory. */
apo_status apo_measure_peaks(void* stream, double* ffma_tflops, double* imad_tops, double* alu_tops);

/* Static text of a status code (never NULL).  The paper has no counterpart:
 * the C ABI's error reporting convention. */
const char* apo_status_string(apo_status status);
const char* apo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* APO_H */
