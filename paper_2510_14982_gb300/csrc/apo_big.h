// apo_big.h -- host/device interface of the large-dimension path
// (apo_big.cu, kSmallMaxDim < D <= kBigMaxDim).  Not part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include "apo_internal.h"

namespace apo {

constexpr int kBigMaxRuns = 8;   // runs sharing one launch sequence
constexpr int kBigMaxPs = 16384; // population (16 sorted chunks of 1024 keys in shared memory)

// Flags of a group of large-dimension runs.
constexpr int kBigInit = 1;       // initialise the population (else: state from X_in / F_in)
constexpr int kBigStepOut = 2;    // write the state after t_end (current order); no best, no curve
constexpr int kBigStateOut = 4;   // also write the state after t_end, with best and curve
constexpr int kBigEval = 8;       // evaluation only: F_out[r] = f(X_in[r])

// One run on the device.  Populations are slot-indexed: slot s's current row
// is X[loc[s]][s]; perm[t & 1] maps the ranks of iteration t to slots.
struct BigRun {
    int D, Dp, Kp, form, s1, s2;
    const float *lb, *ub, *o, *ew;
    float ysc, zsc;
    int ps, np, pair_policy, T;
    uint32_t seed, run;
    const uint32_t* thr_dr;
    const uint32_t* thr_ah;
    const float* fsc;
    const float* nsc;
    const uint32_t* drmask;     // [t_end + 1][ceil(ps / 32)]
    float* X[2];                // [ps][Dp]
    uint8_t* loc;               // [ps]
    float* F;                   // [ps] by slot
    uint32_t* perm[2];          // [ps]
    unsigned long long* keys;   // [nchunk * 1024] sorted chunks of (ord(F), rank)
    int nchunk;
    uint16_t* Yh;               // [rows][Kp] fp16 hi of y = ysc (x - o), row = rank
    uint16_t* Yl;               // [rows][Kp] fp16 lo
    int bn, ntiles;             // GEMM N tile and tiles per row
    float2* part;               // [ps][ntiles] partial sums of the objective
    float2* zedge;              // [ps][ntiles] z at each tile's first and last column
    float* curve;               // indexed by iteration (t - 1 at iteration t's ranking)
    float* best_x;
    double* best_f;
    const float* X_in;          // evaluation input [ps][D]
    float* X_out;               // state output [ps][D]
    float* F_out;               // state / evaluation output [ps]
    int* status;
};

// One run of a launch request.
struct BigSpec {
    const apo_problem* P;
    apo_params prm;   // resolved (max_iter = the run's iterations)
    int ps;           // population (evaluation: rows)
    int t_begin, t_end, flags;
    float* best_x;
    double* best_f;
    float* curve;     // offset so that curve[t - 1] is written at iteration t
    const float* X_in;
    const float* F_in;
    float* X_out;
    float* F_out;
};

// Runs a group of at most kBigMaxRuns runs sharing (t_begin, t_end, flags)
// on `st` (stream-ordered; the workspace is allocated and freed in stream
// order).  err receives a message when the result is not APO_OK.
apo_status big_run_group(const std::vector<BigSpec>& specs, cudaStream_t st, char* err, size_t errlen);

// Stages of an iteration, for the instrumentation timers.
constexpr int kStageRank = 0, kStageGen = 1, kStageGemm = 2, kStageFinal = 3, kBigStages = 4;

// Instrumentation: returns (and clears) the accumulated device time and
// launch count of every stage, then switches the timers on or off.
void big_stage_timing(int on, double* ms, long long* launches);

// Optional timing events around the iteration loops (set by apo_set_timing_events).
cudaEvent_t big_timing_before();
cudaEvent_t big_timing_after();

}  // namespace apo
