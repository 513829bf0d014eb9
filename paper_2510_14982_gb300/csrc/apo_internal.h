// apo_internal.h -- host-side interface between the C ABI (apo_api.cu) and
// the kernel translation units.  Not part of the public ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/apo.h"
#include "apo_device.cuh"

// A problem created by apo_problem_create: device copies of the bounds,
// shifts, (transposed, permuted) rotations, elliptic weights and Otsu tables
// in one allocation `mem`, described by `dev`.
struct apo_problem {
    int device;
    int D, Dp, Np, kind, ncomp;
    int any_rot;
    apo::DevProblem dev;
    void* mem;
};

namespace apo {

// Launches the Dr_index selection (Eq. 11) for every (run, t) of the runs:
// work item w belongs to the run k with offs[k] <= w < offs[k+1], and covers
// iteration runs[k].t_begin + (w - offs[k]).  max_ps_pad sizes shared memory.
cudaError_t launch_dr(const ApoRun* d_runs, const int* d_offs, int n_runs, int n_work,
                      int max_ps_pad, cudaStream_t st);

// Launches the APO iteration loop.  grid_g > 0: cooperative launch of
// n_runs * grid_g CTAs of the grid kernel (512 threads), CTA b serving run
// b / grid_g; with cluster, a plain launch in which the grid_g CTAs of each
// run form one thread-block cluster (grid_g <= 8).  grid_g == 0: a
// persistent work-queue launch of n_ctas CTAs (256 threads) popping runs
// from *d_queue.  fit64 selects float64 fitness (Otsu); qpl is the
// dimension-pair count per lane (1, 2 or 4).
cudaError_t launch_run(const ApoRun* d_runs, int n_runs, int grid_g, int n_ctas, int* d_queue,
                       int* d_status, size_t smem_bytes, bool fit64, int qpl, cudaStream_t st,
                       bool cluster = false);

// Largest number of co-resident CTAs of the work-queue kernel (grid = false)
// or of the cooperative grid kernel (grid = true) for this shared-memory size
// (0 on error).
int run_kernel_capacity(bool fit64, int qpl, size_t smem_bytes, bool grid);

// Evaluation hooks: rows of d_X [n][D]; select != 0 applies Sec. 4.1 step 6
// (clamp d_Xnew in place, evaluate into d_Fnew, greedy into d_X / d_F).
cudaError_t launch_eval(const ApoRun* d_run, int n, const float* d_X, void* d_F, int select,
                        float* d_Xsel, void* d_Fsel, size_t smem_bytes, bool fit64, int qpl,
                        cudaStream_t st);

// Schedule tables of Eq. 4, 9, 12 and 13 (cached per device; allocated on
// first use).
apo_status sched_tables(int ps, int pdr_form, int T, const uint32_t** thr_dr, const uint32_t** thr_ah,
                                const float** fsc, const float** nsc);

// Process-wide device status word (first device-side error wins).
int* device_status_word();

// Barrier self-test launch (see apo_barrier_selftest).
cudaError_t launch_barrier_test(unsigned* d_bar, int launched, int expected, int rounds, int* status,
                                cudaStream_t st);

// Sets the text that apo_last_error() returns on the calling thread.
void set_last_error(const char* msg);

cudaError_t launch_philox(const uint32_t* d_ctr, uint32_t k0, uint32_t k1, int n, uint32_t* d_out,
                          cudaStream_t st);

// Histogram and Otsu prefix tables (apo_hist.cu).
cudaError_t launch_histogram_u8(const uint8_t* d_px, int64_t n_per_image, int n_images,
                                int32_t* d_hist, cudaStream_t st);
cudaError_t launch_otsu_prefix(const int32_t* d_hist, long long* d_P0, long long* d_P1,
                               cudaStream_t st);
cudaError_t launch_otsu_table(const long long* d_P0, const long long* d_P1, double* d_tab, cudaStream_t st);

}  // namespace apo
