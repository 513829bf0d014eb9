// apo_noalloc.cu -- apo_run_device_noalloc: one whole APO run, like
// apo_run_device, for callers that cannot allocate device memory -- callers
// whose device memory is entirely reserved by their own pool or framework
// (so a cudaMalloc would fail or take memory the pool accounts for), and
// callers in latency-critical loops that cannot accept the device-wide
// synchronisation that cudaFree implies.
//
// Instead of a per-call workspace, every call uses one file-scope device
// array of kScratchBytes (8 MiB).  Each device that loads the library holds
// that array until the process exits.  Its device address is looked up with
// cudaGetSymbolAddress on the first call made with a device (and context)
// current and cached for that context; a call after cudaDeviceReset, which
// brings a new context, looks it up again.  That first call should come
// before any stream capture.  Every call reuses the same array, which keeps
// the previous call's contents: the words that must start at zero (status,
// work-queue counter, barrier words) are cleared by every call, and two calls
// whose work overlaps on the GPU (from two host threads, or on two streams)
// race on the array.  The call returns after its run has finished.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.h"
#include "apo_plan.h"

using namespace apo;

// Shared scratch of every apo_run_device_noalloc call (see above).
static __device__ __align__(256) unsigned char apo_noalloc_scratch[8u << 20];

namespace {

constexpr size_t kScratchBytes = 8u << 20;
constexpr int kQueueMaxPsNA = 1024;
constexpr int kGridMinRowsNA = 8;
constexpr int kMaxDevices = 64;

std::mutex g_na_mu;
void* g_na_addr[kMaxDevices] = {};
void* g_na_ctx[kMaxDevices] = {};   // the context the cached address belongs to

thread_local char g_na_err[256] = "";

size_t al(size_t v, size_t a) { return (v + a - 1) / a * a; }

// The current driver context (nullptr when the driver entry point is not
// available), so that a cached address is never used in a later context.
void* current_context()
{
    using Fn = int (*)(void**);
    static Fn fn = []() -> Fn {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return nullptr;
        return reinterpret_cast<Fn>(f);
    }();
    void* ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Device address of the scratch array on the current device and context.
apo_status scratch_address(int dev, unsigned char** out)
{
    if (dev < 0 || dev >= kMaxDevices) {
        snprintf(g_na_err, sizeof(g_na_err), "device ordinal %d out of range", dev);
        return APO_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    void* ctx = current_context();
    if (!g_na_addr[dev] || !ctx || ctx != g_na_ctx[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, apo_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            snprintf(g_na_err, sizeof(g_na_err), "cudaGetSymbolAddress of the scratch array failed: %s",
                     cudaGetErrorString(e));
            return APO_ERR_CUDA;
        }
        g_na_addr[dev] = p;
        g_na_ctx[dev] = ctx;
    }
    *out = static_cast<unsigned char*>(g_na_addr[dev]);
    return APO_OK;
}

}  // namespace

extern "C" apo_status apo_run_device_noalloc(const apo_problem* P, const apo_params* p_in, void* stream,
                                             float* d_best_x, double* d_best_f, float* d_curve)
{
    auto fail = [](apo_status s, const char* msg) {
        apo::set_last_error(msg);
        return s;
    };
    if (!P || !p_in || !d_best_x || !d_best_f) return fail(APO_ERR_INVALID_ARG, "NULL problem, params or output");
    apo_params q;
    if (const char* why = normalize_params(p_in, &q)) return fail(APO_ERR_INVALID_ARG, why);
    const apo_params* p = &q;
    if (P->D > kSmallMaxDim) return fail(APO_ERR_UNSUPPORTED, "apo_run_device_noalloc supports D <= 256");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != P->device)
        return fail(APO_ERR_INVALID_ARG, "the problem belongs to another device");
    int smem_optin = 0;
    if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return fail(APO_ERR_CUDA, "cannot read the shared-memory limit");
    // the kernels keep less than 2 KB of static shared memory beside the plan
    const size_t kSmemMaxNA = (size_t)smem_optin - 2048;
    unsigned char* base = nullptr;
    apo_status rc = scratch_address(dev, &base);
    if (rc != APO_OK) return fail(rc, g_na_err);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    const int ps = p->ps, T = p->max_iter, Dp = P->Dp;
    const bool fit64 = P->kind == APO_OBJ_OTSU;
    const int qpl = fit64 ? 1 : (P->D <= 64 ? 1 : (P->D <= 128 ? 2 : 4));
    const bool grid = ps > kQueueMaxPsNA || ps >= 128;   // same rule as a lone apo_run_device
    SmemPlan plan = grid ? choose_plan(P, ps, false, true, kSmemMaxNA) : choose_plan(P, ps, true, false, kSmemMaxNA);
    if (!grid && plan.total > kSmemMaxNA) plan = choose_plan(P, ps, false, false, kSmemMaxNA);
    if (plan.total > kSmemMaxNA) return fail(APO_ERR_UNSUPPORTED, "problem needs too much shared memory");

    // scratch layout
    const size_t fsz = fit64 ? 8 : 4;
    const int W = (ps + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = al(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t o_ctrl = take(256), o_run = take(sizeof(ApoRun)), o_offs = take(2 * sizeof(int));
    const size_t o_thr = take((size_t)ps * 4), o_ah = take((size_t)(T + 1) * 4), o_fs = take((size_t)(T + 1) * 4),
                 o_ns = take((size_t)(T + 1) * 4);
    const size_t o_dr = take((size_t)(T + 1) * W * 4);
    const bool glob = !plan.resident;
    const size_t o_x0 = glob ? take((size_t)ps * Dp * 4) : 0, o_x1 = glob ? take((size_t)ps * Dp * 4) : 0;
    const size_t o_f0 = glob ? take(ps * fsz) : 0, o_f1 = glob ? take(ps * fsz) : 0;
    const size_t o_pg = grid ? take((size_t)ps * 4) : 0, o_kg = grid ? take((size_t)ps * (fit64 ? 16 : 8)) : 0;
    if (off > kScratchBytes) {
        char msg[200];
        snprintf(msg, sizeof(msg), "this run needs %zu bytes of scratch; apo_run_device_noalloc is limited to "
                 "%zu bytes (use apo_run_device)", off, kScratchBytes);
        return fail(APO_ERR_UNSUPPORTED, msg);
    }

    // schedule tables of Eq. 4, 9, 12 and 13 (the same helper as apo_run_device)
    std::vector<uint32_t> thr(ps), ah(T + 1);
    std::vector<float> fs(T + 1), ns(T + 1);
    fill_sched_tables(ps, p->pdr_form, T, thr.data(), ah.data(), fs.data(), ns.data());

    int g = 1;
    if (grid) {
        const int cap = run_kernel_capacity(fit64, qpl, plan.total, true);
        if (cap <= 0) return fail(APO_ERR_UNSUPPORTED, "grid kernel cannot be resident");
        g = std::max(1, std::min(std::min(cap, kMaxGridCtas), (ps + kGridMinRowsNA - 1) / kGridMinRowsNA));
    }
    ApoRun R;
    std::memset(&R, 0, sizeof(R));
    R.prob = P->dev;
    R.plan = plan;
    R.ps = ps; R.np = p->np; R.T = T; R.pdr_form = p->pdr_form; R.pf_max = p->pf_max;
    R.pair_policy = p->pair_policy;
    R.seed = p->seed; R.run = p->run; R.t_begin = 1; R.t_end = T; R.flags = kFlagInit; R.g = g;
    R.thr_dr = reinterpret_cast<const uint32_t*>(base + o_thr);
    R.thr_ah = reinterpret_cast<const uint32_t*>(base + o_ah);
    R.fsc = reinterpret_cast<const float*>(base + o_fs);
    R.nsc = reinterpret_cast<const float*>(base + o_ns);
    R.drmask = reinterpret_cast<const uint32_t*>(base + o_dr);
    if (glob) {
        R.X[0] = reinterpret_cast<float*>(base + o_x0);
        R.X[1] = reinterpret_cast<float*>(base + o_x1);
        R.F[0] = base + o_f0;
        R.F[1] = base + o_f1;
    }
    R.best_x = d_best_x; R.best_f = d_best_f; R.curve = d_curve;
    R.bar = reinterpret_cast<unsigned*>(base + o_ctrl + 16);
    if (grid) {
        R.perm_g = reinterpret_cast<uint32_t*>(base + o_pg);
        R.keys_g = base + o_kg;
    }
    const int offs[2] = {0, T};
    int* status = reinterpret_cast<int*>(base + o_ctrl);
    int* queue = reinterpret_cast<int*>(base + o_ctrl + 4);

    cudaError_t e = cudaMemsetAsync(base + o_ctrl, 0, 256, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_run, &R, sizeof(R), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_offs, offs, sizeof(offs), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_thr, thr.data(), (size_t)ps * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ah, ah.data(), (size_t)(T + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_fs, fs.data(), (size_t)(T + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ns, ns.data(), (size_t)(T + 1) * 4, cudaMemcpyHostToDevice, st);
    const ApoRun* d_run = reinterpret_cast<const ApoRun*>(base + o_run);
    if (e == cudaSuccess) e = launch_dr(d_run, reinterpret_cast<const int*>(base + o_offs), 1, T, plan.ps_pad, st);
    if (e == cudaSuccess)
        e = launch_run(d_run, 1, grid ? g : 0, 1, queue, status, plan.total, fit64, qpl, st);
    int host_status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_status, status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        char msg[200];
        snprintf(msg, sizeof(msg), "apo_run_device_noalloc: %s", cudaGetErrorString(e));
        return fail(APO_ERR_CUDA, msg);
    }
    if (host_status != 0) return fail((apo_status)host_status, "a device-side wait exceeded its limit");
    return APO_OK;
}
