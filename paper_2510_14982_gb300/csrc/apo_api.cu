// apo_api.cu -- the C ABI of libapo.so (declared in include/apo.h): argument
// validation, problem objects, the per-iteration schedule tables of Eq. 4,
// Eq. 9, Eq. 12 and Eq. 13, run planning (shared-memory resident work-queue
// launch or cooperative grid launch), workspace management and launches.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

#include "../../include/apo.h"
#include "apo_internal.h"
#include "apo_plan.h"

using namespace apo;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

#define APO_CUDA(expr)                                                                   \
    do {                                                                                 \
        const cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                         \
            set_err("%s failed: %s", #expr, cudaGetErrorString(e_));                    \
            return e_ == cudaErrorMemoryAllocation ? APO_ERR_OOM : APO_ERR_CUDA;         \
        }                                                                                \
    } while (0)

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
int next_pow2(int v)
{
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

// Largest dynamic shared memory per CTA on sm_100-class parts.
constexpr size_t kSmemMax = 232448;
// Runs with a larger population go to the cooperative grid launch.
constexpr int kQueueMaxPs = 1024;
// Minimum protozoa per CTA in grid mode.
constexpr int kGridMinRows = 8;

// Optional timing events around the iteration-loop kernels.
cudaEvent_t g_ev_before = nullptr, g_ev_after = nullptr;

}  // namespace


// ------------------------------------------------------------ errors
extern "C" const char* apo_status_string(apo_status s)
{
    switch (s) {
    case APO_OK: return "ok";
    case APO_ERR_INVALID_ARG: return "invalid argument";
    case APO_ERR_CUDA: return "CUDA error";
    case APO_ERR_OOM: return "out of memory";
    case APO_ERR_TIMEOUT: return "device wait timed out";
    case APO_ERR_UNSUPPORTED: return "unsupported";
    case APO_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

extern "C" const char* apo_last_error(void) { return g_err; }

void apo::set_last_error(const char* msg) { set_err("%s", msg); }

// ---------------------------------------------------------- problems
namespace {

int form_of_component(int kind, int k) { return kind == APO_OBJ_COMPOSITION ? 1 + (k % 4) : kind; }

// ceil(0.3 D) / ceil(0.3 D) / rest split of the hybrid form.
void hybrid_sizes(int D, int* n1, int* n2)
{
    int a = (3 * D + 9) / 10, b = (3 * D + 9) / 10;
    if (a > D) a = D;
    if (b > D - a) b = D - a;
    *n1 = a;
    *n2 = b;
}

bool valid_perm(const int32_t* p, int D)
{
    std::vector<char> seen(D, 0);
    for (int i = 0; i < D; ++i) {
        if (p[i] < 0 || p[i] >= D || seen[p[i]]) return false;
        seen[p[i]] = 1;
    }
    return true;
}

}  // namespace

extern "C" apo_status apo_problem_create(int D, const double* lb, const double* ub, const apo_objective_desc* obj,
                                         apo_problem** out)
{
    if (!out) { set_err("out is NULL"); return APO_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!obj || !lb || !ub) { set_err("obj, lb and ub must not be NULL"); return APO_ERR_INVALID_ARG; }
    const int kind = obj->kind;
    if (kind < APO_OBJ_SPHERE || kind > APO_OBJ_OTSU) { set_err("unknown objective kind %d", kind); return APO_ERR_INVALID_ARG; }
    if (D < 1) { set_err("D must be >= 1"); return APO_ERR_INVALID_ARG; }
    if (kind == APO_OBJ_OTSU ? D > APO_MAX_OTSU_THRESHOLDS : D > APO_MAX_DIM) {
        set_err("D = %d exceeds the supported maximum", D);
        return APO_ERR_UNSUPPORTED;
    }
    for (int d = 0; d < D; ++d) {
        if (!std::isfinite(lb[d]) || !std::isfinite(ub[d]) || !(lb[d] < ub[d])) {
            set_err("bounds must be finite with lb < ub (dim %d)", d);
            return APO_ERR_INVALID_ARG;
        }
    }
    const int ncomp = kind == APO_OBJ_COMPOSITION ? obj->n_comp : (kind == APO_OBJ_OTSU ? 0 : 1);
    if (kind == APO_OBJ_COMPOSITION) {
        if (ncomp < 1 || ncomp > APO_MAX_COMPONENTS) { set_err("n_comp must be 1..%d", APO_MAX_COMPONENTS); return APO_ERR_INVALID_ARG; }
        if (!obj->shift || !obj->rotation || !obj->comp_sigma || !obj->comp_bias) {
            set_err("composition needs shift, rotation, comp_sigma and comp_bias");
            return APO_ERR_INVALID_ARG;
        }
        for (int k = 0; k < ncomp; ++k)
            if (!(obj->comp_sigma[k] > 0.0) || !std::isfinite(obj->comp_bias[k])) {
                set_err("comp_sigma must be > 0 and comp_bias finite");
                return APO_ERR_INVALID_ARG;
            }
    }
    for (int k = 0; k < ncomp; ++k) {
        if (form_of_component(kind, k) == APO_OBJ_HYBRID) {
            if (!obj->perm) { set_err("hybrid form needs perm"); return APO_ERR_INVALID_ARG; }
            if (!valid_perm(obj->perm + (size_t)(kind == APO_OBJ_COMPOSITION ? k : 0) * D, D)) {
                set_err("perm is not a permutation of 0..D-1");
                return APO_ERR_INVALID_ARG;
            }
        }
    }
    if (kind == APO_OBJ_OTSU && !obj->hist) { set_err("Otsu needs hist"); return APO_ERR_INVALID_ARG; }
    if (kind == APO_OBJ_OTSU && !obj->hist_on_device) {
        long long n = 0;
        for (int v = 0; v < 256; ++v) {
            if (obj->hist[v] < 0) { set_err("negative histogram count"); return APO_ERR_INVALID_ARG; }
            n += obj->hist[v];
        }
        if (n <= 0) { set_err("empty histogram"); return APO_ERR_INVALID_ARG; }
    }

    const int Dp = (D + 3) & ~3;
    const int Np = (D + 15) & ~15;
    // Host image of every device array, laid out in one allocation.
    std::vector<std::pair<size_t, std::vector<unsigned char>>> pieces;
    size_t off = 0;
    auto add = [&](const void* src, size_t bytes) -> size_t {
        off = align_up(off, 256);
        const size_t at = off;
        std::vector<unsigned char> v(bytes);
        if (src) std::memcpy(v.data(), src, bytes);
        pieces.emplace_back(at, std::move(v));
        off += bytes;
        return at;
    };
    std::vector<float> lbf(Dp, 0.f), ubf(Dp, 0.f);
    for (int d = 0; d < D; ++d) { lbf[d] = (float)lb[d]; ubf[d] = (float)ub[d]; }
    const size_t off_lb = add(lbf.data(), Dp * 4), off_ub = add(ubf.data(), Dp * 4);
    size_t off_o[kMaxComp] = {}, off_mt[kMaxComp] = {}, off_ew[kMaxComp] = {};
    bool has_mt[kMaxComp] = {};
    DevComp comps[kMaxComp] = {};
    int any_rot = 0;
    for (int k = 0; k < ncomp; ++k) {
        const int form = form_of_component(kind, k);
        const float* M = obj->rotation ? obj->rotation + (size_t)(kind == APO_OBJ_COMPOSITION ? k : 0) * D * D : nullptr;
        const int32_t* perm = obj->perm ? obj->perm + (size_t)(kind == APO_OBJ_COMPOSITION ? k : 0) * D : nullptr;
        std::vector<float> o(Dp, 0.f);
        if (obj->shift)
            for (int d = 0; d < D; ++d) o[d] = obj->shift[(size_t)(kind == APO_OBJ_COMPOSITION ? k : 0) * D + d];
        off_o[k] = add(o.data(), Dp * 4);
        // z'_c = z_{perm[c]} for the hybrid form: rows of M are permuted, so
        // MT[j][c] = M[perm[c]][j]; otherwise MT = M^T.
        const bool perm_rows = form == APO_OBJ_HYBRID;
        if (M || perm_rows) {
            std::vector<float> mt((size_t)Dp * Np, 0.f);
            for (int c = 0; c < D; ++c) {
                const int row = perm_rows ? perm[c] : c;
                for (int j = 0; j < D; ++j)
                    mt[(size_t)j * Np + c] = M ? M[(size_t)row * D + j] : (j == row ? 1.f : 0.f);
            }
            off_mt[k] = add(mt.data(), (size_t)Dp * Np * 4);
            has_mt[k] = true;
            any_rot = 1;
        }
        int s1 = 0, s2 = 0, nell = 0;
        switch (form) {
        case APO_OBJ_SPHERE: s1 = D; s2 = D; nell = 0; break;
        case APO_OBJ_ELLIPTIC: s1 = D; s2 = D; nell = D; break;
        case APO_OBJ_ROSENBROCK: s1 = 0; s2 = D; break;
        case APO_OBJ_RASTRIGIN: s1 = 0; s2 = 0; break;
        case APO_OBJ_HYBRID: {
            int n1, n2;
            hybrid_sizes(D, &n1, &n2);
            s1 = n1; s2 = n1 + n2; nell = n1;
            break;
        }
        default: break;
        }
        std::vector<float> ew(Dp, 1.f);
        for (int d = 0; d < nell; ++d)
            ew[d] = nell > 1 ? (float)std::pow(10.0, 6.0 * (double)d / (double)(nell - 1)) : 1.f;
        off_ew[k] = add(ew.data(), Dp * 4);
        comps[k].s1 = s1;
        comps[k].s2 = s2;
        if (kind == APO_OBJ_COMPOSITION) {
            const double sg = obj->comp_sigma[k];
            comps[k].inv_2Dsig2 = (float)(1.0 / (2.0 * (double)D * sg * sg));
            comps[k].bias = (float)obj->comp_bias[k];
        }
    }
    size_t off_p0 = 0, off_p1 = 0, off_hist = 0;
    if (kind == APO_OBJ_OTSU) {
        std::vector<long long> p0(256, 0), p1(256, 0);
        if (!obj->hist_on_device) {
            long long a = 0, b = 0;
            for (int v = 0; v < 256; ++v) {
                a += obj->hist[v];
                b += (long long)v * obj->hist[v];
                p0[v] = a;
                p1[v] = b;
            }
        }
        off_p0 = add(p0.data(), 256 * 8);
        off_p1 = add(p1.data(), 256 * 8);
        if (obj->hist_on_device) off_hist = add(nullptr, 256 * 4);
    }

    apo_problem* P = new apo_problem();
    APO_CUDA(cudaGetDevice(&P->device));
    P->D = D; P->Dp = Dp; P->Np = Np; P->kind = kind; P->ncomp = ncomp; P->any_rot = any_rot;
    cudaError_t e = cudaMalloc(&P->mem, std::max<size_t>(off, 256));
    if (e != cudaSuccess) {
        delete P;
        set_err("cudaMalloc of %zu bytes failed: %s", off, cudaGetErrorString(e));
        return APO_ERR_OOM;
    }
    unsigned char* base = static_cast<unsigned char*>(P->mem);
    for (auto& pc : pieces) {
        e = cudaMemcpy(base + pc.first, pc.second.data(), pc.second.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && kind == APO_OBJ_OTSU && obj->hist_on_device) {
        e = cudaMemcpy(base + off_hist, obj->hist, 256 * 4, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = launch_otsu_prefix(reinterpret_cast<int32_t*>(base + off_hist),
                                   reinterpret_cast<long long*>(base + off_p0),
                                   reinterpret_cast<long long*>(base + off_p1), 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e == cudaSuccess) {
            long long n = 0;
            e = cudaMemcpy(&n, base + off_p0 + 255 * 8, 8, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && n <= 0) {
                cudaFree(P->mem);
                delete P;
                set_err("empty histogram");
                return APO_ERR_INVALID_ARG;
            }
        }
    }
    if (e != cudaSuccess) {
        cudaFree(P->mem);
        delete P;
        set_err("problem upload failed: %s", cudaGetErrorString(e));
        return APO_ERR_CUDA;
    }
    DevProblem& dp = P->dev;
    std::memset(&dp, 0, sizeof(dp));
    dp.D = D; dp.Dp = Dp; dp.Np = Np; dp.kind = kind; dp.ncomp = ncomp;
    dp.lb = reinterpret_cast<const float*>(base + off_lb);
    dp.ub = reinterpret_cast<const float*>(base + off_ub);
    for (int k = 0; k < ncomp; ++k) {
        dp.comp[k] = comps[k];
        dp.comp[k].o = reinterpret_cast<const float*>(base + off_o[k]);
        dp.comp[k].MT = has_mt[k] ? reinterpret_cast<const float*>(base + off_mt[k]) : nullptr;
        dp.comp[k].ew = reinterpret_cast<const float*>(base + off_ew[k]);
    }
    if (kind == APO_OBJ_OTSU) {
        dp.P0 = reinterpret_cast<const long long*>(base + off_p0);
        dp.P1 = reinterpret_cast<const long long*>(base + off_p1);
    }
    *out = P;
    return APO_OK;
}

extern "C" void apo_problem_destroy(apo_problem* P)
{
    if (!P) return;
    cudaDeviceSynchronize();
    cudaFree(P->mem);
    delete P;
}

extern "C" int apo_problem_dim(const apo_problem* P) { return P ? P->D : 0; }

// ----------------------------------------------------- schedule tables
namespace {

struct TableCache {
    std::mutex mu;
    std::map<std::pair<int, int>, uint32_t*> dr;     // (ps, pdr_form) -> thr_dr [ps]
    std::map<std::pair<int, int>, void*> sched;      // (T, device)    -> thr_ah | fsc | nsc
};
TableCache& tables()
{
    static TableCache* c = new TableCache();  // never destroyed: device memory lives to exit
    return *c;
}

// Eq. 13 (form 0 as printed, form 1 mirrored) as a 24-bit threshold:
// protozoon of rank i (1-based) goes dormant iff U < p_dr(i), i.e. iff
// ((r >> 8) + 1) < ceil(p_dr(i) 2^24).
apo_status get_thr_dr(int ps, int form, int dev, const uint32_t** out)
{
    TableCache& c = tables();
    std::lock_guard<std::mutex> lk(c.mu);
    const std::pair<int, int> key(ps * 2 + form, dev);
    auto it = c.dr.find(key);
    if (it != c.dr.end()) { *out = it->second; return APO_OK; }
    std::vector<uint32_t> thr(ps);
    for (int i = 1; i <= ps; ++i) {
        const double cv = cos((1.0 - (double)i / (double)ps) * M_PI);
        const double p = form == 0 ? 0.5 * (1.0 - cv) : 0.5 * (1.0 + cv);
        thr[i - 1] = (uint32_t)ceil(p * 16777216.0);
    }
    uint32_t* d = nullptr;
    APO_CUDA(cudaMalloc(&d, sizeof(uint32_t) * ps));
    APO_CUDA(cudaMemcpy(d, thr.data(), sizeof(uint32_t) * ps, cudaMemcpyHostToDevice));
    c.dr[key] = d;
    *out = d;
    return APO_OK;
}

// Eq. 12 threshold ceil(p_ah(t) 2^24), Eq. 4 factor 1 + cos(pi t / T) and
// Eq. 9 factor 1 - t / T for t = 0..T.
apo_status get_sched(int T, int dev, const uint32_t** thr_ah, const float** fsc, const float** nsc)
{
    TableCache& c = tables();
    std::lock_guard<std::mutex> lk(c.mu);
    const std::pair<int, int> key(T, dev);
    auto it = c.sched.find(key);
    void* d = nullptr;
    if (it != c.sched.end()) {
        d = it->second;
    } else {
        std::vector<uint32_t> a(T + 1);
        std::vector<float> f(T + 1), n(T + 1);
        for (int t = 0; t <= T; ++t) {
            const double cv = cos(((double)t / (double)T) * M_PI);
            const double pah = 0.5 * (1.0 + cv);
            a[t] = (uint32_t)ceil(pah * 16777216.0);
            f[t] = (float)(1.0 + cv);
            n[t] = (float)(1.0 - (double)t / (double)T);
        }
        const size_t stride = align_up((size_t)(T + 1) * 4, 256);
        APO_CUDA(cudaMalloc(&d, 3 * stride));
        unsigned char* b = static_cast<unsigned char*>(d);
        APO_CUDA(cudaMemcpy(b, a.data(), (T + 1) * 4, cudaMemcpyHostToDevice));
        APO_CUDA(cudaMemcpy(b + stride, f.data(), (T + 1) * 4, cudaMemcpyHostToDevice));
        APO_CUDA(cudaMemcpy(b + 2 * stride, n.data(), (T + 1) * 4, cudaMemcpyHostToDevice));
        c.sched[key] = d;
    }
    const size_t stride = align_up((size_t)(T + 1) * 4, 256);
    unsigned char* b = static_cast<unsigned char*>(d);
    *thr_ah = reinterpret_cast<const uint32_t*>(b);
    *fsc = reinterpret_cast<const float*>(b + stride);
    *nsc = reinterpret_cast<const float*>(b + 2 * stride);
    return APO_OK;
}

// Process-wide device status word (first device-side error wins).
int* device_status(int dev)
{
    static std::mutex mu;
    static std::map<int, int*> words;
    std::lock_guard<std::mutex> lk(mu);
    auto it = words.find(dev);
    if (it != words.end()) return it->second;
    int* p = nullptr;
    if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
    cudaMemset(p, 0, sizeof(int));
    cudaDeviceSynchronize();
    words[dev] = p;
    return p;
}

apo_status check_params(const apo_problem* P, const apo_params* p)
{
    if (!P || !p) { set_err("problem and params must not be NULL"); return APO_ERR_INVALID_ARG; }
    if (p->ps < 2) { set_err("ps must be >= 2"); return APO_ERR_INVALID_ARG; }
    if (p->np < 1 || 2 * p->np >= p->ps) { set_err("np must satisfy 1 <= np and 2 np < ps"); return APO_ERR_INVALID_ARG; }
    if (!(p->pf_max >= 0.0 && p->pf_max <= 1.0)) { set_err("pf_max must be in [0, 1]"); return APO_ERR_INVALID_ARG; }
    if (p->max_iter < 1) { set_err("max_iter must be >= 1"); return APO_ERR_INVALID_ARG; }
    if (p->pdr_form != 0 && p->pdr_form != 1) { set_err("pdr_form must be 0 or 1"); return APO_ERR_INVALID_ARG; }
    if (p->ps > (1 << 20)) { set_err("ps above 2^20 is not supported"); return APO_ERR_UNSUPPORTED; }
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != P->device) { set_err("problem belongs to device %d, current device is %d", P->device, dev); return APO_ERR_INVALID_ARG; }
    return APO_OK;
}

int qpl_of(const apo_problem* P) { return P->D <= 64 ? 1 : (P->D <= 128 ? 2 : 4); }


// One run of a launch plan.
struct RunSpec {
    const apo_problem* P;
    apo_params prm;
    int t_begin, t_end, flags;
    float* best_x;
    double* best_f;
    float* curve;
    float* X_in;   // step mode: caller state [ps][D]
    void* F_in;
};

struct Group {
    bool fit64;
    int qpl;
    bool grid;
    size_t smem;
    std::vector<int> runs;  // indices into specs
};

// Plans, allocates and launches a set of runs on one stream.
apo_status launch_runs(std::vector<RunSpec>& specs, cudaStream_t st)
{
    const int n = (int)specs.size();
    if (n == 0) return APO_OK;
    int dev = 0, sms = 0;
    APO_CUDA(cudaGetDevice(&dev));
    APO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int* status = device_status(dev);
    if (!status) { set_err("status word allocation failed"); return APO_ERR_OOM; }

    std::vector<ApoRun> runs(n);
    std::vector<char> grid(n, 0);
    std::vector<SmemPlan> plans(n);
    for (int k = 0; k < n; ++k) {
        const RunSpec& s = specs[k];
        const int ps = s.prm.ps;
        const SmemPlan res = choose_plan(s.P, ps, true, false, kSmemMax);
        const SmemPlan nres = choose_plan(s.P, ps, false, false, kSmemMax);
        if (ps > kQueueMaxPs) {
            grid[k] = 1;
            const SmemPlan gp = choose_plan(s.P, ps, false, true, kSmemMax);
            plans[k] = gp;
            if (gp.total > kSmemMax) { set_err("population %d needs too much shared memory", ps); return APO_ERR_UNSUPPORTED; }
            if (nres.total > kSmemMax) { set_err("population %d needs too much shared memory", ps); return APO_ERR_UNSUPPORTED; }
        } else if (res.total <= kSmemMax) {
            plans[k] = res;
        } else {
            plans[k] = nres;
            if (nres.total > kSmemMax) { set_err("problem needs too much shared memory"); return APO_ERR_UNSUPPORTED; }
        }
    }
    // group by kernel instantiation and mode
    std::map<std::tuple<int, int, int>, Group> groups;
    for (int k = 0; k < n; ++k) {
        const bool f64 = specs[k].P->kind == APO_OBJ_OTSU;
        const int q = f64 ? 1 : qpl_of(specs[k].P);
        Group& gr = groups[std::make_tuple((int)f64, q, (int)grid[k])];
        gr.fit64 = f64; gr.qpl = q; gr.grid = grid[k] != 0;
        gr.runs.push_back(k);
        gr.smem = std::max<size_t>(gr.smem, plans[k].total);
    }

    // workspace layout
    size_t off = 0;
    auto take = [&](size_t bytes) -> size_t {
        off = align_up(off, 256);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t off_runs = take(sizeof(ApoRun) * n);
    const size_t off_offs = take(sizeof(int) * (n + 1));
    const size_t off_ctrl = take(sizeof(int) * 64);
    std::vector<size_t> off_dr(n), off_x0(n), off_x1(n), off_f0(n), off_f1(n), off_bar(n), off_pg(n), off_kg(n);
    int n_work = 0;
    std::vector<int> offs(n + 1, 0);
    int max_ps_pad = 1;
    for (int k = 0; k < n; ++k) {
        const RunSpec& s = specs[k];
        const int ps = s.prm.ps, Dp = s.P->Dp;
        const size_t fsz = s.P->kind == APO_OBJ_OTSU ? 8 : 4;
        const int W = (ps + 31) / 32;
        off_dr[k] = take(sizeof(uint32_t) * W * (size_t)(s.t_end + 1));
        const bool need_global = !plans[k].resident || (s.flags & kFlagStepOut);
        off_pg[k] = grid[k] ? take((size_t)ps * 4) : 0;
        off_kg[k] = grid[k] ? take((size_t)ps * (s.P->kind == APO_OBJ_OTSU ? 16 : 8)) : 0;
        off_x0[k] = need_global ? take((size_t)ps * Dp * 4) : 0;
        off_x1[k] = need_global ? take((size_t)ps * Dp * 4) : 0;
        off_f0[k] = need_global ? take(ps * fsz) : 0;
        off_f1[k] = need_global ? take(ps * fsz) : 0;
        off_bar[k] = take(16);
        offs[k] = n_work;
        n_work += s.t_end - s.t_begin + 1;
        max_ps_pad = std::max(max_ps_pad, next_pow2(ps));
    }
    offs[n] = n_work;
    void* ws = nullptr;
    APO_CUDA(cudaMallocAsync(&ws, std::max<size_t>(off, 256), st));
    unsigned char* base = static_cast<unsigned char*>(ws);
    auto fail = [&](apo_status s) {
        cudaFreeAsync(ws, st);
        return s;
    };

    for (int k = 0; k < n; ++k) {
        const RunSpec& s = specs[k];
        ApoRun& R = runs[k];
        std::memset(&R, 0, sizeof(R));
        R.prob = s.P->dev;
        R.plan = plans[k];
        R.ps = s.prm.ps; R.np = s.prm.np; R.T = s.prm.max_iter; R.pdr_form = s.prm.pdr_form;
        R.pf_max = s.prm.pf_max; R.seed = s.prm.seed; R.run = s.prm.run;
        R.t_begin = s.t_begin; R.t_end = s.t_end; R.flags = s.flags;
        R.g = 1;
        const uint32_t* thr_dr = nullptr;
        const uint32_t* thr_ah = nullptr;
        const float *fsc = nullptr, *nsc = nullptr;
        apo_status rc = get_thr_dr(R.ps, R.pdr_form, dev, &thr_dr);
        if (rc == APO_OK) rc = get_sched(R.T, dev, &thr_ah, &fsc, &nsc);
        if (rc != APO_OK) return fail(rc);
        R.thr_dr = thr_dr; R.thr_ah = thr_ah; R.fsc = fsc; R.nsc = nsc;
        R.drmask = reinterpret_cast<const uint32_t*>(base + off_dr[k]);
        if (off_x0[k] || off_x1[k]) {
            R.X[0] = reinterpret_cast<float*>(base + off_x0[k]);
            R.X[1] = reinterpret_cast<float*>(base + off_x1[k]);
            R.F[0] = base + off_f0[k];
            R.F[1] = base + off_f1[k];
        }
        R.X_out = s.X_in;
        R.F_out = s.F_in;
        R.best_x = s.best_x; R.best_f = s.best_f; R.curve = s.curve;
        R.bar = reinterpret_cast<unsigned*>(base + off_bar[k]);
        if (grid[k]) {
            R.perm_g = reinterpret_cast<uint32_t*>(base + off_pg[k]);
            R.keys_g = base + off_kg[k];
        }
    }
    // grid group sizes: g CTAs per run, all co-resident
    std::vector<std::pair<Group*, std::vector<int>>> launches;  // (group, run subset)
    for (auto& kv : groups) {
        Group& gr = kv.second;
        if (!gr.grid) {
            launches.emplace_back(&gr, gr.runs);
            continue;
        }
        const int cap = run_kernel_capacity(gr.fit64, gr.qpl, gr.smem, true);
        if (cap <= 0) { set_err("grid kernel cannot be resident with %zu B of shared memory", gr.smem); return fail(APO_ERR_UNSUPPORTED); }
        // split into launches of at most `cap` runs (one CTA each at least)
        for (size_t i = 0; i < gr.runs.size(); i += (size_t)cap) {
            std::vector<int> sub(gr.runs.begin() + i, gr.runs.begin() + std::min(gr.runs.size(), i + (size_t)cap));
            const int per = std::min(kMaxGridCtas, cap / (int)sub.size());
            for (int k : sub) {
                const int want = (specs[k].prm.ps + kGridMinRows - 1) / kGridMinRows;
                runs[k].g = std::max(1, std::min(per, want));
            }
            // one g per launch: the smallest over the subset
            int g = per;
            for (int k : sub) g = std::min(g, runs[k].g);
            for (int k : sub) runs[k].g = g;
            launches.emplace_back(&gr, sub);
        }
    }

    APO_CUDA(cudaMemcpyAsync(base + off_runs, runs.data(), sizeof(ApoRun) * n, cudaMemcpyHostToDevice, st));
    APO_CUDA(cudaMemcpyAsync(base + off_offs, offs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st));
    APO_CUDA(cudaMemsetAsync(base + off_ctrl, 0, sizeof(int) * 64, st));
    for (int k = 0; k < n; ++k) {
        APO_CUDA(cudaMemsetAsync(base + off_bar[k], 0, 16, st));
        const RunSpec& s = specs[k];
        if (s.flags & kFlagStepOut) {
            const size_t fsz = s.P->kind == APO_OBJ_OTSU ? 8 : 4;
            APO_CUDA(cudaMemcpy2DAsync(base + off_x0[k], (size_t)s.P->Dp * 4, s.X_in, (size_t)s.P->D * 4,
                                       (size_t)s.P->D * 4, s.prm.ps, cudaMemcpyDeviceToDevice, st));
            APO_CUDA(cudaMemcpyAsync(base + off_f0[k], s.F_in, s.prm.ps * fsz, cudaMemcpyDeviceToDevice, st));
        }
    }
    const ApoRun* d_runs = reinterpret_cast<const ApoRun*>(base + off_runs);
    cudaError_t e = launch_dr(d_runs, reinterpret_cast<const int*>(base + off_offs), n, n_work, max_ps_pad, st);
    if (e != cudaSuccess) { set_err("Dr selection launch failed: %s", cudaGetErrorString(e)); return fail(APO_ERR_CUDA); }

    // The run kernels index runs through a per-launch table: lay the runs of
    // each launch out contiguously in a second copy of the descriptors.
    size_t nl = launches.size();
    std::vector<ApoRun> ordered;
    std::vector<int> first(nl, 0);
    for (size_t l = 0; l < nl; ++l) {
        first[l] = (int)ordered.size();
        for (int k : launches[l].second) ordered.push_back(runs[k]);
    }
    ApoRun* d_ordered = nullptr;
    APO_CUDA(cudaMallocAsync(reinterpret_cast<void**>(&d_ordered), sizeof(ApoRun) * ordered.size(), st));
    if (nl > 64) { set_err("too many launch groups"); return fail(APO_ERR_INTERNAL); }
    e = cudaMemcpyAsync(d_ordered, ordered.data(), sizeof(ApoRun) * ordered.size(), cudaMemcpyHostToDevice, st);
    const bool timed = g_ev_before && g_ev_after && !(specs[0].flags & kFlagStepOut);
    if (timed && e == cudaSuccess) e = cudaEventRecord(g_ev_before, st);
    for (size_t l = 0; l < nl && e == cudaSuccess; ++l) {
        Group& gr = *launches[l].first;
        const int cnt = (int)launches[l].second.size();
        int* queue = reinterpret_cast<int*>(base + off_ctrl) + (int)l;
        if (gr.grid) {
            e = launch_run(d_ordered + first[l], cnt, ordered[first[l]].g, 0, queue, status, gr.smem, gr.fit64,
                           gr.qpl, st);
        } else {
            const int cap = run_kernel_capacity(gr.fit64, gr.qpl, gr.smem, false);
            if (cap <= 0) { e = cudaErrorInvalidConfiguration; break; }
            e = launch_run(d_ordered + first[l], cnt, 0, std::min(cap, cnt), queue, status, gr.smem, gr.fit64,
                           gr.qpl, st);
        }
    }
    if (timed && e == cudaSuccess) e = cudaEventRecord(g_ev_after, st);
    cudaFreeAsync(d_ordered, st);
    if (e != cudaSuccess) { set_err("run launch failed: %s", cudaGetErrorString(e)); return fail(APO_ERR_CUDA); }
    APO_CUDA(cudaFreeAsync(ws, st));
    return APO_OK;
}

apo_status read_device_status(int dev)
{
    int* s = device_status(dev);
    if (!s) return APO_ERR_OOM;
    int v = 0;
    APO_CUDA(cudaMemcpy(&v, s, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        cudaMemset(s, 0, sizeof(int));
        set_err("a device-side wait exceeded its limit");
        return (apo_status)v;
    }
    return APO_OK;
}

}  // namespace

// ----------------------------------------------------------------- runs
extern "C" apo_status apo_run_device(const apo_problem* P, const apo_params* p, void* stream, float* d_best_x,
                                     double* d_best_f, float* d_curve)
{
    apo_status rc = check_params(P, p);
    if (rc != APO_OK) return rc;
    if (!d_best_x || !d_best_f) { set_err("d_best_x and d_best_f must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    s.P = P; s.prm = *p; s.t_begin = 1; s.t_end = p->max_iter; s.flags = kFlagInit;
    s.best_x = d_best_x; s.best_f = d_best_f; s.curve = d_curve; s.X_in = nullptr; s.F_in = nullptr;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

extern "C" apo_status apo_run(const apo_problem* P, const apo_params* p, void* stream, float* best_x,
                              double* best_f, float* curve)
{
    apo_status rc = check_params(P, p);
    if (rc != APO_OK) return rc;
    if (!best_x || !best_f) { set_err("best_x and best_f must not be NULL"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bx = align_up((size_t)P->D * 4, 256), bc = (size_t)(p->max_iter + 1) * 4;
    void* out = nullptr;
    APO_CUDA(cudaMallocAsync(&out, bx + 256 + bc, st));
    unsigned char* b = static_cast<unsigned char*>(out);
    rc = apo_run_device(P, p, stream, reinterpret_cast<float*>(b), reinterpret_cast<double*>(b + bx),
                        curve ? reinterpret_cast<float*>(b + bx + 256) : nullptr);
    if (rc == APO_OK) {
        cudaError_t e = cudaMemcpyAsync(best_x, b, (size_t)P->D * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(best_f, b + bx, 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && curve) e = cudaMemcpyAsync(curve, b + bx + 256, bc, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { set_err("result copy failed: %s", cudaGetErrorString(e)); rc = APO_ERR_CUDA; }
    }
    cudaFreeAsync(out, st);
    if (rc == APO_OK) {
        cudaStreamSynchronize(st);
        rc = read_device_status(P->device);
    }
    return rc;
}

extern "C" apo_status apo_run_batch(const apo_problem* const* probs, const apo_params* params, int n_runs,
                                    void* stream, float* d_best_x, int x_stride, double* d_best_f,
                                    float* d_curves, int curve_stride)
{
    if (n_runs < 0 || (n_runs > 0 && (!probs || !params || !d_best_x || !d_best_f))) {
        set_err("invalid batch arguments");
        return APO_ERR_INVALID_ARG;
    }
    std::vector<RunSpec> specs(n_runs);
    for (int k = 0; k < n_runs; ++k) {
        apo_status rc = check_params(probs[k], &params[k]);
        if (rc != APO_OK) return rc;
        if (x_stride < probs[k]->D || (d_curves && curve_stride < params[k].max_iter + 1)) {
            set_err("x_stride / curve_stride too small for run %d", k);
            return APO_ERR_INVALID_ARG;
        }
        RunSpec& s = specs[k];
        s.P = probs[k]; s.prm = params[k]; s.t_begin = 1; s.t_end = params[k].max_iter; s.flags = kFlagInit;
        s.best_x = d_best_x + (size_t)k * x_stride;
        s.best_f = d_best_f + k;
        s.curve = d_curves ? d_curves + (size_t)k * curve_stride : nullptr;
        s.X_in = nullptr; s.F_in = nullptr;
    }
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

extern "C" apo_status apo_step(const apo_problem* P, const apo_params* p, int iter, void* stream, float* d_X,
                               void* d_F)
{
    apo_status rc = check_params(P, p);
    if (rc != APO_OK) return rc;
    if (iter < 1 || iter > p->max_iter) { set_err("iter must be in 1..max_iter"); return APO_ERR_INVALID_ARG; }
    if (!d_X || !d_F) { set_err("d_X and d_F must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    s.P = P; s.prm = *p; s.t_begin = iter; s.t_end = iter; s.flags = kFlagStepOut;
    s.best_x = nullptr; s.best_f = nullptr; s.curve = nullptr; s.X_in = d_X; s.F_in = d_F;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

namespace {

apo_status eval_common(const apo_problem* P, void* stream, int n, const float* d_X, void* d_F, int select,
                       float* d_Xsel, void* d_Fsel)
{
    if (!P || n < 0 || (n > 0 && (!d_X || !d_F))) { set_err("invalid evaluation arguments"); return APO_ERR_INVALID_ARG; }
    if (n == 0) return APO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    ApoRun R;
    std::memset(&R, 0, sizeof(R));
    R.prob = P->dev;
    R.plan = choose_plan(P, 0, false, false, kSmemMax);
    R.g = 1;
    void* d = nullptr;
    APO_CUDA(cudaMallocAsync(&d, sizeof(ApoRun), st));
    cudaError_t e = cudaMemcpyAsync(d, &R, sizeof(ApoRun), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_eval(static_cast<const ApoRun*>(d), n, d_X, d_F, select, d_Xsel, d_Fsel, R.plan.total,
                        P->kind == APO_OBJ_OTSU, 1, st);
    cudaFreeAsync(d, st);
    if (e != cudaSuccess) { set_err("evaluation launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    return APO_OK;
}

}  // namespace

extern "C" apo_status apo_evaluate(const apo_problem* P, void* stream, const float* d_X, int n, void* d_F)
{
    return eval_common(P, stream, n, d_X, d_F, 0, nullptr, nullptr);
}

extern "C" apo_status apo_clamp_eval_select(const apo_problem* P, void* stream, int n, float* d_X, void* d_F,
                                            float* d_Xnew, void* d_Fnew)
{
    if (n > 0 && (!d_X || !d_F || !d_Xnew || !d_Fnew)) { set_err("NULL buffer"); return APO_ERR_INVALID_ARG; }
    return eval_common(P, stream, n, d_Xnew, d_Fnew, 1, d_X, d_F);
}

extern "C" apo_status apo_histogram_u8(const uint8_t* d_pixels, int64_t n_pixels_per_image, int n_images,
                                       int32_t* d_hist, void* stream)
{
    if (n_images < 0 || n_pixels_per_image < 0 || n_pixels_per_image >= (1ll << 31)) {
        set_err("invalid histogram sizes");
        return APO_ERR_INVALID_ARG;
    }
    if (n_images > 65535) { set_err("at most 65535 images per call"); return APO_ERR_UNSUPPORTED; }
    if (n_images > 0 && (!d_hist || (n_pixels_per_image > 0 && !d_pixels))) { set_err("NULL buffer"); return APO_ERR_INVALID_ARG; }
    if (n_images == 0) return APO_OK;
    const cudaError_t e = launch_histogram_u8(d_pixels, n_pixels_per_image, n_images, d_hist,
                                              static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { set_err("histogram launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    return APO_OK;
}

extern "C" apo_status apo_set_timing_events(void* before, void* after)
{
    if ((before == nullptr) != (after == nullptr)) { set_err("set both events or neither"); return APO_ERR_INVALID_ARG; }
    g_ev_before = static_cast<cudaEvent_t>(before);
    g_ev_after = static_cast<cudaEvent_t>(after);
    return APO_OK;
}

extern "C" apo_status apo_philox4x32_10(const uint32_t* d_ctr, uint32_t key0, uint32_t key1, int n, uint32_t* d_out,
                                        void* stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) { set_err("invalid Philox arguments"); return APO_ERR_INVALID_ARG; }
    const cudaError_t e = launch_philox(d_ctr, key0, key1, n, d_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { set_err("Philox launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    return APO_OK;
}
