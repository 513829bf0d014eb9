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

#include <cuda_fp16.h>

#include "../../include/apo.h"
#include "apo_big.h"
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
constexpr size_t kSmemMax = 232448 - 2048;  // dynamic part; the kernels use < 1 KB of static shared memory
// Runs with a larger population go to the cooperative grid launch.
constexpr int kQueueMaxPs = 1024;
// Minimum protozoa per CTA in grid mode.
constexpr int kGridMinRows = 8;
// A run launched alone uses the grid kernel from this population size on.
constexpr int kGridSingleMinPs = 128;
// barrier words of different runs on different L2 lines (their CTAs poll them)
constexpr size_t kBarStride = 256;

// Optional timing events around the iteration-loop kernels.
cudaEvent_t g_ev_before = nullptr, g_ev_after = nullptr;

}  // namespace

cudaEvent_t apo::big_timing_before() { return g_ev_before; }
cudaEvent_t apo::big_timing_after() { return g_ev_after; }


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

namespace {
apo_status get_thr_dr(int ps, int form, int dev, const uint32_t** out);
apo_status get_sched(int T, int dev, const uint32_t** thr_ah, const float** fsc, const float** nsc);
int* device_status(int dev);
}  // namespace

apo_status apo::sched_tables(int ps, int pdr_form, int T, const uint32_t** thr_dr, const uint32_t** thr_ah,
                      const float** fsc, const float** nsc)
{
    int dev = 0;
    cudaGetDevice(&dev);
    apo_status rc = get_thr_dr(ps, pdr_form, dev, thr_dr);
    if (rc == APO_OK) rc = get_sched(T, dev, thr_ah, fsc, nsc);
    return rc;
}

int* apo::device_status_word()
{
    int dev = 0;
    cudaGetDevice(&dev);
    return device_status(dev);
}

void apo::set_last_error(const char* msg) { set_err("%s", msg); }

// ---------------------------------------------------------- problems
namespace {

// 2^(target - e) for v < 2^e: brings max |value| = v just below 2^target
// (1 for v == 0).  A power of two, so scaling by it is exact.
float pow2_scale(double v, int target)
{
    if (!(v > 0.0)) return 1.f;
    int e = 0;
    std::frexp(v, &e);
    e = std::min(std::max(target - e, -100), 100);
    return (float)std::ldexp(1.0, e);
}

uint16_t half_bits(__half h)
{
    const __half_raw r = h;
    return r.x;
}

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
    if (kind < APO_OBJ_SPHERE || kind > APO_OBJ_GRIEWANK) { set_err("unknown objective kind %d", kind); return APO_ERR_INVALID_ARG; }
    if (D < 1) { set_err("D must be >= 1"); return APO_ERR_INVALID_ARG; }
    if (kind == APO_OBJ_OTSU ? D > APO_MAX_OTSU_THRESHOLDS : D > APO_MAX_DIM) {
        set_err("D = %d exceeds the supported maximum", D);
        return APO_ERR_UNSUPPORTED;
    }
    // dimensions above kSmallMaxDim take the large-dimension path
    const bool big = D > kSmallMaxDim;
    if (big && kind == APO_OBJ_COMPOSITION) {
        set_err("the composition objective supports D <= %d", kSmallMaxDim);
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
    const int Kp = (D + 63) & ~63;
    const int bws = split_words(D);
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
    size_t off_o[kMaxComp] = {}, off_mt[kMaxComp] = {}, off_ew[kMaxComp] = {}, off_bh[kMaxComp] = {},
           off_bl[kMaxComp] = {}, off_th[kMaxComp] = {}, off_tl[kMaxComp] = {}, off_gh = 0, off_gl = 0;
    bool has_mt[kMaxComp] = {}, has_tc[kMaxComp] = {};
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
        if (big) {
            // the large-dimension GEMM operand: B = msc M' (M' = M with the
            // hybrid's rows permuted, the identity when M is absent) split
            // into fp16 hi + lo, row n = output dimension, K-contiguous [D][Kp]
            double mmax = 0.0, ymax = 0.0;
            if (M)
                for (size_t i = 0; i < (size_t)D * D; ++i) mmax = std::max(mmax, (double)std::fabs(M[i]));
            else
                mmax = 1.0;
            for (int d = 0; d < D; ++d)
                ymax = std::max(ymax, std::max(std::fabs((double)ubf[d] - (double)o[d]),
                                               std::fabs((double)lbf[d] - (double)o[d])));
            const float msc = pow2_scale(mmax, 12), ysc = pow2_scale(ymax, 10);
            std::vector<uint16_t> gh((size_t)D * Kp, 0), gl((size_t)D * Kp, 0);
            for (int n = 0; n < D; ++n) {
                const int row = perm_rows ? perm[n] : n;
                for (int kk = 0; kk < D; ++kk) {
                    const float v = (M ? M[(size_t)row * D + kk] : (kk == row ? 1.f : 0.f)) * msc;
                    const __half hh = __float2half_rn(v);
                    const __half ll = __float2half_rn(v - __half2float(hh));
                    gh[(size_t)n * Kp + kk] = half_bits(hh);
                    gl[(size_t)n * Kp + kk] = half_bits(ll);
                }
            }
            off_gh = add(gh.data(), gh.size() * 2);
            off_gl = add(gl.data(), gl.size() * 2);
            comps[k].ysc = ysc;
            comps[k].zsc = 1.f / (ysc * msc);
            any_rot = 1;
        } else if (M || perm_rows) {
            std::vector<float> mt((size_t)Dp * Np, 0.f);
            for (int c = 0; c < D; ++c) {
                const int row = perm_rows ? perm[c] : c;
                for (int j = 0; j < D; ++j)
                    mt[(size_t)j * Np + c] = M ? M[(size_t)row * D + j] : (j == row ? 1.f : 0.f);
            }
            off_mt[k] = add(mt.data(), (size_t)Dp * Np * 4);
            has_mt[k] = true;
            any_rot = 1;
            // The tensor-core copy: B[k][n] = msc MT[k][n] split into fp16
            // hi + lo, per column n as k pairs (lower half = even k) in the
            // fragment order of pair_word.  msc
            // brings max |B| below 2^12 and ysc the largest |x - o| over the
            // box below 2^10 (64x headroom for points outside the box), so
            // every part and product stays inside the fp16 / fp32 ranges.
            double mmax = 0.0, ymax = 0.0;
            for (float v : mt) mmax = std::max(mmax, (double)std::fabs(v));
            for (int d = 0; d < D; ++d)
                ymax = std::max(ymax, std::max(std::fabs((double)ubf[d] - (double)o[d]),
                                               std::fabs((double)lbf[d] - (double)o[d])));
            const float msc = pow2_scale(mmax, 12), ysc = pow2_scale(ymax, 10);
            // A single component with D <= kTcM also gets the parts in the
            // canonical UMMA layout (rows n, columns k; Np x Np each).
            const bool tc = ncomp == 1 && Np <= kTcM;
            std::vector<uint32_t> bh((size_t)Np * bws, 0u), bl((size_t)Np * bws, 0u);
            std::vector<uint16_t> th(tc ? (size_t)Np * Np : 0, 0), tl(tc ? (size_t)Np * Np : 0, 0);
            for (int n = 0; n < D; ++n)
                for (int kk = 0; kk < D; ++kk) {
                    const float v = mt[(size_t)kk * Np + n] * msc;
                    const __half hh = __float2half_rn(v);
                    const __half ll = __float2half_rn(v - __half2float(hh));
                    const uint32_t sh = (kk & 1) ? 16u : 0u;
                    bh[(size_t)n * bws + pair_word(kk / 2)] |= (uint32_t)half_bits(hh) << sh;
                    bl[(size_t)n * bws + pair_word(kk / 2)] |= (uint32_t)half_bits(ll) << sh;
                    if (tc) {
                        th[umma_off(n, kk, Np) / 2] = half_bits(hh);
                        tl[umma_off(n, kk, Np) / 2] = half_bits(ll);
                    }
                }
            off_bh[k] = add(bh.data(), bh.size() * 4);
            off_bl[k] = add(bl.data(), bl.size() * 4);
            if (tc) {
                off_th[k] = add(th.data(), th.size() * 2);
                off_tl[k] = add(tl.data(), tl.size() * 2);
                has_tc[k] = true;
            }
            comps[k].ysc = ysc;
            comps[k].zsc = 1.f / (ysc * msc);   // a power of two: exact
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
        case APO_OBJ_BENTCIGAR: s1 = D; s2 = D; nell = 0; break;   // weights 1, 10^6, 10^6, ...
        default: break;   // HGBat, Griewank: their own epilogue (form)
        }
        std::vector<float> ew(Dp, 1.f);
        for (int d = 0; d < nell; ++d)
            ew[d] = nell > 1 ? (float)std::pow(10.0, 6.0 * (double)d / (double)(nell - 1)) : 1.f;
        if (form == APO_OBJ_BENTCIGAR)
            for (int d = 1; d < D; ++d) ew[d] = 1e6f;
        if (form == APO_OBJ_GRIEWANK)   // cos(y / sqrt(i)) = cospi(y / (pi sqrt(i)))
            for (int d = 0; d < D; ++d) ew[d] = (float)(1.0 / (M_PI * std::sqrt((double)(d + 1))));
        comps[k].form = form;
        off_ew[k] = add(ew.data(), Dp * 4);
        comps[k].s1 = s1;
        comps[k].s2 = s2;
        if (kind == APO_OBJ_COMPOSITION) {
            const double sg = obj->comp_sigma[k];
            comps[k].inv_2Dsig2 = (float)(1.0 / (2.0 * (double)D * sg * sg));
            comps[k].bias = (float)obj->comp_bias[k];
        }
    }
    size_t off_p0 = 0, off_p1 = 0, off_hist = 0, off_tab = 0;
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
        off_tab = add(nullptr, (size_t)kOtsuTabSize * 8);
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
    if (e == cudaSuccess && kind == APO_OBJ_OTSU) {
        e = launch_otsu_table(reinterpret_cast<const long long*>(base + off_p0),
                              reinterpret_cast<const long long*>(base + off_p1),
                              reinterpret_cast<double*>(base + off_tab), 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cudaFree(P->mem);
        delete P;
        set_err("problem upload failed: %s", cudaGetErrorString(e));
        return APO_ERR_CUDA;
    }
    DevProblem& dp = P->dev;
    std::memset(&dp, 0, sizeof(dp));
    dp.D = D; dp.Dp = Dp; dp.Np = Np; dp.kind = kind; dp.ncomp = ncomp; dp.bws = bws; dp.Kp = Kp;
    dp.lb = reinterpret_cast<const float*>(base + off_lb);
    dp.ub = reinterpret_cast<const float*>(base + off_ub);
    for (int k = 0; k < ncomp; ++k) {
        dp.comp[k] = comps[k];
        dp.comp[k].o = reinterpret_cast<const float*>(base + off_o[k]);
        dp.comp[k].MT = has_mt[k] ? reinterpret_cast<const float*>(base + off_mt[k]) : nullptr;
        dp.comp[k].Bh = has_mt[k] ? reinterpret_cast<const uint32_t*>(base + off_bh[k]) : nullptr;
        dp.comp[k].Bl = has_mt[k] ? reinterpret_cast<const uint32_t*>(base + off_bl[k]) : nullptr;
        dp.comp[k].Th = has_tc[k] ? reinterpret_cast<const uint4*>(base + off_th[k]) : nullptr;
        dp.comp[k].Tl = has_tc[k] ? reinterpret_cast<const uint4*>(base + off_tl[k]) : nullptr;
        dp.comp[k].ew = reinterpret_cast<const float*>(base + off_ew[k]);
    }
    if (big) {
        dp.comp[0].Gh = reinterpret_cast<const uint16_t*>(base + off_gh);
        dp.comp[0].Gl = reinterpret_cast<const uint16_t*>(base + off_gl);
    }
    if (kind == APO_OBJ_OTSU) {
        dp.P0 = reinterpret_cast<const long long*>(base + off_p0);
        dp.P1 = reinterpret_cast<const long long*>(base + off_p1);
        dp.otsu_tab = reinterpret_cast<const double*>(base + off_tab);
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
    fill_sched_tables(ps, form, 0, thr.data(), nullptr, nullptr, nullptr);
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
        fill_sched_tables(0, 0, T, nullptr, a.data(), f.data(), n.data());
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

// Validates a problem and its params (normalize_params) and writes the
// resolved params (max_fes turned into max_iter) to *q.
apo_status check_params(const apo_problem* P, const apo_params* p, apo_params* q)
{
    if (!P || !p) { set_err("problem and params must not be NULL"); return APO_ERR_INVALID_ARG; }
    if (const char* why = normalize_params(p, q)) { set_err("%s", why); return APO_ERR_INVALID_ARG; }
    if (q->ps > (1 << 20)) { set_err("ps above 2^20 is not supported"); return APO_ERR_UNSUPPORTED; }
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

// One kernel launch of a prepared set of runs.
struct LaunchInfo {
    int first, count;   // runs [first, first + count) of the launch-ordered descriptors
    bool grid, fit64;
    int qpl, g, ctas;
    size_t smem;
    bool cluster;       // grid kernel with one thread-block cluster of g CTAs per run
};

// Everything a set of runs needs on the device, planned and uploaded once;
// launching it then only clears control words and launches kernels.
struct Prepared {
    void* ws = nullptr;         // workspace (descriptors, Dr masks, state, barriers)
    bool ws_async = false;      // allocated with cudaMallocAsync
    ApoRun* d_runs = nullptr;   // launch-ordered descriptors
    int* d_offs = nullptr;
    int* d_ctrl = nullptr;      // queue counters (one per launch)
    unsigned char* d_bars = nullptr;  // barrier words, one 256-byte line per run
    int n = 0, n_work = 0, max_ps_pad = 1;
    std::vector<LaunchInfo> launches;
    std::vector<RunSpec> order;           // specs in launch order
    std::vector<size_t> x0_off, f0_off;   // step mode: state copies
    size_t queue_smem_cap = 0;            // work-queue shared-memory budget used
};

void release_prepared(Prepared& PR, cudaStream_t st);

// Plans the launches: runs with ps > kQueueMaxPs go to the cooperative grid
// kernel; the others to the work-queue kernel, resident in shared memory when
// their layout fits `queue_budget` bytes.  queue_ctas_per_sm limits the
// persistent work-queue grid (0 = occupancy limit).
apo_status prepare_runs(const std::vector<RunSpec>& specs_in, cudaStream_t st, bool async_alloc,
                        size_t queue_budget, int queue_ctas_per_sm, Prepared* out, int cluster_ps = 0,
                        int cluster_size = 0)
{
    Prepared& PR = *out;
    const int n = (int)specs_in.size();
    PR.n = n;
    if (n == 0) return APO_OK;
    int dev = 0, sms = 0;
    APO_CUDA(cudaGetDevice(&dev));
    APO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (queue_budget == 0 || queue_budget > kSmemMax) queue_budget = kSmemMax;

    // per-run layout and kernel class
    struct Cls { bool grid, fit64; int qpl; bool cluster; };
    std::vector<SmemPlan> plans(n);
    std::vector<Cls> cls(n);
    for (int k = 0; k < n; ++k) {
        const RunSpec& s = specs_in[k];
        const int ps = s.prm.ps;
        const bool f64 = s.P->kind == APO_OBJ_OTSU;
        if (s.P->D > kSmallMaxDim) {
            set_err("prepared batches support D <= %d (run D = %d with apo_run_batch)", kSmallMaxDim, s.P->D);
            return APO_ERR_UNSUPPORTED;
        }
        // a lone run of a large population spreads over many CTAs; runs of
        // at least cluster_ps protozoa in a batch take a cluster of
        // cluster_size CTAs each (the grid kernel, launched as clusters)
        const bool big_pop = ps > kQueueMaxPs || (n == 1 && ps >= kGridSingleMinPs);
        const bool cl = !big_pop && cluster_ps > 0 && cluster_size >= 2 && ps >= cluster_ps;
        cls[k] = {big_pop || cl, f64, f64 ? 1 : qpl_of(s.P), cl};
        if (cls[k].grid) {
            plans[k] = choose_plan(s.P, ps, false, true, kSmemMax);
        } else {
            plans[k] = choose_plan(s.P, ps, true, false, queue_budget);
            if (plans[k].total > queue_budget) plans[k] = choose_plan(s.P, ps, false, false, queue_budget);
        }
        if (plans[k].total > kSmemMax) { set_err("problem needs too much shared memory (ps %d)", ps); return APO_ERR_UNSUPPORTED; }
    }
    // launch groups: one per kernel class; work-queue runs longest first
    std::map<std::tuple<int, int, int, int>, std::vector<int>> groups;
    for (int k = 0; k < n; ++k)
        groups[std::make_tuple((int)cls[k].grid, (int)cls[k].cluster, (int)cls[k].fit64, cls[k].qpl)].push_back(k);
    std::vector<int> order;
    for (auto& kv : groups) {
        std::vector<int>& v = kv.second;
        const Cls c = cls[v[0]];
        size_t smem = 0;
        for (int k : v) smem = std::max<size_t>(smem, plans[k].total);
        if (!c.grid) {
            auto cost = [&](int k) {
                const double D = specs_in[k].P->D;
                return (double)specs_in[k].prm.ps * (D * D + 40.0 * D) * (specs_in[k].t_end - specs_in[k].t_begin + 1);
            };
            std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return cost(a) > cost(b); });
            int cap = run_kernel_capacity(c.fit64, c.qpl, smem, false);
            if (cap <= 0) { set_err("work-queue kernel cannot be resident with %zu B of shared memory", smem); return APO_ERR_UNSUPPORTED; }
            if (queue_ctas_per_sm > 0) cap = std::min(cap, queue_ctas_per_sm * sms);
            PR.launches.push_back({(int)order.size(), (int)v.size(), false, c.fit64, c.qpl, 1, std::min(cap, (int)v.size()), smem,
                                   false});
            order.insert(order.end(), v.begin(), v.end());
            PR.queue_smem_cap = std::max(PR.queue_smem_cap, smem);
            continue;
        }
        if (c.cluster) {
            // longest first, as in the work queue: clusters are scheduled in order
            auto cost = [&](int k) {
                const double D = specs_in[k].P->D;
                return (double)specs_in[k].prm.ps * (D * D + 40.0 * D) * (specs_in[k].t_end - specs_in[k].t_begin + 1);
            };
            std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return cost(a) > cost(b); });
            PR.launches.push_back({(int)order.size(), (int)v.size(), true, c.fit64, c.qpl, cluster_size,
                                   (int)v.size() * cluster_size, smem, true});
            order.insert(order.end(), v.begin(), v.end());
            continue;
        }
        const int cap = run_kernel_capacity(c.fit64, c.qpl, smem, true);
        if (cap <= 0) { set_err("grid kernel cannot be resident with %zu B of shared memory", smem); return APO_ERR_UNSUPPORTED; }
        for (size_t i = 0; i < v.size(); i += (size_t)cap) {
            const int cnt = (int)std::min(v.size() - i, (size_t)cap);
            int g = std::min(kMaxGridCtas, cap / cnt);
            for (int j = 0; j < cnt; ++j) {
                const int want = (specs_in[v[i + j]].prm.ps + kGridMinRows - 1) / kGridMinRows;
                g = std::max(1, std::min(g, want));
            }
            PR.launches.push_back({(int)order.size(), cnt, true, c.fit64, c.qpl, g, cnt * g, smem, false});
            order.insert(order.end(), v.begin() + i, v.begin() + i + cnt);
        }
    }
    PR.order.resize(n);
    for (int i = 0; i < n; ++i) PR.order[i] = specs_in[order[i]];
    const std::vector<RunSpec>& specs = PR.order;

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
    const size_t off_ctrl = take(sizeof(int) * std::max<size_t>(PR.launches.size(), 1));
    const size_t off_bars = take(kBarStride * (size_t)n);
    std::vector<size_t> off_dr(n), off_x0(n), off_x1(n), off_f0(n), off_f1(n), off_pg(n), off_kg(n);
    std::vector<int> offs(n + 1, 0);
    for (int i = 0; i < n; ++i) {
        const RunSpec& s = specs[i];
        const int k = order[i];
        const int ps = s.prm.ps, Dp = s.P->Dp;
        const size_t fsz = s.P->kind == APO_OBJ_OTSU ? 8 : 4;
        const int W = (ps + 31) / 32;
        off_dr[i] = take(sizeof(uint32_t) * W * (size_t)(s.t_end + 1));
        // a run that starts from a given state reads it from global memory
        const bool need_global = !plans[k].resident || !(s.flags & kFlagInit);
        off_x0[i] = need_global ? take((size_t)ps * Dp * 4) : 0;
        off_x1[i] = need_global ? take((size_t)ps * Dp * 4) : 0;
        off_f0[i] = need_global ? take(ps * fsz) : 0;
        off_f1[i] = need_global ? take(ps * fsz) : 0;
        off_pg[i] = cls[k].grid ? take((size_t)ps * 4) : 0;
        off_kg[i] = cls[k].grid ? take((size_t)ps * (fsz == 8 ? 16 : 8)) : 0;
        offs[i] = PR.n_work;
        PR.n_work += s.t_end - s.t_begin + 1;
        PR.max_ps_pad = std::max(PR.max_ps_pad, next_pow2(ps));
    }
    offs[n] = PR.n_work;
    if (async_alloc) {
        APO_CUDA(cudaMallocAsync(&PR.ws, std::max<size_t>(off, 256), st));
    } else {
        APO_CUDA(cudaMalloc(&PR.ws, std::max<size_t>(off, 256)));
    }
    PR.ws_async = async_alloc;
    unsigned char* base = static_cast<unsigned char*>(PR.ws);
    PR.d_runs = reinterpret_cast<ApoRun*>(base + off_runs);
    PR.d_offs = reinterpret_cast<int*>(base + off_offs);
    PR.d_ctrl = reinterpret_cast<int*>(base + off_ctrl);
    PR.d_bars = base + off_bars;

    std::vector<ApoRun> runs(n);
    std::vector<int> g_of(n, 1);
    for (const LaunchInfo& L : PR.launches)
        for (int i = L.first; i < L.first + L.count; ++i) g_of[i] = L.g;
    for (int i = 0; i < n; ++i) {
        const RunSpec& s = specs[i];
        const int k = order[i];
        ApoRun& R = runs[i];
        std::memset(&R, 0, sizeof(R));
        R.prob = s.P->dev;
        R.plan = plans[k];
        R.ps = s.prm.ps; R.np = s.prm.np; R.T = s.prm.max_iter; R.pdr_form = s.prm.pdr_form;
        R.pair_policy = s.prm.pair_policy;
        R.pf_max = s.prm.pf_max; R.seed = s.prm.seed; R.run = s.prm.run;
        R.t_begin = s.t_begin; R.t_end = s.t_end; R.flags = s.flags;
        R.g = g_of[i];
        const uint32_t* thr_dr = nullptr;
        const uint32_t* thr_ah = nullptr;
        const float *fsc = nullptr, *nsc = nullptr;
        apo_status rc = get_thr_dr(R.ps, R.pdr_form, dev, &thr_dr);
        if (rc == APO_OK) rc = get_sched(R.T, dev, &thr_ah, &fsc, &nsc);
        if (rc != APO_OK) { release_prepared(PR, st); return rc; }
        R.thr_dr = thr_dr; R.thr_ah = thr_ah; R.fsc = fsc; R.nsc = nsc;
        R.drmask = reinterpret_cast<const uint32_t*>(base + off_dr[i]);
        if (off_x0[i] || off_x1[i]) {
            R.X[0] = reinterpret_cast<float*>(base + off_x0[i]);
            R.X[1] = reinterpret_cast<float*>(base + off_x1[i]);
            R.F[0] = base + off_f0[i];
            R.F[1] = base + off_f1[i];
        }
        R.X_out = s.X_in;
        R.F_out = s.F_in;
        R.best_x = s.best_x; R.best_f = s.best_f; R.curve = s.curve;
        R.bar = reinterpret_cast<unsigned*>(PR.d_bars + kBarStride * (size_t)i);
        if (cls[k].grid) {
            R.perm_g = reinterpret_cast<uint32_t*>(base + off_pg[i]);
            R.keys_g = base + off_kg[i];
        }
    }
    PR.x0_off = off_x0;
    PR.f0_off = off_f0;
    cudaError_t e;
    if (async_alloc) {
        e = cudaMemcpyAsync(PR.d_runs, runs.data(), sizeof(ApoRun) * n, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(PR.d_offs, offs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, st);
    } else {
        e = cudaMemcpy(PR.d_runs, runs.data(), sizeof(ApoRun) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(PR.d_offs, offs.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        set_err("descriptor upload failed: %s", cudaGetErrorString(e));
        release_prepared(PR, st);
        return APO_ERR_CUDA;
    }
    return APO_OK;
}

// Clears the control words and launches the Dr_index and iteration-loop
// kernels of a prepared set of runs on `st` (no allocation, no host copy:
// capturable in a CUDA graph when no run is in step mode).
apo_status launch_prepared(const Prepared& PR, cudaStream_t st)
{
    if (PR.n == 0) return APO_OK;
    int dev = 0;
    APO_CUDA(cudaGetDevice(&dev));
    int* status = device_status(dev);
    if (!status) { set_err("status word allocation failed"); return APO_ERR_OOM; }
    unsigned char* base = static_cast<unsigned char*>(PR.ws);
    APO_CUDA(cudaMemsetAsync(PR.d_ctrl, 0, sizeof(int) * std::max<size_t>(PR.launches.size(), 1), st));
    APO_CUDA(cudaMemsetAsync(PR.d_bars, 0, kBarStride * (size_t)PR.n, st));
    for (int i = 0; i < PR.n; ++i) {
        const RunSpec& s = PR.order[i];
        if ((s.flags & kFlagInit) || !s.X_in) continue;   // runs from a given state: copy it in
        const size_t fsz = s.P->kind == APO_OBJ_OTSU ? 8 : 4;
        APO_CUDA(cudaMemcpy2DAsync(base + PR.x0_off[i], (size_t)s.P->Dp * 4, s.X_in, (size_t)s.P->D * 4,
                                   (size_t)s.P->D * 4, s.prm.ps, cudaMemcpyDeviceToDevice, st));
        APO_CUDA(cudaMemcpyAsync(base + PR.f0_off[i], s.F_in, s.prm.ps * fsz, cudaMemcpyDeviceToDevice, st));
    }
    cudaError_t e = launch_dr(PR.d_runs, PR.d_offs, PR.n, PR.n_work, PR.max_ps_pad, st);
    if (e != cudaSuccess) { set_err("Dr selection launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    const bool timed = g_ev_before && g_ev_after && !(PR.order[0].flags & (kFlagStepOut | kFlagStateOut));
    if (timed) APO_CUDA(cudaEventRecord(g_ev_before, st));
    for (size_t l = 0; l < PR.launches.size() && e == cudaSuccess; ++l) {
        const LaunchInfo& L = PR.launches[l];
        e = launch_run(PR.d_runs + L.first, L.count, L.grid ? L.g : 0, L.ctas, PR.d_ctrl + l, status, L.smem,
                       L.fit64, L.qpl, st, L.cluster);
    }
    if (e != cudaSuccess) { set_err("run launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    if (timed) APO_CUDA(cudaEventRecord(g_ev_after, st));
    return APO_OK;
}

void release_prepared(Prepared& PR, cudaStream_t st)
{
    if (PR.ws) {
        if (PR.ws_async) cudaFreeAsync(PR.ws, st);
        else cudaFree(PR.ws);
    }
    PR.ws = nullptr;
}

// The large-dimension runs of a request (D > kSmallMaxDim), in groups of at
// most kBigMaxRuns sharing (t_begin, t_end, flags), on the stage sequence of
// apo_big.cu.
apo_status launch_big_runs(const std::vector<RunSpec>& specs, cudaStream_t st)
{
    std::vector<BigSpec> all;
    for (const RunSpec& s : specs) {
        if (s.prm.ps > kBigMaxPs) {
            set_err("ps = %d: the large-dimension path supports ps <= %d", s.prm.ps, kBigMaxPs);
            return APO_ERR_UNSUPPORTED;
        }
        BigSpec b{};
        b.P = s.P; b.prm = s.prm; b.ps = s.prm.ps; b.t_begin = s.t_begin; b.t_end = s.t_end;
        b.flags = ((s.flags & kFlagInit) ? kBigInit : 0) | ((s.flags & kFlagStepOut) ? kBigStepOut : 0) |
                  ((s.flags & kFlagStateOut) ? kBigStateOut : 0);
        b.best_x = s.best_x; b.best_f = s.best_f; b.curve = s.curve;
        b.X_in = s.X_in; b.F_in = static_cast<const float*>(s.F_in);
        b.X_out = s.X_in; b.F_out = static_cast<float*>(s.F_in);
        all.push_back(b);
    }
    std::vector<char> done(all.size(), 0);
    for (size_t i = 0; i < all.size(); ++i) {
        if (done[i]) continue;
        std::vector<BigSpec> group;
        for (size_t j = i; j < all.size() && (int)group.size() < kBigMaxRuns; ++j) {
            if (done[j] || all[j].t_begin != all[i].t_begin || all[j].t_end != all[i].t_end ||
                all[j].flags != all[i].flags)
                continue;
            group.push_back(all[j]);
            done[j] = 1;
        }
        char msg[256] = "";
        const apo_status rc = big_run_group(group, st, msg, sizeof(msg));
        if (rc != APO_OK) { set_err("%s", msg); return rc; }
    }
    return APO_OK;
}

// Plans, allocates (stream-ordered) and launches a set of runs on one stream.
apo_status launch_runs(std::vector<RunSpec>& specs_in, cudaStream_t st)
{
    std::vector<RunSpec> specs, big;
    for (const RunSpec& s : specs_in) (s.P->D > kSmallMaxDim ? big : specs).push_back(s);
    apo_status rc = APO_OK;
    if (!specs.empty()) {
        Prepared PR;
        rc = prepare_runs(specs, st, true, 0, 0, &PR);
        if (rc != APO_OK) return rc;
        rc = launch_prepared(PR, st);
        release_prepared(PR, st);
    }
    if (rc == APO_OK && !big.empty()) rc = launch_big_runs(big, st);
    return rc;
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
    apo_params q;
    apo_status rc = check_params(P, p, &q);
    if (rc != APO_OK) return rc;
    if (!d_best_x || !d_best_f) { set_err("d_best_x and d_best_f must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    s.P = P; s.prm = q; s.t_begin = 1; s.t_end = q.max_iter; s.flags = kFlagInit;
    s.best_x = d_best_x; s.best_f = d_best_f; s.curve = d_curve; s.X_in = nullptr; s.F_in = nullptr;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

extern "C" apo_status apo_run(const apo_problem* P, const apo_params* p, void* stream, float* best_x,
                              double* best_f, float* curve)
{
    apo_params q;
    apo_status rc = check_params(P, p, &q);
    if (rc != APO_OK) return rc;
    if (!best_x || !best_f) { set_err("best_x and best_f must not be NULL"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bx = align_up((size_t)P->D * 4, 256), bc = (size_t)(q.max_iter + 1) * 4;
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
    // (planning as in apo_batch_create, with a stream-ordered workspace)
    if (n_runs < 0 || (n_runs > 0 && (!probs || !params || !d_best_x || !d_best_f))) {
        set_err("invalid batch arguments");
        return APO_ERR_INVALID_ARG;
    }
    std::vector<RunSpec> specs(n_runs);
    for (int k = 0; k < n_runs; ++k) {
        apo_params q;
        apo_status rc = check_params(probs[k], &params[k], &q);
        if (rc != APO_OK) return rc;
        if (x_stride < probs[k]->D || (d_curves && curve_stride < q.max_iter + 1)) {
            set_err("x_stride / curve_stride too small for run %d", k);
            return APO_ERR_INVALID_ARG;
        }
        RunSpec& s = specs[k];
        s.P = probs[k]; s.prm = q; s.t_begin = 1; s.t_end = q.max_iter; s.flags = kFlagInit;
        s.best_x = d_best_x + (size_t)k * x_stride;
        s.best_f = d_best_f + k;
        s.curve = d_curves ? d_curves + (size_t)k * curve_stride : nullptr;
        s.X_in = nullptr; s.F_in = nullptr;
    }
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

struct apo_batch {
    std::vector<RunSpec> specs;
    apo_batch_options opt;
    Prepared prep;
};

namespace {

apo_status batch_specs(const apo_problem* const* probs, const apo_params* params, int n_runs, float* d_best_x,
                       int x_stride, double* d_best_f, float* d_curves, int curve_stride,
                       std::vector<RunSpec>& specs)
{
    if (n_runs < 0 || (n_runs > 0 && (!probs || !params || !d_best_x || !d_best_f))) {
        set_err("invalid batch arguments");
        return APO_ERR_INVALID_ARG;
    }
    specs.resize(n_runs);
    for (int k = 0; k < n_runs; ++k) {
        apo_params q;
        apo_status rc = check_params(probs[k], &params[k], &q);
        if (rc != APO_OK) return rc;
        if (x_stride < probs[k]->D || (d_curves && curve_stride < q.max_iter + 1)) {
            set_err("x_stride / curve_stride too small for run %d", k);
            return APO_ERR_INVALID_ARG;
        }
        RunSpec& s = specs[k];
        s.P = probs[k]; s.prm = q; s.t_begin = 1; s.t_end = q.max_iter; s.flags = kFlagInit;
        s.best_x = d_best_x + (size_t)k * x_stride;
        s.best_f = d_best_f + k;
        s.curve = d_curves ? d_curves + (size_t)k * curve_stride : nullptr;
        s.X_in = nullptr; s.F_in = nullptr;
    }
    return APO_OK;
}

}  // namespace

extern "C" apo_status apo_batch_create(const apo_problem* const* probs, const apo_params* params, int n_runs,
                                       float* d_best_x, int x_stride, double* d_best_f, float* d_curves,
                                       int curve_stride, const apo_batch_options* opt, apo_batch** out)
{
    if (!out) { set_err("out is NULL"); return APO_ERR_INVALID_ARG; }
    *out = nullptr;
    apo_batch* B = new apo_batch();
    apo_status rc = batch_specs(probs, params, n_runs, d_best_x, x_stride, d_best_f, d_curves, curve_stride, B->specs);
    if (rc != APO_OK) { delete B; return rc; }
    B->opt.smem_budget = opt ? opt->smem_budget : 0;
    B->opt.ctas_per_sm = opt ? opt->ctas_per_sm : 0;
    B->opt.cluster_ps = opt ? opt->cluster_ps : 0;
    B->opt.cluster_size = opt ? opt->cluster_size : 0;
    if (B->opt.cluster_ps < 0 || (B->opt.cluster_ps > 0 && (B->opt.cluster_size < 2 || B->opt.cluster_size > 8))) {
        delete B;
        set_err("cluster_size must be 2..8 when cluster_ps > 0");
        return APO_ERR_INVALID_ARG;
    }
    rc = prepare_runs(B->specs, 0, false, B->opt.smem_budget, B->opt.ctas_per_sm, &B->prep, B->opt.cluster_ps,
                      B->opt.cluster_size);
    if (rc != APO_OK) { delete B; return rc; }
    int dev = 0;
    cudaGetDevice(&dev);
    if (!device_status(dev)) { release_prepared(B->prep, 0); delete B; set_err("status word allocation failed"); return APO_ERR_OOM; }
    *out = B;
    return APO_OK;
}

extern "C" apo_status apo_batch_launch(apo_batch* B, void* stream)
{
    if (!B) { set_err("batch is NULL"); return APO_ERR_INVALID_ARG; }
    return launch_prepared(B->prep, static_cast<cudaStream_t>(stream));
}

extern "C" void apo_batch_destroy(apo_batch* B)
{
    if (!B) return;
    cudaDeviceSynchronize();
    release_prepared(B->prep, 0);
    delete B;
}

extern "C" apo_status apo_batch_autotune(apo_batch* B, void* stream, int probe_iters, apo_batch_options* chosen)
{
    if (!B || probe_iters < 1) { set_err("invalid autotune arguments"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<RunSpec> probe = B->specs;
    for (RunSpec& s : probe) s.t_end = std::min(s.t_end, probe_iters);
    // candidates: the work-queue budget for 1 to 4 CTAs per SM, each with
    // every run in the work queue (one CTA per run) or with the larger runs
    // on one cluster of 2 or 4 CTAs each
    const size_t budgets[4] = {kSmemMax, 113 * 1024, 75 * 1024, 56 * 1024};
    const int clusters[4][2] = {{0, 0}, {256, 2}, {256, 4}, {384, 4}};
    cudaEvent_t e0, e1;
    APO_CUDA(cudaEventCreate(&e0));
    APO_CUDA(cudaEventCreate(&e1));
    float best_ms = 1e30f;
    apo_batch_options best = B->opt;
    for (size_t cand = 0; cand < 16; ++cand) {
        const size_t c = cand / 4;
        const int cps = clusters[cand % 4][0], csz = clusters[cand % 4][1];
        Prepared PR;
        if (prepare_runs(probe, st, false, budgets[c], 0, &PR, cps, csz) != APO_OK) continue;
        float ms = 1e30f;
        bool ok = launch_prepared(PR, st) == APO_OK;   // warm-up
        for (int rep = 0; rep < 2 && ok; ++rep) {
            cudaEventRecord(e0, st);
            ok = launch_prepared(PR, st) == APO_OK;
            cudaEventRecord(e1, st);
            if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                ms = std::min(ms, t);
            }
        }
        cudaStreamSynchronize(st);
        release_prepared(PR, st);
        if (ok && ms < best_ms) {
            best_ms = ms;
            best.smem_budget = budgets[c];
            best.ctas_per_sm = 0;
            best.cluster_ps = cps;
            best.cluster_size = csz;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms >= 1e30f) { set_err("no autotune candidate ran"); return APO_ERR_INTERNAL; }
    cudaStreamSynchronize(st);
    release_prepared(B->prep, st);
    B->prep = Prepared();
    B->opt = best;
    apo_status rc = prepare_runs(B->specs, st, false, best.smem_budget, best.ctas_per_sm, &B->prep, best.cluster_ps,
                                 best.cluster_size);
    if (rc != APO_OK) return rc;
    if (chosen) *chosen = best;
    return APO_OK;
}

extern "C" apo_status apo_step(const apo_problem* P, const apo_params* p, int iter, void* stream, float* d_X,
                               void* d_F)
{
    apo_params q;
    apo_status rc = check_params(P, p, &q);
    if (rc != APO_OK) return rc;
    if (iter < 1 || iter > q.max_iter) { set_err("iter must be in 1..max_iter"); return APO_ERR_INVALID_ARG; }
    if (!d_X || !d_F) { set_err("d_X and d_F must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    s.P = P; s.prm = q; s.t_begin = iter; s.t_end = iter; s.flags = kFlagStepOut;
    s.best_x = nullptr; s.best_f = nullptr; s.curve = nullptr; s.X_in = d_X; s.F_in = d_F;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

extern "C" int apo_effective_iterations(const apo_params* p)
{
    apo_params q;
    if (normalize_params(p, &q)) return -1;
    return q.max_iter;
}

extern "C" apo_status apo_init_state(const apo_problem* P, const apo_params* p, void* stream, float* d_X, void* d_F)
{
    apo_params q;
    apo_status rc = check_params(P, p, &q);
    if (rc != APO_OK) return rc;
    if (!d_X || !d_F) { set_err("d_X and d_F must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    // no iteration: initialisation, then the state in protozoon order
    s.P = P; s.prm = q; s.t_begin = 1; s.t_end = 0; s.flags = kFlagInit | kFlagStateOut;
    s.best_x = nullptr; s.best_f = nullptr; s.curve = nullptr; s.X_in = d_X; s.F_in = d_F;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

extern "C" apo_status apo_run_from_state(const apo_problem* P, const apo_params* p, int t_begin, int t_end,
                                         void* stream, float* d_X, void* d_F, float* d_best_x, double* d_best_f,
                                         float* d_curve)
{
    apo_params q;
    apo_status rc = check_params(P, p, &q);
    if (rc != APO_OK) return rc;
    if (t_begin < 1 || t_end < t_begin - 1 || t_end > q.max_iter) {
        set_err("need 1 <= t_begin and t_begin - 1 <= t_end <= T (T = %d)", q.max_iter);
        return APO_ERR_INVALID_ARG;
    }
    if (!d_X || !d_F) { set_err("d_X and d_F must not be NULL"); return APO_ERR_INVALID_ARG; }
    std::vector<RunSpec> specs(1);
    RunSpec& s = specs[0];
    s.P = P; s.prm = q; s.t_begin = t_begin; s.t_end = t_end; s.flags = kFlagStateOut;
    // the kernels write curve[t - 1] for t = t_begin .. t_end + 1: index the
    // caller's array from iteration t_begin - 1
    s.curve = d_curve ? reinterpret_cast<float*>(reinterpret_cast<uintptr_t>(d_curve) -
                                                 sizeof(float) * (size_t)(t_begin - 1))
                      : nullptr;
    s.best_x = d_best_x; s.best_f = d_best_f; s.X_in = d_X; s.F_in = d_F;
    return launch_runs(specs, static_cast<cudaStream_t>(stream));
}

namespace {

apo_status eval_common(const apo_problem* P, void* stream, int n, const float* d_X, void* d_F, int select,
                       float* d_Xsel, void* d_Fsel)
{
    if (!P || n < 0 || (n > 0 && (!d_X || !d_F))) { set_err("invalid evaluation arguments"); return APO_ERR_INVALID_ARG; }
    if (n == 0) return APO_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (P->D > kSmallMaxDim) {
        if (select) { set_err("apo_clamp_eval_select supports D <= %d", kSmallMaxDim); return APO_ERR_UNSUPPORTED; }
        if (n > kBigMaxPs) { set_err("at most %d rows per evaluation at D > %d", kBigMaxPs, kSmallMaxDim); return APO_ERR_UNSUPPORTED; }
        BigSpec b{};
        b.P = P; b.ps = n; b.flags = kBigEval; b.X_in = d_X; b.F_out = static_cast<float*>(d_F);
        b.prm.ps = n; b.prm.np = 1; b.prm.max_iter = 1;
        char msg[256] = "";
        const apo_status rc = big_run_group(std::vector<BigSpec>{b}, st, msg, sizeof(msg));
        if (rc != APO_OK) set_err("%s", msg);
        return rc;
    }
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

extern "C" apo_status apo_large_stage_timing(int on, double* ms, long long* launches)
{
    big_stage_timing(on, ms, launches);
    return APO_OK;
}

extern "C" apo_status apo_set_timing_events(void* before, void* after)
{
    if ((before == nullptr) != (after == nullptr)) { set_err("set both events or neither"); return APO_ERR_INVALID_ARG; }
    g_ev_before = static_cast<cudaEvent_t>(before);
    g_ev_after = static_cast<cudaEvent_t>(after);
    return APO_OK;
}

extern "C" apo_status apo_barrier_selftest(int ctas_launched, int ctas_expected, int rounds, void* stream)
{
    if (ctas_launched < 1 || ctas_expected < 1 || ctas_launched > ctas_expected || ctas_expected > 1024 ||
        rounds < 1 || rounds > 100000) {
        set_err("barrier self-test: 1 <= launched <= expected <= 1024, 1 <= rounds <= 100000");
        return APO_ERR_INVALID_ARG;
    }
    int dev = 0;
    APO_CUDA(cudaGetDevice(&dev));
    int* status = device_status(dev);
    if (!status) { set_err("status word allocation failed"); return APO_ERR_OOM; }
    // every launched CTA must be resident at once for the barrier to complete
    int sms = 0;
    APO_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (ctas_launched > sms) { set_err("barrier self-test: at most one CTA per SM"); return APO_ERR_INVALID_ARG; }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* bar = nullptr;
    APO_CUDA(cudaMalloc(&bar, 256));
    cudaError_t e = cudaMemsetAsync(bar, 0, 256, st);
    if (e == cudaSuccess) e = launch_barrier_test(bar, ctas_launched, ctas_expected, rounds, status, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(bar);
    if (e != cudaSuccess) { set_err("barrier self-test launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    return read_device_status(dev);
}

extern "C" apo_status apo_philox4x32_10(const uint32_t* d_ctr, uint32_t key0, uint32_t key1, int n, uint32_t* d_out,
                                        void* stream)
{
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) { set_err("invalid Philox arguments"); return APO_ERR_INVALID_ARG; }
    const cudaError_t e = launch_philox(d_ctr, key0, key1, n, d_out, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) { set_err("Philox launch failed: %s", cudaGetErrorString(e)); return APO_ERR_CUDA; }
    return APO_OK;
}
