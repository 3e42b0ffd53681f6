// fpt_abi.cu -- the C ABI of libfpt.so (declared in include/fpt.h).
//
// Owns the device state of a context: packed noise tables, model and run
// descriptors, per-trajectory result arrays, histogram scratch, a private
// stream and the cache of captured CUDA graphs (one per launch shape).
#include "fpt_internal.h"
#include "fpt_mlp.cuh"

#include <cuda_runtime.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <unordered_map>
#include <mutex>
#include <new>
#include <set>
#include <stdexcept>
#include <string>
#include <tuple>
#include <vector>

using namespace fpt_dev;

namespace {

std::mutex g_err_mu;
std::string g_init_err = "no error";

struct TableHost {
    bool ready = false;
    bool n_indexed = false;    // grid in time since the start (noise window)
    bool rank2 = false;        // full-rank 2-D noise: S = S_phiphi, T = S_phipi, C = S_pipi
    int M = 0;
    double lo = 0, h = 0;
    std::vector<double> S, T, C;
    // float4 entries on the device: M (1-D: value + slope) or M + 1 (2-D: values)
    int entries() const { return rank2 ? M + 1 : M; }
};

using GraphKey = std::tuple<int, int, int, int, size_t, int, int, int, long long, int>;

// A captured fpt_run. The stepper takes its EmParams by value (Philox round
// keys, launch-uniform model constants), and a graph keeps the values it was
// captured with; before a replay whose parameters differ, the stepper node of
// the executable graph is given the new ones.
struct RunGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t stepper = nullptr;
    EmParams params;
};

}  // namespace

struct fpt_ctx {
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    std::string err = "no error";

    std::vector<fpt_model> models;
    std::vector<fpt_model_info> infos;
    std::vector<TableHost> tables;

    // device buffers
    ModelDev *d_models = nullptr;
    float4 *d_tables = nullptr;
    size_t tables_cap = 0;
    std::vector<int> table_offset;
    std::vector<int> region_entries;   // float4 entries per model: noise table (+ drift table)
    std::vector<ModelDev> h_models;    // host copy of the device model descriptors
    RunDev *d_runs = nullptr;
    RunDev *h_runs = nullptr;           // pinned staging
    unsigned long long *d_cursor = nullptr;
    int *d_flags = nullptr;             // launch flag words (kFlag* in fpt_internal.h)
    int *h_flags = nullptr;             // pinned copy
    int32_t *d_nsteps = nullptr;
    double *d_logw = nullptr;
    uint8_t *d_status = nullptr;
    double *d_N = nullptr;
    long long unit_cap = 0;

    // histogram scratch
    unsigned long long *d_hmax = nullptr;
    double *d_hmom = nullptr;
    double *d_hscal = nullptr;
    double *d_hout = nullptr;
    double *h_hout = nullptr;
    // caller-data histogram scratch
    int32_t *d_xn = nullptr;
    double *d_xlw = nullptr;
    uint8_t *d_xst = nullptr;
    long long x_cap = 0;

    // last run
    std::vector<RunDev> last_runs;
    int last_n_runs = 0;
    long long last_total = 0;
    bool last_valid = false;
    cudaStream_t last_stream = nullptr;
    cudaEvent_t run_done = nullptr;

    fpt_launch launch{512, 0, 32, 1, 0.0};
    std::map<GraphKey, RunGraph> graphs;

    // learned-proposal training scratch
    float *d_records = nullptr;
    long long rec_cap = 0;
    unsigned long long *d_rec_cursor = nullptr;
    bool record_mode = false;
    double *d_Y = nullptr;
    long long y_cap = 0;
    float *d_coef = nullptr;
    long long coef_cap = 0;
    double *d_acc = nullptr;
    float *d_grad = nullptr;
    float *d_tmp = nullptr;
    long long tmp_cap = 0;
    // deterministic backward: per-block partial gradients, record order
    float *d_gpart = nullptr;
    uint32_t *d_perm = nullptr;
    long long perm_cap = 0;
    int *d_cnt = nullptr;
    long long cnt_cap = 0;
    long long *d_off = nullptr;
    long long off_cap = 0;
    int *d_rec_err = nullptr;

    // device memory of the context, counted against an optional limit
    std::unordered_map<void *, size_t> dev_sizes;
    size_t dev_bytes = 0;
    size_t dev_limit = 0;           // 0: no limit
    size_t refused_bytes = 0;       // last request the limit refused
};

static fpt_status fail(fpt_ctx *c, fpt_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else {
        std::lock_guard<std::mutex> g(g_err_mu);
        g_init_err = msg;
    }
    return s;
}

static fpt_status cuda_fail(fpt_ctx *c, cudaError_t e, const char *what)
{
    fpt_status s = (e == cudaErrorMemoryAllocation) ? FPT_E_NOMEM : FPT_E_CUDA;
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    if (c && e == cudaErrorMemoryAllocation && c->refused_bytes) {
        msg += " (context memory limit " + std::to_string(c->dev_limit) + " bytes: " +
               std::to_string(c->dev_bytes) + " in use, " + std::to_string(c->refused_bytes) + " requested)";
        c->refused_bytes = 0;
    }
    return fail(c, s, msg);
}

#ifdef FPT_CHECKS
// A failed device bounds check makes the call that observes it (fpt_sync, a
// histogram) return FPT_E_STATE.
static fpt_status take_checks(fpt_ctx *c)
{
    int word = 0;
    const cudaError_t e = checks_take(&word);
    if (e != cudaSuccess) return cuda_fail(c, e, "reading the bounds-check word");
    if (!word) return FPT_OK;
    std::string what;
    if (word & kCheckTable) what += " noise-table index;";
    if (word & kCheckDriftTable) what += " drift-table index;";
    if (word & kCheckUnit) what += " trajectory index;";
    if (word & kCheckBin) what += " histogram bin;";
    return fail(c, FPT_E_STATE, "device bounds check failed (FPT_CHECKS):" + what + " results are invalid");
}
#endif

// Device allocations of a context: counted, and refused like an out-of-memory
// cudaMalloc when they would take the context past its limit.
template <class T>
static cudaError_t dev_malloc(fpt_ctx *ctx, T **p, size_t bytes)
{
    if (ctx->dev_limit && ctx->dev_bytes + bytes > ctx->dev_limit) {
        ctx->refused_bytes = bytes;
        return cudaErrorMemoryAllocation;
    }
    const cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), bytes);
    if (e == cudaSuccess) {
        ctx->dev_sizes[*p] = bytes;
        ctx->dev_bytes += bytes;
    }
    return e;
}

static void dev_free(fpt_ctx *ctx, void *p)
{
    if (!p) return;
    auto it = ctx->dev_sizes.find(p);
    if (it != ctx->dev_sizes.end()) {
        ctx->dev_bytes -= it->second;
        ctx->dev_sizes.erase(it);
    }
    cudaFree(p);
}

#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

static void clear_graphs(fpt_ctx *ctx)
{
    for (auto &kv : ctx->graphs) {
        cudaGraphExecDestroy(kv.second.exec);
        cudaGraphDestroy(kv.second.graph);
    }
    ctx->graphs.clear();
}

static void free_all(fpt_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    clear_graphs(ctx);
    dev_free(ctx, ctx->d_models);
    dev_free(ctx, ctx->d_tables);
    dev_free(ctx, ctx->d_runs);
    cudaFreeHost(ctx->h_runs);
    dev_free(ctx, ctx->d_cursor);
    dev_free(ctx, ctx->d_flags);
    cudaFreeHost(ctx->h_flags);
    dev_free(ctx, ctx->d_nsteps);
    dev_free(ctx, ctx->d_logw);
    dev_free(ctx, ctx->d_status);
    dev_free(ctx, ctx->d_N);
    dev_free(ctx, ctx->d_hmax);
    dev_free(ctx, ctx->d_hmom);
    dev_free(ctx, ctx->d_hscal);
    dev_free(ctx, ctx->d_hout);
    cudaFreeHost(ctx->h_hout);
    dev_free(ctx, ctx->d_records);
    dev_free(ctx, ctx->d_rec_cursor);
    dev_free(ctx, ctx->d_Y);
    dev_free(ctx, ctx->d_coef);
    dev_free(ctx, ctx->d_acc);
    dev_free(ctx, ctx->d_grad);
    dev_free(ctx, ctx->d_tmp);
    dev_free(ctx, ctx->d_gpart);
    dev_free(ctx, ctx->d_perm);
    dev_free(ctx, ctx->d_cnt);
    dev_free(ctx, ctx->d_off);
    dev_free(ctx, ctx->d_rec_err);
    dev_free(ctx, ctx->d_xn);
    dev_free(ctx, ctx->d_xlw);
    dev_free(ctx, ctx->d_xst);
    if (ctx->run_done) cudaEventDestroy(ctx->run_done);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
}

static size_t hout_doubles() { return (size_t)10 * kMaxBins + 16; }

template <class T>
static fpt_status ensure_dev(fpt_ctx *ctx, T *&ptr, long long &cap, long long need)
{
    if (need <= cap) return FPT_OK;
    CK(cudaStreamSynchronize(ctx->stream));
    dev_free(ctx, ptr);
    ptr = nullptr;
    cap = 0;
    CK(dev_malloc(ctx, &ptr, sizeof(T) * need));
    cap = need;
    return FPT_OK;
}

__global__ void grad_norm_kernel(const float *g, int n, double *out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += (double)g[i] * g[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
        *out = t;
    }
}

extern "C" {

#ifdef FPT_CHECKS
const char *fpt_version(void) { return "fpt-gb300 0.1 (sm_103a, FPT_CHECKS)"; }
#else
const char *fpt_version(void) { return "fpt-gb300 0.1 (sm_103a)"; }
#endif

const char *fpt_last_error(const fpt_ctx *ctx)
{
    if (ctx) return ctx->err.c_str();
    std::lock_guard<std::mutex> g(g_err_mu);
    return g_init_err.c_str();
}

fpt_status fpt_resolve_model(const fpt_model *model, fpt_model_info *out)
{
    if (!model || !out) return fail(nullptr, FPT_E_INVALID, "null argument");
    std::string v = fpt_host::validate_model(*model);
    if (!v.empty()) return fail(nullptr, FPT_E_INVALID, v);
    try {
        *out = fpt_host::resolve(*model);
    } catch (const std::exception &e) {
        return fail(nullptr, FPT_E_INVALID, e.what());
    }
    if (!(out->phi_in > out->phi_end)) return fail(nullptr, FPT_E_INVALID, "resolved phi_in <= phi_end");
    return FPT_OK;
}

static fpt_status table_args(int kind, int n_points, double sigma, double phi_lo, double phi_hi,
                             const double *uS, const double *uT, std::string &msg)
{
    if (kind != FPT_TABLE_DESITTER && kind != FPT_TABLE_BESSEL && kind != FPT_TABLE_USER &&
        kind != FPT_TABLE_BESSEL_N && kind != FPT_TABLE_USER_N) {
        msg = "unknown table kind";
        return FPT_E_INVALID;
    }
    if ((kind == FPT_TABLE_BESSEL_N || kind == FPT_TABLE_USER_N) &&
        (std::isnan(phi_lo) || !(phi_lo >= 0.0))) {
        msg = "N-indexed tables need 0 <= N_lo < N_hi";
        return FPT_E_INVALID;
    }
    if (n_points < 2 || n_points > kMaxTablePoints) { msg = "n_points out of [2, 8192]"; return FPT_E_INVALID; }
    if (std::isnan(phi_lo) != std::isnan(phi_hi)) { msg = "phi_lo and phi_hi must both be set or both NaN"; return FPT_E_INVALID; }
    if (!std::isnan(phi_lo) && !(phi_hi > phi_lo && std::isfinite(phi_lo) && std::isfinite(phi_hi))) {
        msg = "need finite phi_lo < phi_hi";
        return FPT_E_INVALID;
    }
    if ((kind == FPT_TABLE_BESSEL || kind == FPT_TABLE_BESSEL_N) && !(sigma > 0 && sigma <= 10)) {
        msg = "sigma out of (0, 10]";
        return FPT_E_INVALID;
    }
    if (kind == FPT_TABLE_USER || kind == FPT_TABLE_USER_N) {
        if (!uS || !uT) { msg = "USER tables need user_S and user_Spi"; return FPT_E_INVALID; }
        for (int j = 0; j < n_points; ++j)
            if (!(uS[j] >= 0) || !std::isfinite(uS[j]) || !std::isfinite(uT[j])) {
                msg = "USER table values must be finite with S >= 0";
                return FPT_E_INVALID;
            }
    }
    return FPT_OK;
}

static fpt_status build_host_table(const fpt_model &m, const fpt_model_info &info, int kind,
                                   int n_points, double sigma, double phi_lo, double phi_hi,
                                   const double *uS, const double *uT, TableHost &t, std::string &msg)
{
    try {
        if (kind == FPT_TABLE_USER || kind == FPT_TABLE_USER_N) {
            double lo = std::isnan(phi_lo) ? info.phi_end : phi_lo;
            double hi = std::isnan(phi_hi) ? info.phi_in : phi_hi;
            if (!(hi > lo)) { msg = "need phi_hi > phi_lo"; return FPT_E_INVALID; }
            t.S.assign(uS, uS + n_points);
            t.T.assign(uT, uT + n_points);
            t.lo = lo;
            t.h = (hi - lo) / (n_points - 1);
        } else {
            fpt_host::build_table(m, kind, n_points, sigma, phi_lo, phi_hi, t.S, t.T, t.lo, t.h);
        }
    } catch (const std::exception &e) {
        msg = e.what();
        return FPT_E_INVALID;
    }
    t.M = n_points;
    t.ready = true;
    t.n_indexed = (kind == FPT_TABLE_BESSEL_N || kind == FPT_TABLE_USER_N);
    return FPT_OK;
}

fpt_status fpt_table_build(const fpt_model *model, int32_t kind, int32_t n_points, double sigma,
                           double phi_lo, double phi_hi, double *out_S, double *out_Spi)
{
    if (!model || !out_S || !out_Spi) return fail(nullptr, FPT_E_INVALID, "null argument");
    std::string msg;
    if (kind == FPT_TABLE_USER || kind == FPT_TABLE_USER_N)
        return fail(nullptr, FPT_E_INVALID, "USER tables are not built");
    fpt_status s = table_args(kind, n_points, sigma, phi_lo, phi_hi, nullptr, nullptr, msg);
    if (s != FPT_OK) return fail(nullptr, s, msg);
    fpt_model_info info;
    if ((s = fpt_resolve_model(model, &info)) != FPT_OK) return s;
    TableHost t;
    s = build_host_table(*model, info, kind, n_points, sigma, phi_lo, phi_hi, nullptr, nullptr, t, msg);
    if (s != FPT_OK) return fail(nullptr, s, msg);
    std::copy(t.S.begin(), t.S.end(), out_S);
    std::copy(t.T.begin(), t.T.end(), out_Spi);
    return FPT_OK;
}

// Full-rank (2-D) tables: arguments, host build and the copy-out of the
// three planes (S_phiphi, S_phipi, S_pipi).
static fpt_status table2_args(int kind, int n_points, double sigma, double phi_lo, double phi_hi,
                              const double *uS, std::string &msg)
{
    if (kind != FPT_TABLE_NUMERIC && kind != FPT_TABLE_USER2) { msg = "unknown 2-D table kind"; return FPT_E_INVALID; }
    if (n_points < 2 || n_points > kMaxTablePoints) { msg = "n_points out of [2, 8192]"; return FPT_E_INVALID; }
    if (std::isnan(phi_lo) != std::isnan(phi_hi)) { msg = "phi_lo and phi_hi must both be set or both NaN"; return FPT_E_INVALID; }
    if (!std::isnan(phi_lo) && !(phi_hi > phi_lo && std::isfinite(phi_lo) && std::isfinite(phi_hi))) {
        msg = "need finite phi_lo < phi_hi";
        return FPT_E_INVALID;
    }
    if (kind == FPT_TABLE_NUMERIC && !(sigma > 0 && sigma <= 10)) { msg = "sigma out of (0, 10]"; return FPT_E_INVALID; }
    if (kind == FPT_TABLE_USER2) {
        if (!uS) { msg = "USER2 tables need user_S"; return FPT_E_INVALID; }
        for (int j = 0; j < 3 * n_points; ++j)
            if (!std::isfinite(uS[j])) { msg = "USER2 table values must be finite"; return FPT_E_INVALID; }
    }
    return FPT_OK;
}

static fpt_status build_host_table2(const fpt_model &m, const fpt_model_info &info, int kind,
                                    int n_points, double sigma, double phi_lo, double phi_hi,
                                    const double *uS, TableHost &t, std::string &msg)
{
    try {
        if (kind == FPT_TABLE_USER2) {
            double lo = std::isnan(phi_lo) ? info.phi_end : phi_lo;
            double hi = std::isnan(phi_hi) ? info.phi_in : phi_hi;
            if (!(hi > lo)) { msg = "need phi_hi > phi_lo"; return FPT_E_INVALID; }
            t.S.assign(uS, uS + n_points);
            t.T.assign(uS + n_points, uS + 2 * n_points);
            t.C.assign(uS + 2 * n_points, uS + 3 * n_points);
            t.lo = lo;
            t.h = (hi - lo) / (n_points - 1);
        } else {
            fpt_host::build_table2(m, kind, n_points, sigma, phi_lo, phi_hi, t.S, t.T, t.C, t.lo, t.h);
        }
    } catch (const std::exception &e) {
        msg = e.what();
        return FPT_E_INVALID;
    }
    t.M = n_points;
    t.ready = true;
    t.rank2 = true;
    return FPT_OK;
}

static void copy_planes(const TableHost &t, double *out)
{
    std::copy(t.S.begin(), t.S.end(), out);
    std::copy(t.T.begin(), t.T.end(), out + t.M);
    std::copy(t.C.begin(), t.C.end(), out + 2 * t.M);
}

fpt_status fpt_table_build2(const fpt_model *model, int32_t kind, int32_t n_points, double sigma,
                            double phi_lo, double phi_hi, double *out_S)
{
    if (!model || !out_S) return fail(nullptr, FPT_E_INVALID, "null argument");
    if (kind != FPT_TABLE_NUMERIC) return fail(nullptr, FPT_E_INVALID, "only NUMERIC tables are built");
    std::string msg;
    fpt_status s = table2_args(kind, n_points, sigma, phi_lo, phi_hi, nullptr, msg);
    if (s != FPT_OK) return fail(nullptr, s, msg);
    fpt_model_info info;
    if ((s = fpt_resolve_model(model, &info)) != FPT_OK) return s;
    TableHost t;
    s = build_host_table2(*model, info, kind, n_points, sigma, phi_lo, phi_hi, nullptr, t, msg);
    if (s != FPT_OK) return fail(nullptr, s, msg);
    copy_planes(t, out_S);
    return FPT_OK;
}

// ---------------------------------------------------------------------------
// Classical delta N (host only)
// ---------------------------------------------------------------------------
fpt_status fpt_power_spectrum(const fpt_model *model, double sigma, int32_t n, const double *N_s,
                              double N_eval, double *out_PR)
{
    if (!model || !N_s || !out_PR || n < 0) return fail(nullptr, FPT_E_INVALID, "null argument or negative n");
    if (!(sigma > 0 && sigma <= 10)) return fail(nullptr, FPT_E_INVALID, "sigma out of (0, 10]");
    fpt_model_info info;
    fpt_status s = fpt_resolve_model(model, &info);
    if (s != FPT_OK) return s;
    try {
        fpt_host::power_spectrum(*model, sigma, n, N_s, N_eval, out_PR);
    } catch (const std::exception &e) {
        return fail(nullptr, FPT_E_INVALID, e.what());
    }
    return FPT_OK;
}

fpt_status fpt_classical_dn(const fpt_model *model, double sigma, int32_t n_k, double N_eval,
                            fpt_classical *out)
{
    if (!model || !out) return fail(nullptr, FPT_E_INVALID, "null argument");
    if (n_k < 3 || n_k > 4097 || !(n_k & 1)) return fail(nullptr, FPT_E_INVALID, "n_k must be odd in [3, 4097]");
    if (!(sigma > 0 && sigma <= 10)) return fail(nullptr, FPT_E_INVALID, "sigma out of (0, 10]");
    fpt_model_info info;
    fpt_status s = fpt_resolve_model(model, &info);
    if (s != FPT_OK) return s;
    try {
        fpt_host::classical_dn(*model, sigma, n_k, N_eval, out->sigma_R2, out->eps2_in, out->eps2_end,
                               out->N_in, out->N_end);
    } catch (const std::exception &e) {
        return fail(nullptr, FPT_E_INVALID, e.what());
    }
    return FPT_OK;
}

// Eq. (2.20); eps2 = 0 is the Gaussian limit.
static double classical_pdf_one(double dN, double s2, double eps2)
{
    const double c = 1.0 / std::sqrt(2.0 * 3.14159265358979323846 * s2);
    if (eps2 == 0.0) return c * std::exp(-dN * dN / (2.0 * s2));
    const double R = -(2.0 / eps2) * -std::expm1(-0.5 * eps2 * dN);
    return c * std::exp(-R * R / (2.0 * s2) - 0.5 * eps2 * dN);
}

fpt_status fpt_classical_pdf(const double *dN, int64_t n, double sigma_R2, double eps2, double *out)
{
    if ((!dN || !out) && n > 0) return fail(nullptr, FPT_E_INVALID, "null argument");
    if (n < 0 || !(sigma_R2 > 0) || !std::isfinite(sigma_R2) || !std::isfinite(eps2))
        return fail(nullptr, FPT_E_INVALID, "need n >= 0, sigma_R2 > 0 and finite eps2");
    for (int64_t i = 0; i < n; ++i) out[i] = classical_pdf_one(dN[i], sigma_R2, eps2);
    return FPT_OK;
}

// chi^2 of ln P: sum over bins with pdf > 0 and se > 0 of
// ((ln pdf_b - ln P(dN_b; sigma_R2, eps2)) / (se_b / pdf_b))^2.
static double fit_chi2(const double *dN, const double *pdf, const double *se, int n, double s2, double e2,
                       int *used)
{
    double chi2 = 0.0;
    int k = 0;
    for (int b = 0; b < n; ++b) {
        if (!(pdf[b] > 0) || !(se[b] > 0)) continue;
        const double lp = std::log(classical_pdf_one(dN[b], s2, e2));
        const double r = (std::log(pdf[b]) - lp) * pdf[b] / se[b];
        chi2 += r * r;
        ++k;
    }
    if (used) *used = k;
    return chi2;
}

fpt_status fpt_fit_eps2(const double *dN, const double *pdf, const double *se, int32_t n_bins,
                        double sigma_R2, double eps2_lo, double eps2_hi, double *eps2_out,
                        double *chi2_out, int32_t *bins_used)
{
    if (!dN || !pdf || !se || !eps2_out || n_bins < 1) return fail(nullptr, FPT_E_INVALID, "null argument or no bins");
    if (!(sigma_R2 > 0) || !(eps2_hi > eps2_lo) || !std::isfinite(eps2_lo) || !std::isfinite(eps2_hi))
        return fail(nullptr, FPT_E_INVALID, "need sigma_R2 > 0 and eps2_lo < eps2_hi");
    // golden-section search for the minimum of chi^2 on [eps2_lo, eps2_hi]
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double a = eps2_lo, b = eps2_hi;
    double c = b - g * (b - a), d = a + g * (b - a);
    double fc = fit_chi2(dN, pdf, se, n_bins, sigma_R2, c, nullptr);
    double fd = fit_chi2(dN, pdf, se, n_bins, sigma_R2, d, nullptr);
    for (int it = 0; it < 200 && b - a > 1e-12 * std::max(1.0, std::fabs(a)); ++it) {
        if (fc < fd) { b = d; d = c; fd = fc; c = b - g * (b - a); fc = fit_chi2(dN, pdf, se, n_bins, sigma_R2, c, nullptr); }
        else { a = c; c = d; fc = fd; d = a + g * (b - a); fd = fit_chi2(dN, pdf, se, n_bins, sigma_R2, d, nullptr); }
    }
    const double e = 0.5 * (a + b);
    int used = 0;
    const double chi2 = fit_chi2(dN, pdf, se, n_bins, sigma_R2, e, &used);
    if (used == 0) return fail(nullptr, FPT_E_INVALID, "no bin with pdf > 0 and se > 0");
    *eps2_out = e;
    if (chi2_out) *chi2_out = chi2;
    if (bins_used) *bins_used = used;
    return FPT_OK;
}

fpt_status fpt_init_model(fpt_ctx **pctx, const fpt_model *models, int32_t n_models, int32_t device)
{
    if (!pctx) return fail(nullptr, FPT_E_INVALID, "null ctx pointer");
    *pctx = nullptr;
    if (!models || n_models < 1 || n_models > kMaxModels)
        return fail(nullptr, FPT_E_INVALID, "n_models out of [1, 64]");
    std::vector<fpt_model_info> infos(n_models);
    for (int i = 0; i < n_models; ++i) {
        fpt_status s = fpt_resolve_model(&models[i], &infos[i]);
        if (s != FPT_OK) {
            std::lock_guard<std::mutex> g(g_err_mu);
            g_init_err = "model " + std::to_string(i) + ": " + g_init_err;
            return s;
        }
    }
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0)
        return fail(nullptr, FPT_E_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    if (device < 0 || device >= ndev) return fail(nullptr, FPT_E_INVALID, "device index out of range");
    fpt_ctx *ctx = new (std::nothrow) fpt_ctx;
    if (!ctx) return fail(nullptr, FPT_E_NOMEM, "host allocation failed");
    ctx->device = device;
    ctx->models.assign(models, models + n_models);
    ctx->infos = infos;
    ctx->tables.resize(n_models);
    ctx->table_offset.assign(n_models, 0);
    ctx->region_entries.assign(n_models, 0);
    auto bail = [&](cudaError_t err, const char *what) {
        fpt_status s = (err == cudaErrorMemoryAllocation) ? FPT_E_NOMEM : FPT_E_CUDA;
        fail(nullptr, s, std::string(what) + ": " + cudaGetErrorString(err));
        free_all(ctx);
        delete ctx;
        return s;
    };
    if ((e = cudaSetDevice(device))) return bail(e, "cudaSetDevice");
    if ((e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device))) return bail(e, "attribute");
    if ((e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking))) return bail(e, "stream");
    if ((e = cudaEventCreateWithFlags(&ctx->run_done, cudaEventDisableTiming))) return bail(e, "event");
    if ((e = dev_malloc(ctx, &ctx->d_models, sizeof(ModelDev) * kMaxModels))) return bail(e, "cudaMalloc models");
    if ((e = dev_malloc(ctx, &ctx->d_runs, sizeof(RunDev) * kMaxRuns))) return bail(e, "cudaMalloc runs");
    if ((e = cudaMallocHost(&ctx->h_runs, sizeof(RunDev) * kMaxRuns))) return bail(e, "cudaMallocHost runs");
    if ((e = dev_malloc(ctx, &ctx->d_cursor, 64))) return bail(e, "cudaMalloc cursor");
    if ((e = dev_malloc(ctx, &ctx->d_flags, 64))) return bail(e, "cudaMalloc flags");
    if ((e = cudaMallocHost(&ctx->h_flags, 64))) return bail(e, "cudaMallocHost flags");
    if ((e = dev_malloc(ctx, &ctx->d_hmax, sizeof(unsigned long long) * (kMaxBins + 2)))) return bail(e, "cudaMalloc hist");
    if ((e = dev_malloc(ctx, &ctx->d_hmom, sizeof(double) * (size_t)kJackknife * kMaxBins * 5))) return bail(e, "cudaMalloc hist");
    if ((e = dev_malloc(ctx, &ctx->d_hscal, sizeof(double) * kJackknife * 16))) return bail(e, "cudaMalloc hist");
    if ((e = dev_malloc(ctx, &ctx->d_hout, sizeof(double) * hout_doubles()))) return bail(e, "cudaMalloc hist");
    if ((e = cudaMallocHost(&ctx->h_hout, sizeof(double) * hout_doubles()))) return bail(e, "cudaMallocHost hist");
    std::memset(ctx->h_flags, 0, 64);
    *pctx = ctx;
    return FPT_OK;
}

fpt_status fpt_model_get_info(const fpt_ctx *ctx, int32_t model, fpt_model_info *out)
{
    if (!ctx || !out) return FPT_E_INVALID;
    if (model < 0 || model >= (int)ctx->models.size())
        return fail(const_cast<fpt_ctx *>(ctx), FPT_E_INVALID, "model index out of range");
    *out = ctx->infos[model];
    return FPT_OK;
}

// Re-pack every ready table into one float4 array and refresh the model
// descriptors. 1-D tables: entry j = ((S_j + S_{j+1})/2, S_{j+1} - S_j,
// (T_j + T_{j+1})/2, T_{j+1} - T_j) times sqrt(dN), in FP32 (midpoint form,
// see table_at); 2-D tables: the values (S_phiphi, S_phipi, S_pipi, 0) times
// sqrt(dN) at the grid points, entry M repeating entry M - 1.
// Cubic table of V'/V for the Gaussian bump (see drift_vpv in fpt_kernels.cu):
// kDriftIntervals intervals over x = phi - phi_end in [0, X], X = 16 (phi_in -
// phi_end), capped at the background start; Hermite coefficients from the FP64
// values v and slopes v' = V''/V - (V'/V)^2 at the nodes.
static const int kDriftIntervals = 1024;

static double drift_top(const fpt_model &m, const fpt_model_info &inf)
{
    double X = 16.0 * (inf.phi_in - inf.phi_end);
    if (!std::isnan(m.n_in)) X = std::min(X, m.bg_phi0 - inf.phi_end);
    return X;
}

static void drift_table(const fpt_model &m, const fpt_model_info &inf, float4 *out)
{
    const double X = drift_top(m, inf), h = X / kDriftIntervals;
    std::vector<double> v(kDriftIntervals + 1), dv(kDriftIntervals + 1);
    for (int j = 0; j <= kDriftIntervals; ++j) {
        const double phi = inf.phi_end + h * j;
        v[j] = fpt_host::dlnV(m, phi, 0);
        dv[j] = fpt_host::d2V_over_V(m, phi) - v[j] * v[j];
    }
    for (int j = 0; j < kDriftIntervals; ++j) {
        const double v0 = v[j], v1 = v[j + 1], d0 = h * dv[j], d1 = h * dv[j + 1];
        out[j] = make_float4((float)v0, (float)d0, (float)(3.0 * (v1 - v0) - 2.0 * d0 - d1),
                             (float)(2.0 * (v0 - v1) + d0 + d1));
    }
    out[kDriftIntervals] = make_float4((float)v[kDriftIntervals], 0.0f, 0.0f, 0.0f);
}

static fpt_status upload_tables(fpt_ctx *ctx)
{
    size_t total = 0;
    for (size_t i = 0; i < ctx->tables.size(); ++i) {
        ctx->table_offset[i] = (int)total;
        int e = 0;
        if (ctx->tables[i].ready)
            e = ctx->tables[i].entries() + (ctx->models[i].kind == FPT_POT_BUMP ? kDriftIntervals + 1 : 0);
        ctx->region_entries[i] = e;
        total += e;
    }
    std::vector<float4> packed(std::max<size_t>(total, 1));
    std::vector<ModelDev> md(ctx->models.size());
    for (size_t i = 0; i < ctx->models.size(); ++i) {
        const fpt_model &m = ctx->models[i];
        const fpt_model_info &inf = ctx->infos[i];
        const TableHost &t = ctx->tables[i];
        ModelDev &d = md[i];
        std::memset(&d, 0, sizeof(d));
        d.x_star = (float)(m.phi_star - inf.phi_end);
        d.x_star_lo = (float)((m.phi_star - inf.phi_end) - (double)d.x_star);
        // V'/V = 1 / (1/a + c (phi - phi_star)); a zero slope gives 1/a = inf and V'/V = 0
        auto inv = [](double a) { return a == 0.0 ? INFINITY : (float)(1.0 / a); };
        if (m.kind == FPT_POT_EXP) {
            d.inv_a_plus = d.inv_a_minus = inv(m.mu);
            d.drift_c = 0.0f;
            d.x_star = 0.0f;
            d.x_star_lo = 0.0f;
        } else {
            d.inv_a_plus = inv(m.a_plus);
            d.inv_a_minus = inv(m.a_minus);
            d.drift_c = 1.0f;
        }
        d.x_in = (float)(inf.phi_in - inf.phi_end);
        d.pi_in = (float)inf.pi_in;
        d.dtab = -1;
        if (m.kind == FPT_POT_BUMP && t.ready) {
            d.dtab = t.entries();
            d.d_scale = (float)(kDriftIntervals / drift_top(m, inf));
            d.d_umax = (float)kDriftIntervals;
            d.bump_m2 = (float)(m.bump_m * m.bump_m);
            d.bump_phi_end = (float)inf.phi_end;
            d.bump_dphi0 = (float)(inf.phi_end - m.bump_phi0);
            d.bump_inv_w2 = (float)(1.0 / (m.bump_width * m.bump_width));
            d.bump_K = (float)m.bump_K;
            drift_table(m, inf, &packed[ctx->table_offset[i] + t.entries()]);
        }
        d.dN = (float)m.dN;
        d.sqrt_dN = (float)std::sqrt(m.dN);
        d.half_dN = 0.5f * d.dN;       // the same FP32 products the steppers form from dN
        d.m3dN = -3.0f * d.dN;
        d.max_steps = (int32_t)m.max_steps;
        d.table_offset = ctx->table_offset[i];
        if (t.ready) {
            d.M = t.M;
            d.u_umax = (float)(t.M - 1);
            if (t.n_indexed) {
                // u = (n dN - N_lo)/h; window of steps as in the oracle's definition
                d.nidx = 1;
                d.u_scale = (float)(m.dN / t.h);
                d.u_shift = (float)(-t.lo / t.h);
                const double lo_s = std::ceil(t.lo / m.dN - 1e-9);
                const double hi_s = std::floor((t.lo + t.h * (t.M - 1)) / m.dN + 1e-9);
                d.win_lo = (int32_t)std::max(0.0, std::min(lo_s, 2147483647.0));
                d.win_hi = (int32_t)std::max(-1.0, std::min(hi_s, 2147483647.0));
            } else {
                d.u_scale = (float)(1.0 / t.h);
                d.u_shift = (float)((inf.phi_end - t.lo) / t.h);
            }
            if (!t.rank2) {
                // 1-D tables are read at the interval midpoints: u' = u - 1/2 in [-1/2, M - 3/2]
                if (t.n_indexed) d.u_shift = (float)(-t.lo / t.h - 0.5);
                else d.u_shift = (float)((inf.phi_end - t.lo) / t.h - 0.5);
                d.u_umax = (float)(t.M - 1.5);
            }
            const double sq = std::sqrt(m.dN);
            d.rank2 = t.rank2 ? 1 : 0;
            if (t.rank2) {
                // (S_phiphi, S_phipi, S_pipi, 0) sqrt(dN); entry M repeats entry M - 1
                for (int j = 0; j <= t.M; ++j) {
                    const int k = std::min(j, t.M - 1);
                    packed[ctx->table_offset[i] + j] =
                        make_float4((float)(t.S[k] * sq), (float)(t.T[k] * sq), (float)(t.C[k] * sq), 0.0f);
                }
                continue;
            }
            for (int j = 0; j < t.M; ++j) {
                const int k = std::min(j + 1, t.M - 1);
                float4 e;
                e.x = (float)(0.5 * (t.S[j] + t.S[k]) * sq);       // interval midpoint value
                e.y = (float)((t.S[k] - t.S[j]) * sq);             // slope per grid interval
                e.z = (float)(0.5 * (t.T[j] + t.T[k]) * sq);
                e.w = (float)((t.T[k] - t.T[j]) * sq);
                packed[ctx->table_offset[i] + j] = e;
            }
        }
    }
    if (packed.size() > ctx->tables_cap) {
        dev_free(ctx, ctx->d_tables);
        ctx->d_tables = nullptr;
        ctx->tables_cap = 0;
        CK(dev_malloc(ctx, &ctx->d_tables, sizeof(float4) * packed.size()));
        ctx->tables_cap = packed.size();
        clear_graphs(ctx);
    }
    CK(cudaMemcpyAsync(ctx->d_tables, packed.data(), sizeof(float4) * packed.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_models, md.data(), sizeof(ModelDev) * md.size(),
                       cudaMemcpyHostToDevice, ctx->stream));
    ctx->h_models = md;
    CK(cudaStreamSynchronize(ctx->stream));
    return FPT_OK;
}

fpt_status fpt_noise_table(fpt_ctx *ctx, int32_t model, int32_t kind, int32_t n_points,
                           double sigma, double phi_lo, double phi_hi, const double *user_S,
                           const double *user_Spi, double *out_S, double *out_Spi)
{
    if (!ctx) return FPT_E_INVALID;
    if (model < 0 || model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "model index out of range");
    std::string msg;
    fpt_status s = table_args(kind, n_points, sigma, phi_lo, phi_hi, user_S, user_Spi, msg);
    if (s != FPT_OK) return fail(ctx, s, msg);
    TableHost t;
    s = build_host_table(ctx->models[model], ctx->infos[model], kind, n_points, sigma, phi_lo, phi_hi,
                         user_S, user_Spi, t, msg);
    if (s != FPT_OK) return fail(ctx, s, msg);
    CK(cudaSetDevice(ctx->device));
    if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
    ctx->tables[model] = t;
    if ((s = upload_tables(ctx)) != FPT_OK) return s;
    if (out_S) std::copy(t.S.begin(), t.S.end(), out_S);
    if (out_Spi) std::copy(t.T.begin(), t.T.end(), out_Spi);
    return FPT_OK;
}

fpt_status fpt_noise_table2(fpt_ctx *ctx, int32_t model, int32_t kind, int32_t n_points,
                            double sigma, double phi_lo, double phi_hi, const double *user_S,
                            double *out_S)
{
    if (!ctx) return FPT_E_INVALID;
    if (model < 0 || model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "model index out of range");
    std::string msg;
    fpt_status s = table2_args(kind, n_points, sigma, phi_lo, phi_hi, user_S, msg);
    if (s != FPT_OK) return fail(ctx, s, msg);
    TableHost t;
    s = build_host_table2(ctx->models[model], ctx->infos[model], kind, n_points, sigma, phi_lo, phi_hi,
                          user_S, t, msg);
    if (s != FPT_OK) return fail(ctx, s, msg);
    CK(cudaSetDevice(ctx->device));
    if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
    ctx->tables[model] = t;
    if ((s = upload_tables(ctx)) != FPT_OK) return s;
    if (out_S) copy_planes(t, out_S);
    return FPT_OK;
}

fpt_status fpt_set_launch(fpt_ctx *ctx, const fpt_launch *l)
{
    if (!ctx || !l) return FPT_E_INVALID;
    if (l->block && l->block != 128 && l->block != 192 && l->block != 256 && l->block != 384 && l->block != 512)
        return fail(ctx, FPT_E_INVALID, "block must be 128, 192, 256, 384 or 512");
    if (l->blocks_per_sm < 0 || l->blocks_per_sm > 16) return fail(ctx, FPT_E_INVALID, "blocks_per_sm out of [0, 16]");
    if (l->check_steps < 0 || (l->check_steps % 4) || l->check_steps > 4096)
        return fail(ctx, FPT_E_INVALID, "check_steps must be a multiple of 4 in [4, 4096]");
    if (!(l->deadline_s >= 0) || !std::isfinite(l->deadline_s)) return fail(ctx, FPT_E_INVALID, "bad deadline");
    ctx->launch.block = l->block ? l->block : 512;
    ctx->launch.blocks_per_sm = l->blocks_per_sm;
    ctx->launch.check_steps = l->check_steps ? l->check_steps : 32;
    ctx->launch.use_graph = l->use_graph;
    ctx->launch.deadline_s = l->deadline_s;
    return FPT_OK;
}

fpt_status fpt_get_launch(const fpt_ctx *ctx, fpt_launch *l)
{
    if (!ctx || !l) return FPT_E_INVALID;
    *l = ctx->launch;
    return FPT_OK;
}

fpt_status fpt_set_memory_limit(fpt_ctx *ctx, int64_t max_bytes)
{
    if (!ctx) return FPT_E_INVALID;
    if (max_bytes < 0) return fail(ctx, FPT_E_INVALID, "memory limit must be >= 0");
    ctx->dev_limit = (size_t)max_bytes;
    return FPT_OK;
}

fpt_status fpt_memory_in_use(const fpt_ctx *ctx, int64_t *in_use, int64_t *max_bytes)
{
    if (!ctx) return FPT_E_INVALID;
    if (in_use) *in_use = (int64_t)ctx->dev_bytes;
    if (max_bytes) *max_bytes = (int64_t)ctx->dev_limit;
    return FPT_OK;
}

static fpt_status ensure_units(fpt_ctx *ctx, long long total)
{
    if (total <= ctx->unit_cap) return FPT_OK;
    long long cap = std::max<long long>(total, 1 << 16);
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
    dev_free(ctx, ctx->d_nsteps); dev_free(ctx, ctx->d_logw); dev_free(ctx, ctx->d_status); dev_free(ctx, ctx->d_N);
    ctx->d_nsteps = nullptr; ctx->d_logw = nullptr; ctx->d_status = nullptr; ctx->d_N = nullptr;
    ctx->unit_cap = 0;
    clear_graphs(ctx);
    CK(dev_malloc(ctx, &ctx->d_nsteps, sizeof(int32_t) * cap));
    CK(dev_malloc(ctx, &ctx->d_logw, sizeof(double) * cap));
    CK(dev_malloc(ctx, &ctx->d_status, cap));
    ctx->unit_cap = cap;
    return FPT_OK;
}

// Enqueue: descriptor upload, counter reset, status pre-fill, stepper launch,
// flag read-back.
static cudaError_t enqueue_run(fpt_ctx *ctx, const EmParams &p, EmVariant v, int grid,
                               int block, size_t smem_bytes, int n_runs, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ctx->d_runs, ctx->h_runs, sizeof(RunDev) * n_runs,
                             cudaMemcpyHostToDevice, s)))
        return e;
    if ((e = cudaMemsetAsync(ctx->d_cursor, 0, 64, s))) return e;
    if ((e = cudaMemsetAsync(ctx->d_flags, 0, 64, s))) return e;
    if ((e = cudaMemsetAsync(ctx->d_status, FPT_TRAJ_ABORTED, (size_t)p.total_units, s))) return e;
    if (v.rec && (e = cudaMemsetAsync(ctx->d_rec_cursor, 0, sizeof(unsigned long long), s))) return e;
    if ((e = em_launch(p, v, grid, block, smem_bytes, s))) return e;
    return cudaMemcpyAsync(ctx->h_flags, ctx->d_flags, kFlagWords * sizeof(int), cudaMemcpyDeviceToHost, s);
}

fpt_status fpt_run(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs, fpt_traj_out *out,
                   void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!runs || n_runs < 1 || n_runs > kMaxRuns) return fail(ctx, FPT_E_INVALID, "n_runs out of [1, 128]");
    std::set<int> used_models;
    bool mnet = false;   // MLP runs with different networks (or normalisations, clamps)
    long long total = 0;
    bool weighted = false;
    bool nidx = false;
    int rank2 = -1;
    int bump = -1;
    int mlp_run = -1;
    for (int r = 0; r < n_runs; ++r) {
        const fpt_run_desc &d = runs[r];
        if (d.model < 0 || d.model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "run model out of range");
        if (!ctx->tables[d.model].ready) return fail(ctx, FPT_E_STATE, "no noise table for the run's model");
        if (d.bias_kind != FPT_BIAS_NONE && d.bias_kind != FPT_BIAS_CONST && d.bias_kind != FPT_BIAS_MLP)
            return fail(ctx, FPT_E_INVALID, "unknown bias kind");
        if (d.bias_kind == FPT_BIAS_MLP) {
            if (!d.mlp || (reinterpret_cast<uintptr_t>(d.mlp) & 15))
                return fail(ctx, FPT_E_INVALID, "MLP runs need a 16-byte aligned device weight blob");
            if (d.mlp_segment < 4 || d.mlp_segment > 4096 || (d.mlp_segment % 4))
                return fail(ctx, FPT_E_INVALID, "mlp_segment must be a multiple of 4 in [4, 4096]");
            if (!(d.alpha_max > 0.0f) || !std::isfinite(d.alpha_max))
                return fail(ctx, FPT_E_INVALID, "alpha_max must be positive");
            for (int k = 0; k < 3; ++k)
                if (!std::isfinite(d.mlp_shift[k]) || !std::isfinite(d.mlp_scale[k]))
                    return fail(ctx, FPT_E_INVALID, "MLP input shift/scale must be finite");
            if (mlp_run < 0) mlp_run = r;
            const fpt_run_desc &q = runs[mlp_run];
            if (d.mlp_flags & ~FPT_MLP_LOG_X) return fail(ctx, FPT_E_INVALID, "unknown mlp_flags bits");
            // the held-alpha segment is the launch's refill interval: shared by all MLP runs
            if (d.mlp_segment != q.mlp_segment)
                return fail(ctx, FPT_E_INVALID, "all MLP runs of one call must share mlp_segment");
            if (!std::isfinite(d.mlp_x_floor)) return fail(ctx, FPT_E_INVALID, "mlp_x_floor must be finite");
            if (d.mlp != q.mlp || d.alpha_max != q.alpha_max || d.mlp_flags != q.mlp_flags ||
                d.mlp_x_floor != q.mlp_x_floor ||
                std::memcmp(d.mlp_shift, q.mlp_shift, sizeof(q.mlp_shift)) ||
                std::memcmp(d.mlp_scale, q.mlp_scale, sizeof(q.mlp_scale)))
                mnet = true;
        }
        if (d.bias_kind == FPT_BIAS_CONST && (!std::isfinite(d.A) || !std::isfinite(d.A2)))
            return fail(ctx, FPT_E_INVALID, "A and A2 must be finite");
        if (d.n_traj > 0) {
            const bool bp = ctx->models[d.model].kind == FPT_POT_BUMP;
            if (bump < 0) bump = bp ? 1 : 0;
            else if (bump != (bp ? 1 : 0))
                return fail(ctx, FPT_E_INVALID, "runs of one call must all use the bump potential or none");
            if (bp && ctx->tables[d.model].n_indexed)
                return fail(ctx, FPT_E_INVALID, "the bump potential needs a phi-indexed noise table");
            const bool r2 = ctx->tables[d.model].rank2;
            if (rank2 < 0) rank2 = r2 ? 1 : 0;
            else if (rank2 != (r2 ? 1 : 0))
                return fail(ctx, FPT_E_INVALID, "runs of one call must all use 1-D or all use 2-D noise tables");
            if (!r2 && d.bias_kind == FPT_BIAS_CONST && d.A2 != 0.0)
                return fail(ctx, FPT_E_INVALID, "A2 needs a 2-D noise table");
        }
        if (d.n_traj < 0 || d.traj_offset < 0 || d.traj_offset + d.n_traj > (1LL << 32))
            return fail(ctx, FPT_E_INVALID, "trajectory ids must lie in [0, 2^32)");
        if (d.seed != runs[0].seed) return fail(ctx, FPT_E_INVALID, "all runs of one call must share the seed");
        if (d.n_traj > 0) used_models.insert(d.model);
        if ((d.bias_kind == FPT_BIAS_CONST && (d.A != 0.0 || d.A2 != 0.0)) || d.bias_kind == FPT_BIAS_MLP)
            weighted = true;
        if (d.n_traj > 0 && ctx->tables[d.model].n_indexed) {
            if (d.bias_kind == FPT_BIAS_MLP)
                return fail(ctx, FPT_E_INVALID, "learned-proposal runs need a phi-indexed noise table");
            nidx = true;
        }
        total += d.n_traj;
    }
    if (total > (1LL << 32)) return fail(ctx, FPT_E_INVALID, "more than 2^32 trajectories in one call");
    // the learned-proposal steppers index every table by the field: a call with
    // an MLP run cannot also carry a run on a time-indexed (noise-window) table
    if (mlp_run >= 0 && nidx)
        return fail(ctx, FPT_E_INVALID, "a call with a learned-proposal run needs phi-indexed tables for all its runs");
    if (mnet && (rank2 == 1 || bump == 1))
        return fail(ctx, FPT_E_INVALID,
                    "MLP runs with different networks need 1-D noise tables and the piecewise-linear or "
                    "exponential potential");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    fpt_status st = ensure_units(ctx, std::max<long long>(total, 1));
    if (st != FPT_OK) return st;

    long long begin = 0;
    ctx->last_runs.resize(n_runs);
    for (int r = 0; r < n_runs; ++r) {
        const fpt_run_desc &d = runs[r];
        const fpt_model &m = ctx->models[d.model];
        RunDev &rd = ctx->last_runs[r];
        std::memset(&rd, 0, sizeof(rd));
        const double A = d.bias_kind == FPT_BIAS_CONST ? d.A : 0.0;
        const double A2 = d.bias_kind == FPT_BIAS_CONST ? d.A2 : 0.0;
        rd.model = d.model;
        rd.bias_kind = d.bias_kind;
        rd.cb = (float)(A * std::sqrt(m.dN));
        rd.cb_b = (float)(A2 * std::sqrt(m.dN));
        rd.half_cb2 = (float)(0.5 * (A * A + A2 * A2) * m.dN);
        rd.n_traj = d.n_traj;
        rd.traj_offset = d.traj_offset;
        rd.unit_begin = begin;
        rd.run_id = d.run_id;
        rd.sqrt_dN = (float)std::sqrt(m.dN);
        rd.dN = (float)m.dN;
        if (d.bias_kind == FPT_BIAS_MLP) {
            rd.segment = d.mlp_segment;
            rd.mlp = d.mlp;
            for (int k = 0; k < 3; ++k) { rd.shift[k] = d.mlp_shift[k]; rd.scale[k] = d.mlp_scale[k]; }
            rd.alpha_max = d.alpha_max;
            rd.mlp_flags = d.mlp_flags;
            rd.x_floor = d.mlp_x_floor > 0.0f ? d.mlp_x_floor : 1e-30f;
        }
        begin += d.n_traj;
    }
    // the stepper is the only reader of h_runs: wait for the previous launch
    if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
    std::memcpy(ctx->h_runs, ctx->last_runs.data(), sizeof(RunDev) * n_runs);

    const bool smem = used_models.size() == 1;
    const int smem_model = smem ? *used_models.begin() : 0;
    const bool mlp = mlp_run >= 0;
    const EmVariant var{weighted, smem, mlp, mlp && ctx->record_mode, nidx && !mlp, rank2 == 1, bump == 1,
                        mlp && mnet};
    const size_t smem_bytes = em_smem_bytes(var, smem ? ctx->region_entries[smem_model] : 0, n_runs,
                                            (int)ctx->models.size());
    // the learned-proposal steppers are compiled for at most kMlpMaxBlock threads
    const int block = mlp ? std::min(ctx->launch.block, kMlpMaxBlock) : ctx->launch.block;
    int occ = em_occupancy(var, block, smem_bytes);
    if (occ < 1) return fail(ctx, FPT_E_CUDA, "stepper does not fit on an SM with this shape");
    const int bps = ctx->launch.blocks_per_sm ? std::min(ctx->launch.blocks_per_sm, occ) : occ;
    const int grid = std::max(1, bps * ctx->sm_count);
    // the learned proposal is re-evaluated at every refill point
    const int check_steps = mlp ? runs[mlp_run].mlp_segment : ctx->launch.check_steps;

    EmParams p;
    std::memset(&p, 0, sizeof(p));
    p.models = ctx->d_models;
    p.runs = ctx->d_runs;
    p.n_models = (int)ctx->models.size();
    p.n_runs = n_runs;
    p.tables = ctx->d_tables;
    p.smem_table_offset = smem ? ctx->table_offset[smem_model] : 0;
    if (smem) p.m0 = ctx->h_models[smem_model];
    p.smem_table_points = smem ? ctx->region_entries[smem_model] : 0;
    p.total_units = total;
    p.cursor = ctx->d_cursor;
    p.flags = ctx->d_flags;
    p.nsteps = ctx->d_nsteps;
    p.logw = ctx->d_logw;
    p.status = ctx->d_status;
    {
        // Philox4x32-10 key schedule (Weyl increments 0x9E3779B9, 0xBB67AE85)
        uint32_t k0 = (uint32_t)runs[0].seed, k1 = (uint32_t)(runs[0].seed >> 32);
        for (int r = 0; r < 10; ++r) {
            p.rk[2 * r] = k0;
            p.rk[2 * r + 1] = k1;
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    p.groups_per_check = check_steps / 4;
    p.mlp_run = mlp ? mlp_run : 0;
    p.records = ctx->d_records;
    p.rec_cursor = ctx->d_rec_cursor;
    p.rec_cap = ctx->rec_cap;
    p.budget_ns = ctx->launch.deadline_s > 0.0 ? (unsigned long long)(ctx->launch.deadline_s * 1e9) + 1ull : 0ull;
    p.t0 = reinterpret_cast<unsigned long long *>(ctx->d_flags + kFlagT0);   // zeroed with the flags
    const bool graph = ctx->launch.use_graph && p.budget_ns == 0;

    if (total > 0) {
        if (graph) {
            GraphKey key{weighted, smem, grid, block, smem_bytes, p.groups_per_check, n_runs,
                         smem ? smem_model : -1, total,
                         (mlp ? 1 : 0) + (var.rec ? 2 : 0) + (var.nidx ? 4 : 0) + (var.rank2 ? 8 : 0) +
                             (var.dtab ? 16 : 0) + (var.mnet ? 32 : 0) + 64 * p.mlp_run};
            auto it = ctx->graphs.find(key);
            if (it == ctx->graphs.end()) {
                RunGraph rg;
                CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
                cudaError_t e = enqueue_run(ctx, p, var, grid, block, smem_bytes, n_runs, ctx->stream);
                cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &rg.graph);
                if (e != cudaSuccess) {
                    if (e2 == cudaSuccess) cudaGraphDestroy(rg.graph);
                    return cuda_fail(ctx, e, "capture");
                }
                if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "cudaStreamEndCapture");
                // the one kernel node of the capture is the stepper
                size_t n_nodes = 0;
                e = cudaGraphGetNodes(rg.graph, nullptr, &n_nodes);
                std::vector<cudaGraphNode_t> nodes(n_nodes);
                if (e == cudaSuccess && n_nodes) e = cudaGraphGetNodes(rg.graph, nodes.data(), &n_nodes);
                int n_kernels = 0;
                for (size_t i = 0; e == cudaSuccess && i < n_nodes; ++i) {
                    cudaGraphNodeType t;
                    e = cudaGraphNodeGetType(nodes[i], &t);
                    if (e == cudaSuccess && t == cudaGraphNodeTypeKernel) {
                        rg.stepper = nodes[i];
                        ++n_kernels;
                    }
                }
                if (e == cudaSuccess && n_kernels != 1) e = cudaErrorInvalidValue;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&rg.exec, rg.graph, 0);
                if (e != cudaSuccess) {
                    cudaGraphDestroy(rg.graph);
                    return cuda_fail(ctx, e, "graph of the run");
                }
                it = ctx->graphs.emplace(key, rg).first;
                std::memcpy(&it->second.params, &p, sizeof(EmParams));   // padding included
            } else if (std::memcmp(&it->second.params, &p, sizeof(EmParams)) != 0) {
                cudaKernelNodeParams kp;
                CK(cudaGraphKernelNodeGetParams(it->second.stepper, &kp));
                void *args[] = {&p};
                kp.kernelParams = args;
                kp.extra = nullptr;
                CK(cudaGraphExecKernelNodeSetParams(it->second.exec, it->second.stepper, &kp));
                std::memcpy(&it->second.params, &p, sizeof(EmParams));
            }
            CK(cudaGraphLaunch(it->second.exec, s));
        } else {
            cudaError_t e = enqueue_run(ctx, p, var, grid, block, smem_bytes, n_runs, s);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "run launch");
        }
    } else {
        std::memset(ctx->h_flags, 0, kFlagWords * sizeof(int));
    }
    CK(cudaEventRecord(ctx->run_done, s));
    ctx->last_n_runs = n_runs;
    ctx->last_total = total;
    ctx->last_valid = true;
    ctx->last_stream = s;

    if (out) {
        bool host_dst = false;
        for (int r = 0; r < n_runs; ++r) {
            const RunDev &rd = ctx->last_runs[r];
            const long long n = rd.n_traj;
            if (n == 0) continue;
            const fpt_traj_out &o = out[r];
            if (o.nsteps) CK(cudaMemcpyAsync(o.nsteps, ctx->d_nsteps + rd.unit_begin, sizeof(int32_t) * n, cudaMemcpyDefault, s));
            if (o.logw) CK(cudaMemcpyAsync(o.logw, ctx->d_logw + rd.unit_begin, sizeof(double) * n, cudaMemcpyDefault, s));
            if (o.status) CK(cudaMemcpyAsync(o.status, ctx->d_status + rd.unit_begin, n, cudaMemcpyDefault, s));
            if (o.N) {
                if (!ctx->d_N) CK(dev_malloc(ctx, &ctx->d_N, sizeof(double) * ctx->unit_cap));
                CK(n_of_steps_launch(ctx->d_nsteps + rd.unit_begin, n, ctx->models[rd.model].dN,
                                     ctx->d_N + rd.unit_begin, s));
                CK(cudaMemcpyAsync(o.N, ctx->d_N + rd.unit_begin, sizeof(double) * n, cudaMemcpyDefault, s));
            }
            for (const void *ptr : {(const void *)o.N, (const void *)o.logw, (const void *)o.nsteps, (const void *)o.status}) {
                if (!ptr) continue;
                cudaPointerAttributes a;
                if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess || a.type != cudaMemoryTypeDevice) host_dst = true;
                cudaGetLastError();
            }
        }
        if (host_dst) return fpt_sync(ctx);
    }
    return FPT_OK;
}

fpt_status fpt_sync(fpt_ctx *ctx)
{
    if (!ctx) return FPT_E_INVALID;
    CK(cudaSetDevice(ctx->device));
    if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
    CK(cudaStreamSynchronize(ctx->stream));
#ifdef FPT_CHECKS
    {
        const fpt_status cs = take_checks(ctx);
        if (cs != FPT_OK) return cs;
    }
#endif
    if (!ctx->last_valid) return FPT_OK;
    if (ctx->h_flags[0]) return fail(ctx, FPT_E_TIMEOUT, "kernel deadline passed; run aborted");
    if (ctx->h_flags[1] > 0) {
        ctx->err = std::to_string(ctx->h_flags[1]) + " trajectories hit max_steps";
        return FPT_W_CAPPED;
    }
    return FPT_OK;
}

static fpt_status hist_args(fpt_ctx *ctx, double N_lo, double N_hi, int32_t n_bins, double N_tail)
{
    if (n_bins < 1 || n_bins > kMaxBins) return fail(ctx, FPT_E_INVALID, "n_bins out of [1, 4096]");
    if (!(N_hi > N_lo) || !std::isfinite(N_lo) || !std::isfinite(N_hi))
        return fail(ctx, FPT_E_INVALID, "need finite N_lo < N_hi");
    if (!((N_hi - N_lo) / n_bins >= DBL_MIN) || !std::isfinite(N_hi - N_lo))
        return fail(ctx, FPT_E_INVALID, "bin width (N_hi - N_lo) / n_bins must be a positive normal number");
    if (!std::isnan(N_tail) && !std::isfinite(N_tail)) return fail(ctx, FPT_E_INVALID, "N_tail must be finite or NaN");
    return FPT_OK;
}

// Launch the histogram kernels on per-trajectory device arrays and unpack the
// FP64 results into the caller's fpt_hist.
static fpt_status hist_run(fpt_ctx *ctx, const int32_t *nsteps, const double *logw,
                           const uint8_t *status, long long unit_begin, long long n, double dN,
                           double N_lo, double N_hi, int32_t n_bins, double N_tail, fpt_hist *out,
                           cudaStream_t s)
{
    HistParams p;
    std::memset(&p, 0, sizeof(p));
    p.nsteps = nsteps;
    p.logw = logw;
    p.status = status;
    p.unit_begin = unit_begin;
    p.n = n;
    p.dN = dN;
    p.N_lo = N_lo;
    p.db = (N_hi - N_lo) / n_bins;
    p.N_tail = N_tail;
    p.n_bins = n_bins;
    p.chunk = 4096;
    p.maxkey = ctx->d_hmax;
    p.mom = ctx->d_hmom;
    p.scal = ctx->d_hscal;
    cudaError_t e = hist_launch(p, ctx->d_hout, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "histogram launch");
    const size_t nd = (size_t)10 * n_bins + 16;
    CK(cudaMemcpyAsync(ctx->h_hout, ctx->d_hout, sizeof(double) * nd, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
#ifdef FPT_CHECKS
    {
        const fpt_status cs = take_checks(ctx);
        if (cs != FPT_OK) return cs;
    }
#endif
    const double *h = ctx->h_hout;
    for (int b = 0; b < n_bins; ++b) {
        if (out->count) out->count[b] = (int64_t)h[b];
        if (out->log_sum_w) out->log_sum_w[b] = h[1 * n_bins + b];
        if (out->log_sum_w2) out->log_sum_w2[b] = h[2 * n_bins + b];
        if (out->sum_lw) out->sum_lw[b] = h[3 * n_bins + b];
        if (out->sum_lw2) out->sum_lw2[b] = h[4 * n_bins + b];
        if (out->pdf) out->pdf[b] = h[5 * n_bins + b];
        if (out->se_w) out->se_w[b] = h[6 * n_bins + b];
        if (out->pdf_ln) out->pdf_ln[b] = h[7 * n_bins + b];
        if (out->se_ln) out->se_ln[b] = h[8 * n_bins + b];
        if (out->se_jk) out->se_jk[b] = h[9 * n_bins + b];
    }
    const double *sc = h + 10 * n_bins;
    out->n_total = (int64_t)sc[0];
    out->n_passed = (int64_t)sc[1];
    out->n_under = (int64_t)sc[2];
    out->n_over = (int64_t)sc[3];
    out->n_capped = (int64_t)sc[4];
    out->n_tail = (int64_t)sc[5];
    out->N_mean = sc[6];
    out->N_mean_w = sc[7];
    out->ess_tail = sc[8];
    out->p_tail = sc[9];
    out->log_max_w = sc[10];
    return FPT_OK;
}

fpt_status fpt_histogram(fpt_ctx *ctx, int32_t run, double N_lo, double N_hi, int32_t n_bins,
                         double N_tail, fpt_hist *out, void *cuda_stream)
{
    if (!ctx || !out) return FPT_E_INVALID;
    if (!ctx->last_valid) return fail(ctx, FPT_E_STATE, "no run to histogram");
    if (run < 0 || run >= ctx->last_n_runs) return fail(ctx, FPT_E_INVALID, "run index out of range");
    fpt_status st = hist_args(ctx, N_lo, N_hi, n_bins, N_tail);
    if (st != FPT_OK) return st;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    CK(cudaStreamWaitEvent(s, ctx->run_done, 0));
    const RunDev &rd = ctx->last_runs[run];
    st = hist_run(ctx, ctx->d_nsteps, ctx->d_logw, ctx->d_status, rd.unit_begin, rd.n_traj,
                  ctx->models[rd.model].dN, N_lo, N_hi, n_bins, N_tail, out, s);
    if (st != FPT_OK) return st;
    if (ctx->h_flags[0]) return fail(ctx, FPT_E_STATE, "the run was aborted by its deadline");
    return FPT_OK;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a;
    bool dev = cudaPointerGetAttributes(&a, p) == cudaSuccess &&
               (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    return dev;
}

fpt_status fpt_histogram_data(fpt_ctx *ctx, const int32_t *nsteps, const double *logw,
                              const uint8_t *status, int64_t n, double dN, double N_lo,
                              double N_hi, int32_t n_bins, double N_tail, fpt_hist *out,
                              void *cuda_stream)
{
    if (!ctx || !out) return FPT_E_INVALID;
    if (!nsteps || !logw || !status || n < 1) return fail(ctx, FPT_E_INVALID, "need n >= 1 and three arrays");
    if (!(dN > 0) || !std::isfinite(dN)) return fail(ctx, FPT_E_INVALID, "dN must be positive");
    fpt_status st = hist_args(ctx, N_lo, N_hi, n_bins, N_tail);
    if (st != FPT_OK) return st;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    const bool dev = is_device_ptr(nsteps) && is_device_ptr(logw) && is_device_ptr(status);
    if (!dev) {
        if (n > ctx->x_cap) {
            CK(cudaStreamSynchronize(s));
            dev_free(ctx, ctx->d_xn); dev_free(ctx, ctx->d_xlw); dev_free(ctx, ctx->d_xst);
            ctx->d_xn = nullptr; ctx->d_xlw = nullptr; ctx->d_xst = nullptr; ctx->x_cap = 0;
            CK(dev_malloc(ctx, &ctx->d_xn, sizeof(int32_t) * n));
            CK(dev_malloc(ctx, &ctx->d_xlw, sizeof(double) * n));
            CK(dev_malloc(ctx, &ctx->d_xst, n));
            ctx->x_cap = n;
        }
        CK(cudaMemcpyAsync(ctx->d_xn, nsteps, sizeof(int32_t) * n, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(ctx->d_xlw, logw, sizeof(double) * n, cudaMemcpyDefault, s));
        CK(cudaMemcpyAsync(ctx->d_xst, status, n, cudaMemcpyDefault, s));
        return hist_run(ctx, ctx->d_xn, ctx->d_xlw, ctx->d_xst, 0, n, dN, N_lo, N_hi, n_bins, N_tail, out, s);
    }
    return hist_run(ctx, nsteps, logw, status, 0, n, dN, N_lo, N_hi, n_bins, N_tail, out, s);
}

fpt_status fpt_autotune(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs, double fraction,
                        fpt_launch *chosen)
{
    if (!ctx) return FPT_E_INVALID;
    if (!runs || n_runs < 1 || n_runs > kMaxRuns) return fail(ctx, FPT_E_INVALID, "n_runs out of [1, 128]");
    if (!(fraction > 0.0 && fraction <= 1.0)) return fail(ctx, FPT_E_INVALID, "fraction out of (0, 1]");
    std::vector<fpt_run_desc> sub(runs, runs + n_runs);
    for (auto &d : sub)
        if (d.n_traj > 0) d.n_traj = std::max<int64_t>(32, (int64_t)std::llround(d.n_traj * fraction));
    const fpt_launch keep = ctx->launch;
    CK(cudaSetDevice(ctx->device));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    fpt_launch best = keep;
    float best_ms = -1.0f;
    fpt_status st = FPT_OK;
    for (int block : {128, 256, 384, 512}) {
        for (int check : {8, 32, 128}) {
            ctx->launch.block = block;
            ctx->launch.blocks_per_sm = 0;
            ctx->launch.check_steps = check;
            ctx->launch.use_graph = keep.use_graph;
            ctx->launch.deadline_s = 0.0;
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && st == FPT_OK; ++rep) {
                cudaEventRecord(e0, ctx->stream);
                st = fpt_run(ctx, sub.data(), n_runs, nullptr, nullptr);
                cudaEventRecord(e1, ctx->stream);
                if (st == FPT_OK) {
                    fpt_status s2 = fpt_sync(ctx);
                    if (s2 != FPT_OK && s2 != FPT_W_CAPPED) st = s2;
                }
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (st != FPT_OK) break;
            if (best_ms < 0.0f || ms < best_ms) {
                best_ms = ms;
                best = ctx->launch;
            }
        }
        if (st != FPT_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    best.use_graph = keep.use_graph;
    best.deadline_s = keep.deadline_s;
    ctx->launch = (st == FPT_OK) ? best : keep;
    if (st != FPT_OK) return st;
    if (chosen) *chosen = ctx->launch;
    return FPT_OK;
}

// ---------------------------------------------------------------------------
// learned proposal
// ---------------------------------------------------------------------------
fpt_status fpt_mlp_pack(fpt_ctx *ctx, const float *params, void *blob, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!params || !blob || (reinterpret_cast<uintptr_t>(blob) & 15) || !is_device_ptr(blob))
        return fail(ctx, FPT_E_INVALID, "need parameters and a 16-byte aligned device blob");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    const float *dp = params;
    if (!is_device_ptr(params)) {
        fpt_status st = ensure_dev(ctx, ctx->d_tmp, ctx->tmp_cap, kMlpParams);
        if (st != FPT_OK) return st;
        CK(cudaMemcpyAsync(ctx->d_tmp, params, sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
        dp = ctx->d_tmp;
        CK(mlp_pack_launch(dp, blob, s));
        CK(cudaStreamSynchronize(s));     // the staging buffer is reused
        return FPT_OK;
    }
    CK(mlp_pack_launch(dp, blob, s));
    return FPT_OK;
}

// Per-block partial gradients of the backward (fixed size per device).
static fpt_status ensure_gpart(fpt_ctx *ctx)
{
    if (ctx->d_gpart) return FPT_OK;
    CK(dev_malloc(ctx, &ctx->d_gpart, sizeof(float) * (size_t)mlp_bwd_max_blocks(ctx->sm_count) * kMlpParams));
    return FPT_OK;
}

fpt_status fpt_mlp_eval(fpt_ctx *ctx, const void *blob, const float *s_in, const float *tan_t, int64_t n,
                        float alpha_max, float *alpha, float *o, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!blob || !s_in || !tan_t || !alpha || n < 1) return fail(ctx, FPT_E_INVALID, "null buffer or n < 1");
    if (!(alpha_max > 0.0f)) return fail(ctx, FPT_E_INVALID, "alpha_max must be positive");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    fpt_status st = ensure_dev(ctx, ctx->d_tmp, ctx->tmp_cap, 7 * n);
    if (st != FPT_OK) return st;
    float *ds = ctx->d_tmp, *dt = ds + 3 * n, *da = dt + n, *dout = da + n;
    CK(cudaMemcpyAsync(ds, s_in, sizeof(float) * 3 * n, cudaMemcpyDefault, s));
    CK(cudaMemcpyAsync(dt, tan_t, sizeof(float) * n, cudaMemcpyDefault, s));
    CK(mlp_eval_launch(blob, ds, dt, n, alpha_max, da, dout, s));
    CK(cudaMemcpyAsync(alpha, da, sizeof(float) * n, cudaMemcpyDefault, s));
    if (o) CK(cudaMemcpyAsync(o, dout, sizeof(float) * 2 * n, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return FPT_OK;
}

fpt_status fpt_mlp_grad(fpt_ctx *ctx, const float *params, const float *s_in, const float *tan_t,
                        const float *dalpha, int64_t n, float alpha_max, float *grad, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!params || !s_in || !tan_t || !dalpha || !grad || n < 1) return fail(ctx, FPT_E_INVALID, "null buffer or n < 1");
    if (!(alpha_max > 0.0f)) return fail(ctx, FPT_E_INVALID, "alpha_max must be positive");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    // records (in0, in1, in2, t, -, -, -, -) and the direct dalpha, built on the host
    std::vector<float> hs(3 * n), ht(n), hd(n), hrec(8 * n, 0.0f), hp(kMlpParams);
    CK(cudaMemcpy(hs.data(), s_in, sizeof(float) * 3 * n, cudaMemcpyDefault));
    CK(cudaMemcpy(ht.data(), tan_t, sizeof(float) * n, cudaMemcpyDefault));
    CK(cudaMemcpy(hd.data(), dalpha, sizeof(float) * n, cudaMemcpyDefault));
    CK(cudaMemcpy(hp.data(), params, sizeof(float) * kMlpParams, cudaMemcpyDefault));
    for (int64_t i = 0; i < n; ++i) {
        hrec[8 * i] = hs[3 * i]; hrec[8 * i + 1] = hs[3 * i + 1]; hrec[8 * i + 2] = hs[3 * i + 2];
        hrec[8 * i + 3] = ht[i];
    }
    fpt_status st = ensure_dev(ctx, ctx->d_tmp, ctx->tmp_cap, 9 * n + 2 * kMlpParams);
    if (st != FPT_OK) return st;
    if ((st = ensure_gpart(ctx)) != FPT_OK) return st;
    float *drec = ctx->d_tmp, *dd = drec + 8 * n, *dp = dd + n, *dg = dp + kMlpParams;
    CK(cudaMemcpyAsync(drec, hrec.data(), sizeof(float) * 8 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dd, hd.data(), sizeof(float) * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dp, hp.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dg, 0, sizeof(float) * kMlpParams, s));
    CK(mlp_bwd_launch(dp, drec, n, nullptr, 0.0f, alpha_max, dd, dg, ctx->sm_count, s, nullptr, ctx->d_gpart));
    CK(cudaMemcpyAsync(grad, dg, sizeof(float) * kMlpParams, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return FPT_OK;
}

fpt_status fpt_mlp_grad2(fpt_ctx *ctx, const float *params, const float *s_in, const float *dbeta, int64_t n,
                         float alpha_max, float *grad, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!params || !s_in || !dbeta || !grad || n < 1) return fail(ctx, FPT_E_INVALID, "null buffer or n < 1");
    if (!(alpha_max > 0.0f)) return fail(ctx, FPT_E_INVALID, "alpha_max must be positive");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    // records (in0, in1, in2, -, ...) and the direct output gradients, built on the host
    std::vector<float> hs(3 * n), hd(2 * n), hrec(8 * n, 0.0f), hp(kMlpParams);
    CK(cudaMemcpy(hs.data(), s_in, sizeof(float) * 3 * n, cudaMemcpyDefault));
    CK(cudaMemcpy(hd.data(), dbeta, sizeof(float) * 2 * n, cudaMemcpyDefault));
    CK(cudaMemcpy(hp.data(), params, sizeof(float) * kMlpParams, cudaMemcpyDefault));
    for (int64_t i = 0; i < n; ++i) {
        hrec[8 * i] = hs[3 * i]; hrec[8 * i + 1] = hs[3 * i + 1]; hrec[8 * i + 2] = hs[3 * i + 2];
    }
    fpt_status st = ensure_dev(ctx, ctx->d_tmp, ctx->tmp_cap, 10 * n + 2 * kMlpParams);
    if (st != FPT_OK) return st;
    if ((st = ensure_gpart(ctx)) != FPT_OK) return st;
    float *drec = ctx->d_tmp, *dd = drec + 8 * n, *dp = dd + 2 * n, *dg = dp + kMlpParams;
    CK(cudaMemcpyAsync(drec, hrec.data(), sizeof(float) * 8 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dd, hd.data(), sizeof(float) * 2 * n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(dp, hp.data(), sizeof(float) * kMlpParams, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(dg, 0, sizeof(float) * kMlpParams, s));
    CK(mlp_bwd_launch(dp, drec, n, nullptr, 0.0f, alpha_max, dd, dg, ctx->sm_count, s, nullptr, ctx->d_gpart, 1));
    CK(cudaMemcpyAsync(grad, dg, sizeof(float) * kMlpParams, cudaMemcpyDefault, s));
    CK(cudaStreamSynchronize(s));
    return FPT_OK;
}

fpt_status fpt_run_records(fpt_ctx *ctx, const fpt_run_desc *run, int64_t cap, float *records,
                           int64_t *n_records, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!run || !n_records || cap < 0 || (cap > 0 && !records)) return fail(ctx, FPT_E_INVALID, "null argument");
    if (run->bias_kind != FPT_BIAS_MLP) return fail(ctx, FPT_E_INVALID, "segment records need an MLP run");
    if (run->model < 0 || run->model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "run model out of range");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    const fpt_model &m = ctx->models[run->model];
    const long long want = std::min<long long>(std::max<long long>(1, run->n_traj) * (m.max_steps / std::max(4, run->mlp_segment) + 2),
                                               1LL << 29);
    if (want > ctx->rec_cap) {
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, ctx->d_records);
        ctx->d_records = nullptr;
        ctx->rec_cap = 0;
        clear_graphs(ctx);
        CK(dev_malloc(ctx, &ctx->d_records, sizeof(float) * 8 * want));
        ctx->rec_cap = want;
    }
    if (!ctx->d_rec_cursor) CK(dev_malloc(ctx, &ctx->d_rec_cursor, 64));
    ctx->record_mode = true;
    fpt_status st = fpt_run(ctx, run, 1, nullptr, s);
    ctx->record_mode = false;
    if (st != FPT_OK) return st;
    st = fpt_sync(ctx);
    if (st == FPT_E_TIMEOUT) return st;
    if (ctx->h_flags[3]) return fail(ctx, FPT_E_NOMEM, "segment records exceed the record buffer");
    unsigned long long n_rec = 0;
    CK(cudaMemcpy(&n_rec, ctx->d_rec_cursor, sizeof(n_rec), cudaMemcpyDeviceToHost));
    *n_records = (int64_t)n_rec;
    const long long k = std::min<long long>((long long)n_rec, cap);
    if (k > 0) CK(cudaMemcpy(records, ctx->d_records, sizeof(float) * 8 * k, cudaMemcpyDefault));
    return st;
}

fpt_status fpt_mlp_train_round(fpt_ctx *ctx, const fpt_run_desc *run, int64_t chunk, double lambda,
                               double N_cut, const fpt_adam *adam, float *params, float *adam_m,
                               float *adam_v, void *blob, fpt_train_stats *stats, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!run || !adam || !params || !adam_m || !adam_v || !blob)
        return fail(ctx, FPT_E_INVALID, "null argument");
    if (run->bias_kind != FPT_BIAS_MLP || run->mlp != blob)
        return fail(ctx, FPT_E_INVALID, "the run must use the MLP proposal stored in blob");
    if (run->n_traj < 2 || chunk < 1) return fail(ctx, FPT_E_INVALID, "need n_traj >= 2 and chunk >= 1");
    if (!std::isfinite(lambda) || !(N_cut > 0)) return fail(ctx, FPT_E_INVALID, "bad lambda or N_cut");
    if (!(adam->lr > 0) || adam->step < 1) return fail(ctx, FPT_E_INVALID, "bad Adam settings");
    if (run->model < 0 || run->model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "run model out of range");
    if (!is_device_ptr(params) || !is_device_ptr(adam_m) || !is_device_ptr(adam_v))
        return fail(ctx, FPT_E_INVALID, "params and Adam moments must be device buffers");
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    const fpt_model &m = ctx->models[run->model];
    const long long n_total = run->n_traj;
    const long long ch = std::min<long long>(chunk, n_total);
    const long long seg_per_traj = m.max_steps / run->mlp_segment + 2;
    const long long want = std::min<long long>(ch * seg_per_traj, 1LL << 29);
    if (want > ctx->rec_cap) {
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, ctx->d_records);
        ctx->d_records = nullptr;
        ctx->rec_cap = 0;
        clear_graphs(ctx);
        CK(dev_malloc(ctx, &ctx->d_records, sizeof(float) * 8 * want));
        ctx->rec_cap = want;
    }
    if (!ctx->d_rec_cursor) CK(dev_malloc(ctx, &ctx->d_rec_cursor, 64));
    if (!ctx->d_acc) CK(dev_malloc(ctx, &ctx->d_acc, sizeof(double) * mlp_coef_scratch_doubles()));
    if (!ctx->d_grad) CK(dev_malloc(ctx, &ctx->d_grad, sizeof(float) * kMlpParams));
    if (!ctx->d_rec_err) CK(dev_malloc(ctx, &ctx->d_rec_err, 64));
    fpt_status st = ensure_dev(ctx, ctx->d_coef, ctx->coef_cap, ch);
    if (st != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_Y, ctx->y_cap, ch)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_perm, ctx->perm_cap, ctx->rec_cap)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_cnt, ctx->cnt_cap, ch)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_off, ctx->off_cap, ch)) != FPT_OK) return st;
    if ((st = ensure_gpart(ctx)) != FPT_OK) return st;
    CK(cudaMemsetAsync(ctx->d_grad, 0, sizeof(float) * kMlpParams, s));
    double sumY = 0, sumY2 = 0, sumN = 0;
    long long n_rec_total = 0, n_capped = 0, n_passed = 0;
    for (long long off = 0; off < n_total; off += ch) {
        fpt_run_desc sub = *run;
        sub.n_traj = std::min(ch, n_total - off);
        sub.traj_offset = run->traj_offset + off;
        ctx->record_mode = true;
        st = fpt_run(ctx, &sub, 1, nullptr, s);
        ctx->record_mode = false;
        if (st != FPT_OK) return st;
        st = fpt_sync(ctx);
        if (st == FPT_E_TIMEOUT) return st;
        if (ctx->h_flags[3]) return fail(ctx, FPT_E_NOMEM, "segment records exceed the record buffer; use a smaller chunk");
        n_capped += ctx->h_flags[1];
        unsigned long long n_rec = 0;
        CK(cudaMemcpy(&n_rec, ctx->d_rec_cursor, sizeof(n_rec), cudaMemcpyDeviceToHost));
        CK(mlp_coef_launch(ctx->d_nsteps, ctx->d_logw, sub.n_traj, m.dN, lambda, N_cut, 2.0 / (double)n_total,
                           ctx->d_Y, ctx->d_acc, ctx->d_coef, s));
        // records in a fixed order (by trajectory, then segment), so that the
        // gradient does not depend on the order the stepper appended them in
        CK(rec_order_launch(ctx->d_records, (long long)n_rec, sub.n_traj, run->mlp_segment, ctx->d_cnt,
                            ctx->d_off, ctx->d_perm, ctx->d_rec_err, s));
        CK(mlp_bwd_launch(params, ctx->d_records, (long long)n_rec, ctx->d_coef, (float)m.dN, run->alpha_max,
                          nullptr, ctx->d_grad, ctx->sm_count, s, ctx->d_perm, ctx->d_gpart,
                          ctx->tables[run->model].rank2 ? 1 : 0));
        double acc[2];
        int rec_err = 0;
        CK(cudaMemcpyAsync(acc, ctx->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&rec_err, ctx->d_rec_err, sizeof(int), cudaMemcpyDeviceToHost, s));
        // mean first-passage time of the chunk
        fpt_hist h;
        std::memset(&h, 0, sizeof(h));
        st = hist_run(ctx, ctx->d_nsteps, ctx->d_logw, ctx->d_status, 0, sub.n_traj, m.dN, 0.0,
                      (double)m.max_steps * m.dN + 1.0, 1, NAN, &h, s);
        if (st != FPT_OK) return st;
        if (rec_err) return fail(ctx, FPT_E_STATE, "segment records out of order (code " + std::to_string(rec_err) + ")");
        sumY += acc[0];
        sumY2 += acc[1];
        sumN += h.N_mean * (double)h.n_passed;
        n_passed += h.n_passed;
        n_rec_total += (long long)n_rec;
    }
    double gn2 = 0.0;
    CK(cudaMemsetAsync(ctx->d_acc, 0, sizeof(double), s));
    grad_norm_kernel<<<1, 256, 0, s>>>(ctx->d_grad, kMlpParams, ctx->d_acc);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(&gn2, ctx->d_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(mlp_adam_launch(params, ctx->d_grad, adam_m, adam_v, kMlpParams, adam->lr, adam->beta1, adam->beta2,
                       adam->eps, adam->step, adam->clip, s));
    CK(mlp_pack_launch(params, blob, s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        const double mY = sumY / (double)n_total;
        stats->loss = sumY2 / (double)n_total - mY * mY;
        stats->mean_Y = mY;
        stats->mean_N = n_passed ? sumN / (double)n_passed : NAN;
        stats->n_traj = n_total;
        stats->n_records = n_rec_total;
        stats->n_capped = n_capped;
        stats->grad_norm = std::sqrt(gn2);
    }
    return FPT_OK;
}

fpt_status fpt_mlp_train_batch(fpt_ctx *ctx, const fpt_run_desc *runs, int32_t n_runs, double lambda,
                               const double *N_cut, const fpt_adam *adam, float *params, float *adam_m,
                               float *adam_v, void *blobs, fpt_train_stats *stats, void *cuda_stream)
{
    if (!ctx) return FPT_E_INVALID;
    if (!runs || n_runs < 1 || n_runs > kMaxRuns || !N_cut || !adam || !params || !adam_m || !adam_v || !blobs)
        return fail(ctx, FPT_E_INVALID, "null argument or n_runs out of [1, 128]");
    if (!(adam->lr > 0) || adam->step < 1) return fail(ctx, FPT_E_INVALID, "bad Adam settings");
    if (!std::isfinite(lambda)) return fail(ctx, FPT_E_INVALID, "bad lambda");
    if (!is_device_ptr(params) || !is_device_ptr(adam_m) || !is_device_ptr(adam_v) || !is_device_ptr(blobs))
        return fail(ctx, FPT_E_INVALID, "params, Adam moments and blobs must be device buffers");
    long long total = 0;
    std::vector<long long> begin(n_runs + 1, 0);
    for (int k = 0; k < n_runs; ++k) {
        const fpt_run_desc &d = runs[k];
        if (d.bias_kind != FPT_BIAS_MLP ||
            d.mlp != static_cast<const char *>(blobs) + (size_t)k * kMlpBlobBytes)
            return fail(ctx, FPT_E_INVALID, "run k must be an MLP run on blob k (blobs + k FPT_MLP_BLOB_BYTES)");
        if (d.model < 0 || d.model >= (int)ctx->models.size()) return fail(ctx, FPT_E_INVALID, "run model out of range");
        if (!(N_cut[k] > 0)) return fail(ctx, FPT_E_INVALID, "N_cut must be positive");
        if (d.n_traj < 2) return fail(ctx, FPT_E_INVALID, "every run needs n_traj >= 2");
        begin[k] = total;
        total += d.n_traj;
    }
    begin[n_runs] = total;
    CK(cudaSetDevice(ctx->device));
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : ctx->stream;
    // record buffer: every run's paths' segments
    long long want = 0;
    for (int k = 0; k < n_runs; ++k)
        want += runs[k].n_traj * (ctx->models[runs[k].model].max_steps / std::max(4, runs[k].mlp_segment) + 2);
    want = std::min<long long>(want, 1LL << 29);
    if (want > ctx->rec_cap) {
        CK(cudaStreamSynchronize(s));
        dev_free(ctx, ctx->d_records);
        ctx->d_records = nullptr;
        ctx->rec_cap = 0;
        clear_graphs(ctx);
        CK(dev_malloc(ctx, &ctx->d_records, sizeof(float) * 8 * want));
        ctx->rec_cap = want;
    }
    const size_t acc_doubles = mlp_coef_scratch_doubles();
    if (!ctx->d_rec_cursor) CK(dev_malloc(ctx, &ctx->d_rec_cursor, 64));
    if (!ctx->d_rec_err) CK(dev_malloc(ctx, &ctx->d_rec_err, 64));
    fpt_status st;
    if ((st = ensure_dev(ctx, ctx->d_coef, ctx->coef_cap, total)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_Y, ctx->y_cap, total)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_perm, ctx->perm_cap, ctx->rec_cap)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_cnt, ctx->cnt_cap, total)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_off, ctx->off_cap, total)) != FPT_OK) return st;
    if ((st = ensure_dev(ctx, ctx->d_tmp, ctx->tmp_cap, (long long)n_runs * kMlpParams)) != FPT_OK) return st;
    if ((st = ensure_gpart(ctx)) != FPT_OK) return st;
    double *d_accs = nullptr;
    CK(dev_malloc(ctx, &d_accs, sizeof(double) * acc_doubles * n_runs));
    struct Free { fpt_ctx *c; double *p; ~Free() { dev_free(c, p); } } free_accs{ctx, d_accs};

    // one launch generates every run's paths with segment records
    ctx->record_mode = true;
    st = fpt_run(ctx, runs, n_runs, nullptr, s);
    ctx->record_mode = false;
    if (st != FPT_OK) return st;
    st = fpt_sync(ctx);
    if (st == FPT_E_TIMEOUT) return st;
    if (ctx->h_flags[3]) return fail(ctx, FPT_E_NOMEM, "segment records exceed the record buffer; use fewer paths");
    unsigned long long n_rec = 0;
    CK(cudaMemcpy(&n_rec, ctx->d_rec_cursor, sizeof(n_rec), cudaMemcpyDeviceToHost));
    // records in (trajectory, segment) order: run k's records are one contiguous range
    CK(rec_order_launch(ctx->d_records, (long long)n_rec, total, runs[0].mlp_segment, ctx->d_cnt, ctx->d_off,
                        ctx->d_perm, ctx->d_rec_err, s));
    std::vector<long long> off(total);
    std::vector<int32_t> nsteps(total);
    std::vector<uint8_t> status(total);
    CK(cudaMemcpyAsync(off.data(), ctx->d_off, sizeof(long long) * total, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(nsteps.data(), ctx->d_nsteps, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(status.data(), ctx->d_status, total, cudaMemcpyDeviceToHost, s));
    int rec_err = 0;
    CK(cudaMemcpyAsync(&rec_err, ctx->d_rec_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (rec_err) return fail(ctx, FPT_E_STATE, "segment records out of order (code " + std::to_string(rec_err) + ")");
    float *d_grads = ctx->d_tmp;
    CK(cudaMemsetAsync(d_grads, 0, sizeof(float) * (size_t)n_runs * kMlpParams, s));
    for (int k = 0; k < n_runs; ++k) {
        const fpt_run_desc &d = runs[k];
        const fpt_model &m = ctx->models[d.model];
        const long long b = begin[k], n = d.n_traj;
        const long long r0 = off[b], r1 = (k + 1 < n_runs) ? off[begin[k + 1]] : (long long)n_rec;
        // coefficients of run k's paths at their launch units (the backward indexes coef by unit)
        CK(mlp_coef_launch(ctx->d_nsteps + b, ctx->d_logw + b, n, m.dN, lambda, N_cut[k], 2.0 / (double)n,
                           ctx->d_Y + b, d_accs + (size_t)k * acc_doubles, ctx->d_coef + b, s));
        CK(mlp_bwd_launch(params + (size_t)k * kMlpParams, ctx->d_records, r1 - r0, ctx->d_coef, (float)m.dN,
                          d.alpha_max, nullptr, d_grads + (size_t)k * kMlpParams, ctx->sm_count, s,
                          ctx->d_perm + r0, ctx->d_gpart, 0, (long long)n_rec));
        CK(mlp_adam_launch(params + (size_t)k * kMlpParams, d_grads + (size_t)k * kMlpParams,
                           adam_m + (size_t)k * kMlpParams, adam_v + (size_t)k * kMlpParams, kMlpParams, adam->lr,
                           adam->beta1, adam->beta2, adam->eps, adam->step, adam->clip, s));
        CK(mlp_pack_launch(params + (size_t)k * kMlpParams, static_cast<char *>(blobs) + (size_t)k * kMlpBlobBytes, s));
        if (stats) {
            stats[k].n_traj = n;
            stats[k].n_records = r1 - r0;
        }
    }
    std::vector<double> accs(acc_doubles * n_runs);
    CK(cudaMemcpyAsync(accs.data(), d_accs, sizeof(double) * accs.size(), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (stats) {
        for (int k = 0; k < n_runs; ++k) {
            const long long b = begin[k], n = runs[k].n_traj;
            const double dN = ctx->models[runs[k].model].dN;
            const double mY = accs[k * acc_doubles] / (double)n;
            stats[k].loss = accs[k * acc_doubles + 1] / (double)n - mY * mY;
            stats[k].mean_Y = mY;
            double sN = 0.0;
            long long passed = 0, capped = 0;
            for (long long i = b; i < b + n; ++i) {
                if (status[i] == FPT_TRAJ_PASSED) { sN += nsteps[i] * dN; ++passed; }
                else if (status[i] == FPT_TRAJ_CAPPED) ++capped;
            }
            stats[k].mean_N = passed ? sN / (double)passed : NAN;
            stats[k].n_capped = capped;
            stats[k].grad_norm = NAN;
        }
    }
    return FPT_OK;
}

fpt_status fpt_histogram_noalloc(const int32_t *nsteps, const double *logw, const uint8_t *status,
                                 int64_t n, double dN, double N_lo, double N_hi, int32_t n_bins,
                                 double N_tail, double *out, void *cuda_stream)
{
    if (!nsteps || !logw || !status || !out || n < 1)
        return fail(nullptr, FPT_E_INVALID, "need n >= 1, three input arrays and an output array");
    if (n_bins < 1 || n_bins > kNoAllocMaxBins)
        return fail(nullptr, FPT_E_INVALID, "n_bins out of [1, FPT_NOALLOC_MAX_BINS = 1024]");
    if (!(dN > 0) || !std::isfinite(dN)) return fail(nullptr, FPT_E_INVALID, "dN must be positive");
    if (!(N_hi > N_lo) || !std::isfinite(N_lo) || !std::isfinite(N_hi))
        return fail(nullptr, FPT_E_INVALID, "need finite N_lo < N_hi");
    if (!((N_hi - N_lo) / n_bins >= DBL_MIN) || !std::isfinite(N_hi - N_lo))
        return fail(nullptr, FPT_E_INVALID, "bin width (N_hi - N_lo) / n_bins must be a positive normal number");
    if (!std::isnan(N_tail) && !std::isfinite(N_tail)) return fail(nullptr, FPT_E_INVALID, "N_tail must be finite or NaN");
    HistParams p;
    std::memset(&p, 0, sizeof(p));
    p.nsteps = nsteps;
    p.logw = logw;
    p.status = status;
    p.unit_begin = 0;
    p.n = n;
    p.dN = dN;
    p.N_lo = N_lo;
    p.db = (N_hi - N_lo) / n_bins;
    p.N_tail = N_tail;
    p.n_bins = n_bins;
    p.chunk = 4096;
    cudaError_t e = hist_noalloc_launch(p, out, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "fpt_histogram_noalloc");
    return FPT_OK;
}

void fpt_destroy(fpt_ctx *ctx)
{
    if (!ctx) return;
    free_all(ctx);
    delete ctx;
}

}  // extern "C"
