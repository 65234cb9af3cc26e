// Host side of the C ABI declared in include/speedup.h.
//
// A plan holds everything that does not depend on the samples: the validated
// arguments, the level-p coefficient tables of every sampled level (generated
// on the host, uploaded once), the launch configuration and the level-0 value.
// Executing a plan launches the sampler (one bisection path per thread) and
// the block combine; finalizing turns the per-block log-sum-exp tuples into
// amplitudes and errors (Sec. 4.1: mean of the normalised e^{-S} and its
// error, here from contiguous sample blocks).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <numeric>
#include <random>
#include <string>
#include <tuple>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/speedup.h"
#include "generator.h"
#include "mlp.cuh"
#include "proposal.h"
#include "fixed_shapes.h"
#include "sampler.h"
#include "spectrum.h"
#include "train.h"

namespace {

thread_local std::string g_err;

// launch shapes stored by su_autotune, per (precision, model, p, s)
struct TuneKey {
    int precision, model, p, s;
    bool operator<(const TuneKey &o) const {
        return std::tie(precision, model, p, s) < std::tie(o.precision, o.model, o.p, o.s);
    }
};
std::mutex g_tune_mu;
std::map<TuneKey, su_tuning> g_tune;

// register segments stored by su_batch_autotune, per (precision, model, p, s, hierarchy)
struct BatchTuneKey {
    int precision, model, p, s, hier;
    bool operator<(const BatchTuneKey &o) const {
        return std::tie(precision, model, p, s, hier) < std::tie(o.precision, o.model, o.p, o.s, o.hier);
    }
};
std::map<BatchTuneKey, int> g_btune;

bool tuned_shape(int precision, int model, int p, int s, su_tuning &out) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({precision, model, p, s});
    if (it == g_tune.end()) return false;
    out = it->second;
    return true;
}

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();   // not sticky: clear it for the next call
        return fail(SU_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(SU_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// ---- fault injection (test support; every hook off unless su_fault_inject
// turned it on)
std::atomic<int64_t> g_fault_alloc{0};     // > 0: that allocation from now fails
std::atomic<int> g_fault_table_nan{0};     // the next coefficient table gets a NaN
std::atomic<int64_t> g_fault_queue{0};     // > 0: batched launches stop after that many items
std::atomic<int> g_fault_mma{0};           // the next proposal launch withholds its MMA commit

bool take_alloc_fault() {
    int64_t c = g_fault_alloc.load();
    while (c > 0) {
        if (g_fault_alloc.compare_exchange_weak(c, c - 1)) return c == 1;
    }
    return false;
}

// device allocations of this file go through these two (with the hook)
cudaError_t dmalloc(void **p, size_t bytes) {
    if (take_alloc_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dmalloc_async(void **p, size_t bytes, cudaStream_t st) {
    if (take_alloc_fault()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

template <typename T>
cudaError_t dmalloc(T **p, size_t bytes) {
    return dmalloc(reinterpret_cast<void **>(p), bytes);
}
template <typename T>
cudaError_t dmalloc_async(T **p, size_t bytes, cudaStream_t st) {
    return dmalloc_async(reinterpret_cast<void **>(p), bytes, st);
}

#define CU(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr int64_t kMaxSamples = (int64_t)1 << 40;
constexpr int64_t kMaxBlocks = (int64_t)1 << 20;

double log_A_free(double a, double b, double T) {
    return -0.5 * std::log(2.0 * M_PI * T) - (b - a) * (b - a) / (2.0 * T);
}

}  // namespace

struct su_plan {
    int model = 0;
    std::vector<double> params;
    double a = 0, b = 0, T = 1;
    int p = 1, s = 0;
    int64_t n_mc = 1;
    uint64_t seed = 0;
    su_options opt{};
    su::Effective E;
    double w0 = 0;            // level-0 log-weight -T W_p((a+b)/2, (b-a)/2; T)
    double laf = 0;           // log of the free amplitude
    int levels = 0;           // sampled levels
    int64_t n_blocks = 1;
    su::SamplerParams P{};
    void *d_tables = nullptr;
    int device = 0;
    int grid = 0;
    size_t smem = 0;
    int64_t tuple_bytes = 0, scratch_bytes = 0, partial_bytes = 0;
    int64_t slice_actions = 0;
    double cancel_ratio = 1;  // largest sum|terms| / |sum| in the table collapse
    // SU_GENERAL: the monomial program of W_p, the potential's families and
    // their device image (GeneralDev | nodes)
    std::shared_ptr<const su::GeneralEffective> G;
    su::GeneralPotential V{};
    void *d_general = nullptr;
    // systems of several coordinates (su_plan_create_nd): d, the program, the
    // kernel's parameters and the bytes of its path scratch
    int nd = 0;
    std::vector<double> nd_a, nd_b;
    su::NdEffective N;
    su::NdParams Q{};
    int64_t path_bytes = 0;
};

namespace {

// The monomial program of W_p for a general potential depends on p only;
// built once per p (milliseconds at p = 12) and shared.
std::shared_ptr<const su::GeneralEffective> general_program(int p, int &rc, std::string &err) {
    static std::mutex mu;
    static std::map<int, std::shared_ptr<const su::GeneralEffective>> cache;
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(p);
    if (it != cache.end()) {
        rc = SU_OK;
        return it->second;
    }
    auto G = std::make_shared<su::GeneralEffective>();
    rc = su::build_general(p, *G, err);
    if (rc) return nullptr;
    cache.emplace(p, G);
    return G;
}

}  // namespace

extern "C" {

void su_options_default(su_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->precision = SU_FP64;
    o->n_blocks = 64;
    o->hierarchy = 1;
    o->instance = 0;
    o->width_factor = 1.0;
    o->stream = nullptr;
    o->sample0 = 0;
}

const char *su_last_error(void) { return g_err.c_str(); }

int su_version(char *buf, int cap) {
    if (!buf || cap <= 0) return fail(SU_EINVAL, "buffer missing");
    int rt = 0, drv = 0, dev = -1, n = 0;
    cudaRuntimeGetVersion(&rt);
    cudaDriverGetVersion(&drv);
    std::string s = "speedup-gb300 1 (sm_103a); cudart " + std::to_string(rt) + ", driver " +
                    std::to_string(drv);
    if (cudaGetDeviceCount(&n) == cudaSuccess && n > 0 && cudaGetDevice(&dev) == cudaSuccess) {
        cudaDeviceProp pr;
        if (cudaGetDeviceProperties(&pr, dev) == cudaSuccess)
            s += std::string("; device ") + pr.name + ", " + std::to_string(pr.multiProcessorCount) +
                 " SMs, cc " + std::to_string(pr.major) + "." + std::to_string(pr.minor);
    } else {
        cudaGetLastError();
        s += "; no CUDA device";
    }
    std::snprintf(buf, (size_t)cap, "%s", s.c_str());
    return SU_OK;
}

int speedup_generate_coeffs(int model, const double *params, int n_params, int p, double eps,
                            double *table, int capacity, int *shape, int *n_terms) {
    if (!(eps > 0) || !std::isfinite(eps)) return fail(SU_EINVAL, "eps must be finite and > 0");
    if (!table || !shape || !n_terms || capacity < 0) return fail(SU_EINVAL, "output missing");
    if (model == SU_GENERAL) return fail(SU_ENOTSUP, "the general potential has no collapsed table");
    su::Effective E;
    std::string err;
    int rc = su::build_effective(model, params, n_params, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    std::vector<double> P;
    su::collapse(E, eps, P);
    *n_terms = (int)P.size();
    shape[0] = E.shape.ncol;
    shape[1] = E.shape.ring;
    for (int j = 0; j < SU_MAX_P; ++j) shape[2 + j] = j < E.shape.ncol ? E.shape.len[j] : 0;
    if ((int)P.size() > capacity) return fail(SU_ENOTSUP, "table needs %d entries", (int)P.size());
    for (size_t i = 0; i < P.size(); ++i) {
        if (!std::isfinite(P[i])) return fail(SU_ENONFINITE, "non-finite coefficient");
        table[i] = P[i];
    }
    return SU_OK;
}

static int validate(int model, const double *params, int n_params, double a, double b, double T,
                    int p, int s, int64_t n_mc, const su_options &o) {
    (void)params;
    (void)n_params;
    if (!std::isfinite(a) || !std::isfinite(b)) return fail(SU_EINVAL, "a and b must be finite");
    if (!(T > 0) || !std::isfinite(T)) return fail(SU_EINVAL, "T must be finite and > 0");
    if (p < 1 || p > SU_MAX_P) return fail(SU_EINVAL, "p must be in 1..%d", SU_MAX_P);
    if (s < 0 || s > SU_MAX_S) return fail(SU_EINVAL, "s must be in 0..%d", SU_MAX_S);
    if (n_mc < 1 || n_mc > kMaxSamples) return fail(SU_EINVAL, "n_mc must be in 1..2^40");
    if (o.precision != SU_FP64 && o.precision != SU_FP32) return fail(SU_EINVAL, "unknown precision");
    if (o.n_blocks < 1 || o.n_blocks > kMaxBlocks) return fail(SU_EINVAL, "n_blocks must be in 1..2^20");
    if (!(o.width_factor > 0) || !std::isfinite(o.width_factor))
        return fail(SU_EINVAL, "width_factor must be finite and > 0");
    if (o.sample0 < 0 || o.sample0 + n_mc > kMaxSamples) return fail(SU_EINVAL, "sample0 out of range");
    if (o.seg_log2 < 0 || o.seg_log2 > su::kMaxFine) return fail(SU_EINVAL, "seg_log2 must be in 0..5");
    if (o.rounds < 0 || o.rounds > 8) return fail(SU_EINVAL, "rounds must be in 0..8");
    if (o.kernel != 0 && o.kernel != 1) return fail(SU_EINVAL, "kernel must be 0 or 1");
    if (model == SU_GENERAL) {
        if (p > su::kGenMaxP) return fail(SU_ENOTSUP, "the general potential supports p <= %d", su::kGenMaxP);
        if (o.precision != SU_FP64) return fail(SU_ENOTSUP, "the general potential is evaluated in double only");
    }
    return SU_OK;
}

// Device image of the general program and potential: one allocation holding
// GeneralDev and the depth-first nodes.
static int general_image(const su::GeneralEffective &G, const su::GeneralPotential &V, void **d_out) {
    using namespace su;
    *d_out = nullptr;
    GeneralDev D;
    std::memset(&D, 0, sizeof D);
    D.J = G.J;
    D.K = G.K;
    D.n_nodes = (int)G.depth.size();
    D.n_entries = (int)G.entry_k.size();
    D.ng = V.ng;
    D.ns = V.ns;
    D.ne = V.ne;
    for (int q = 0; q < V.ne; ++q)
        for (int r = 0; r < 3; ++r) D.expo[q][r] = V.expo[q][r];
    if (G.J >= kGenMaxSym || G.K > kGenMaxP) return fail(SU_EINVAL, "internal: general program out of range");
    std::vector<GeneralNode> nodes((size_t)D.n_nodes);
    for (int t = 0; t < D.n_nodes; ++t) {
        if (G.depth[(size_t)t] > kGenMaxDepth || G.count[(size_t)t] > 65535)
            return fail(SU_EINVAL, "internal: general program node out of range");
        nodes[(size_t)t].depth = (unsigned char)G.depth[(size_t)t];
        nodes[(size_t)t].sym = (unsigned char)G.sym[(size_t)t];
        nodes[(size_t)t].count = (unsigned short)G.count[(size_t)t];
        nodes[(size_t)t].first = G.first[(size_t)t];
    }
    for (int t = 0; t < D.n_nodes; ++t)   // the device takes a node's entries as vs^0, vs^2, ..
        for (int e = 0; e < G.count[(size_t)t]; ++e)
            if (G.entry_k[(size_t)(G.first[(size_t)t] + e)] != e)
                return fail(SU_EINVAL, "internal: general program entries out of order");
    for (int j = 0; j <= std::min(G.J, 8); ++j)   // V^(j) of the polynomial: a_i i!/(i-j)!
        for (int i = j; i <= 8; ++i) {
            double f = 1.0;
            for (int r = 0; r < j; ++r) f *= (double)(i - r);
            D.poly_der[j][i] = V.a[i] * f;
        }
    for (int g = 0; g < V.ng; ++g) {
        for (int r = 0; r < 3; ++r) D.gauss[g][r] = V.gauss[g][r];
        D.gauss[g][3] = std::sqrt(V.gauss[g][1]);
    }
    for (int q = 0; q < V.ns; ++q) {
        for (int r = 0; r < 3; ++r) D.sech[q][r] = V.sech[q][r];
        double sc = V.sech[q][0];                  // B alpha^n (n+1)!
        for (int n = 0; n <= G.J; ++n) {
            sc *= (double)(n + 1);
            D.sech_scale[q][n] = sc;
            sc *= V.sech[q][1];
        }
    }
    for (int n = 1; n <= kGenMaxSym; ++n) D.inv[n] = 1.0 / (double)n;
    const size_t o_nodes = (sizeof(GeneralDev) + 15) & ~(size_t)15;
    const size_t bytes = o_nodes + nodes.size() * sizeof(GeneralNode);
    CU(dmalloc(d_out, bytes), "device allocation (general program)");
    char *base = static_cast<char *>(*d_out);
    D.nodes = reinterpret_cast<const GeneralNode *>(base + o_nodes);
    std::vector<unsigned char> blob(bytes, 0);
    std::memcpy(blob.data(), &D, sizeof D);
    std::memcpy(blob.data() + o_nodes, nodes.data(), nodes.size() * sizeof(GeneralNode));
    CU(cudaMemcpy(*d_out, blob.data(), bytes, cudaMemcpyHostToDevice), "upload general program");
    return SU_OK;
}

static int upload_general(su_plan &pl) { return general_image(*pl.G, pl.V, &pl.d_general); }

// The level tables of a plan (rows d = 0..S-1 for levels n = S..1), each
// scaled for the kernel and rounded to its precision: host work only.
static int plan_tables(su_plan &pl, std::vector<unsigned char> &blob) {
    using namespace su;
    const int S = pl.s;
    const int prec = pl.opt.precision;
    const size_t rs = prec == SU_FP32 ? sizeof(float) : sizeof(double);
    const bool general = pl.model == SU_GENERAL;
    const int M = general ? (int)pl.G->entry_k.size() : pl.E.shape.M;
    std::vector<double> tabd((size_t)std::max(S, 1) * M, 0.0);
    for (int d = 0; d < S; ++d) {
        const int n = S - d;
        const double eps = pl.T / std::ldexp(1.0, n);
        std::vector<double> t;
        if (general)
            su::general_table(*pl.G, eps, t);
        else
            pl.cancel_ratio = std::max(pl.cancel_ratio, su::kernel_table(pl.E, eps, t));
        if (g_fault_table_nan.exchange(0)) t[0] = NAN;   // fault injection
        for (int i = 0; i < M; ++i) {
            if (!std::isfinite(t[i]) || (prec == SU_FP32 && !std::isfinite((float)t[i])))
                return fail(SU_ENONFINITE, "non-finite coefficient at level %d", n);
            tabd[(size_t)d * M + i] = t[i];
        }
    }
    blob.assign(tabd.size() * rs, 0);
    if (prec == SU_FP32)
        for (size_t i = 0; i < tabd.size(); ++i) reinterpret_cast<float *>(blob.data())[i] = (float)tabd[i];
    else
        std::memcpy(blob.data(), tabd.data(), blob.size());
    return SU_OK;
}

// Work decomposition of a plan for `rounds` paths per thread per item:
// items of 128 * rounds samples, the persistent grid and the buffer sizes.
// Returns the resident CTAs per SM (0 when the shared memory does not fit).
static int plan_rounds(su_plan &pl, int rounds, int sms, int smem_max) {
    using namespace su;
    SamplerParams &P = pl.P;
    const int prec = pl.opt.precision;
    P.rounds = rounds;
    const int chunk = kThreads * rounds;
    const int64_t bsz = (pl.n_mc + pl.n_blocks - 1) / pl.n_blocks;
    P.items_per_block = (bsz + chunk - 1) / chunk;
    P.n_items = P.items_per_block * pl.n_blocks;
    pl.smem = sampler_smem_bytes(P, prec);
    const int occ = pl.smem > (size_t)smem_max ? 0 : sampler_occupancy(P, prec, pl.smem);
    pl.grid = (int)std::min<int64_t>(P.n_items, (int64_t)sms * std::max(occ, 1));
    pl.partial_bytes = P.n_items * pl.levels * 4 * (int64_t)sizeof(double);
    pl.scratch_bytes = ((pl.partial_bytes + 255) / 256) * 256 + 256;
    return occ;
}

// The sampler's parameters and launch shape of a plan (everything but the
// device pointers): host work and occupancy queries only, no allocation.
static int plan_shape(su_plan &pl, int sms, int smem_max) {
    using namespace su;
    SamplerParams &P = pl.P;
    const int S = pl.s;
    const int prec = pl.opt.precision;
    const bool general = pl.model == SU_GENERAL;
    const int M = general ? (int)pl.G->entry_k.size() : pl.E.shape.M;
    std::memset(&P, 0, sizeof P);
    P.a = pl.a;
    P.b = pl.b;
    for (int n = 1; n <= S; ++n) P.sigma[n] = pl.opt.width_factor * std::sqrt(pl.T / std::ldexp(1.0, n + 1));
    // launch shape: explicit, else stored by su_autotune, else the rule
    su_tuning tuned{};
    const bool have_tuned = tuned_shape(prec, pl.model, pl.p, S, tuned);
    // rule: 16-slice register segments in double (measured 1-5 % faster than
    // 32 at 2 CTAs per SM), 32 in single precision and for the general
    // potential (4 CTAs per SM; 32 beat 8 and 16 by 25 % and 11 % at N = 1024)
    const int seg_rule = (general || prec != SU_FP64) ? kMaxFine : 4;
    int seg = pl.opt.seg_log2 > 0 ? pl.opt.seg_log2 : (have_tuned ? tuned.seg_log2 : seg_rule);
    P.S = S;
    P.F = std::min(S, std::max(1, seg));
    P.levels = pl.levels;
    P.wf_on = pl.opt.width_factor != 1.0;
    P.lwf = std::log(pl.opt.width_factor);
    P.hcoef = 0.5 * (1.0 - pl.opt.width_factor * pl.opt.width_factor);
    P.ring = general ? RING_GENERAL : pl.E.shape.ring;
    P.ncol = general ? 0 : pl.E.shape.ncol;
    P.M = M;
    for (int j = 0; j < P.ncol; ++j) P.len[j] = pl.E.shape.len[j];
    P.alpha = general ? 0.0 : pl.E.shape.alpha;
    P.seed = pl.seed;
    P.instance = pl.opt.instance;
    P.n_mc = pl.n_mc;
    P.sample0 = pl.opt.sample0;
    P.n_blocks = pl.n_blocks;

    // tables too large to stage next to the rest (the highest levels) are
    // read from global memory instead
    P.rounds = 1;
    P.tab_global = 0;
    P.generic = pl.opt.kernel == 1;
    if (sampler_smem_bytes(P, prec) > (size_t)smem_max) {
        if (prec != SU_FP64) return fail(SU_ENOTSUP, "the level tables do not fit shared memory in single precision");
        P.tab_global = 1;
    }
    // launch shape: one path per thread, persistent grid over items of
    // 128 * rounds samples
    const int occ1 = plan_rounds(pl, 1, sms, smem_max);
    if (pl.smem > (size_t)smem_max)
        return fail(SU_ENOTSUP, "shared memory %zu exceeds %d bytes", pl.smem, smem_max);
    if (occ1 < 1) return fail(SU_ECUDA, "sampler cannot be resident (%s)", cudaGetErrorString(cudaGetLastError()));
    // rule: one path per thread per item (the per-item reduction is cheap next
    // to the sampling, and small items leave no tail), more only to keep the
    // per-item tuples under 512 MB, and only while as many CTAs stay resident
    int rounds = 1;
    while (rounds < 8 && P.n_items * pl.levels * 32 > ((int64_t)512 << 20)) plan_rounds(pl, rounds *= 2, sms, smem_max);
    while (rounds > 1 && plan_rounds(pl, rounds, sms, smem_max) < occ1) rounds /= 2;
    if (pl.opt.rounds > 0 || (have_tuned && tuned.rounds > 0)) {
        rounds = pl.opt.rounds > 0 ? pl.opt.rounds : tuned.rounds;
        if (plan_rounds(pl, rounds, sms, smem_max) < 1)
            return fail(SU_ENOTSUP, "rounds = %d does not fit (shared memory %zu bytes)", rounds, pl.smem);
    }
    plan_rounds(pl, rounds, sms, smem_max);
    pl.tuple_bytes = pl.n_blocks * pl.levels * 4 * (int64_t)sizeof(double);
    const int64_t N = (int64_t)1 << S;
    pl.slice_actions = pl.n_mc * (pl.levels > 1 ? 2 * N - 2 : N);
    if (S == 0) pl.slice_actions = 0;
    return SU_OK;
}

// The current device's SM count and opt-in shared memory per CTA.
static int device_limits(int &dev, int &sms, int &smem_max) {
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SU_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    CU(cudaGetDevice(&dev), "cudaGetDevice");
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem limit");
    return SU_OK;
}

static int configure(su_plan &pl) {
    std::vector<unsigned char> blob;
    int rc = plan_tables(pl, blob);
    if (rc) return rc;
    int sms = 0, smem_max = 0;
    rc = device_limits(pl.device, sms, smem_max);
    if (rc) return rc;
    rc = plan_shape(pl, sms, smem_max);
    if (rc) return rc;
    CU(dmalloc(&pl.d_tables, blob.size()), "device allocation (tables)");
    CU(cudaMemcpy(pl.d_tables, blob.data(), blob.size(), cudaMemcpyHostToDevice), "upload tables");
    if (pl.model == SU_GENERAL) {
        rc = upload_general(pl);
        if (rc) return rc;
    }
    pl.P.tables = pl.d_tables;
    pl.P.general = static_cast<const su::GeneralDev *>(pl.d_general);
    return SU_OK;
}

// Validated arguments, the effective action and the level-0 value of a plan
// (host only).
static int plan_init(su_plan &pl, int model, const double *params, int n_params, double a, double b, double T,
                     int p, int s, int64_t n_mc, uint64_t seed, const su_options &o) {
    int rc = validate(model, params, n_params, a, b, T, p, s, n_mc, o);
    if (rc) return rc;
    std::string err;
    if (model == SU_GENERAL) {
        rc = su::general_potential(params, n_params, pl.V, err);
        if (!rc) pl.G = general_program(p, rc, err);
    } else {
        rc = su::build_effective(model, params, n_params, p, pl.E, err);
    }
    if (rc) return fail(rc, "%s", err.c_str());
    pl.model = model;
    pl.params.assign(params, params + n_params);
    pl.a = a;
    pl.b = b;
    pl.T = T;
    pl.p = p;
    pl.s = s;
    pl.n_mc = n_mc;
    pl.seed = seed;
    pl.opt = o;
    pl.levels = s == 0 ? 0 : (o.hierarchy ? s : 1);
    pl.n_blocks = std::min<int64_t>(o.n_blocks, n_mc);
    pl.w0 = model == SU_GENERAL ? -T * su::general_wp_host(*pl.G, pl.V, 0.5 * (a + b), 0.5 * (b - a), T)
                                : -T * su::wp_host(pl.E, 0.5 * (a + b), 0.5 * (b - a), T);
    pl.laf = log_A_free(a, b, T);
    if (!std::isfinite(pl.w0) && !(std::isinf(pl.w0) && pl.w0 < 0))
        return fail(SU_ENONFINITE, "level-0 weight is not finite");
    return SU_OK;
}

int su_plan_create(int model, const double *params, int n_params, double a, double b, double T,
                   int p, int s, int64_t n_mc, uint64_t seed, const su_options *opt, su_plan **out) {
    if (!out) return fail(SU_EINVAL, "plan pointer missing");
    *out = nullptr;
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    std::unique_ptr<su_plan> pl(new (std::nothrow) su_plan);
    if (!pl) return fail(SU_ENOMEM, "host allocation failed");
    int rc = plan_init(*pl, model, params, n_params, a, b, T, p, s, n_mc, seed, o);
    if (rc) return rc;
    rc = configure(*pl);
    if (rc) {
        if (pl->d_tables) cudaFree(pl->d_tables);
        if (pl->d_general) cudaFree(pl->d_general);
        return rc;
    }
    *out = pl.release();
    return SU_OK;
}

// Tables, program and launch shape of a system of several coordinates.
static int configure_nd(su_plan &pl) {
    using namespace su;
    const int S = pl.s;
    const int M = (int)pl.N.hi.size();
    const int prec = pl.opt.precision;
    std::vector<double> tabd((size_t)std::max(S, 1) * M, 0.0);
    for (int d = 0; d < S; ++d) {
        const double eps = pl.T / std::ldexp(1.0, S - d);
        std::vector<double> t;
        nd_table(pl.N, eps, t);
        if (g_fault_table_nan.exchange(0)) t[0] = NAN;   // fault injection
        for (int i = 0; i < M; ++i) {
            if (!std::isfinite(t[(size_t)i]) || (prec == SU_FP32 && !std::isfinite((float)t[(size_t)i])))
                return fail(SU_ENONFINITE, "non-finite coefficient at level %d", S - d);
            tabd[(size_t)d * M + i] = t[(size_t)i];
        }
    }
    const size_t rs = prec == SU_FP32 ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> blob(tabd.size() * rs);
    if (prec == SU_FP32)
        for (size_t i = 0; i < tabd.size(); ++i) reinterpret_cast<float *>(blob.data())[i] = (float)tabd[i];
    else
        std::memcpy(blob.data(), tabd.data(), blob.size());
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SU_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    CU(cudaGetDevice(&pl.device), "cudaGetDevice");
    int sms = 0;
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, pl.device), "SM count");
    CU(dmalloc(&pl.d_tables, blob.size()), "device allocation (tables)");
    CU(cudaMemcpy(pl.d_tables, blob.data(), blob.size(), cudaMemcpyHostToDevice), "upload tables");
    std::vector<GeneralNode> nodes(pl.N.depth.size());
    for (size_t t = 0; t < nodes.size(); ++t) {
        if (pl.N.count[t] > 65535) return fail(SU_ENOTSUP, "a monomial group has more than 65535 entries");
        nodes[t].depth = (unsigned char)pl.N.depth[t];
        nodes[t].sym = (unsigned char)pl.N.sym[t];
        nodes[t].count = (unsigned short)pl.N.count[t];
        nodes[t].first = pl.N.first[t];
    }
    CU(dmalloc(&pl.d_general, nodes.size() * sizeof(GeneralNode)), "device allocation (program)");
    CU(cudaMemcpy(pl.d_general, nodes.data(), nodes.size() * sizeof(GeneralNode), cudaMemcpyHostToDevice),
       "upload program");

    SamplerParams &P = pl.P;
    std::memset(&P, 0, sizeof P);
    for (int n = 1; n <= S; ++n) P.sigma[n] = std::sqrt(pl.T / std::ldexp(1.0, n + 1));
    P.S = S;
    P.F = 0;
    P.rounds = 1;
    P.levels = pl.levels;
    P.M = M;
    P.tables = pl.d_tables;
    P.seed = pl.seed;
    P.instance = pl.opt.instance;
    P.n_mc = pl.n_mc;
    P.sample0 = pl.opt.sample0;
    P.n_blocks = pl.n_blocks;
    const int64_t bsz = (pl.n_mc + pl.n_blocks - 1) / pl.n_blocks;
    P.items_per_block = (bsz + kThreads - 1) / kThreads;
    P.n_items = P.items_per_block * pl.n_blocks;
    NdParams &Q = pl.Q;
    std::memset(&Q, 0, sizeof Q);
    Q.base = P;
    Q.D = pl.nd;
    Q.H = pl.N.H;
    Q.G = pl.N.G;
    Q.n_nodes = (int)nodes.size();
    Q.nodes = static_cast<const GeneralNode *>(pl.d_general);
    for (int c = 0; c < pl.nd; ++c) {
        Q.a[c] = pl.nd_a[(size_t)c];
        Q.b[c] = pl.nd_b[(size_t)c];
    }
    pl.smem = nd_smem_bytes(Q, prec);
    const int occ = nd_occupancy(Q, prec, pl.smem);
    if (occ < 1) return fail(SU_ECUDA, "sampler cannot be resident (%s)", cudaGetErrorString(cudaGetLastError()));
    pl.grid = (int)std::min<int64_t>(P.n_items, (int64_t)sms * occ);
    Q.pstride = (int64_t)pl.grid * kThreads;
    pl.path_bytes = Q.pstride * (((int64_t)1 << (S - std::min(S, kNdSeg))) + 1) * pl.nd * (int64_t)rs;
    pl.partial_bytes = P.n_items * pl.levels * 4 * (int64_t)sizeof(double);
    pl.scratch_bytes = ((pl.partial_bytes + 255) / 256) * 256 + ((pl.path_bytes + 255) / 256) * 256 + 256;
    pl.tuple_bytes = pl.n_blocks * pl.levels * 4 * (int64_t)sizeof(double);
    const int64_t N = (int64_t)1 << S;
    pl.slice_actions = S == 0 ? 0 : pl.n_mc * (pl.levels > 1 ? 2 * N - 2 : N);
    return SU_OK;
}

int su_plan_create_nd(int d, const int *exps, const double *coefs, int n_terms, const double *a, const double *b,
                      double T, int p, int s, int64_t n_mc, uint64_t seed, const su_options *opt, su_plan **out) {
    if (!out) return fail(SU_EINVAL, "plan pointer missing");
    *out = nullptr;
    if (d < 1 || d > su::kNdMaxDim) return fail(SU_EINVAL, "d must be in 1..%d", su::kNdMaxDim);
    if (!a || !b) return fail(SU_EINVAL, "endpoints missing");
    for (int c = 0; c < d; ++c)
        if (!std::isfinite(a[c]) || !std::isfinite(b[c])) return fail(SU_EINVAL, "a and b must be finite");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    int rc = validate(-1, nullptr, 0, a[0], b[0], T, p, s, n_mc, o);
    if (rc) return rc;
    if (p > su::kNdMaxP) return fail(SU_ENOTSUP, "systems of several coordinates support p <= %d", su::kNdMaxP);
    if (o.width_factor != 1.0) return fail(SU_ENOTSUP, "systems of several coordinates sample the exact bridge only");
    if (o.seg_log2 != 0 || o.rounds > 1) return fail(SU_ENOTSUP, "systems of several coordinates have one launch shape");
    std::unique_ptr<su_plan> pl(new (std::nothrow) su_plan);
    if (!pl) return fail(SU_ENOMEM, "host allocation failed");
    std::string err;
    rc = su::build_nd(d, exps, coefs, n_terms, p, pl->N, err);
    if (rc) return fail(rc, "%s", err.c_str());
    pl->model = -1;
    pl->nd = d;
    pl->nd_a.assign(a, a + d);
    pl->nd_b.assign(b, b + d);
    pl->a = a[0];
    pl->b = b[0];
    pl->T = T;
    pl->p = p;
    pl->s = s;
    pl->n_mc = n_mc;
    pl->seed = seed;
    pl->opt = o;
    pl->levels = s == 0 ? 0 : (o.hierarchy ? s : 1);
    pl->n_blocks = std::min<int64_t>(o.n_blocks, n_mc);
    double xm[su::kNdMaxDim], xh[su::kNdMaxDim];
    pl->laf = 0.0;
    for (int c = 0; c < d; ++c) {
        xm[c] = 0.5 * (a[c] + b[c]);
        xh[c] = 0.5 * (b[c] - a[c]);
        pl->laf += log_A_free(a[c], b[c], T);
    }
    pl->w0 = -T * su::nd_wp_host(pl->N, xm, xh, T);
    if (!std::isfinite(pl->w0) && !(std::isinf(pl->w0) && pl->w0 < 0))
        return fail(SU_ENONFINITE, "level-0 weight is not finite");
    rc = configure_nd(*pl);
    if (rc) {
        if (pl->d_tables) cudaFree(pl->d_tables);
        if (pl->d_general) cudaFree(pl->d_general);
        return rc;
    }
    *out = pl.release();
    return SU_OK;
}

int su_plan_destroy(su_plan *pl) {
    if (!pl) return SU_OK;
    if (pl->d_tables) cudaFree(pl->d_tables);
    if (pl->d_general) cudaFree(pl->d_general);
    delete pl;
    return SU_OK;
}

int su_plan_sizes(const su_plan *pl, int64_t *tuple_bytes, int64_t *scratch_bytes, int *levels,
                  int64_t *slice_actions) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (tuple_bytes) *tuple_bytes = pl->tuple_bytes;
    if (scratch_bytes) *scratch_bytes = pl->scratch_bytes;
    if (levels) *levels = pl->levels;
    if (slice_actions) *slice_actions = pl->slice_actions;
    return SU_OK;
}

int su_plan_shape(const su_plan *pl, int *seg_log2, int *rounds) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (seg_log2) *seg_log2 = pl->s > 0 ? pl->P.F : 0;
    if (rounds) *rounds = pl->s > 0 ? pl->P.rounds : 0;
    return SU_OK;
}

int su_plan_kernel(const su_plan *pl, int *fixed_shape) {
    if (!pl || !fixed_shape) return fail(SU_EINVAL, "plan or output missing");
    *fixed_shape = pl->s > 0 ? su::sampler_fixed_shape(pl->P, pl->opt.precision) : -1;
    return SU_OK;
}

int su_fixed_shape(int model, const double *params, int n_params, int p, int *index) {
    if (!index) return fail(SU_EINVAL, "output missing");
    if (model == SU_GENERAL) return fail(SU_ENOTSUP, "the general potential has no collapsed table");
    su::Effective E;
    std::string err;
    const int rc = su::build_effective(model, params, n_params, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    *index = E.shape.ring == su::RING_EVEN ? su::fixed_shape_index(E.shape.ncol, E.shape.len.data()) : -1;
    return SU_OK;
}

int su_plan_execute(su_plan *pl, void *d_tuples, void *d_scratch, void *stream, int *launches) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    return su_plan_execute_range(pl, 0, pl->n_blocks, d_tuples, d_scratch, stream, launches);
}

int su_plan_execute_range(su_plan *pl, int64_t b0, int64_t b1, void *d_tuples, void *d_scratch, void *stream,
                          int *launches) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (launches) *launches = 0;
    if (b0 < 0 || b1 > pl->n_blocks || b0 > b1) return fail(SU_EINVAL, "block range out of 0..%lld", (long long)pl->n_blocks);
    if (pl->s == 0 || b0 == b1) return SU_OK;  // level 0 is analytic: nothing to sample
    if (!d_tuples || !d_scratch) return fail(SU_EINVAL, "device buffers missing");
    cudaStream_t st = (cudaStream_t)stream;
    su::SamplerParams P = pl->P;
    P.item0 = b0 * P.items_per_block;
    P.n_items = b1 * P.items_per_block;
    const int grid = (int)std::min<int64_t>(pl->grid, P.n_items - P.item0);
    P.partial = static_cast<double *>(d_scratch);
    P.flags = reinterpret_cast<int *>(static_cast<char *>(d_scratch) + pl->scratch_bytes - 256);
    P.w_out = nullptr;
    CU(cudaMemsetAsync(P.flags, 0, sizeof(int), st), "clear flags");
    if (pl->nd) {
        su::NdParams Q = pl->Q;
        Q.base = P;
        Q.paths = static_cast<char *>(d_scratch) + ((pl->partial_bytes + 255) / 256) * 256;
        CU(su::launch_nd(Q, pl->opt.precision, grid, pl->smem, st), "sampler launch");
    } else {
        CU(su::launch_sampler(P, pl->opt.precision, grid, pl->smem, st), "sampler launch");
    }
    CU(su::launch_combine(P.partial, static_cast<double *>(d_tuples), b0, b1 - b0, pl->levels, P.items_per_block,
                          st),
       "combine launch");
    if (launches) *launches = 2;
    return SU_OK;
}

int su_plan_execute_timed(su_plan *pl, void *d_tuples, void *d_scratch, void *stream, int *launches, float *ms) {
    if (!ms) return fail(SU_EINVAL, "ms missing");
    cudaStream_t st = (cudaStream_t)stream;
    struct Ev {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Ev() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    CU(cudaEventCreate(&ev.e[0]), "event");
    CU(cudaEventCreate(&ev.e[1]), "event");
    CU(cudaEventRecord(ev.e[0], st), "event record");
    const int rc = su_plan_execute(pl, d_tuples, d_scratch, stream, launches);
    if (rc) return rc;
    CU(cudaEventRecord(ev.e[1], st), "event record");
    CU(cudaEventSynchronize(ev.e[1]), "event synchronize");
    CU(cudaEventElapsedTime(ms, ev.e[0], ev.e[1]), "event time");
    return SU_OK;
}

static void level_result(double laf, const double *tup, int64_t nb, int levels, int d,
                         su_level_result *r) {
    double M = -INFINITY;
    int64_t n = 0;
    for (int64_t b = 0; b < nb; ++b) {
        const double *t = tup + 4 * (b * levels + d);
        n += (int64_t)t[3];
        if (t[3] > 0 && t[0] > M) M = t[0];
    }
    r->n = n;
    if (!(M > -INFINITY)) {
        r->amp = 0;
        r->log_amp = -INFINITY;
        r->err = r->err_naive = 0;
        r->rel_err = NAN;
        r->ess = 0;
        r->max_share = NAN;
        return;
    }
    double S = 0, Q = 0;
    std::vector<double> mu;
    for (int64_t b = 0; b < nb; ++b) {
        const double *t = tup + 4 * (b * levels + d);
        if (!(t[3] > 0)) continue;
        const double f = t[0] > -INFINITY ? std::exp(t[0] - M) : 0.0;
        S += t[1] * f;
        Q += t[2] * f * f;
        mu.push_back(t[1] * f / t[3]);
    }
    const double mean = S / (double)n;
    double err_b = NAN;
    if (mu.size() > 1) {
        double m = 0;
        for (double v : mu) m += v;
        m /= (double)mu.size();
        double ss = 0;
        for (double v : mu) ss += (v - m) * (v - m);
        err_b = std::sqrt(ss / (double)(mu.size() - 1)) / std::sqrt((double)mu.size());
    }
    const double var = std::max(Q / (double)n - mean * mean, 0.0);
    const double err_n = n > 1 ? std::sqrt(var / (double)(n - 1)) : NAN;
    const double scale = std::exp(laf + M);
    r->amp = scale * mean;
    r->log_amp = laf + M + std::log(mean);
    r->err = scale * err_b;
    r->rel_err = err_b / mean;
    r->err_naive = scale * err_n;
    r->ess = S * S / Q;
    r->max_share = 1.0 / S;
}

int su_plan_finalize(const su_plan *pl, const double *h_tuples, const void *d_scratch,
                     su_level_result *out) {
    if (!pl || !out) return fail(SU_EINVAL, "plan or output missing");
    if (pl->s > 0 && d_scratch) {
        int flags = 0;
        CU(cudaMemcpy(&flags, static_cast<const char *>(d_scratch) + pl->scratch_bytes - 256, sizeof(int),
                      cudaMemcpyDeviceToHost),
           "read flags");
        if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    }
    su_level_result &r0 = out[0];
    r0.amp = std::exp(pl->laf + pl->w0);
    r0.log_amp = pl->laf + pl->w0;
    r0.err = r0.err_naive = r0.rel_err = 0;
    r0.ess = (double)pl->n_mc;
    r0.max_share = 1.0 / (double)pl->n_mc;
    r0.n = pl->n_mc;
    if (pl->s == 0) return SU_OK;
    if (!h_tuples) return fail(SU_EINVAL, "tuples missing");
    for (int d = 0; d < pl->levels; ++d)
        level_result(pl->laf, h_tuples, pl->n_blocks, pl->levels, d, &out[pl->s - d]);
    if (out[pl->s].n != pl->n_mc)
        return fail(SU_ECUDA, "%lld of %lld samples reduced", (long long)out[pl->s].n, (long long)pl->n_mc);
    return SU_OK;
}

// Sample a plan once and finalize: scratch on the plan's stream, tuples and
// the flag word back to the host, the plan destroyed by the caller.
static int amplitude_of_plan(su_plan *pl, su_level_result *out, float *ms = nullptr) {
    if (ms) *ms = 0;
    if (pl->s == 0) return su_plan_finalize(pl, nullptr, nullptr, out);
    cudaStream_t st = (cudaStream_t)pl->opt.stream;
    void *dbuf = nullptr;
    const int64_t tb = pl->tuple_bytes, sb = pl->scratch_bytes;
    CU(dmalloc_async(&dbuf, (size_t)(tb + sb), st), "cudaMallocAsync");
    std::vector<double> h((size_t)(tb / sizeof(double)) + 32);
    void *d_tup = dbuf;
    void *d_scr = static_cast<char *>(dbuf) + tb;
    int rc = ms ? su_plan_execute_timed(pl, d_tup, d_scr, st, nullptr, ms) : su_plan_execute(pl, d_tup, d_scr, st, nullptr);
    cudaError_t e = cudaSuccess;
    if (rc == SU_OK) {
        e = cudaMemcpyAsync(h.data(), d_tup, (size_t)tb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h.data() + tb / sizeof(double), static_cast<char *>(d_scr) + sb - 256,
                                sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(dbuf, st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "sampling");
    int flags = 0;
    std::memcpy(&flags, h.data() + tb / sizeof(double), sizeof(int));
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return su_plan_finalize(pl, h.data(), nullptr, out);
}

int speedup_amplitude(int model, const double *params, int n_params, double a, double b, double T,
                      int p, int s, int64_t n_mc, uint64_t seed, const su_options *opt,
                      su_level_result *out) {
    if (!out) return fail(SU_EINVAL, "output missing");
    su_plan *pl = nullptr;
    int rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_mc, seed, opt, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    return amplitude_of_plan(pl, out);
}

int speedup_amplitude_nd(int d, const int *exps, const double *coefs, int n_terms, const double *a, const double *b,
                         double T, int p, int s, int64_t n_mc, uint64_t seed, const su_options *opt,
                         su_level_result *out) {
    if (!out) return fail(SU_EINVAL, "output missing");
    su_plan *pl = nullptr;
    int rc = su_plan_create_nd(d, exps, coefs, n_terms, a, b, T, p, s, n_mc, seed, opt, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    return amplitude_of_plan(pl, out);
}

int speedup_logweights_nd(int d, const int *exps, const double *coefs, int n_terms, const double *a, const double *b,
                          double T, int p, int s, int64_t sample0, int64_t n_samples, uint64_t seed,
                          const su_options *opt, double *d_w) {
    if (s < 1) return fail(SU_EINVAL, "s must be >= 1 for per-sample weights");
    if (!d_w) return fail(SU_EINVAL, "output missing");
    if (sample0 < 0 || n_samples < 1 || sample0 + n_samples > kMaxSamples)
        return fail(SU_EINVAL, "sample range out of bounds");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    o.hierarchy = 1;
    o.n_blocks = 1;
    su_plan *pl = nullptr;
    int rc = su_plan_create_nd(d, exps, coefs, n_terms, a, b, T, p, s, n_samples, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    cudaStream_t st = (cudaStream_t)o.stream;
    su::NdParams Q = pl->Q;
    Q.base.w_out = d_w;
    Q.base.sample0 = sample0;
    Q.base.partial = nullptr;
    const size_t smem = su::nd_smem_bytes(Q, o.precision);
    void *buf = nullptr;
    const int64_t pb = ((pl->path_bytes + 255) / 256) * 256;
    CU(dmalloc_async(&buf, (size_t)(pb + 256), st), "cudaMallocAsync");
    Q.paths = buf;
    Q.base.flags = reinterpret_cast<int *>(static_cast<char *>(buf) + pb);
    cudaError_t e = cudaMemsetAsync(Q.base.flags, 0, sizeof(int), st);
    if (e == cudaSuccess) e = su::launch_nd(Q, o.precision, pl->grid, smem, st);
    int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, Q.base.flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "per-sample weights");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return SU_OK;
}

int su_fit_continuum(const su_level_result *levels, int s, int p, int n_min, int n_terms, double *A, double *A_err,
                     double *chi2) {
    if (!levels || !A) return fail(SU_EINVAL, "levels or output missing");
    if (s < 1 || s > SU_MAX_S) return fail(SU_EINVAL, "s must be in 1..%d", SU_MAX_S);
    if (p < 1 || p > SU_MAX_P) return fail(SU_EINVAL, "p must be in 1..%d", SU_MAX_P);
    if (n_terms != 2 && n_terms != 3) return fail(SU_EINVAL, "n_terms must be 2 or 3");
    if (n_min < 1 || s - n_min + 1 < n_terms)
        return fail(SU_EINVAL, "need levels n_min..s, n_min >= 1 (level 0 has no statistical error), at least n_terms");
    const int m = s - n_min + 1, k = n_terms;
    // weighted design matrix sqrt(w_n) (1, N^-p, N^-(p+1)), N = 2^n, each column
    // scaled to unit maximum; modified Gram-Schmidt QR
    double a[3][SU_MAX_S + 1], y[SU_MAX_S + 1], c[3];
    for (int i = 0; i < m; ++i) {
        const su_level_result &r = levels[n_min + i];
        if (!(r.err > 0) || !std::isfinite(r.err) || !std::isfinite(r.amp))
            return fail(SU_EINVAL, "level %d has no finite positive error", n_min + i);
        const double sw = 1.0 / r.err, lN = (double)(n_min + i) * std::log(2.0);
        a[0][i] = sw;
        a[1][i] = sw * std::exp(-p * lN);
        if (k == 3) a[2][i] = sw * std::exp(-(p + 1) * lN);
        y[i] = sw * r.amp;
    }
    for (int j = 0; j < k; ++j) {
        double mx = 0;
        for (int i = 0; i < m; ++i) mx = std::max(mx, std::fabs(a[j][i]));
        c[j] = 1.0 / mx;
        for (int i = 0; i < m; ++i) a[j][i] *= c[j];
    }
    double R[3][3] = {{0}}, z[3];
    for (int j = 0; j < k; ++j) {
        for (int l = 0; l < j; ++l) {
            double d = 0;
            for (int i = 0; i < m; ++i) d += a[l][i] * a[j][i];
            R[l][j] = d;
            for (int i = 0; i < m; ++i) a[j][i] -= d * a[l][i];
        }
        double nn = 0;
        for (int i = 0; i < m; ++i) nn += a[j][i] * a[j][i];
        R[j][j] = std::sqrt(nn);
        if (!(R[j][j] > 0)) return fail(SU_EINVAL, "the fit's columns are dependent");
        for (int i = 0; i < m; ++i) a[j][i] /= R[j][j];
        double d = 0;
        for (int i = 0; i < m; ++i) d += a[j][i] * y[i];
        z[j] = d;
        for (int i = 0; i < m; ++i) y[i] -= d * a[j][i];
    }
    double res = 0;
    for (int i = 0; i < m; ++i) res += y[i] * y[i];
    // R beta = z, and the first row of R^-1 for the variance of the constant
    double beta[3], Ri[3][3] = {{0}};
    for (int j = k - 1; j >= 0; --j) {
        double t = z[j];
        for (int l = j + 1; l < k; ++l) t -= R[j][l] * beta[l];
        beta[j] = t / R[j][j];
    }
    for (int j = 0; j < k; ++j) {
        Ri[j][j] = 1.0 / R[j][j];
        for (int l = j - 1; l >= 0; --l) {
            double t = 0;
            for (int q = l + 1; q <= j; ++q) t += R[l][q] * Ri[q][j];
            Ri[l][j] = -t / R[l][l];
        }
    }
    double v = 0;
    for (int j = 0; j < k; ++j) v += Ri[0][j] * Ri[0][j];
    *A = c[0] * beta[0];
    if (A_err) *A_err = c[0] * std::sqrt(v);
    if (chi2) *chi2 = res;
    return SU_OK;
}

int speedup_generate_nd(int d, const int *exps, const double *coefs, int n_terms, int p, double eps, int *out_exps,
                        double *out_w, int capacity, int *n_out) {
    if (!(eps > 0) || !std::isfinite(eps)) return fail(SU_EINVAL, "eps must be finite and > 0");
    if (!out_exps || !out_w || !n_out || capacity < 0) return fail(SU_EINVAL, "output missing");
    su::NdEffective E;
    std::string err;
    int rc = su::build_nd(d, exps, coefs, n_terms, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    std::vector<double> T;
    su::nd_table(E, eps, T);
    int n = 0;
    for (size_t e = 0; e < T.size(); ++e) {
        bool any = false;
        for (double v : E.hi[e]) any |= v != 0.0;
        if (!any) continue;   // a zero pad of the Horner groups
        if (n < capacity) {
            for (int v = 0; v < 2 * d; ++v) out_exps[(size_t)n * 2 * d + (size_t)v] = E.mono[e][(size_t)v];
            out_w[n] = -T[e] / eps;
        }
        ++n;
    }
    *n_out = n;
    if (n > capacity) return fail(SU_ENOTSUP, "the effective potential has %d terms", n);
    return SU_OK;
}

int speedup_wp(int model, const double *params, int n_params, int p, double eps, const double *x, const double *xb,
               int64_t n_points, double *w) {
    if (!(eps > 0) || !std::isfinite(eps)) return fail(SU_EINVAL, "eps must be finite and > 0");
    if (p < 1 || p > SU_MAX_P) return fail(SU_EINVAL, "p must be in 1..%d", SU_MAX_P);
    if (n_points < 0) return fail(SU_EINVAL, "n_points must be >= 0");
    if (n_points > 0 && (!x || !xb || !w)) return fail(SU_EINVAL, "points or output missing");
    std::string err;
    int rc = SU_OK;
    if (model == SU_GENERAL) {
        if (p > su::kGenMaxP) return fail(SU_ENOTSUP, "the general potential supports p <= %d", su::kGenMaxP);
        su::GeneralPotential V;
        rc = su::general_potential(params, n_params, V, err);
        if (rc) return fail(rc, "%s", err.c_str());
        const auto G = general_program(p, rc, err);
        if (rc) return fail(rc, "%s", err.c_str());
        su::general_wp_points(*G, V, eps, x, xb, n_points, w);
        return SU_OK;
    }
    su::Effective E;
    rc = su::build_effective(model, params, n_params, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    su::wp_host_points(E, eps, x, xb, n_points, w);
    return SU_OK;
}

int speedup_wp_nd(int d, const int *exps, const double *coefs, int n_terms, int p, double eps, const double *x,
                  const double *xb, int64_t n_points, double *w) {
    if (!(eps > 0) || !std::isfinite(eps)) return fail(SU_EINVAL, "eps must be finite and > 0");
    if (n_points < 0) return fail(SU_EINVAL, "n_points must be >= 0");
    if (n_points > 0 && (!x || !xb || !w)) return fail(SU_EINVAL, "points or output missing");
    su::NdEffective E;
    std::string err;
    const int rc = su::build_nd(d, exps, coefs, n_terms, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    su::nd_wp_points(E, eps, x, xb, n_points, w);
    return SU_OK;
}

// ------------------------------------------------------ fault injection
int su_fault_inject(int kind, int64_t arg) {
    switch (kind) {
        case SU_FAULT_CLEAR:
            g_fault_alloc = 0;
            g_fault_table_nan = 0;
            g_fault_queue = 0;
            g_fault_mma = 0;
            return SU_OK;
        case SU_FAULT_ALLOC:
            if (arg < 1) return fail(SU_EINVAL, "the failing allocation is counted from 1");
            g_fault_alloc = arg;
            return SU_OK;
        case SU_FAULT_TABLE_NAN:
            g_fault_table_nan = 1;
            return SU_OK;
        case SU_FAULT_QUEUE_STOP:
            if (arg < 1) return fail(SU_EINVAL, "the queue keeps at least one item");
            g_fault_queue = arg;
            return SU_OK;
        case SU_FAULT_WITHHOLD_MMA:
            g_fault_mma = 1;
            return SU_OK;
        default:
            return fail(SU_EINVAL, "unknown fault kind %d", kind);
    }
}

// ------------------------------------------------------- evolution operator
// The level-p table of the single-slice weight at eps = t (kernel precision)
// and the sampler parameters that evaluate it, for the evolution operator.
static int evolution_setup(int model, const double *params, int n_params, int p, double t, double L, int n,
                           int precision, std::vector<unsigned char> &blob, su::SamplerParams &P,
                           void **d_general) {
    *d_general = nullptr;
    if (!(t > 0) || !std::isfinite(t)) return fail(SU_EINVAL, "t must be finite and > 0");
    if (!(L > 0) || !std::isfinite(L)) return fail(SU_EINVAL, "L must be finite and > 0");
    if (n < 2 || n > 65536) return fail(SU_EINVAL, "n must be in 2..65536");
    if (p < 1 || p > SU_MAX_P) return fail(SU_EINVAL, "p must be in 1..%d", SU_MAX_P);
    if (precision != SU_FP64 && precision != SU_FP32) return fail(SU_EINVAL, "unknown precision");
    if (model == SU_GENERAL) {
        // the derivative-symbol program of W_p for a general potential (double only)
        if (precision != SU_FP64) return fail(SU_ENOTSUP, "the general potential is evaluated in double only");
        if (p > su::kGenMaxP) return fail(SU_ENOTSUP, "the general potential supports p <= %d", su::kGenMaxP);
        su::GeneralPotential V;
        std::string err;
        int rc = su::general_potential(params, n_params, V, err);
        std::shared_ptr<const su::GeneralEffective> G;
        if (!rc) G = general_program(p, rc, err);
        if (rc) return fail(rc, "%s", err.c_str());
        std::vector<double> T;
        su::general_table(*G, t, T);
        for (double v : T)
            if (!std::isfinite(v)) return fail(SU_ENONFINITE, "a coefficient of W_p is not finite at t = %g", t);
        blob.assign(T.size() * sizeof(double), 0);
        std::memcpy(blob.data(), T.data(), blob.size());
        std::memset(&P, 0, sizeof P);
        P.ring = su::RING_GENERAL;
        P.M = (int)T.size();
        rc = general_image(*G, V, d_general);
        if (rc) return rc;
        P.general = static_cast<const su::GeneralDev *>(*d_general);
        return SU_OK;
    }
    su::Effective E;
    std::string err;
    int rc = su::build_effective(model, params, n_params, p, E, err);
    if (rc) return fail(rc, "%s", err.c_str());
    std::vector<double> T;
    su::kernel_table(E, t, T);
    const size_t rs = precision == SU_FP32 ? sizeof(float) : sizeof(double);
    blob.assign(T.size() * rs, 0);
    for (size_t i = 0; i < T.size(); ++i) {
        if (!std::isfinite(T[i]) || (precision == SU_FP32 && !std::isfinite((float)T[i])))
            return fail(SU_ENONFINITE, "a coefficient of W_p is not representable at t = %g", t);
        if (precision == SU_FP32) {
            const float f = (float)T[i];
            std::memcpy(blob.data() + i * rs, &f, rs);
        } else {
            std::memcpy(blob.data() + i * rs, &T[i], rs);
        }
    }
    std::memset(&P, 0, sizeof P);
    P.ring = E.shape.ring;
    P.ncol = E.shape.ncol;
    P.M = E.shape.M;
    for (int j = 0; j < E.shape.ncol; ++j) P.len[j] = E.shape.len[j];
    P.alpha = E.shape.alpha;
    return SU_OK;
}

int speedup_evolution_matrix(int model, const double *params, int n_params, int p, double t, double L, int n,
                             int precision, double *d_U, void *stream) {
    if (!d_U) return fail(SU_EINVAL, "output missing");
    std::vector<unsigned char> blob;
    su::SamplerParams P;
    void *d_gen = nullptr;
    int rc = evolution_setup(model, params, n_params, p, t, L, n, precision, blob, P, &d_gen);
    std::unique_ptr<void, cudaError_t (*)(void *)> gen_guard(d_gen, cudaFree);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void *d_tab = nullptr;
    CU(dmalloc_async(&d_tab, blob.size(), st), "device allocation (table)");
    cudaError_t e = cudaMemcpyAsync(d_tab, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    const double delta = 2.0 * L / (double)(n - 1);
    const double lognorm = std::log(delta) - 0.5 * std::log(2.0 * M_PI * t);
    if (e == cudaSuccess) e = su::launch_evolution(P, precision, d_tab, L, delta, n, t, lognorm, d_U, st);
    // the host copy of the table must outlive the asynchronous upload
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_tab, st);
    if (e != cudaSuccess) return cuda_fail(e, "evolution matrix");
    return SU_OK;
}

int su_evolution_band_size(double t, double L, int n, int *half_width, int64_t *pitch) {
    if (!(t > 0) || !std::isfinite(t) || !(L > 0) || !std::isfinite(L) || n < 2 || n > 65536)
        return fail(SU_EINVAL, "t, L must be finite and > 0, n in 2..65536");
    const double delta = 2.0 * L / (double)(n - 1);
    // (x_j - x_i)^2 / (2t) <= 40 needs |j - i| Delta <= sqrt(80 t); two more
    // diagonals cover the rounding of the grid points (zero there anyway)
    const int w = (int)std::min<double>(n - 1, std::floor(std::sqrt(80.0 * t) / delta) + 2.0);
    if (half_width) *half_width = w;
    if (pitch) *pitch = ((int64_t)n + 31) / 32 * 32;
    return SU_OK;
}

int speedup_evolution_band(int model, const double *params, int n_params, int p, double t, double L, int n,
                           int precision, double *d_band, int64_t capacity, void *stream) {
    int w = 0;
    int64_t pitch = 0;
    int rc = su_evolution_band_size(t, L, n, &w, &pitch);
    if (rc) return rc;
    if (!d_band) return fail(SU_EINVAL, "output missing");
    const int64_t need = (int64_t)(w + 1) * pitch * (int64_t)sizeof(double);
    if (capacity < need) return fail(SU_EINVAL, "the band needs %lld bytes, %lld given", (long long)need, (long long)capacity);
    std::vector<unsigned char> blob;
    su::SamplerParams P;
    void *d_gen = nullptr;
    rc = evolution_setup(model, params, n_params, p, t, L, n, precision, blob, P, &d_gen);
    std::unique_ptr<void, cudaError_t (*)(void *)> gen_guard(d_gen, cudaFree);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    void *d_tab = nullptr;
    CU(dmalloc_async(&d_tab, blob.size(), st), "device allocation (table)");
    cudaError_t e = cudaMemcpyAsync(d_tab, blob.data(), blob.size(), cudaMemcpyHostToDevice, st);
    const double delta = 2.0 * L / (double)(n - 1);
    const double lognorm = std::log(delta) - 0.5 * std::log(2.0 * M_PI * t);
    if (e == cudaSuccess) e = su::launch_band(P, precision, d_tab, L, delta, n, t, lognorm, w, pitch, d_band, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_tab, st);
    if (e != cudaSuccess) return cuda_fail(e, "evolution band");
    return SU_OK;
}

int speedup_evolution_spectrum(int model, const double *params, int n_params, int p, double t, double L, int n,
                               int precision, int nev, double *energies, double *residuals, double *d_vectors,
                               su_spectrum_info *info, void *stream) {
    if (!energies) return fail(SU_EINVAL, "energies missing");
    int w = 0;
    int64_t pitch = 0;
    int rc = su_evolution_band_size(t, L, n, &w, &pitch);
    if (rc) return rc;
    if (nev < 1 || nev > 26 || nev > n / 2) return fail(SU_EINVAL, "nev must be in 1..26 and at most n/2");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t bytes = (int64_t)(w + 1) * pitch * (int64_t)sizeof(double);
    void *d_band = nullptr;
    CU(dmalloc(&d_band, (size_t)bytes), "device allocation (band)");
    std::unique_ptr<void, cudaError_t (*)(void *)> guard(d_band, cudaFree);
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    struct EvGuard {
        cudaEvent_t *e;
        ~EvGuard() {
            for (int i = 0; i < 3; ++i)
                if (e[i]) cudaEventDestroy(e[i]);
        }
    } eg{ev};
    for (auto &x : ev) CU(cudaEventCreate(&x), "event");
    CU(cudaEventRecord(ev[0], st), "event record");
    rc = speedup_evolution_band(model, params, n_params, p, t, L, n, precision, static_cast<double *>(d_band), bytes,
                                stream);
    if (rc) return rc;
    CU(cudaEventRecord(ev[1], st), "event record");
    const double delta = 2.0 * L / (double)(n - 1);
    su::SpectrumResult R;
    std::string err;
    rc = su::band_spectrum(static_cast<const double *>(d_band), pitch, n, w, nev, 12, 1e-11, 60, 20110505ULL,
                           d_vectors, 1.0 / std::sqrt(delta), st, R, err);
    if (rc) return fail(rc, "%s", err.c_str());
    CU(cudaEventRecord(ev[2], st), "event record");
    CU(cudaEventSynchronize(ev[2]), "event synchronize");
    for (int k = 0; k < nev; ++k) {
        energies[k] = R.theta[(size_t)k] > 0 ? -std::log(R.theta[(size_t)k]) / t : NAN;
        if (residuals) residuals[k] = R.resid[(size_t)k];
    }
    if (info) {
        std::memset(info, 0, sizeof *info);
        info->half_width = w;
        info->band_bytes = bytes;
        info->block = R.block;
        info->iterations = R.iterations;
        info->matvecs = R.matvecs;
        info->converged = R.converged;
        info->block_matvecs = R.block_matvecs;
        info->block_matvec_ms = R.block_matvec_ms;
        info->lower = R.lower;
        info->upper = R.upper;
        float ms = 0;
        CU(cudaEventElapsedTime(&ms, ev[0], ev[1]), "event time");
        info->band_ms = ms;
        CU(cudaEventElapsedTime(&ms, ev[1], ev[2]), "event time");
        info->solve_ms = ms;
    }
    if (!R.converged) return fail(SU_ENOTSUP, "the eigensolver did not reach its residual tolerance in 60 rounds");
    return SU_OK;
}

// ------------------------------------------------------------ autotuner
int su_autotune_clear(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
    g_btune.clear();
    return SU_OK;
}

int su_autotune(int model, const double *params, int n_params, double a, double b, double T, int p, int s,
                int64_t n_probe, uint64_t seed, const su_options *opt, su_tuning *best, su_tuning *all,
                int cap, int *n_all) {
    if (!best) return fail(SU_EINVAL, "best missing");
    if (n_all) *n_all = 0;
    if (s < 1) return fail(SU_EINVAL, "s must be >= 1 to tune the sampler");
    if (cap < 0 || (cap > 0 && !all)) return fail(SU_EINVAL, "all and cap inconsistent");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    o.seg_log2 = 0;
    o.rounds = 0;
    int rc = validate(model, params, n_params, a, b, T, p, s, n_probe, o);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.stream;
    struct Res {
        void *buf = nullptr;
        size_t cap = 0;
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Res() {
            if (buf) cudaFree(buf);
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } res;
    CU(cudaEventCreate(&res.e[0]), "event");
    CU(cudaEventCreate(&res.e[1]), "event");
    std::vector<su_tuning> got;
    for (int F = 1; F <= std::min(s, su::kMaxFine); ++F) {
        for (int r : {1, 2, 4, 8}) {
            su_options oc = o;
            oc.seg_log2 = F;
            oc.rounds = r;
            su_plan *pl = nullptr;
            rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_probe, seed, &oc, &pl);
            if (rc == SU_ENOTSUP) continue;   // this shape's shared memory does not fit
            if (rc) return rc;
            std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
            const size_t need = (size_t)(pl->tuple_bytes + pl->scratch_bytes);
            if (need > res.cap) {
                if (res.buf) cudaFree(res.buf);
                res.buf = nullptr;
                res.cap = 0;
                CU(dmalloc(&res.buf, need), "device allocation (probe buffers)");
                res.cap = need;
            }
            void *d_tup = res.buf, *d_scr = static_cast<char *>(res.buf) + pl->tuple_bytes;
            rc = su_plan_execute(pl, d_tup, d_scr, st, nullptr);   // warm-up
            if (rc) return rc;
            float ms_best = INFINITY;
            for (int k = 0; k < 2; ++k) {
                CU(cudaEventRecord(res.e[0], st), "event record");
                rc = su_plan_execute(pl, d_tup, d_scr, st, nullptr);
                if (rc) return rc;
                CU(cudaEventRecord(res.e[1], st), "event record");
                CU(cudaEventSynchronize(res.e[1]), "probe");
                float ms = 0;
                CU(cudaEventElapsedTime(&ms, res.e[0], res.e[1]), "event time");
                ms_best = std::min(ms_best, ms);
            }
            got.push_back({pl->P.F, pl->P.rounds, (double)ms_best});
        }
    }
    if (got.empty()) return fail(SU_ENOTSUP, "no launch shape fits this device");
    const su_tuning top = *std::min_element(got.begin(), got.end(),
                                            [](const su_tuning &x, const su_tuning &y) { return x.ms < y.ms; });
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune[{o.precision, model, p, s}] = top;
    }
    *best = top;
    for (int i = 0; i < (int)got.size() && i < cap; ++i) all[i] = got[(size_t)i];
    if (n_all) *n_all = (int)got.size();
    g_err.clear();
    return SU_OK;
}

int speedup_logweights(int model, const double *params, int n_params, double a, double b, double T,
                       int p, int s, int64_t sample0, int64_t n_samples, uint64_t seed,
                       const su_options *opt, double *d_w) {
    if (s < 1) return fail(SU_EINVAL, "s must be >= 1 for per-sample weights");
    if (!d_w) return fail(SU_EINVAL, "output missing");
    if (sample0 < 0 || n_samples < 1 || sample0 + n_samples > kMaxSamples)
        return fail(SU_EINVAL, "sample range out of bounds");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    o.hierarchy = 1;
    o.n_blocks = 1;
    su_plan *pl = nullptr;
    int rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_samples, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    cudaStream_t st = (cudaStream_t)o.stream;
    su::SamplerParams P = pl->P;
    P.w_out = d_w;
    P.sample0 = sample0;
    P.partial = nullptr;
    const size_t smem = su::sampler_smem_bytes(P, o.precision);
    if (su::sampler_occupancy(P, o.precision, smem) < 1) return fail(SU_ECUDA, "sampler not resident");
    int *d_flag = nullptr;
    CU(dmalloc_async(&d_flag, sizeof(int), st), "cudaMallocAsync");
    P.flags = d_flag;
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = su::launch_sampler(P, o.precision, pl->grid, smem, st);
    int flags = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_flag, st);
    if (e != cudaSuccess) return cuda_fail(e, "per-sample weights");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return SU_OK;
}

int speedup_normals(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                    int n_normals, int precision, double *d_out, void *stream) {
    if (!d_out || sample0 < 0 || n_samples < 0 || n_normals < 0) return fail(SU_EINVAL, "bad arguments");
    if (precision != SU_FP64 && precision != SU_FP32) return fail(SU_EINVAL, "unknown precision");
    CU(su::launch_normals(seed, instance, sample0, n_samples, n_normals, precision, d_out,
                          (cudaStream_t)stream),
       "normals launch");
    return SU_OK;
}

// ----------------------------------------------------------------- batch

}  // extern "C"

struct su_batch_plan {
    int p = 1;
    int model = 0;
    int64_t n_inst = 0, n_mc = 1;
    su_options opt{};
    std::map<int, su::Effective> E;   // per level p
    // the general potential: its terms, and per level p the program and its device image
    su::GeneralPotential V{};
    std::map<int, std::shared_ptr<const su::GeneralEffective>> G;
    std::vector<void *> d_general;
    su::BatchParams B{};
    void *d_inst = nullptr, *d_items = nullptr, *d_tables = nullptr, *d_shapes = nullptr;
    // per instance
    std::vector<int> S, L, F, K, NB, hier, from;
    std::vector<int64_t> N, tup, out_off;
    std::vector<double> laf, w0;      // log A_free and the level-0 weight
    int64_t n_results = 0;
    int grid = 0;
    size_t smem = 0;
    int64_t tuple_bytes = 0, scratch_bytes = 256, slice_actions = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void *g_tuples = nullptr, *g_scratch = nullptr;
    // the launches: the items [item0, item0 + n) of each group, one kernel per
    // group (a compiled table shape, or the generic kernel: fixed = -1), each
    // with its own queue head (scratch int `counter`)
    struct Group {
        int fixed, src, counter, grid;
        int64_t item0;
        int n;
    };
    std::vector<Group> groups;
};

static void batch_free(su_batch_plan *pl) {
    if (!pl) return;
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->d_inst) cudaFree(pl->d_inst);
    if (pl->d_items) cudaFree(pl->d_items);
    if (pl->d_tables) cudaFree(pl->d_tables);
    if (pl->d_shapes) cudaFree(pl->d_shapes);
    for (void *g : pl->d_general)
        if (g) cudaFree(g);
    delete pl;
}

namespace {

// one instance's resolved arguments
struct BatchArg {
    double a, b, T;
    int s, p, hier;
    int64_t n;
};

int batch_args(int p, const su_instance *inst, int64_t n_inst, int64_t n_mc, std::vector<BatchArg> &out) {
    out.resize((size_t)n_inst);
    for (int64_t i = 0; i < n_inst; ++i) {
        const su_instance &q = inst[i];
        if (q.hierarchy != 0 && q.hierarchy != 1)
            return fail(SU_EINVAL, "instance %lld: hierarchy must be 0 or 1", (long long)i);
        if (q.p < 0 || q.n_mc < 0) return fail(SU_EINVAL, "instance %lld: negative p or n_mc", (long long)i);
        out[(size_t)i] = {q.a, q.b, q.T, q.s, q.p ? q.p : p, q.hierarchy, q.n_mc ? q.n_mc : n_mc};
    }
    return SU_OK;
}

}  // namespace

// The batch plan with every instance's register segment either automatic
// (force_F = 0: the stored shape of its class, else the rule) or force_F.
static int batch_create(int model, const double *params, int n_params, int p, const su_instance *inst,
                        int64_t n_inst, int64_t n_mc, uint64_t seed, const su_options *opt, int force_F,
                        su_batch_plan **out) {
    using namespace su;
    if (!out) return fail(SU_EINVAL, "plan pointer missing");
    *out = nullptr;
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    if (!inst || n_inst < 1 || n_inst > (1LL << 24)) return fail(SU_EINVAL, "n_inst must be in 1..2^24");
    if ((uint64_t)o.instance + (uint64_t)n_inst > (1ULL << 32))
        return fail(SU_EINVAL, "instance ids exceed 32 bits");
    if (o.width_factor != 1.0) return fail(SU_ENOTSUP, "the batched path samples the exact bridge only");
    const bool general = model == SU_GENERAL;
    std::vector<BatchArg> arg;
    int rc = batch_args(p, inst, n_inst, n_mc, arg);
    if (rc) return rc;
    for (int64_t i = 0; i < n_inst; ++i) {
        const BatchArg &q = arg[(size_t)i];
        rc = validate(model, params, n_params, q.a, q.b, q.T, q.p, q.s, q.n, o);
        if (rc) {
            const std::string why = g_err;
            return fail(rc, "instance %lld: %s", (long long)i, why.c_str());
        }
    }
    if (o.sample0 != 0) return fail(SU_ENOTSUP, "sample0 must be 0 for a batch");
    std::unique_ptr<su_batch_plan, void (*)(su_batch_plan *)> pl(new (std::nothrow) su_batch_plan, batch_free);
    if (!pl) return fail(SU_ENOMEM, "host allocation failed");
    pl->p = p;
    pl->model = model;
    pl->n_inst = n_inst;
    pl->n_mc = n_mc;
    pl->opt = o;
    const int prec = o.precision;

    // effective actions and table shapes, one per distinct level p (the
    // general potential: a monomial program per p, uploaded with the
    // potential's terms; its shape has no columns, M = the program's entries)
    std::map<int, int> shape_of;
    std::vector<BatchShape> shapes;
    if (general) {
        std::string err;
        rc = general_potential(params, n_params, pl->V, err);
        if (rc) return fail(rc, "%s", err.c_str());
    }
    for (const BatchArg &q : arg) {
        if (shape_of.count(q.p)) continue;
        std::string err;
        BatchShape sh;
        std::memset(&sh, 0, sizeof sh);
        if (general) {
            auto G = general_program(q.p, rc, err);
            if (rc) return fail(rc, "%s", err.c_str());
            pl->G[q.p] = G;
            void *d = nullptr;
            rc = general_image(*G, pl->V, &d);
            pl->d_general.push_back(d);
            if (rc) return rc;
            sh.M = (int)G->entry_k.size();
            sh.general = static_cast<const GeneralDev *>(d);
        } else {
            Effective &E = pl->E[q.p];
            rc = build_effective(model, params, n_params, q.p, E, err);
            if (rc) return fail(rc, "%s", err.c_str());
            sh.ncol = E.shape.ncol;
            sh.M = E.shape.M;
            for (int j = 0; j < E.shape.ncol; ++j) sh.len[j] = E.shape.len[j];
        }
        shape_of[q.p] = (int)shapes.size();
        shapes.push_back(sh);
    }
    const double alpha = general ? 0.0 : pl->E.begin()->second.shape.alpha;
    const int ring = general ? RING_GENERAL : pl->E.begin()->second.shape.ring;

    int dev = 0, sms = 0, smem_max = 0;
    rc = device_limits(dev, sms, smem_max);
    if (rc) return rc;

    // per instance: path, tables (one set per (p, T, s, levels)), level 0, shape
    std::map<std::tuple<int, double, int, int>, int64_t> tab_of;
    std::map<std::pair<int, double>, std::vector<double>> coll;
    std::vector<double> tabd;
    std::vector<BatchInstance> hin((size_t)n_inst);
    const size_t ni = (size_t)n_inst;
    pl->S.resize(ni);
    pl->L.resize(ni);
    pl->F.resize(ni);
    pl->K.resize(ni, 1);
    pl->NB.resize(ni);
    pl->hier.resize(ni);
    pl->from.resize(ni, 0);
    pl->N.resize(ni);
    pl->tup.resize(ni, 0);
    pl->out_off.resize(ni);
    pl->laf.resize(ni);
    pl->w0.resize(ni);
    int S_max = 0, C_max = 1, L_max = 1;
    int64_t tab_max = 1;
    for (size_t i = 0; i < ni; ++i) {
        const BatchArg &q = arg[i];
        const Effective *E = general ? nullptr : &pl->E[q.p];
        const GeneralEffective *G = general ? pl->G[q.p].get() : nullptr;
        BatchInstance &h = hin[i];
        std::memset(&h, 0, sizeof h);
        h.a = q.a;
        h.b = q.b;
        h.S = q.s;
        h.L = q.s == 0 ? 0 : (q.hier ? q.s : 1);
        h.shape = shape_of[q.p];
        h.n_mc = q.n;
        h.n_blocks = (int)std::min<int64_t>(o.n_blocks, q.n);
        for (int n = 1; n <= q.s; ++n) h.sigma[n] = std::sqrt(q.T / std::ldexp(1.0, n + 1));
        pl->S[i] = q.s;
        pl->L[i] = h.L;
        pl->NB[i] = h.n_blocks;
        pl->hier[i] = q.hier;
        pl->N[i] = q.n;
        pl->out_off[i] = pl->n_results;
        pl->n_results += q.hier ? q.s + 1 : 1;
        pl->laf[i] = log_A_free(q.a, q.b, q.T);
        if (general) {
            pl->w0[i] = -q.T * general_wp_host(*G, pl->V, 0.5 * (q.a + q.b), 0.5 * (q.b - q.a), q.T);
        } else {
            auto c = coll.find({q.p, q.T});
            if (c == coll.end()) {
                std::vector<double> P;
                collapse(*E, q.T, P);
                c = coll.emplace(std::make_pair(q.p, q.T), std::move(P)).first;
            }
            pl->w0[i] = -q.T * wp_collapsed(E->shape, c->second, 0.5 * (q.a + q.b), 0.5 * (q.b - q.a));
        }
        if (!std::isfinite(pl->w0[i]) && !(std::isinf(pl->w0[i]) && pl->w0[i] < 0))
            return fail(SU_ENONFINITE, "instance %lld: level-0 weight is not finite", (long long)i);
        if (q.s == 0) continue;
        // shape: forced, else stored for the class, else the rule (as the
        // single-instance plans: 16-slice segments in double, 32 in single
        // precision and for the general potential)
        int F = (prec == SU_FP64 && !general) ? 4 : kMaxFine;
        if (force_F > 0) {
            F = force_F;
        } else {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_btune.find({prec, model, q.p, q.s, q.hier});
            if (it != g_btune.end()) {
                F = it->second;
                pl->from[i] = 1;
            }
        }
        h.F = std::min(q.s, std::max(1, F));
        pl->F[i] = h.F;
        const auto key = std::make_tuple(q.p, q.T, q.s, h.L);
        auto t = tab_of.find(key);
        if (t == tab_of.end()) {
            const int64_t offset = (int64_t)tabd.size();
            for (int d = 0; d < h.L; ++d) {
                std::vector<double> row;
                const double eps = q.T / std::ldexp(1.0, q.s - d);
                if (general)
                    general_table(*G, eps, row);
                else
                    kernel_table(*E, eps, row);
                if (g_fault_table_nan.exchange(0)) row[0] = NAN;   // fault injection
                for (double v : row)
                    if (!std::isfinite(v) || (prec == SU_FP32 && !std::isfinite((float)v)))
                        return fail(SU_ENONFINITE, "non-finite coefficient at p = %d, eps = %g", q.p,
                                    q.T / std::ldexp(1.0, q.s - d));
                tabd.insert(tabd.end(), row.begin(), row.end());
            }
            t = tab_of.emplace(key, offset).first;
        }
        h.tab = t->second;
        S_max = std::max(S_max, q.s);
        C_max = std::max(C_max, 1 << (q.s - h.F));
        L_max = std::max(L_max, h.L);
        tab_max = std::max(tab_max, (int64_t)h.L * shapes[(size_t)h.shape].M);
        const int64_t Nn = (int64_t)1 << q.s;
        pl->slice_actions += q.n * (h.L > 1 ? 2 * Nn - 2 : Nn);
    }

    BatchParams &B = pl->B;
    std::memset(&B, 0, sizeof B);
    SamplerParams &P = B.base;
    P.levels = 1;
    P.ring = ring;
    P.alpha = alpha;
    P.seed = seed;
    P.instance = o.instance;
    B.S_max = S_max;
    B.C_max = C_max;
    B.L_max = L_max;
    B.tab_max = tab_max;
    B.fixed_shape = -1;   // the generic kernel; the compiled-shape groups are set up below
    B.fixed_src = 0;
    pl->smem = batch_smem_bytes(B, prec);
    if (pl->smem > (size_t)smem_max)
        return fail(SU_ENOTSUP, "shared memory %zu exceeds %d (tables of %lld entries, %d levels)", pl->smem, smem_max,
                    (long long)tab_max, L_max);
    // the work items (and so the order of every sum) come from the generic
    // kernel's residency, so that the compiled-shape kernels, which run at
    // other occupancies, give the same bits
    const int occ_gen = batch_occupancy(B, prec, pl->smem);
    if (occ_gen < 1) return fail(SU_ECUDA, "batched kernel cannot be resident");
    const int64_t work_slots = (int64_t)sms * occ_gen;

    // work items (instance, block, chunk).  Cost of an instance's block:
    // samples x slices x (table entries + the per-slice formation and RNG
    // share); blocks are split into chunks where the whole batch has fewer
    // than about eight items of the average cost per resident CTA
    std::vector<double> bcost(ni, 0.0);
    double total = 0;
    for (size_t i = 0; i < ni; ++i) {
        if (pl->S[i] == 0) continue;
        const int64_t Nn = (int64_t)1 << pl->S[i];
        const double slices = (double)(pl->L[i] > 1 ? 2 * Nn - 2 : Nn);
        bcost[i] = ((double)pl->N[i] / pl->NB[i]) * slices * (double)(shapes[(size_t)hin[i].shape].M + 12);
        total += bcost[i] * pl->NB[i];
    }
    const double target = total / (8.0 * (double)work_slots);
    int64_t n_items = 0, n_tup = 0;
    for (size_t i = 0; i < ni; ++i) {
        if (pl->S[i] == 0) continue;
        const int64_t bmin = pl->N[i] / pl->NB[i];                 // smallest block
        int64_t k = target > 0 ? (int64_t)std::ceil(bcost[i] / target) : 1;
        k = std::max<int64_t>(1, std::min<int64_t>(k, std::max<int64_t>(1, bmin / kThreads)));
        pl->K[i] = (int)k;
        hin[i].chunks = (int)k;
        hin[i].tup = n_tup;
        pl->tup[i] = n_tup;
        n_tup += (int64_t)pl->NB[i] * k * pl->L[i];
        n_items += (int64_t)pl->NB[i] * k;
    }
    if (n_items > (1LL << 31) - 1) return fail(SU_ENOTSUP, "too many work items");
    // costliest items first: an instance's items are alike, so order the instances
    std::vector<int64_t> order;
    for (size_t i = 0; i < ni; ++i)
        if (pl->S[i] >= 1) order.push_back((int64_t)i);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
        return bcost[(size_t)x] / pl->K[(size_t)x] > bcost[(size_t)y] / pl->K[(size_t)y];
    });
    // kernels: in single precision (even ring) every level p whose table shape
    // is compiled in gets that shape's kernel, the other levels the generic
    // one; the items grouped by kernel, each group in cost order
    std::vector<int> kshape(shapes.size(), -1);
    if (prec == SU_FP32 && ring == RING_EVEN && o.kernel != 1)
        for (size_t k = 0; k < shapes.size(); ++k) kshape[k] = fixed_shape_index(shapes[k].ncol, shapes[k].len);
    std::map<int, int> src_of;          // compiled shape -> its index in shapes
    for (size_t k = 0; k < shapes.size(); ++k)
        if (kshape[k] >= 0) src_of[kshape[k]] = (int)k;
    std::vector<int> keys;              // group order: the generic kernel (-1) first, then by shape
    for (int64_t i : order) {
        const int key = kshape[(size_t)hin[(size_t)i].shape];
        if (std::find(keys.begin(), keys.end(), key) == keys.end()) keys.push_back(key);
    }
    std::sort(keys.begin(), keys.end());
    std::vector<int2> items;
    items.reserve((size_t)n_items);
    pl->groups.clear();
    for (int key : keys) {
        su_batch_plan::Group g{};
        g.fixed = key;
        g.src = key >= 0 ? src_of[key] : 0;
        g.item0 = (int64_t)items.size();
        for (int64_t i : order) {
            if (kshape[(size_t)hin[(size_t)i].shape] != key) continue;
            for (int u = 0; u < pl->NB[(size_t)i] * pl->K[(size_t)i]; ++u) items.push_back(make_int2((int)i, u));
        }
        g.n = (int)((int64_t)items.size() - g.item0);
        // queue heads: group 0 at scratch int 0, the flags at int 1, group k >= 1 at int k + 1
        g.counter = pl->groups.empty() ? 0 : (int)pl->groups.size() + 1;
        BatchParams Bg = B;
        Bg.fixed_shape = g.fixed;
        Bg.fixed_src = g.src;
        const int occ = batch_occupancy(Bg, prec, pl->smem);
        if (occ < 1) return fail(SU_ECUDA, "batched kernel cannot be resident");
        g.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * occ, std::max(g.n, 1)));
        pl->groups.push_back(g);
    }

    const size_t rs = prec == SU_FP32 ? sizeof(float) : sizeof(double);
    std::vector<unsigned char> blob(std::max<size_t>(tabd.size(), 1) * rs, 0);
    if (prec == SU_FP32)
        for (size_t i = 0; i < tabd.size(); ++i) reinterpret_cast<float *>(blob.data())[i] = (float)tabd[i];
    else if (!tabd.empty())
        std::memcpy(blob.data(), tabd.data(), tabd.size() * sizeof(double));
    CU(dmalloc(&pl->d_tables, blob.size()), "device allocation (tables)");
    CU(cudaMemcpy(pl->d_tables, blob.data(), blob.size(), cudaMemcpyHostToDevice), "upload tables");
    CU(dmalloc(&pl->d_inst, sizeof(BatchInstance) * hin.size()), "device allocation (instances)");
    CU(cudaMemcpy(pl->d_inst, hin.data(), sizeof(BatchInstance) * hin.size(), cudaMemcpyHostToDevice),
       "upload instances");
    CU(dmalloc(&pl->d_shapes, sizeof(BatchShape) * shapes.size()), "device allocation (shapes)");
    CU(cudaMemcpy(pl->d_shapes, shapes.data(), sizeof(BatchShape) * shapes.size(), cudaMemcpyHostToDevice),
       "upload shapes");
    if (!items.empty()) {
        CU(dmalloc(&pl->d_items, sizeof(int2) * items.size()), "device allocation (items)");
        CU(cudaMemcpy(pl->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice),
           "upload items");
    }
    P.tables = pl->d_tables;
    B.inst = static_cast<const BatchInstance *>(pl->d_inst);
    B.shapes = static_cast<const BatchShape *>(pl->d_shapes);
    B.items = static_cast<const int2 *>(pl->d_items);
    B.n_items = (int)items.size();
    pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>(work_slots, std::max(B.n_items, 1)));
    pl->tuple_bytes = std::max<int64_t>(n_tup, 1) * 4 * (int64_t)sizeof(double);
    pl->scratch_bytes = 256;
    *out = pl.release();
    return SU_OK;
}

extern "C" {

int su_batch_plan_create(int model, const double *params, int n_params, int p, const su_instance *inst,
                         int64_t n_inst, int64_t n_mc, uint64_t seed, const su_options *opt,
                         su_batch_plan **out) {
    return batch_create(model, params, n_params, p, inst, n_inst, n_mc, seed, opt, 0, out);
}

int su_batch_plan_destroy(su_batch_plan *pl) {
    batch_free(pl);
    return SU_OK;
}

int su_batch_plan_sizes(const su_batch_plan *pl, int64_t *tuple_bytes, int64_t *scratch_bytes,
                        int64_t *slice_actions, int64_t *n_results) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (tuple_bytes) *tuple_bytes = pl->tuple_bytes;
    if (scratch_bytes) *scratch_bytes = pl->scratch_bytes;
    if (slice_actions) *slice_actions = pl->slice_actions;
    if (n_results) *n_results = pl->n_results;
    return SU_OK;
}

int su_batch_plan_shape(const su_batch_plan *pl, int64_t i, int *seg_log2, int *chunks, int *from) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (i < 0 || i >= pl->n_inst) return fail(SU_EINVAL, "instance %lld out of range", (long long)i);
    if (seg_log2) *seg_log2 = pl->F[(size_t)i];
    if (chunks) *chunks = pl->K[(size_t)i];
    if (from) *from = pl->from[(size_t)i];
    return SU_OK;
}

int su_batch_plan_kernel(const su_batch_plan *pl, int *fixed_shape) {
    if (!pl || !fixed_shape) return fail(SU_EINVAL, "plan or output missing");
    bool any_fixed = false;
    for (const auto &g : pl->groups) any_fixed = any_fixed || g.fixed >= 0;
    *fixed_shape = pl->groups.size() == 1 ? pl->groups[0].fixed : (any_fixed ? -2 : -1);
    return SU_OK;
}

int su_batch_plan_execute(su_batch_plan *pl, void *d_tuples, void *d_scratch, void *stream, int *launches) {
    if (!pl) return fail(SU_EINVAL, "plan missing");
    if (!d_tuples || !d_scratch) return fail(SU_EINVAL, "device buffers missing");
    if (launches) *launches = 0;
    cudaStream_t st = (cudaStream_t)stream;
    // instances with s = 0 have no samples and no tuples
    if (pl->B.n_items == 0) return SU_OK;
    su::BatchParams B = pl->B;
    B.tuples = static_cast<double *>(d_tuples);
    B.counter = static_cast<int *>(d_scratch);
    B.base.flags = static_cast<int *>(d_scratch) + 1;
    const int64_t stop = g_fault_queue.exchange(0);
    if (stop > 0) {   // fault injection: the queue (all items, generic kernel) ends after `stop` items
        const void *fn = su::batch_fn(B, pl->opt.precision);
        void *args[] = {&B};
        B.n_items = (int)std::min<int64_t>(B.n_items, stop);
        CU(cudaMemsetAsync(d_tuples, 0, (size_t)pl->tuple_bytes, st), "clear tuples");
        CU(cudaMemsetAsync(d_scratch, 0, 8, st), "clear queue");
        CU(cudaLaunchKernel(fn, dim3(pl->grid), dim3(su::kThreads), args, pl->smem, st), "batch launch");
        if (launches) *launches = 1;
        return SU_OK;
    }
    if (!pl->exec) {
        // one graph per plan: clear the queue heads and the flags, then one
        // persistent kernel per group (independent: disjoint items, heads and
        // tuples)
        CU(cudaGraphCreate(&pl->graph, 0), "graph create");
        cudaMemsetParams mp{};
        mp.dst = d_scratch;
        mp.value = 0;
        mp.elementSize = 4;
        mp.width = pl->groups.size() + 1;
        mp.height = 1;
        cudaGraphNode_t mnode;
        CU(cudaGraphAddMemsetNode(&mnode, pl->graph, nullptr, 0, &mp), "graph memset node");
        for (const auto &g : pl->groups) {
            su::BatchParams Bg = B;
            Bg.items = B.items + g.item0;
            Bg.n_items = g.n;
            Bg.counter = static_cast<int *>(d_scratch) + g.counter;
            Bg.fixed_shape = g.fixed;
            Bg.fixed_src = g.src;
            void *args[] = {&Bg};
            cudaKernelNodeParams kp{};
            kp.func = const_cast<void *>(su::batch_fn(Bg, pl->opt.precision));
            kp.gridDim = dim3(g.grid);
            kp.blockDim = dim3(su::kThreads);
            kp.sharedMemBytes = (unsigned)pl->smem;
            kp.kernelParams = args;   // copied into the node
            cudaGraphNode_t knode;
            CU(cudaGraphAddKernelNode(&knode, pl->graph, &mnode, 1, &kp), "graph kernel node");
        }
        CU(cudaGraphInstantiate(&pl->exec, pl->graph, 0), "graph instantiate");
        pl->g_tuples = d_tuples;
        pl->g_scratch = d_scratch;
    } else if (pl->g_tuples != d_tuples || pl->g_scratch != d_scratch) {
        // new buffers: rebuild (the memset node's destination changes too)
        cudaGraphExecDestroy(pl->exec);
        cudaGraphDestroy(pl->graph);
        pl->exec = nullptr;
        pl->graph = nullptr;
        return su_batch_plan_execute(pl, d_tuples, d_scratch, stream, launches);
    }
    CU(cudaGraphLaunch(pl->exec, st), "graph launch");
    if (launches) *launches = 1;
    return SU_OK;
}

int su_batch_plan_finalize(const su_batch_plan *pl, const double *h_tuples, const void *d_scratch,
                           su_level_result *out) {
    if (!pl || !out || !h_tuples) return fail(SU_EINVAL, "plan, tuples or output missing");
    if (d_scratch) {
        int flags = 0;
        CU(cudaMemcpy(&flags, static_cast<const int *>(d_scratch) + 1, sizeof(int), cudaMemcpyDeviceToHost),
           "read flags");
        if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    }
    std::vector<double> blk;
    for (int64_t i = 0; i < pl->n_inst; ++i) {
        const size_t k = (size_t)i;
        su_level_result *o = out + pl->out_off[k];
        su_level_result r0;
        r0.amp = std::exp(pl->laf[k] + pl->w0[k]);
        r0.log_amp = pl->laf[k] + pl->w0[k];
        r0.err = r0.err_naive = r0.rel_err = 0;
        r0.ess = (double)pl->N[k];
        r0.max_share = 1.0 / (double)pl->N[k];
        r0.n = pl->N[k];
        if (pl->S[k] == 0) {
            o[0] = r0;
            continue;
        }
        // merge each block's chunks in order: tuples [block][level]
        const int L = pl->L[k], K = pl->K[k], nb = pl->NB[k];
        const double *t = h_tuples + 4 * pl->tup[k];
        blk.assign((size_t)nb * L * 4, 0.0);
        for (int b = 0; b < nb; ++b)
            for (int d = 0; d < L; ++d) {
                double M = -INFINITY, S = 0, Q = 0, n = 0;
                for (int c = 0; c < K; ++c) {
                    const double *x = t + 4 * (((int64_t)b * K + c) * L + d);
                    n += x[3];
                    if (!(x[0] > -INFINITY)) continue;
                    if (x[0] > M) {
                        const double f = std::exp(M - x[0]);
                        S = S * f + x[1];
                        Q = Q * f * f + x[2];
                        M = x[0];
                    } else {
                        const double f = std::exp(x[0] - M);
                        S += x[1] * f;
                        Q += x[2] * f * f;
                    }
                }
                double *y = blk.data() + 4 * ((int64_t)b * L + d);
                y[0] = M;
                y[1] = S;
                y[2] = Q;
                y[3] = n;
            }
        for (int d = 0; d < L; ++d) {
            su_level_result r;
            level_result(pl->laf[k], blk.data(), nb, L, d, &r);
            if (r.n != pl->N[k])
                return fail(SU_ECUDA, "instance %lld: %lld of %lld samples reduced (the work queue ended early)",
                            (long long)i, (long long)r.n, (long long)pl->N[k]);
            if (pl->hier[k])
                o[pl->S[k] - d] = r;
            else
                o[0] = r;
        }
        if (pl->hier[k]) o[0] = r0;
    }
    return SU_OK;
}

int speedup_amplitude_batch(int model, const double *params, int n_params, int p, const su_instance *inst,
                            int64_t n_inst, int64_t n_mc, uint64_t seed, const su_options *opt,
                            su_level_result *out) {
    if (!out) return fail(SU_EINVAL, "output missing");
    su_batch_plan *pl = nullptr;
    int rc = su_batch_plan_create(model, params, n_params, p, inst, n_inst, n_mc, seed, opt, &pl);
    if (rc) return rc;
    std::unique_ptr<su_batch_plan, int (*)(su_batch_plan *)> guard(pl, su_batch_plan_destroy);
    cudaStream_t st = (cudaStream_t)pl->opt.stream;
    void *dbuf = nullptr;
    CU(dmalloc_async(&dbuf, (size_t)(pl->tuple_bytes + pl->scratch_bytes), st), "cudaMallocAsync");
    std::vector<double> h((size_t)(pl->tuple_bytes / sizeof(double)) + 32);
    void *d_scr = static_cast<char *>(dbuf) + pl->tuple_bytes;
    rc = su_batch_plan_execute(pl, dbuf, d_scr, st, nullptr);
    cudaError_t e = cudaSuccess;
    int flags = 0;
    if (rc == SU_OK && pl->B.n_items > 0) {
        e = cudaMemcpyAsync(h.data(), dbuf, (size_t)pl->tuple_bytes, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&flags, static_cast<int *>(d_scr) + 1, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFreeAsync(dbuf, st);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "batched sampling");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return su_batch_plan_finalize(pl, h.data(), nullptr, out);
}

int su_batch_autotune(int model, const double *params, int n_params, int p, const su_instance *inst,
                      int64_t n_inst, int64_t n_mc, uint64_t seed, const su_options *opt, int max_probe,
                      su_batch_tuning *best, int cap, int *n_best) {
    using namespace su;
    if (n_best) *n_best = 0;
    if (max_probe < 1) return fail(SU_EINVAL, "max_probe must be >= 1");
    if (cap < 0 || (cap > 0 && !best)) return fail(SU_EINVAL, "best and cap inconsistent");
    if (!inst || n_inst < 1 || n_inst > (1LL << 24)) return fail(SU_EINVAL, "n_inst must be in 1..2^24");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    std::vector<BatchArg> arg;
    int rc = batch_args(p, inst, n_inst, n_mc, arg);
    if (rc) return rc;
    // the classes (p, s, hierarchy) and their first max_probe instances
    std::map<std::tuple<int, int, int>, std::vector<su_instance>> cls;
    for (int64_t i = 0; i < n_inst; ++i) {
        const BatchArg &q = arg[(size_t)i];
        if (q.s < 1) continue;
        auto &v = cls[std::make_tuple(q.p, q.s, q.hier)];
        if ((int)v.size() < max_probe) {
            su_instance x = inst[i];
            x.p = q.p;
            x.n_mc = q.n;
            v.push_back(x);
        }
    }
    cudaStream_t st = (cudaStream_t)o.stream;
    struct Res {
        void *buf = nullptr;
        size_t cap = 0;
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Res() {
            if (buf) cudaFree(buf);
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } res;
    CU(cudaEventCreate(&res.e[0]), "event");
    CU(cudaEventCreate(&res.e[1]), "event");
    int done = 0;
    for (auto &kv : cls) {
        const int cp = std::get<0>(kv.first), cs = std::get<1>(kv.first), ch = std::get<2>(kv.first);
        su_batch_tuning top{cp, cs, ch, 0, INFINITY};
        for (int F = 1; F <= std::min(cs, kMaxFine); ++F) {
            su_batch_plan *pl = nullptr;
            rc = batch_create(model, params, n_params, p, kv.second.data(), (int64_t)kv.second.size(), n_mc, seed, &o,
                              F, &pl);
            if (rc == SU_ENOTSUP) continue;   // this segment's shared memory does not fit
            if (rc) return rc;
            std::unique_ptr<su_batch_plan, int (*)(su_batch_plan *)> guard(pl, su_batch_plan_destroy);
            const size_t need = (size_t)(pl->tuple_bytes + pl->scratch_bytes);
            if (need > res.cap) {
                if (res.buf) cudaFree(res.buf);
                res.buf = nullptr;
                res.cap = 0;
                CU(dmalloc(&res.buf, need), "device allocation (probe buffers)");
                res.cap = need;
            }
            void *d_tup = res.buf, *d_scr = static_cast<char *>(res.buf) + pl->tuple_bytes;
            rc = su_batch_plan_execute(pl, d_tup, d_scr, st, nullptr);   // warm-up (and the graph)
            if (rc) return rc;
            float ms_best = INFINITY;
            for (int k = 0; k < 2; ++k) {
                CU(cudaEventRecord(res.e[0], st), "event record");
                rc = su_batch_plan_execute(pl, d_tup, d_scr, st, nullptr);
                if (rc) return rc;
                CU(cudaEventRecord(res.e[1], st), "event record");
                CU(cudaEventSynchronize(res.e[1]), "probe");
                float ms = 0;
                CU(cudaEventElapsedTime(&ms, res.e[0], res.e[1]), "event time");
                ms_best = std::min(ms_best, ms);
            }
            const double ns = (double)ms_best * 1e6 / (double)std::max<int64_t>(pl->slice_actions, 1);
            if (ns < top.ns_per_slice) {
                top.seg_log2 = F;
                top.ns_per_slice = ns;
            }
        }
        if (top.seg_log2 == 0) return fail(SU_ENOTSUP, "no register segment fits class p = %d, s = %d", cp, cs);
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_btune[{o.precision, model, cp, cs, ch}] = top.seg_log2;
        }
        if (done < cap) best[done] = top;
        ++done;
    }
    if (n_best) *n_best = done;
    g_err.clear();
    return SU_OK;
}

int speedup_philox_words(uint64_t seed, uint32_t instance, int64_t sample0, int64_t n_samples,
                         int n_calls, uint32_t *d_out, void *stream) {
    if (!d_out || sample0 < 0 || n_samples < 0 || n_calls < 0) return fail(SU_EINVAL, "bad arguments");
    CU(su::launch_philox_words(seed, instance, sample0, n_samples, n_calls, d_out, (cudaStream_t)stream),
       "philox launch");
    return SU_OK;
}

}  // extern "C"

// ------------------------------------------------------ learned proposal

static int64_t up256(int64_t x) { return (x + 255) / 256 * 256; }

struct su_proposal {
    void *d_blob = nullptr;
};

extern "C" int su_proposal_create(const float *theta, int n_params, su_proposal **out) {
    if (!out || !theta) return fail(SU_EINVAL, "arguments missing");
    *out = nullptr;
    if (n_params != su::mlp::kParams) return fail(SU_EINVAL, "the network has %d parameters", su::mlp::kParams);
    for (int i = 0; i < n_params; ++i)
        if (!std::isfinite(theta[i])) return fail(SU_ENONFINITE, "non-finite network parameter %d", i);
    std::vector<unsigned char> blob(su::mlp::kBlobBytes);
    su::mlp::pack_blob(theta, blob.data());
    std::unique_ptr<su_proposal> pr(new (std::nothrow) su_proposal);
    if (!pr) return fail(SU_ENOMEM, "host allocation failed");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return fail(SU_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(e));
    }
    CU(dmalloc(&pr->d_blob, blob.size()), "device allocation (network)");
    e = cudaMemcpy(pr->d_blob, blob.data(), blob.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(pr->d_blob);
        return cuda_fail(e, "upload network");
    }
    *out = pr.release();
    return SU_OK;
}

extern "C" int su_proposal_destroy(su_proposal *pr) {
    if (!pr) return SU_OK;
    if (pr->d_blob) cudaFree(pr->d_blob);
    delete pr;
    return SU_OK;
}

extern "C" int su_mlp_forward(const su_proposal *pr, const float *d_X, int64_t n, float *d_Y, void *stream) {
    if (!pr || !d_X || !d_Y || n < 0) return fail(SU_EINVAL, "arguments missing");
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev), "cudaGetDevice");
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    if (n == 0) return SU_OK;
    CU(su::launch_mlp_forward(static_cast<const unsigned char *>(pr->d_blob), d_X, n, d_Y, sms,
                              (cudaStream_t)stream),
       "network launch");
    return SU_OK;
}

// plan + proposal parameters with 128-sample items (one path per thread of
// the first 128 threads of a 256-thread CTA)
static int proposal_setup(su_plan *pl, const su_proposal *pr, su::ProposalParams &Q, int &grid, size_t &smem) {
    using namespace su;
    std::memset(&Q, 0, sizeof Q);
    Q.base = pl->P;
    Q.blob = static_cast<const unsigned char *>(pr->d_blob);
    Q.T = pl->T;
    SamplerParams &P = Q.base;
    P.rounds = 1;
    const int64_t bsz = (pl->n_mc + pl->n_blocks - 1) / pl->n_blocks;
    P.items_per_block = (bsz + mlp::kRows - 1) / mlp::kRows;
    P.n_items = P.items_per_block * pl->n_blocks;
    smem = proposal_smem_bytes(Q);
    int dev = 0, sms = 0, smem_max = 0;
    CU(cudaGetDevice(&dev), "cudaGetDevice");
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    CU(cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), "smem limit");
    if (smem > (size_t)smem_max) return fail(SU_ENOTSUP, "shared memory %zu exceeds %d bytes", smem, smem_max);
    const int occ = proposal_occupancy(Q, smem);
    if (occ < 1) return fail(SU_ECUDA, "proposal kernel cannot be resident");
    grid = (int)std::min<int64_t>(P.n_items, (int64_t)sms * occ);
    return SU_OK;
}

static int proposal_check(const su_options &o, int s, const su_proposal *pr) {
    if (!pr) return fail(SU_EINVAL, "proposal missing");
    if (o.precision != SU_FP32) return fail(SU_ENOTSUP, "the learned proposal runs the single-precision path");
    if (s > 6) return fail(SU_ENOTSUP, "the learned proposal supports s <= 6 (N <= 64)");
    if (o.width_factor != 1.0) return fail(SU_ENOTSUP, "the learned proposal replaces the width factor");
    return SU_OK;
}

// Sample plan pl's paths from the proposal and finalize (out: s+1 levels);
// *ms (may be NULL) = device time of the sampling launches (CUDA events).
static int proposal_amplitude_of_plan(su_plan *pl, const su_proposal *pr, su_level_result *out, float *ms) {
    if (ms) *ms = 0;
    if (pl->s == 0) return su_plan_finalize(pl, nullptr, nullptr, out);
    su::ProposalParams Q;
    std::memset(&Q, 0, sizeof Q);
    int grid = 0;
    size_t smem = 0;
    int rc = proposal_setup(pl, pr, Q, grid, smem);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)pl->opt.stream;
    const int64_t part_bytes = up256(Q.base.n_items * pl->levels * 4 * (int64_t)sizeof(double));
    const int64_t tb = pl->tuple_bytes;
    struct Ev {
        cudaEvent_t e[2] = {nullptr, nullptr};
        ~Ev() {
            for (cudaEvent_t x : e)
                if (x) cudaEventDestroy(x);
        }
    } ev;
    if (ms) {
        CU(cudaEventCreate(&ev.e[0]), "event");
        CU(cudaEventCreate(&ev.e[1]), "event");
    }
    void *dbuf = nullptr;
    CU(dmalloc_async(&dbuf, (size_t)(part_bytes + tb + 256), st), "cudaMallocAsync");
    Q.base.partial = static_cast<double *>(dbuf);
    double *d_tup = reinterpret_cast<double *>(static_cast<char *>(dbuf) + part_bytes);
    Q.base.flags = reinterpret_cast<int *>(static_cast<char *>(dbuf) + part_bytes + tb);
    Q.withhold = g_fault_mma.exchange(0);
    Q.base.w_out = nullptr;
    Q.outs = nullptr;
    std::vector<double> h((size_t)(tb / sizeof(double)));
    int flags = 0;
    cudaError_t e = cudaMemsetAsync(Q.base.flags, 0, sizeof(int), st);
    if (e == cudaSuccess && ms) e = cudaEventRecord(ev.e[0], st);
    if (e == cudaSuccess) e = su::launch_proposal(Q, grid, smem, st);
    if (e == cudaSuccess)
        e = su::launch_combine(Q.base.partial, d_tup, 0, pl->n_blocks, pl->levels, Q.base.items_per_block, st);
    if (e == cudaSuccess && ms) e = cudaEventRecord(ev.e[1], st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d_tup, (size_t)tb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, Q.base.flags, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, ev.e[0], ev.e[1]);
    cudaFreeAsync(dbuf, st);
    if (e != cudaSuccess) return cuda_fail(e, "proposal sampling");
    if (flags & 4) return fail(SU_ETIMEOUT, "a tensor-core MMA of the proposal network did not complete");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return su_plan_finalize(pl, h.data(), nullptr, out);
}

extern "C" int speedup_amplitude_proposal(int model, const double *params, int n_params, double a, double b,
                                          double T, int p, int s, int64_t n_mc, uint64_t seed,
                                          const su_options *opt, const su_proposal *pr, su_level_result *out) {
    if (!out) return fail(SU_EINVAL, "output missing");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    int rc = proposal_check(o, s, pr);
    if (rc) return rc;
    su_plan *pl = nullptr;
    rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_mc, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    return proposal_amplitude_of_plan(pl, pr, out, nullptr);
}

// The judge's view of one pilot run: usable when its top-level estimate is
// finite and positive and rests on at least kJudgeMinEss effective samples.
static constexpr double kJudgeMinEss = 10.0;

static void judge_arm(const su_level_result &r, int64_t n, float ms, double target, int arm, su_judge *j) {
    j->pilot_amp[arm] = r.amp;
    j->pilot_err[arm] = r.err;
    j->pilot_ess[arm] = r.ess;
    j->pilot_s[arm] = ms / 1e3;
    const bool ok = std::isfinite(r.amp) && r.amp > 0 && std::isfinite(r.err) && r.ess >= kJudgeMinEss;
    // per-sample relative variance Var(f) / E[f]^2 = n / ESS - 1 (the pilot's own sums)
    j->pilot_relvar[arm] = ok ? std::max((double)n / r.ess - 1.0, 0.0) : INFINITY;
    j->t_target[arm] = ok ? (ms / 1e3) / (double)n * j->pilot_relvar[arm] / (target * target) : INFINITY;
}

extern "C" int speedup_amplitude_judged(int model, const double *params, int n_params, double a, double b,
                                        double T, int p, int s, int64_t n_mc, uint64_t seed,
                                        const su_options *opt, const su_proposal *pr, int64_t n_pilot,
                                        double target_rel_err, su_level_result *out, su_judge *judge) {
    if (!out || !judge) return fail(SU_EINVAL, "output or judge missing");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    int rc = proposal_check(o, s, pr);
    if (rc) return rc;
    if (s < 1) return fail(SU_EINVAL, "the judge compares sampled levels: s must be >= 1");
    if (n_pilot < 2 || !(target_rel_err > 0) || !std::isfinite(target_rel_err))
        return fail(SU_EINVAL, "n_pilot must be >= 2 and target_rel_err finite and > 0");
    std::memset(judge, 0, sizeof *judge);
    judge->target_rel_err = target_rel_err;
    // pilots on the samples after the run's own range, so the main run is
    // the one speedup_amplitude (or _proposal) would make
    su_options op = o;
    op.sample0 = o.sample0 + n_mc;
    op.hierarchy = 0;
    std::vector<su_level_result> pil((size_t)s + 1);
    for (int arm = 0; arm < 2; ++arm) {
        su_plan *pl = nullptr;
        rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_pilot, seed, &op, &pl);
        if (rc) return rc;
        std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
        float ms = 0;
        rc = arm == 0 ? amplitude_of_plan(pl, pil.data(), &ms) : proposal_amplitude_of_plan(pl, pr, pil.data(), &ms);
        if (rc == SU_ENONFINITE) {   // a non-finite weight: this arm cannot estimate the amplitude
            su_level_result bad{};
            bad.amp = NAN;
            bad.err = NAN;
            judge_arm(bad, n_pilot, ms, target_rel_err, arm, judge);
            continue;
        }
        if (rc) return rc;
        judge_arm(pil[(size_t)s], n_pilot, ms, target_rel_err, arm, judge);
    }
    const bool ok0 = std::isfinite(judge->t_target[0]), ok1 = std::isfinite(judge->t_target[1]);
    const double sig = std::hypot(judge->pilot_err[0], judge->pilot_err[1]);
    judge->z = (ok0 && ok1 && sig > 0) ? (judge->pilot_amp[1] - judge->pilot_amp[0]) / sig : NAN;
    // the proposal is taken only where the plain sampler confirms it and it is faster
    if (!ok1)
        judge->reason = SU_JUDGE_PROPOSAL_UNUSABLE;
    else if (!ok0)
        judge->reason = SU_JUDGE_PLAIN_UNUSABLE;
    else if (!(std::fabs(judge->z) <= 5.0))
        judge->reason = SU_JUDGE_DISAGREE;
    else
        judge->reason = judge->t_target[1] < judge->t_target[0] ? SU_JUDGE_PROPOSAL_FASTER : SU_JUDGE_PLAIN_FASTER;
    judge->chosen = judge->reason == SU_JUDGE_PROPOSAL_FASTER ? 1 : 0;
    su_plan *pl = nullptr;
    rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_mc, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    float ms = 0;
    rc = judge->chosen ? proposal_amplitude_of_plan(pl, pr, out, &ms) : amplitude_of_plan(pl, out, &ms);
    judge->run_s = ms / 1e3;
    return rc;
}

extern "C" int speedup_proposal_logweights(int model, const double *params, int n_params, double a, double b,
                                           double T, int p, int s, int64_t sample0, int64_t n_samples,
                                           uint64_t seed, const su_options *opt, const su_proposal *pr,
                                           double *d_w, float *d_outs) {
    if (s < 1) return fail(SU_EINVAL, "s must be >= 1 for per-sample weights");
    if (!d_w) return fail(SU_EINVAL, "output missing");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    o.hierarchy = 1;
    o.n_blocks = 1;
    o.sample0 = sample0;
    int rc = proposal_check(o, s, pr);
    if (rc) return rc;
    su_plan *pl = nullptr;
    rc = su_plan_create(model, params, n_params, a, b, T, p, s, n_samples, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    su::ProposalParams Q;
    std::memset(&Q, 0, sizeof Q);
    int grid = 0;
    size_t smem = 0;
    rc = proposal_setup(pl, pr, Q, grid, smem);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.stream;
    int *d_flag = nullptr;
    CU(dmalloc_async(&d_flag, sizeof(int), st), "cudaMallocAsync");
    Q.base.flags = d_flag;
    Q.withhold = g_fault_mma.exchange(0);
    Q.base.w_out = d_w;
    Q.base.partial = nullptr;
    Q.outs = d_outs;
    int flags = 0;
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = su::launch_proposal(Q, grid, smem, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFreeAsync(d_flag, st);
    if (e != cudaSuccess) return cuda_fail(e, "proposal per-sample weights");
    if (flags & 4) return fail(SU_ETIMEOUT, "a tensor-core MMA of the proposal network did not complete");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    return SU_OK;
}

// ------------------------------------------------------- proposal training

extern "C" void su_train_options_default(su_train_options *t) {
    if (!t) return;
    std::memset(t, 0, sizeof *t);
    t->n_train = 1000000;
    t->steps = 2000;
    t->batch_paths = 512;
    t->lr = 1e-3;
    t->clip_quantile = 0.999;
    t->seed = 1;
}

extern "C" int su_mlp_loss_grad(const float *theta, const float *d_X, const float *d_u, const float *d_rw,
                                int64_t n, double *loss, float *grad) {
    if (!theta || !d_X || !d_u || !d_rw || !loss || !grad || n < 1 || n > (1 << 22))
        return fail(SU_EINVAL, "bad arguments");
    const int R = (int)((n + 31) / 32 * 32);
    su::train::Workspace ws;
    CU(ws.reserve(R), "training workspace");
    cudaStream_t st = nullptr;
    double norm = 0;
    {
        std::vector<float> rw((size_t)n);
        CU(cudaMemcpy(rw.data(), d_rw, (size_t)n * 4, cudaMemcpyDeviceToHost), "read weights");
        for (float v : rw) norm += v;
    }
    if (!(norm > 0)) return fail(SU_EINVAL, "row weights must have a positive sum");
    CU(cudaMemcpyAsync(ws.theta, theta, (size_t)su::mlp::kParams * 4, cudaMemcpyHostToDevice, st), "upload theta");
    CU(su::train::rows_from_features(ws, d_X, d_u, d_rw, (int)n, R, st), "rows");
    CU(su::train::loss_grad(ws, R, 1.0 / norm, true, st), "loss and gradient");
    CU(cudaMemcpyAsync(grad, ws.grad, (size_t)su::mlp::kParams * 4, cudaMemcpyDeviceToHost, st), "read gradient");
    CU(cudaMemcpyAsync(loss, ws.loss, 8, cudaMemcpyDeviceToHost, st), "read loss");
    int tstat = 0;
    CU(cudaMemcpyAsync(&tstat, ws.status, sizeof(int), cudaMemcpyDeviceToHost, st), "read status");
    CU(cudaStreamSynchronize(st), "training step");
    if (tstat) return fail(SU_ETIMEOUT, "a tensor-core MMA of the training GEMMs did not complete");
    return SU_OK;
}

extern "C" int speedup_train_proposal(int model, const double *params, int n_params, double a, double b, double T,
                                      int p, int s, uint64_t seed, const su_train_options *topt, float *theta,
                                      double *loss_out) {
    if (!theta) return fail(SU_EINVAL, "theta missing");
    su_train_options to;
    su_train_options_default(&to);
    if (topt) to = *topt;
    if (s < 2 || s > 6) return fail(SU_ENOTSUP, "training supports 2 <= s <= 6");
    if (to.n_train < 64 || to.n_train > (1LL << 26)) return fail(SU_EINVAL, "n_train must be in 64..2^26");
    if (to.steps < 1 || to.batch_paths < 32 || to.batch_paths % 32 != 0 || to.batch_paths > 16384)
        return fail(SU_EINVAL, "steps >= 1, batch_paths a multiple of 32 in 32..16384");
    if (!(to.lr > 0) || !(to.clip_quantile > 0 && to.clip_quantile <= 1)) return fail(SU_EINVAL, "bad lr or clip");
    const int N = 1 << s, np1 = N + 1;
    // 1. plain single-precision paths and their top-level weights
    su_options o;
    su_options_default(&o);
    o.precision = SU_FP32;
    o.hierarchy = 1;
    o.n_blocks = 1;
    su_plan *pl = nullptr;
    int rc = su_plan_create(model, params, n_params, a, b, T, p, s, to.n_train, seed, &o, &pl);
    if (rc) return rc;
    std::unique_ptr<su_plan, int (*)(su_plan *)> guard(pl, su_plan_destroy);
    float *d_paths = nullptr;
    double *d_w = nullptr;
    int *d_flag = nullptr, *d_ids = nullptr;
    float *d_sig = nullptr;
    struct Free {
        std::vector<void *> v;
        ~Free() { for (void *q : v) cudaFree(q); }
    } fr;
    CU(dmalloc(&d_paths, (size_t)to.n_train * np1 * 4), "device allocation (paths)");
    fr.v.push_back(d_paths);
    CU(dmalloc(&d_w, (size_t)to.n_train * s * 8), "device allocation (weights)");
    fr.v.push_back(d_w);
    CU(dmalloc(&d_flag, 4), "device allocation (flag)");
    fr.v.push_back(d_flag);
    CU(dmalloc(&d_ids, (size_t)to.batch_paths * 4), "device allocation (ids)");
    fr.v.push_back(d_ids);
    CU(dmalloc(&d_sig, 16 * 4), "device allocation (sigma)");
    fr.v.push_back(d_sig);
    su::SamplerParams P = pl->P;
    P.w_out = d_w;
    P.q_out = d_paths;
    P.flags = d_flag;
    P.partial = nullptr;
    const size_t smem = su::sampler_smem_bytes(P, SU_FP32);
    if (su::sampler_occupancy(P, SU_FP32, smem) < 1) return fail(SU_ECUDA, "sampler not resident");
    CU(cudaMemset(d_flag, 0, 4), "clear flag");
    CU(su::launch_sampler(P, SU_FP32, pl->grid, smem, nullptr), "path sampling");
    std::vector<double> w((size_t)to.n_train * s);
    CU(cudaMemcpy(w.data(), d_w, w.size() * 8, cudaMemcpyDeviceToHost), "read weights");
    // 2. training weights: top-level log-weights clipped at a quantile (the
    //    weighted likelihood of rare huge weights would fit one path), then
    //    minibatches drawn in proportion to them
    std::vector<double> wt((size_t)to.n_train);
    for (int64_t i = 0; i < to.n_train; ++i) wt[(size_t)i] = w[(size_t)i * s + (s - 1)];
    std::vector<double> srt = wt;
    const size_t qi = std::min(srt.size() - 1, (size_t)(to.clip_quantile * (double)(srt.size() - 1)));
    std::nth_element(srt.begin(), srt.begin() + qi, srt.end());
    const double cap = srt[qi];
    double mx = -INFINITY;
    for (double &v : wt) {
        if (!std::isfinite(v) && v > 0) return fail(SU_ENONFINITE, "a training weight is +Inf or NaN");
        v = std::min(v, cap);
        mx = std::max(mx, v);
    }
    std::vector<double> cdf(wt.size());
    double acc = 0;
    for (size_t i = 0; i < wt.size(); ++i) {
        acc += std::isfinite(wt[i]) ? std::exp(wt[i] - mx) : 0.0;
        cdf[i] = acc;
    }
    if (!(acc > 0)) return fail(SU_ENONFINITE, "all training weights vanish");
    // 3. Adam on minibatches of batch_paths paths x (N-1) midpoints, drawn on
    //    the device from the running sums of the weights; one step (draw, rows,
    //    loss and gradient, Adam, loss record) is captured as a CUDA graph on a
    //    stream of its own and replayed `steps` times
    const int R = to.batch_paths * (N - 1);
    su::train::Workspace ws;
    CU(ws.reserve(R), "training workspace");
    double *d_cdf = nullptr, *d_losses = nullptr;
    int *d_step = nullptr;
    CU(dmalloc(&d_cdf, cdf.size() * sizeof(double)), "device allocation (cdf)");
    fr.v.push_back(d_cdf);
    CU(dmalloc(&d_losses, (size_t)to.steps * sizeof(double)), "device allocation (losses)");
    fr.v.push_back(d_losses);
    CU(dmalloc(&d_step, sizeof(int)), "device allocation (step)");
    fr.v.push_back(d_step);
    struct GraphRes {
        cudaStream_t st = nullptr;
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        ~GraphRes() {
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (st) cudaStreamDestroy(st);
        }
    } gr;
    CU(cudaStreamCreateWithFlags(&gr.st, cudaStreamNonBlocking), "training stream");
    float sig[16] = {0};
    for (int n = 1; n <= s; ++n) sig[n] = (float)std::sqrt(T / std::ldexp(1.0, n + 1));
    CU(cudaMemcpy(d_sig, sig, sizeof sig, cudaMemcpyHostToDevice), "upload sigma");
    CU(cudaMemcpy(d_cdf, cdf.data(), cdf.size() * sizeof(double), cudaMemcpyHostToDevice), "upload cdf");
    CU(cudaMemcpy(ws.theta, theta, (size_t)su::mlp::kParams * 4, cudaMemcpyHostToDevice), "upload theta");
    CU(cudaMemset(ws.m, 0, (size_t)su::mlp::kParams * 8), "clear moments");   // m and v are adjacent
    CU(cudaMemset(d_step, 0, sizeof(int)), "clear step");
    CU(su::train::fill(ws.rw, 1.0f, R, nullptr), "row weights");
    CU(cudaDeviceSynchronize(), "training set-up");
    const int64_t n_train = to.n_train;
    CU(cudaStreamBeginCapture(gr.st, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t ce = su::train::sample_ids(d_cdf, n_train, acc, to.seed, d_step, to.batch_paths, d_ids, gr.st);
    if (ce == cudaSuccess)
        ce = su::train::build_rows(ws, d_paths, np1, d_ids, to.batch_paths, (float)a, (float)b, (float)T, s, d_sig,
                                   gr.st);
    if (ce == cudaSuccess) ce = su::train::loss_grad(ws, R, 1.0 / R, true, gr.st);
    if (ce == cudaSuccess) ce = su::train::adam_step_dev(ws, d_step, (float)to.lr, gr.st);
    if (ce == cudaSuccess) ce = su::train::step_tail(d_step, ws.loss, d_losses, gr.st);
    const cudaError_t ee = cudaStreamEndCapture(gr.st, &gr.g);
    if (ce != cudaSuccess) return cuda_fail(ce, "capturing the training step");
    CU(ee, "end capture");
    CU(cudaGraphInstantiate(&gr.ge, gr.g, 0), "instantiate the training step");
    for (int t = 0; t < to.steps; ++t) CU(cudaGraphLaunch(gr.ge, gr.st), "training step");
    CU(cudaStreamSynchronize(gr.st), "training");
    if (loss_out)
        CU(cudaMemcpy(loss_out, d_losses, (size_t)to.steps * sizeof(double), cudaMemcpyDeviceToHost), "read losses");
    int tstat = 0;
    CU(cudaMemcpy(&tstat, ws.status, sizeof(int), cudaMemcpyDeviceToHost), "read status");
    if (tstat) return fail(SU_ETIMEOUT, "a tensor-core MMA of the training GEMMs did not complete");
    CU(cudaMemcpy(theta, ws.theta, (size_t)su::mlp::kParams * 4, cudaMemcpyDeviceToHost), "read theta");
    return SU_OK;
}

// -------------------------------------------------- allocation-free variant
//
// Some callers must not allocate device memory while they run: code inside a
// memory-capped or pre-partitioned process, a host that drives the GPU from a
// real-time loop where cudaMalloc/cudaFree (and their implicit device
// synchronisation) are forbidden, or a caller whose allocator owns all device
// memory.  speedup_amplitude_noalloc serves them: it keeps its device scratch
// (coefficient tables, per-item and per-block log-sum-exp tuples, the
// non-finite flag) in the library's own static device array below, which
// every GPU that loads the library holds until the process exits.

static __device__ __align__(256) unsigned char g_noalloc_scratch[SU_NOALLOC_SCRATCH_BYTES];

// The array's name is a host-side stand-in in host code; its device address
// comes from cudaGetSymbolAddress with the caller's device current.  It is
// looked up on every call, not cached: a context torn down and rebuilt (for
// example after cudaDeviceReset) loads the module again, possibly elsewhere.
static int noalloc_scratch(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    }
    *out = static_cast<unsigned char *>(p);
    return SU_OK;
}

extern "C" int speedup_amplitude_noalloc(int model, const double *params, int n_params, double a, double b,
                                         double T, int p, int s, int64_t n_mc, uint64_t seed,
                                         const su_options *opt, su_level_result *out) {
    using namespace su;
    if (!out) return fail(SU_EINVAL, "output missing");
    su_options o;
    su_options_default(&o);
    if (opt) o = *opt;
    if (model == SU_GENERAL) return fail(SU_ENOTSUP, "the allocation-free path takes the collapsed-table models only");
    // the plan's host side (arguments, tables, launch shape) as su_plan_create
    // builds it; only the device memory differs
    su_plan pl;
    int rc = plan_init(pl, model, params, n_params, a, b, T, p, s, n_mc, seed, o);
    if (rc) return rc;
    if (s == 0) return su_plan_finalize(&pl, nullptr, nullptr, out);
    std::vector<unsigned char> blob;
    rc = plan_tables(pl, blob);
    if (rc) return rc;
    int dev = 0, sms = 0, smem_max = 0;
    rc = device_limits(dev, sms, smem_max);
    if (rc) return rc;
    rc = plan_shape(pl, sms, smem_max);
    if (rc) return rc;

    // scratch layout: tables | per-item tuples | per-block tuples | flag word;
    // where the per-item tuples do not fit, more paths per item (rounds up to
    // 8, while the shape stays resident), unless the caller fixed rounds
    const int64_t tab_bytes = up256((int64_t)blob.size());
    const int64_t tup_bytes = up256(pl.tuple_bytes);
    auto fits = [&] { return tab_bytes + up256(pl.partial_bytes) + tup_bytes + 256 <= (int64_t)SU_NOALLOC_SCRATCH_BYTES; };
    if (!fits() && o.rounds == 0) {
        int good = pl.P.rounds;
        for (int r = good * 2; r <= 8 && !fits(); r *= 2) {
            if (plan_rounds(pl, r, sms, smem_max) < 1) break;   // shared memory or residency
            good = r;
        }
        plan_rounds(pl, good, sms, smem_max);
    }
    if (!fits())
        return fail(SU_ENOTSUP,
                    "n_mc = %lld with %lld blocks and %d levels needs more than the %u bytes of no-alloc scratch",
                    (long long)n_mc, (long long)pl.n_blocks, pl.levels, (unsigned)SU_NOALLOC_SCRATCH_BYTES);

    unsigned char *base = nullptr;
    rc = noalloc_scratch(&base);
    if (rc) return rc;
    SamplerParams P = pl.P;
    unsigned char *d_tab = base;
    double *d_part = reinterpret_cast<double *>(base + tab_bytes);
    double *d_tup = reinterpret_cast<double *>(base + tab_bytes + up256(pl.partial_bytes));
    int *d_flag = reinterpret_cast<int *>(base + tab_bytes + up256(pl.partial_bytes) + tup_bytes);
    P.tables = d_tab;
    P.partial = d_part;
    P.flags = d_flag;
    P.w_out = nullptr;
    P.item0 = 0;

    cudaStream_t st = (cudaStream_t)o.stream;
    std::vector<double> h((size_t)(pl.tuple_bytes / sizeof(double)));
    int flags = 0;
    CU(cudaMemcpyAsync(d_tab, blob.data(), blob.size(), cudaMemcpyHostToDevice, st), "upload tables");
    CU(cudaMemsetAsync(d_flag, 0, sizeof(int), st), "clear flag");
    CU(launch_sampler(P, o.precision, pl.grid, pl.smem, st), "sampler launch");
    CU(launch_combine(d_part, d_tup, 0, pl.n_blocks, pl.levels, P.items_per_block, st), "combine launch");
    CU(cudaMemcpyAsync(h.data(), d_tup, h.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "read tuples");
    CU(cudaMemcpyAsync(&flags, d_flag, sizeof(int), cudaMemcpyDeviceToHost, st), "read flag");
    CU(cudaStreamSynchronize(st), "sampling");
    if (flags & 1) return fail(SU_ENONFINITE, "a per-sample weight was NaN or +Inf");
    // the same completeness check as su_plan_finalize (every sample reduced)
    return su_plan_finalize(&pl, h.data(), nullptr, out);
}
