// api.cu -- the C-ABI of libmpkm (include/mpkm.h): argument checks, the
// workspace layout, and the launch sequences of the hot path:
//   assign  = quantise X and C (+ statistics) -> tensor-core screening with
//             the fused reliability test and candidate collection ->
//             refinement by the direct formula (fp32, then binary64 where the
//             argmin is still open) -> full-row direct pass for overflowed rows
//   update  = exact fixed-point centroid sums -> means, empty clusters, shift
//   lloyd   = Alg. 3 on top of the two.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <vector>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>

#include "../../include/mpkm.h"
#include "common.cuh"
#include "group.h"
#include "internal.h"
#include "seed.h"
#include "serve.h"

using namespace km;

// Screening-kernel variant per shape class (format, K atoms, 128-column tiles
// of C, fewer row blocks than SMs): set by km_autotune / km_set_screen_variant,
// shared with the context's serving workers.
struct km_tune {
    std::mutex mu;
    std::map<uint64_t, int> v;
    static uint64_t key(int fmt, int kchunks, int k, int64_t n, int num_sms) {
        const uint64_t nt = (uint64_t)((k + 127) / 128);
        const uint64_t small = (n + 127) / 128 < num_sms ? 1 : 0;
        return (uint64_t)fmt | ((uint64_t)kchunks << 4) | (nt << 8) | (small << 40);
    }
};
// km_autotune's trial variant for the calling thread (-1: none)
static thread_local int t_trial_variant = -1;

struct km_ctx {
    int device = 0;
    int num_sms = 148;
    std::string err;
    // last call, for km_get_stats
    DevCounters* last_cnt = nullptr;
    double* last_sse = nullptr;
    cudaStream_t last_stream = nullptr;
    uint64_t last_pairs = 0;
    km_serve* serve = nullptr;
    // phase timing (km_set_profiling) and launch counting
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[KM_NUM_PHASES];
    uint64_t launches = 0;
    // km_lloyd_step_host: two copy streams and the events that order them
    // against the caller's stream (created on first use)
    cudaStream_t copy_st[2] = {nullptr, nullptr};
    std::vector<cudaEvent_t> host_ev;
    // km_lloyd_run's replayed iterations run on this stream when the caller's
    // is a legacy default stream (which cannot be captured)
    cudaStream_t graph_st = nullptr;
    cudaEvent_t graph_ev[2] = {nullptr, nullptr};
    // screening-kernel variants: the context's own table, or (a serving job's
    // context) the owning context's
    km_tune tune_own;
    km_tune* tune = &tune_own;
    ~km_ctx() {
        for (cudaEvent_t e : graph_ev)
            if (e) cudaEventDestroy(e);
        if (graph_st) cudaStreamDestroy(graph_st);
        for (auto& v : ev)
            for (auto& e : v) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        for (cudaEvent_t e : host_ev) cudaEventDestroy(e);
        for (cudaStream_t c : copy_st)
            if (c) cudaStreamDestroy(c);
    }
};

// Records the start / end of a phase on `st` while profiling is on.
struct PhaseScope {
    km_ctx* c;
    int ph;
    cudaStream_t st;
    cudaEvent_t b = nullptr, e = nullptr;
    PhaseScope(km_ctx* c_, int ph_, cudaStream_t st_) : c(c_), ph(ph_), st(st_) {
        if (c->prof && cudaEventCreate(&b) == cudaSuccess && cudaEventCreate(&e) == cudaSuccess) cudaEventRecord(b, st);
        else b = e = nullptr;
    }
    ~PhaseScope() {
        if (b && e) {
            cudaEventRecord(e, st);
            c->ev[ph].emplace_back(b, e);
        }
    }
};

namespace {

constexpr int kSumParts = 1024;

km_status fail(km_ctx* c, km_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CK(expr)                                                                                     \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return fail(ctx, KM_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
    } while (0)

// Launches `n` kernels through `expr` and counts them.
#define KL(n, expr)              \
    do {                         \
        ctx->launches += (n);    \
        CK(expr);                \
    } while (0)

int fmt_of(int low) { return low == KM_FP16 ? 0 : (low == KM_BF16 ? 1 : 2); }
bool is_tc(int low) { return low == KM_FP16 || low == KM_BF16 || low == KM_E4M3; }
double unit_roundoff(int fmt) { return fmt == 0 ? std::ldexp(1.0, -11) : (fmt == 1 ? std::ldexp(1.0, -8) : std::ldexp(1.0, -4)); }
double gamma_m(int m, double u) {
    double mu = m * u;
    return mu >= 1.0 ? INFINITY : mu / (1.0 - mu);
}
int kpad_of(int k) { return ((k + 255) / 256) * 256; }
int ldq_of(int fmt, int d) { return fmt == 2 ? ((d + 15) / 16) * 16 : ((d + 7) / 8) * 8; }

struct Carve {
    char* base;
    size_t off = 0;
    template <typename T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += count * sizeof(T);
        return p;
    }
};

// Workspace of one assignment / distance computation.
struct AssignWs {
    DevCounters* cnt;
    ColMax* colmax;
    void* Xq;
    void* Cq;
    float4* xstat;
    float* xscale;
    float4* cstat;
    float* cscale;
    float* qpad;
    float* spad;
    uint32_t* cand;
    int2* pairs;
    float* v32;
    int2* rowpair;
    int64_t pair_cap;
    int4* rowinfo;
    int32_t* ovf_list;
    int32_t* amb_list;
    double* partials;
    double* sse;
    int2* queue;
    int64_t qcap;
    unsigned long long* qlen;
    float* dxx;   // matrix modes on CUDA cores: Alg. 2's d_xx per row, d_yy per centre
    float* dyy;
};

// Flagged pairs the distance-matrix call queues for the binary64 patch: four
// per row (at least 2^20, at most all n k); more flagged pairs than that are
// found by a scan of D for their marks instead.
int64_t flag_queue_cap(int64_t n, int k) {
    return std::min<int64_t>(n * (int64_t)k, std::max<int64_t>(4 * n, (int64_t)1 << 20));
}

AssignWs carve_assign(Carve& cv, int64_t n, int d, int k, int low, bool distances) {
    AssignWs w{};
    w.cnt = cv.take<DevCounters>(1);
    w.colmax = cv.take<ColMax>(1);
    w.partials = cv.take<double>(kSumParts);
    w.sse = cv.take<double>(1);
    w.amb_list = cv.take<int32_t>((size_t)n);
    if (is_tc(low)) {
        const int fmt = fmt_of(low);
        const int esz = fmt == 2 ? 1 : 2;
        const int ldq = ldq_of(fmt, d);
        w.Xq = cv.take<char>((size_t)n * ldq * esz);
        w.Cq = cv.take<char>((size_t)k * ldq * esz);
        w.xstat = cv.take<float4>((size_t)n);
        w.xscale = cv.take<float>((size_t)n);
        w.cstat = cv.take<float4>((size_t)k);
        w.cscale = cv.take<float>((size_t)k);
        w.qpad = cv.take<float>((size_t)kpad_of(k));
        w.spad = cv.take<float>((size_t)kpad_of(k));
        w.rowinfo = cv.take<int4>((size_t)n * TC_GROUPS);
        w.ovf_list = cv.take<int32_t>((size_t)n);
        if (!distances) {
            w.cand = cv.take<uint32_t>((size_t)n * TC_GROUPS * TC_LIST);
            w.rowpair = cv.take<int2>((size_t)n);
            w.pair_cap = std::min<int64_t>((int64_t)n * TC_PAIRS_PER_ROW, (int64_t)INT32_MAX);
            w.pairs = cv.take<int2>((size_t)w.pair_cap);
            w.v32 = cv.take<float>((size_t)w.pair_cap);
        } else {
            w.qcap = flag_queue_cap(n, k);
            w.queue = cv.take<int2>((size_t)w.qcap);
            w.qlen = cv.take<unsigned long long>(1);
        }
    } else if (distances) {
        w.dxx = cv.take<float>((size_t)n);
        w.dyy = cv.take<float>((size_t)k);
        w.qcap = flag_queue_cap(n, k);
        w.queue = cv.take<int2>((size_t)w.qcap);
        w.qlen = cv.take<unsigned long long>(1);
    }
    return w;
}

struct UpdateWs {
    long long* sums;
    long long* counts;
    unsigned* absmax;
    double* shift;
    void* esel;
    int* iscratch;
    int32_t* perm;
};
UpdateWs carve_update(Carve& cv, int64_t n, int d, int k) {
    UpdateWs u{};
    u.sums = cv.take<long long>((size_t)k * d);
    u.counts = cv.take<long long>((size_t)k);
    u.absmax = cv.take<unsigned>(1);
    u.shift = cv.take<double>(1);
    u.esel = cv.take<unsigned char>(empty_select_bytes(k));
    u.iscratch = cv.take<int>((size_t)4 * k + 2);
    u.perm = cv.take<int32_t>((size_t)n);
    return u;
}

// Device copies of the inputs and outputs of km_lloyd_step_host.
struct HostWs {
    float* X;
    float* C;
    int32_t* labels;
    double* min_dist;
    float* C_new;
    int64_t* counts;
};
HostWs carve_host(Carve& cv, int64_t n, int d, int k) {
    HostWs h{};
    h.X = cv.take<float>((size_t)n * d);
    h.C = cv.take<float>((size_t)k * d);
    h.labels = cv.take<int32_t>((size_t)n);
    h.min_dist = cv.take<double>((size_t)n);
    h.C_new = cv.take<float>((size_t)k * d);
    h.counts = cv.take<int64_t>((size_t)k);
    return h;
}

struct LloydWs {
    AssignWs a;
    UpdateWs u;
    float* C0;
    float* C1;
    double* min_dist;
    double* sse_hist;
    unsigned long long* flag_hist;
    int64_t* counts;
    double* sse_slot;  // a replayed iteration's SSE, appended to sse_hist on the device
    int* hist_len;     // entries of sse_hist / flag_hist written by replayed iterations
};
LloydWs carve_lloyd(Carve& cv, int64_t n, int d, int k, int low, int max_iter) {
    LloydWs L{};
    L.a = carve_assign(cv, n, d, k, low, false);
    L.u = carve_update(cv, n, d, k);
    L.C0 = cv.take<float>((size_t)k * d);
    L.C1 = cv.take<float>((size_t)k * d);
    L.min_dist = cv.take<double>((size_t)n);
    L.sse_hist = cv.take<double>((size_t)max_iter + 1);
    L.flag_hist = cv.take<unsigned long long>((size_t)max_iter + 1);
    L.counts = cv.take<int64_t>((size_t)k);
    L.sse_slot = cv.take<double>(1);
    L.hist_len = cv.take<int>(1);
    return L;
}

km_status check_params(km_ctx* ctx, const km_params* p, int d, int k = 1, bool matrix = false) {
    if (!p) return fail(ctx, KM_EINVAL, "params is NULL");
    if (p->low < KM_FP64_DIRECT || p->low > KM_FP32) return fail(ctx, KM_EINVAL, "unknown low precision %d", p->low);
    if (p->test < KM_TEST_TC || p->test > KM_TEST_OFF) return fail(ctx, KM_EINVAL, "unknown test %d", p->test);
    if (p->empty != KM_EMPTY_KEEP && p->empty != KM_EMPTY_FARTHEST) return fail(ctx, KM_EINVAL, "unknown empty policy");
    if (p->fallback < KM_FB_FP64 || p->fallback > KM_FB_LOW) return fail(ctx, KM_EINVAL, "unknown fallback %d", p->fallback);
    if (!matrix) {
        if (p->low == KM_FP32) return fail(ctx, KM_EUNSUPPORTED, "KM_FP32 is a distance-matrix mode (km_distances)");
        if (p->fallback != KM_FB_FP64)
            return fail(ctx, KM_EUNSUPPORTED, "the assignment certifies in fp32 and binary64: fallback must be KM_FB_FP64");
    }
    if (p->low == KM_FP32) {
        if (p->test == KM_TEST_TC && !(p->rho > 1.0)) return fail(ctx, KM_EINVAL, "rho must exceed 1 for the tc test");
        if (p->test == KM_TEST_PAPER && !(p->rho > 2.0))
            return fail(ctx, KM_EINVAL, "rho must exceed 2 for the paper test (Eq. (quantis-reliability-test))");
        if (p->test == KM_TEST_PAPER && !(p->paper_factor > 0.0)) return fail(ctx, KM_EINVAL, "paper_factor must be positive");
        if (d > 1024) return fail(ctx, KM_EUNSUPPORTED, "KM_FP32 supports d <= 1024");
        return KM_OK;
    }
    if (matrix && !is_tc(p->low)) {
        if (d > 1024) return fail(ctx, KM_EUNSUPPORTED, "the direct distance matrix supports d <= 1024");
        return KM_OK;
    }
    if (p->fallback == KM_FB_LOW && p->low == KM_E4M3)
        return fail(ctx, KM_EUNSUPPORTED, "no same-precision fallback for E4M3 (no E4M3 arithmetic)");
    if (is_tc(p->low)) {
        if (p->test == KM_TEST_TC && !(p->rho > 1.0)) return fail(ctx, KM_EINVAL, "rho must exceed 1 for the tc test");
        if (p->test == KM_TEST_PAPER) {
            if (!(p->rho > 2.0)) return fail(ctx, KM_EINVAL, "rho must exceed 2 for the paper test (Eq. (quantis-reliability-test))");
            if (!(p->paper_factor > 0.0)) return fail(ctx, KM_EINVAL, "paper_factor must be positive");
            if ((d + 2) * unit_roundoff(fmt_of(p->low)) >= 1.0)
                return fail(ctx, KM_EUNSUPPORTED, "gamma^l_{d+2} undefined: (d+2) u_l >= 1 for d=%d", d);
        }
        if (p->low == KM_E4M3 && d < 16) return fail(ctx, KM_EUNSUPPORTED, "E4M3 needs d >= 16");
        if (k > 65535) return fail(ctx, KM_EUNSUPPORTED, "the tensor-core paths support k <= 65535");
        if (tc_smem_bytes(fmt_of(p->low), d, 1) == 0) return fail(ctx, KM_EUNSUPPORTED, "d=%d too large for the tensor-core tiles", d);
    } else {
        if (d > 256) return fail(ctx, KM_EUNSUPPORTED, "direct paths support d <= 256");
    }
    return KM_OK;
}

TestParams make_tp(const km_params* p, int d) {
    TestParams tp{};
    const double u32 = std::ldexp(1.0, -24);
    const int fmt = is_tc(p->low) ? fmt_of(p->low) : 1;
    const double uacc = fmt == 2 ? std::ldexp(1.0, -13) : std::ldexp(1.0, -21);
    tp.test = p->test;
    tp.rho = (float)p->rho;
    tp.kacc = (float)((2.0 * gamma_m(d, uacc) + 4.0 * u32) * (1.0 + 1e-6));
    tp.kn = (float)(4.0 * u32);
    tp.paper_coef = is_tc(p->low) ? (float)(p->rho * p->paper_factor * gamma_m(d + 2, unit_roundoff(fmt))) : 0.0f;
    tp.bsafe = (float)(1.0 + std::ldexp(1.0, -10));
    tp.gamma32 = (float)(gamma_m(d + 2, u32) * 1.01 + std::ldexp(1.0, -22));
    return tp;
}

bool aligned256(const void* p) { return ((uintptr_t)p & 255) == 0; }

// The centres in the low format with their statistics (per-row power-of-two
// scales for E4M3), the column maxima of the bound, q_j and the scales padded
// to the tile width.
km_status prepare_centres(km_ctx* ctx, const float* C, int k, int d, int fmt, const AssignWs& w, cudaStream_t st) {
    KL(1, launch_quantize(C, k, d, fmt, ldq_of(fmt, d), w.Cq, w.cstat, w.cscale, st));
    KL(1, launch_colmax(w.cstat, k, fmt == 2 ? w.cscale : nullptr, w.colmax, w.qpad, w.spad, kpad_of(k), st));
    return KM_OK;
}

// One assignment of X against C into labels/min_dist (all device).
// x_absmax (nullable, zeroed by the caller): max |x| over X, folded out of the
// quantisation pass (tensor-core paths) or of the direct distances.
// The epilogue variant of the screening kernel for this shape: km_autotune's
// trial, else the tuned entry, else the default measured on GB300 (64-column
// steps; half staging, and with it a second A stage, when K is two atoms).
int screen_variant(km_ctx* ctx, int fmt, int kchunks, int k, int64_t n) {
    if (kchunks > 2) return TC_SV_REG;
    if (t_trial_variant >= 0) return t_trial_variant;
    {
        std::lock_guard<std::mutex> lk(ctx->tune->mu);
        auto it = ctx->tune->v.find(km_tune::key(fmt, kchunks, k, n, ctx->num_sms));
        if (it != ctx->tune->v.end()) return it->second;
    }
    return kchunks == 2 ? TC_SV_HALF : TC_SV_FULL;
}

// c_prepared: the workspace already holds C's low-precision copy, statistics
// and column maxima for this C and format (later row chunks of one call).
km_status run_assign(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d, const km_params* p,
                     int32_t* labels, double* min_dist, const AssignWs& w, bool x_prepared, cudaStream_t st,
                     unsigned* x_absmax = nullptr, bool c_prepared = false) {
    const TestParams tp = make_tp(p, d);
    km_status s = KM_OK;
    if (p->low == KM_FP64_DIRECT || p->low == KM_FP32_DIRECT) {
        const bool acc64 = p->low == KM_FP64_DIRECT;
        {
            PhaseScope ps(ctx, KM_PHASE_DIRECT, st);
            KL(1, launch_direct_assign(acc64, X, n, C, k, d, nullptr, nullptr, labels, min_dist, w.amb_list, w.cnt,
                                       tp.gamma32, ctx->num_sms, st, x_absmax));
        }
        if (!acc64) {
            PhaseScope ps(ctx, KM_PHASE_FULLROW, st);
            KL(1, launch_rows_full(false, X, C, k, d, w.amb_list, &w.cnt->amb_count, labels, min_dist, w.cnt,
                                   tp.gamma32, ctx->num_sms, st));
        }
        return KM_OK;
    }
    const int fmt = fmt_of(p->low);
    const int ldq = ldq_of(fmt, d);
    const int esz = fmt == 2 ? 1 : 2;
    {
        PhaseScope ps(ctx, KM_PHASE_QUANTISE, st);
        if (!x_prepared) KL(1, launch_quantize(X, n, d, fmt, ldq, w.Xq, w.xstat, w.xscale, st, x_absmax));
        if (!c_prepared && (s = prepare_centres(ctx, C, k, d, fmt, w, st)) != KM_OK) return s;
    }
    TcArgs a{};
    a.n = n; a.k = k; a.d = d; a.fmt = fmt;
    a.kchunks = (ldq * esz + 127) / 128;
    a.xstat = w.xstat; a.xscale = w.xscale; a.cstat = w.cstat; a.qpad = w.qpad; a.spad = w.spad; a.colmax = w.colmax;
    a.tp = tp; a.mode = 0; a.cand = w.cand; a.rowinfo = w.rowinfo; a.cnt = w.cnt;
    a.variant = screen_variant(ctx, fmt, a.kchunks, k, n);
    int qbits = 0;
    while ((1 << qbits) < (k + 3) / 4) qbits++;  // quad index bits (k <= 65535: at most 14)
    a.ebits = qbits + 4;
    a.pairs = w.pairs; a.pair_cap = w.pair_cap; a.v32 = w.v32; a.rowpair = w.rowpair;
    {
        PhaseScope ps(ctx, KM_PHASE_SCREEN, st);
        KL(1, launch_tc(w.Xq, w.Cq, ldq, a, ctx->num_sms, st));
    }
    {
        PhaseScope ps(ctx, KM_PHASE_REFINE, st);
        CK(cudaMemsetAsync(&w.cnt->npairs, 0, sizeof(unsigned long long), st));
        int nl = 0;
        CK(launch_refine(X, C, a, labels, min_dist, w.ovf_list, w.amb_list, ctx->num_sms, st, &nl));
        ctx->launches += (uint64_t)nl;
    }
    {
        // rows whose candidate list overflowed (all of them when every pair fails
        // the reliability test): fp32 direct distances to every centre with
        // Theorem 4.1's certificate, then binary64 for the rows left open.  The
        // near-tie list was consumed by the refinement and now takes those rows.
        PhaseScope ps(ctx, KM_PHASE_FULLROW, st);
        if (d <= 256) {  // the direct kernel's row tile fits in shared memory
            CK(cudaMemsetAsync(&w.cnt->amb_count, 0, sizeof(int), st));
            KL(1, launch_direct_assign(false, X, n, C, k, d, w.ovf_list, &w.cnt->ovf_count, labels, min_dist,
                                       w.amb_list, w.cnt, tp.gamma32, ctx->num_sms, st));
            KL(1, launch_rows_full(false, X, C, k, d, w.amb_list, &w.cnt->amb_count, labels, min_dist, w.cnt,
                                   tp.gamma32, ctx->num_sms, st));
        } else {  // one block per row
            KL(1, launch_rows_full(true, X, C, k, d, w.ovf_list, &w.cnt->ovf_count, labels, min_dist, w.cnt,
                                   tp.gamma32, ctx->num_sms, st));
        }
    }
    (void)esz;
    return KM_OK;
}

// min_dist of the winners to binary64 accuracy (the FP64 path has it already).
km_status refine_winners(km_ctx* ctx, const float* X, int64_t n, int d, const float* C, const km_params* p,
                         const int32_t* labels, double* md, cudaStream_t st) {
    if (p->low == KM_FP64_DIRECT) return KM_OK;
    PhaseScope ps(ctx, KM_PHASE_REFINE, st);
    KL(1, launch_winner_dist(X, n, d, C, labels, md, ctx->num_sms, st));
    return KM_OK;
}

// The centre update's accumulation; md_wd (nullable) also receives the rows'
// distances to their centres C_wd (the winner refinement, from the same pass
// over X where the kernel allows).
km_status accumulate(km_ctx* ctx, const float* X, int64_t n, int d, const int32_t* labels, int k, const UpdateWs& u,
                     const float* C_wd, double* md_wd, cudaStream_t st) {
    int nl = 0;
    CK(launch_accumulate(X, n, d, labels, k, u.absmax, u.sums, u.counts, u.iscratch, u.perm, ctx->num_sms, st, C_wd,
                         md_wd, &nl));
    ctx->launches += (uint64_t)nl;
    return KM_OK;
}

// Means, empty clusters and (want_shift) the shift of the centre update.
km_status finalize(km_ctx* ctx, const UpdateWs& u, int64_t n, int k, int d, const float* C_old, const km_params* p,
                   const float* X, const double* md, float* C_new, int64_t* counts, DevCounters* cnt, cudaStream_t st,
                   bool want_shift) {
    int nl = 0;
    CK(launch_finalize(u.sums, u.counts, u.absmax, n, k, d, C_old, p->empty, X, md, C_new, counts,
                       want_shift ? u.shift : nullptr, u.esel, &cnt->status, ctx->num_sms, st, &nl));
    ctx->launches += (uint64_t)nl;
    return KM_OK;
}

km_status sync_status(km_ctx* ctx, DevCounters* cnt, cudaStream_t st) {
    CK(cudaStreamSynchronize(st));
    unsigned status = 0;
    CK(cudaMemcpy(&status, &cnt->status, sizeof status, cudaMemcpyDeviceToHost));
    if (status & KM_DEVERR_TIMEOUT) return fail(ctx, KM_ETIMEOUT, "a device-side wait ran out of its budget");
    if (status) return fail(ctx, KM_ECUDA, "device status word 0x%x", status);
    return KM_OK;
}

km_status check_common(km_ctx* ctx, const void* X, int64_t n, const void* C, int k, int d) {
    if (!ctx) return KM_EINVAL;
    if (!X || !C) return fail(ctx, KM_EINVAL, "null input pointer");
    if (n < 1 || d < 1 || k < 1) return fail(ctx, KM_EINVAL, "need n, d, k >= 1 (n=%lld d=%d k=%d)", (long long)n, d, k);
    if ((int64_t)k > n) return fail(ctx, KM_EINVAL, "k=%d exceeds n=%lld", k, (long long)n);
    if (n > (int64_t)INT32_MAX) return fail(ctx, KM_EINVAL, "n too large");
    return KM_OK;
}

}  // namespace

extern "C" {

void km_default_params(km_params* p) {
    if (!p) return;
    p->low = KM_BF16;
    p->test = KM_TEST_TC;
    p->rho = 5.0;
    p->paper_factor = 2.0;
    p->max_iter = 20;
    p->empty = KM_EMPTY_FARTHEST;
    p->tau = 0.0;
    p->fallback = KM_FB_FP64;
}

km_status km_init(km_ctx** out, int device, void* arena, size_t arena_bytes) {
    if (!out) return KM_EINVAL;
    *out = nullptr;
    km_ctx* ctx = new km_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) { delete ctx; return KM_ECUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) == cudaSuccess && sms > 0) ctx->num_sms = sms;
    int major = 0, minor = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, device);
    if (major != 10) { delete ctx; return KM_EUNSUPPORTED; }
    if (arena && arena_bytes) {
        km_status s = serve_create(&ctx->serve, device, ctx->num_sms, ctx->tune, arena, arena_bytes);
        if (s != KM_OK) { delete ctx; return s; }
    }
    *out = ctx;
    return KM_OK;
}

km_status km_destroy(km_ctx* ctx) {
    if (!ctx) return KM_EINVAL;
    if (ctx->serve) serve_destroy(ctx->serve);
    delete ctx;
    return KM_OK;
}

const char* km_last_error(const km_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

km_status km_workspace_size(const km_ctx* cctx, int64_t n, int d, int k, const km_params* p, size_t* bytes) {
    km_ctx* ctx = const_cast<km_ctx*>(cctx);
    if (!ctx || !bytes || !p) return KM_EINVAL;
    if (n < 1 || d < 1 || k < 1) return fail(ctx, KM_EINVAL, "need n, d, k >= 1");
    Carve a{nullptr};
    carve_lloyd(a, n, d, k, p->low, std::max(0, (int)p->max_iter));
    Carve b{nullptr};
    carve_assign(b, n, d, k, p->low, true);
    *bytes = std::max(a.off, b.off) + 256;
    return KM_OK;
}

km_status km_quantize(km_ctx* ctx, const float* X, int64_t n, int d, int32_t low, void* Xq, float* stats,
                      float* scale, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!X || !Xq || !stats || !scale) return fail(ctx, KM_EINVAL, "null argument");
    if (n < 1 || d < 1) return fail(ctx, KM_EINVAL, "need n, d >= 1 (n=%lld d=%d)", (long long)n, d);
    if (n > (int64_t)INT32_MAX) return fail(ctx, KM_EINVAL, "n too large");
    if (!is_tc(low)) return fail(ctx, KM_EUNSUPPORTED, "km_quantize needs a low format (FP16/BF16/E4M3)");
    if (((uintptr_t)stats & 15) != 0) return fail(ctx, KM_EINVAL, "stats must be 16-byte aligned");
    const int fmt = fmt_of(low);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    KL(1, launch_quantize(X, n, d, fmt, ldq_of(fmt, d), Xq, reinterpret_cast<float4*>(stats), scale, st));
    return KM_OK;
}

km_status km_choose_low(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                        double max_overflow_share, int32_t* low_host, double* stats_host, void* ws, size_t ws_bytes,
                        void* stream) {
    km_status s = check_common(ctx, X, n, C, k, d);
    if (s != KM_OK) return s;
    if (!low_host || !ws) return fail(ctx, KM_EINVAL, "null output or workspace");
    if (!(max_overflow_share >= 0.0 && max_overflow_share <= 1.0))
        return fail(ctx, KM_EINVAL, "max_overflow_share must lie in [0, 1]");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    if (k > 65535 || tc_smem_bytes(1, d, 1) == 0)
        return fail(ctx, KM_EUNSUPPORTED, "no tensor-core path for d=%d, k=%d", d, k);
    constexpr int kSample = 2048;
    Carve cv{(char*)ws};
    unsigned long long* acc = cv.take<unsigned long long>(4);
    ColMax* colmax = cv.take<ColMax>(1);
    void* Cq = cv.take<char>((size_t)k * ldq_of(1, d) * 2);
    float4* cstat = cv.take<float4>((size_t)k);
    float* cscale = cv.take<float>((size_t)k);
    float* qpad = cv.take<float>((size_t)kpad_of(k));
    float* spad = cv.take<float>((size_t)kpad_of(k));
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(acc, 0, 4 * sizeof(unsigned long long), st));
    const int fmts[2] = {1, 2};  // bf16, E4M3
    for (int f = 0; f < 2; f++) {
        const int fmt = fmts[f];
        if (fmt == 2 && d < 16) continue;
        km_params q;
        km_default_params(&q);
        q.low = fmt == 2 ? KM_E4M3 : KM_BF16;
        KL(1, launch_quantize(C, k, d, fmt, ldq_of(fmt, d), Cq, cstat, cscale, st));
        KL(1, launch_colmax(cstat, k, fmt == 2 ? cscale : nullptr, colmax, qpad, spad, kpad_of(k), st));
        KL(1, launch_predict_candidates(X, n, d, C, k, fmt, colmax, make_tp(&q, d), kSample, acc + 2 * f,
                                        ctx->num_sms, st));
    }
    unsigned long long h[4];
    CK(cudaMemcpyAsync(h, acc, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const double ns = (double)std::min<int64_t>(kSample, n);
    double stats[4] = {h[0] / ns, h[1] / ns, INFINITY, 1.0};
    if (d >= 16) {
        stats[2] = h[2] / ns;
        stats[3] = h[3] / ns;
    }
    *low_host = (d >= 16 && stats[3] <= max_overflow_share && stats[2] <= stats[0] + 2.0) ? KM_E4M3 : KM_BF16;
    if (stats_host)
        for (int i = 0; i < 4; i++) stats_host[i] = stats[i];
    return KM_OK;
}

km_status km_assign(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d, const km_params* p,
                    int32_t* labels, double* min_dist, uint64_t* n_flagged_host, void* ws, size_t ws_bytes,
                    void* stream) {
    km_status s = check_common(ctx, X, n, C, k, d);
    if (s != KM_OK) return s;
    if ((s = check_params(ctx, p, d, k)) != KM_OK) return s;
    if (!labels || !ws) return fail(ctx, KM_EINVAL, "null output or workspace");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    AssignWs w = carve_assign(cv, n, d, k, p->low, false);
    double* md = min_dist;
    Carve tmp{nullptr};
    carve_assign(tmp, n, d, k, p->low, false);
    size_t need = tmp.off;
    if (!md) {  // scratch min_dist when the caller does not want it
        Carve c2{(char*)ws};
        c2.off = tmp.off;
        md = c2.take<double>((size_t)n);
        need = c2.off;
    }
    if (ws_bytes < need) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, need);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(w.cnt, 0, sizeof(DevCounters), st));
    s = run_assign(ctx, X, n, C, k, d, p, labels, md, w, false, st);
    if (s != KM_OK) return s;
    if ((s = refine_winners(ctx, X, n, d, C, p, labels, md, st)) != KM_OK) return s;
    KL(2, launch_sum_f64(md, n, w.partials, kSumParts, w.sse, st));
    ctx->last_cnt = w.cnt;
    ctx->last_sse = w.sse;
    ctx->last_stream = st;
    ctx->last_pairs = (uint64_t)n * (uint64_t)k;
    if (n_flagged_host) {
        if ((s = sync_status(ctx, w.cnt, st)) != KM_OK) return s;
        unsigned long long f = 0;
        CK(cudaMemcpy(&f, &w.cnt->flagged, sizeof f, cudaMemcpyDeviceToHost));
        *n_flagged_host = f;
    }
    return KM_OK;
}

namespace {
struct TrialVariant {  // km_autotune's trial variant, cleared on every exit
    explicit TrialVariant(int v) { t_trial_variant = v; }
    ~TrialVariant() { t_trial_variant = -1; }
};
}  // namespace

km_status km_autotune(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d, const km_params* p,
                      int32_t* labels, int32_t* variant_host, float* ms_host, void* ws, size_t ws_bytes,
                      void* stream) {
    km_status s = check_common(ctx, X, n, C, k, d);
    if (s != KM_OK) return s;
    if ((s = check_params(ctx, p, d, k)) != KM_OK) return s;
    if (!labels || !variant_host) return fail(ctx, KM_EINVAL, "null argument");
    if (ms_host)
        for (int i = 0; i < 3; i++) ms_host[i] = -1.0f;
    if (!is_tc(p->low)) {  // no screening kernel on the direct paths
        *variant_host = -1;
        return KM_OK;
    }
    const int fmt = fmt_of(p->low);
    const int kchunks = (ldq_of(fmt, d) * (fmt == 2 ? 1 : 2) + 127) / 128;
    if (kchunks > 2) {  // one variant only
        *variant_host = TC_SV_REG;
        return KM_OK;
    }
    const int64_t ns = std::min<int64_t>(n, (int64_t)1 << 20);  // rows timed (n >= k, so ns >= k)
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    cudaEvent_t ev[2];
    CK(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return fail(ctx, KM_ECUDA, "cudaEventCreate failed");
    }
    float best = INFINITY;
    int bv = TC_SV_FULL;
    for (int v = TC_SV_FULL; v <= TC_SV_C32 && s == KM_OK; v++) {
        TrialVariant tv(v);
        s = km_assign(ctx, X, ns, C, k, d, p, labels, nullptr, nullptr, ws, ws_bytes, stream);  // warm-up
        if (s != KM_OK) break;
        cudaEventRecord(ev[0], st);
        for (int r = 0; r < 3 && s == KM_OK; r++)
            s = km_assign(ctx, X, ns, C, k, d, p, labels, nullptr, nullptr, ws, ws_bytes, stream);
        cudaEventRecord(ev[1], st);
        float ms = 0.0f;
        if (cudaEventSynchronize(ev[1]) != cudaSuccess || cudaEventElapsedTime(&ms, ev[0], ev[1]) != cudaSuccess) {
            if (s == KM_OK) s = fail(ctx, KM_ECUDA, "autotune timing failed");
            break;
        }
        ms /= 3.0f;
        if (ms_host) ms_host[v] = ms;
        if (ms < best) { best = ms; bv = v; }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (s != KM_OK) return s;
    if ((s = sync_status(ctx, ctx->last_cnt, st)) != KM_OK) return s;
    {
        std::lock_guard<std::mutex> lk(ctx->tune->mu);
        ctx->tune->v[km_tune::key(fmt, kchunks, k, n, ctx->num_sms)] = bv;
    }
    *variant_host = bv;
    return KM_OK;
}

km_status km_set_screen_variant(km_ctx* ctx, int64_t n, int d, int k, int32_t low, int32_t variant) {
    if (!ctx) return KM_EINVAL;
    if (n < 1 || d < 1 || k < 1) return fail(ctx, KM_EINVAL, "need n, d, k >= 1");
    if (!is_tc(low)) return fail(ctx, KM_EUNSUPPORTED, "no screening kernel for this format");
    if (variant < -1 || variant > TC_SV_C32) return fail(ctx, KM_EINVAL, "variant %d out of range", variant);
    const int fmt = fmt_of(low);
    const int kchunks = (ldq_of(fmt, d) * (fmt == 2 ? 1 : 2) + 127) / 128;
    if (kchunks > 2) return variant == -1 ? KM_OK : fail(ctx, KM_EUNSUPPORTED, "d=%d: one variant only", d);
    std::lock_guard<std::mutex> lk(ctx->tune->mu);
    const uint64_t key = km_tune::key(fmt, kchunks, k, n, ctx->num_sms);
    if (variant == -1) ctx->tune->v.erase(key);
    else ctx->tune->v[key] = variant;
    return KM_OK;
}

km_status km_distances(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d, const km_params* p,
                       float* D, uint32_t* flag_bits, uint64_t* n_flagged_host, void* ws, size_t ws_bytes,
                       void* stream) {
    km_status s = check_common(ctx, X, n, C, k, d);
    if (s != KM_OK) return s;
    if ((s = check_params(ctx, p, d, k, true)) != KM_OK) return s;
    if (!D || !ws) return fail(ctx, KM_EINVAL, "null output or workspace");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    AssignWs w = carve_assign(cv, n, d, k, p->low, true);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(w.cnt, 0, sizeof(DevCounters), st));
    CK(cudaMemsetAsync(w.qlen, 0, sizeof(unsigned long long), st));
    if (flag_bits) CK(cudaMemsetAsync(flag_bits, 0, ((size_t)n * k + 31) / 32 * 4, st));
    if (!is_tc(p->low)) {
        if (p->low == KM_FP32) {
            // Alg. 2 with u_l = 2^-24: E = fl(rho c_A gamma_{d+2}(u_l)) fl(d_xx + d_yy)
            const double u32 = std::ldexp(1.0, -24);
            const float coef = (float)(p->rho * p->paper_factor * gamma_m(d + 2, u32));
            const float kacc = (float)((2.0 * gamma_m(d, u32) + 4.0 * u32) * (1.0 + 1e-6));
            const float kn = (float)(4.0 * u32);
            KL(1, launch_rowdot_fp32(X, n, d, w.dxx, ctx->num_sms, st));
            KL(1, launch_rowdot_fp32(C, k, d, w.dyy, ctx->num_sms, st));
            KL(1, launch_matrix(0, X, n, C, k, d, w.dxx, w.dyy, p->test, (float)p->rho, coef, kacc, kn, D, flag_bits,
                                w.queue, w.qcap, w.qlen, w.cnt, ctx->num_sms, st));
            // the same-precision fallback of binary32 is the binary32 direct formula
            const int fb = p->fallback == KM_FB_FP64 ? 0 : 1;
            KL(1, launch_patch_flagged(fb, 0, X, C, n, k, d, w.queue, w.qlen, w.qcap, D, w.cnt, ctx->num_sms, st));
        } else {
            KL(1, launch_matrix(p->low == KM_FP64_DIRECT ? 1 : 2, X, n, C, k, d, nullptr, nullptr, KM_TEST_OFF, 0.f,
                                0.f, 0.f, 0.f, D, nullptr, w.queue, w.qcap, w.qlen, w.cnt, ctx->num_sms, st));
        }
    } else {
        const int fmt = fmt_of(p->low);
        const int ldq = ldq_of(fmt, d);
        const int esz = fmt == 2 ? 1 : 2;
        KL(1, launch_quantize(X, n, d, fmt, ldq, w.Xq, w.xstat, w.xscale, st));
        if ((s = prepare_centres(ctx, C, k, d, fmt, w, st)) != KM_OK) return s;
        TcArgs a{};
        a.n = n; a.k = k; a.d = d; a.fmt = fmt;
        a.kchunks = (ldq * esz + 127) / 128;
        a.xstat = w.xstat; a.xscale = w.xscale; a.cstat = w.cstat; a.qpad = w.qpad; a.spad = w.spad; a.colmax = w.colmax;
        a.tp = make_tp(p, d); a.mode = 1; a.rowinfo = w.rowinfo; a.cnt = w.cnt;
        a.D = D; a.flag_bits = flag_bits; a.flag_queue = w.queue; a.flag_queue_cap = w.qcap;
        a.flag_queue_len = w.qlen;
        KL(1, launch_tc(w.Xq, w.Cq, ldq, a, ctx->num_sms, st));
        const int fb = p->fallback == KM_FB_FP64 ? 0 : (p->fallback == KM_FB_FP32 ? 1 : 2);
        KL(1, launch_patch_flagged(fb, fmt, X, C, n, k, d, w.queue, w.qlen, w.qcap, D, w.cnt, ctx->num_sms, st));
    }
    ctx->last_cnt = w.cnt;
    ctx->last_sse = nullptr;
    ctx->last_stream = st;
    ctx->last_pairs = (uint64_t)n * (uint64_t)k;
    if (n_flagged_host) {
        if ((s = sync_status(ctx, w.cnt, st)) != KM_OK) return s;
        unsigned long long f = 0;
        CK(cudaMemcpy(&f, &w.cnt->flagged, sizeof f, cudaMemcpyDeviceToHost));
        *n_flagged_host = f;
    }
    return KM_OK;
}

km_status km_update_centroids(km_ctx* ctx, const float* X, int64_t n, int d, const int32_t* labels, int k,
                              const float* C_old, const km_params* p, const double* min_dist, float* C_new,
                              int64_t* counts, double* shift_host, void* ws, size_t ws_bytes, void* stream) {
    km_status s = check_common(ctx, X, n, C_old, k, d);
    if (s != KM_OK) return s;
    if (!p || !labels || !C_new || !ws) return fail(ctx, KM_EINVAL, "null argument");
    if (p->empty != KM_EMPTY_KEEP && p->empty != KM_EMPTY_FARTHEST) return fail(ctx, KM_EINVAL, "unknown empty policy");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    // the update's scratch lies past an assignment's, so the counters of the
    // last assignment on the same workspace stay readable (km_get_stats)
    Carve cv{(char*)ws};
    carve_assign(cv, n, d, k, p->low, false);
    DevCounters* cnt = cv.take<DevCounters>(1);
    UpdateWs u = carve_update(cv, n, d, k);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), st));
    {
        PhaseScope ps(ctx, KM_PHASE_UPDATE, st);
        KL(1, launch_absmax(X, n * (int64_t)d, u.absmax, st));
        if ((s = accumulate(ctx, X, n, d, labels, k, u, nullptr, nullptr, st)) != KM_OK) return s;
        if ((s = finalize(ctx, u, n, k, d, C_old, p, X, min_dist, C_new, counts, cnt, st, shift_host != nullptr)) != KM_OK)
            return s;
    }
    if (shift_host) {
        if ((s = sync_status(ctx, cnt, st)) != KM_OK) return s;
        CK(cudaMemcpy(shift_host, u.shift, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return KM_OK;
}

// ---- row-sharded centre updates (one exchange per Lloyd iteration) ----------
km_status km_absmax(km_ctx* ctx, const float* X, int64_t count, uint32_t* bits_host, void* ws, size_t ws_bytes,
                    void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!X || !bits_host || !ws) return fail(ctx, KM_EINVAL, "null argument");
    if (count < 1) return fail(ctx, KM_EINVAL, "count must be >= 1");
    if (!aligned256(ws) || ws_bytes < 256) return fail(ctx, KM_EINVAL, "workspace: 256 bytes, 256-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    unsigned* slot = reinterpret_cast<unsigned*>(ws);
    KL(1, launch_absmax(X, count, slot, st));
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, slot, sizeof h, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *bits_host = h;
    return KM_OK;
}

km_status km_update_partial(km_ctx* ctx, const float* X, int64_t n, int d, const int32_t* labels, int k,
                            uint32_t absmax_bits, int64_t n_total, int64_t* sums, int64_t* counts, void* ws,
                            size_t ws_bytes, void* stream) {
    km_status s = check_common(ctx, X, n, labels, 1, d);
    if (s != KM_OK) return s;
    if (k < 1 || !sums || !counts || !ws) return fail(ctx, KM_EINVAL, "null output or workspace, or k < 1");
    if (n_total < n) return fail(ctx, KM_EINVAL, "n_total=%lld is below this shard's n=%lld", (long long)n_total, (long long)n);
    if (!(__builtin_isfinite(__builtin_bit_cast(float, absmax_bits))) || (absmax_bits >> 31))
        return fail(ctx, KM_EINVAL, "absmax_bits is not a finite non-negative float");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    DevCounters* cnt = cv.take<DevCounters>(1);
    UpdateWs u = carve_update(cv, n, d, k);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    (void)cnt;
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpyAsync(u.absmax, &absmax_bits, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    int nl = 0;
    CK(launch_accumulate(X, n, d, labels, k, u.absmax, reinterpret_cast<long long*>(sums),
                         reinterpret_cast<long long*>(counts), u.iscratch, u.perm, ctx->num_sms, st, nullptr, nullptr,
                         &nl, n_total));
    ctx->launches += (uint64_t)nl;
    return KM_OK;
}

km_status km_update_finalize(km_ctx* ctx, const int64_t* sums, const int64_t* counts, int k, int d,
                             uint32_t absmax_bits, int64_t n_total, const float* C_old, float* C_new,
                             double* shift_host, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!sums || !counts || !C_old || !C_new || !ws) return fail(ctx, KM_EINVAL, "null argument");
    if (k < 1 || d < 1 || n_total < 1) return fail(ctx, KM_EINVAL, "need k, d, n_total >= 1");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    DevCounters* cnt = cv.take<DevCounters>(1);
    UpdateWs u = carve_update(cv, 1, d, k);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), st));
    CK(cudaMemcpyAsync(u.absmax, &absmax_bits, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    int nl = 0;
    CK(launch_finalize(reinterpret_cast<const long long*>(sums), reinterpret_cast<const long long*>(counts), u.absmax,
                       n_total, k, d, C_old, KM_EMPTY_KEEP, nullptr, nullptr, C_new, nullptr, u.shift, u.esel,
                       &cnt->status, ctx->num_sms, st, &nl, n_total));
    ctx->launches += (uint64_t)nl;
    if (shift_host) {
        km_status s = sync_status(ctx, cnt, st);
        if (s != KM_OK) return s;
        CK(cudaMemcpy(shift_host, u.shift, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return KM_OK;
}

km_status km_farthest_rows(km_ctx* ctx, const double* min_dist, int64_t n, int e, int64_t* rows, double* vals,
                           void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!min_dist || !rows || !vals || !ws) return fail(ctx, KM_EINVAL, "null argument");
    if (n < 1 || e < 1 || (int64_t)e > n) return fail(ctx, KM_EINVAL, "need 1 <= e <= n (e=%d n=%lld)", e, (long long)n);
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    DevCounters* cnt = cv.take<DevCounters>(1);
    void* esel = cv.take<unsigned char>(empty_select_bytes(e));
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), st));
    KL(1, launch_farthest_rows(min_dist, n, e, reinterpret_cast<long long*>(rows), vals, esel, &cnt->status,
                               ctx->num_sms, st));
    return sync_status(ctx, cnt, st);
}

km_status km_lloyd_step(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_old,
                        const km_params* p, int32_t* labels, double* min_dist, float* C_new, int64_t* counts,
                        double* shift_host, void* ws, size_t ws_bytes, void* stream) {
    km_status s = check_common(ctx, X, n, C_old, k, d);
    if (s != KM_OK) return s;
    if ((s = check_params(ctx, p, d, k)) != KM_OK) return s;
    if (!labels || !C_new || !ws) return fail(ctx, KM_EINVAL, "null output or workspace");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    AssignWs w = carve_assign(cv, n, d, k, p->low, false);
    UpdateWs u = carve_update(cv, n, d, k);
    double* md = min_dist ? min_dist : cv.take<double>((size_t)n);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(w.cnt, 0, sizeof(DevCounters), st));
    // assignment (Alg. 3 step 1); its pass over X (quantisation, or the direct
    // distances) also yields max |x|
    CK(cudaMemsetAsync(u.absmax, 0, sizeof(unsigned), st));
    s = run_assign(ctx, X, n, C_old, k, d, p, labels, md, w, false, st, u.absmax);
    if (s != KM_OK) return s;
    // centre update (Eq. (center)) on the labels just computed; its pass over
    // X also refines the winners' distances (min_dist, binary64 accuracy)
    {
        PhaseScope ps(ctx, KM_PHASE_UPDATE, st);
        s = accumulate(ctx, X, n, d, labels, k, u, C_old, p->low == KM_FP64_DIRECT ? nullptr : md, st);
        if (s != KM_OK) return s;
        KL(2, launch_sum_f64(md, n, w.partials, kSumParts, w.sse, st));
        if ((s = finalize(ctx, u, n, k, d, C_old, p, X, md, C_new, counts, w.cnt, st, shift_host != nullptr)) != KM_OK)
            return s;
    }
    ctx->last_cnt = w.cnt;
    ctx->last_sse = w.sse;
    ctx->last_stream = st;
    ctx->last_pairs = (uint64_t)n * (uint64_t)k;
    if (shift_host) {
        if ((s = sync_status(ctx, w.cnt, st)) != KM_OK) return s;
        CK(cudaMemcpy(shift_host, u.shift, sizeof(double), cudaMemcpyDeviceToHost));
    }
    return KM_OK;
}

km_status km_host_workspace_size(const km_ctx* cctx, int64_t n, int d, int k, const km_params* p, size_t* bytes) {
    km_ctx* ctx = const_cast<km_ctx*>(cctx);
    if (!ctx || !bytes || !p) return KM_EINVAL;
    if (n < 1 || d < 1 || k < 1) return fail(ctx, KM_EINVAL, "need n, d, k >= 1");
    Carve a{nullptr};
    carve_host(a, n, d, k);
    carve_assign(a, n, d, k, p->low, false);
    carve_update(a, n, d, k);
    *bytes = a.off + 256;
    return KM_OK;
}

km_status km_lloyd_step_host(km_ctx* ctx, const float* X_host, int64_t n, int d, int k, const float* C_host,
                             const km_params* p, int32_t* labels_host, double* min_dist_host, float* C_new_host,
                             int64_t* counts_host, double* shift_host, void* ws, size_t ws_bytes, void* stream) {
    km_status s = check_common(ctx, X_host, n, C_host, k, d);
    if (s != KM_OK) return s;
    if (!p || !labels_host || !C_new_host || !ws) return fail(ctx, KM_EINVAL, "null params, output or workspace");
    s = check_params(ctx, p, d, k);
    if (s != KM_OK) return s;
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    HostWs h = carve_host(cv, n, d, k);
    AssignWs w = carve_assign(cv, n, d, k, p->low, false);
    UpdateWs u = carve_update(cv, n, d, k);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    // rows in up to kHostChunks chunks of whole 128-row blocks; each chunk is
    // assigned as soon as it has arrived, while the next one is being copied.
    // Each chunk holds about half the rows of the one before (8:4:2:1): a
    // chunk's assignment takes about a third of the time the host link needs
    // for the same rows, so the link stays busy, and the last chunk, whose
    // assignment and the centre update run after the last copy, is small.
    constexpr int kHostChunks = 4;
    constexpr int kChunkWeight[kHostChunks] = {8, 4, 2, 1};
    int64_t cend[kHostChunks];  // end row of each chunk
    int nch = 0;
    {
        const int64_t nblk = (n + 127) / 128;
        int wsum = 0, wall = 0;
        for (int c = 0; c < kHostChunks; c++) wall += kChunkWeight[c];
        int64_t prev = 0;
        for (int c = 0; c < kHostChunks; c++) {
            wsum += kChunkWeight[c];
            const int64_t eb = (nblk * wsum + wall - 1) / wall;  // end block, rounded up
            const int64_t er = std::min<int64_t>(eb * 128, n);
            if (er > prev) cend[nch++] = er;
            prev = er;
        }
    }
    auto chunk_r0 = [&](int c) -> int64_t { return c == 0 ? 0 : cend[c - 1]; };
    for (int i = 0; i < 2; i++)
        if (!ctx->copy_st[i]) CK(cudaStreamCreateWithFlags(&ctx->copy_st[i], cudaStreamNonBlocking));
    while ((int)ctx->host_ev.size() < 3 * kHostChunks + 1) {
        cudaEvent_t e;
        CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->host_ev.push_back(e);
    }
    // everything from the first copy on: any error exit drains the copy
    // streams first, so no copy still reads the caller's buffers after the return
    auto enqueue = [&]() -> km_status {
        km_status s = KM_OK;
        cudaEvent_t ev_start = ctx->host_ev[0];
        cudaEvent_t* ev_in = ctx->host_ev.data() + 1;
        cudaEvent_t* ev_out = ev_in + kHostChunks;
        cudaEvent_t* ev_back = ev_out + kHostChunks;
        // the copies into the workspace wait for earlier work on the stream
        CK(cudaEventRecord(ev_start, st));
        CK(cudaMemcpyAsync(h.C, C_host, sizeof(float) * (size_t)k * d, cudaMemcpyHostToDevice, st));
        // host -> device on copy stream 0 in chunk order (each chunk at the
        // link's full rate), device -> host on copy stream 1
        CK(cudaStreamWaitEvent(ctx->copy_st[0], ev_start, 0));
        CK(cudaStreamWaitEvent(ctx->copy_st[1], ev_start, 0));
        for (int c = 0; c < nch; c++) {
            const int64_t r0 = chunk_r0(c), rows = cend[c] - r0;
            cudaStream_t cs = ctx->copy_st[0];
            CK(cudaMemcpyAsync(h.X + r0 * d, X_host + r0 * d, sizeof(float) * (size_t)rows * d, cudaMemcpyHostToDevice, cs));
            CK(cudaEventRecord(ev_in[c], cs));
        }
        CK(cudaMemsetAsync(w.cnt, 0, sizeof(DevCounters), st));
        CK(cudaMemsetAsync(u.absmax, 0, sizeof(unsigned), st));
        for (int c = 0; c < nch; c++) {
            const int64_t r0 = chunk_r0(c), rows = cend[c] - r0;
            cudaStream_t cs = ctx->copy_st[1];
            CK(cudaStreamWaitEvent(st, ev_in[c], 0));
            CK(cudaMemsetAsync(&w.cnt->amb_count, 0, 2 * sizeof(int), st));
            // the centres are prepared once, with the first chunk
            s = run_assign(ctx, h.X + r0 * d, rows, h.C, k, d, p, h.labels + r0, h.min_dist + r0, w, false, st, u.absmax,
                           c > 0);
            if (s != KM_OK) return s;
            // the chunk's winner distances (binary64 accuracy) while the next
            // chunk is still on its way: the update's pass then only sums
            if ((s = refine_winners(ctx, h.X + r0 * d, rows, d, h.C, p, h.labels + r0, h.min_dist + r0, st)) != KM_OK)
                return s;
            // this chunk's labels and distances go back while the next chunk is assigned
            CK(cudaEventRecord(ev_out[c], st));
            CK(cudaStreamWaitEvent(cs, ev_out[c], 0));
            CK(cudaMemcpyAsync(labels_host + r0, h.labels + r0, sizeof(int32_t) * (size_t)rows, cudaMemcpyDeviceToHost, cs));
            if (min_dist_host)
                CK(cudaMemcpyAsync(min_dist_host + r0, h.min_dist + r0, sizeof(double) * (size_t)rows,
                                   cudaMemcpyDeviceToHost, cs));
            CK(cudaEventRecord(ev_back[c], cs));
        }
        {
            PhaseScope ps(ctx, KM_PHASE_UPDATE, st);
            s = accumulate(ctx, h.X, n, d, h.labels, k, u, h.C, nullptr, st);
            if (s != KM_OK) return s;
            KL(2, launch_sum_f64(h.min_dist, n, w.partials, kSumParts, w.sse, st));
            if ((s = finalize(ctx, u, n, k, d, h.C, p, h.X, h.min_dist, h.C_new, h.counts, w.cnt, st,
                              shift_host != nullptr)) != KM_OK)
                return s;
        }
        CK(cudaMemcpyAsync(C_new_host, h.C_new, sizeof(float) * (size_t)k * d, cudaMemcpyDeviceToHost, st));
        if (counts_host) CK(cudaMemcpyAsync(counts_host, h.counts, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, st));
        for (int c = 0; c < nch; c++) CK(cudaStreamWaitEvent(st, ev_back[c], 0));
        return KM_OK;
    };
    s = enqueue();
    if (s != KM_OK) {
        for (cudaStream_t c2 : ctx->copy_st) cudaStreamSynchronize(c2);
        cudaStreamSynchronize(st);  // and no copy back into them either
        return s;
    }
    ctx->last_cnt = w.cnt;
    ctx->last_sse = w.sse;
    ctx->last_stream = st;
    ctx->last_pairs = (uint64_t)n * (uint64_t)k;
    if ((s = sync_status(ctx, w.cnt, st)) != KM_OK) return s;
    if (shift_host) CK(cudaMemcpy(shift_host, u.shift, sizeof(double), cudaMemcpyDeviceToHost));
    return KM_OK;
}

static km_status lloyd_impl(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_init,
                            const km_params* p, float* C_out, int32_t* labels, double* sse_per_iter,
                            double* eta_per_iter, int* iters_done, void* ws, size_t ws_bytes, void* stream,
                            const volatile int* cancel, bool allow_graphs);

km_status km_lloyd_run_batch(km_ctx* ctx, const km_batch_job* jobs, int njobs, const km_params* p, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!jobs || !p || njobs < 0) return fail(ctx, KM_EINVAL, "null argument");
    if (p->low != KM_FP32_DIRECT) return fail(ctx, KM_EUNSUPPORTED, "batched runs take low = KM_FP32_DIRECT");
    if (p->max_iter < 0) return fail(ctx, KM_EINVAL, "max_iter must be >= 0");
    km_status s;
    for (int q = 0; q < njobs; q++) {
        const km_batch_job& b = jobs[q];
        if (!b.X || !b.C_init || !b.C_out || !b.labels || !b.sse_per_iter || !b.iters || !b.scratch)
            return fail(ctx, KM_EINVAL, "job %d: null pointer", q);
        if (b.d < 1 || b.d > GROUP_MAX_D || b.k < 1 || b.k > GROUP_MAX_K || b.n < b.k || b.n > GROUP_MAX_N)
            return fail(ctx, KM_EUNSUPPORTED, "job %d: batched runs take d <= 8, 1 <= k <= 64, k <= n <= 16384", q);
        if ((s = check_params(ctx, p, b.d, b.k)) != KM_OK) return s;
    }
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    for (int d = 1; d <= GROUP_MAX_D; d++) {
        GroupArgs a{};
        a.max_iter = p->max_iter;
        a.empty_farthest = p->empty == KM_EMPTY_FARTHEST ? 1 : 0;
        a.tau = p->tau;
        a.gamma32 = make_tp(p, d).gamma32;
        int m = 0;
        for (int q = 0; q <= njobs; q++) {
            if (q < njobs && jobs[q].d == d) {
                const km_batch_job& b = jobs[q];
                a.job[m++] = GroupJob{b.X, b.C_init, b.C_out, b.labels, b.scratch, b.sse_per_iter, b.iters,
                                      (int)b.n, b.k};
            }
            if (m == GROUP_MAX || (q == njobs && m > 0)) {
                KL(1, launch_group_lloyd(a, m, d, st));
                m = 0;
            }
        }
    }
    return KM_OK;
}

km_status km_lloyd_run(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_init,
                       const km_params* p, float* C_out, int32_t* labels, double* sse_per_iter,
                       double* eta_per_iter, int* iters_done, void* ws, size_t ws_bytes, void* stream) {
    return lloyd_impl(ctx, X, n, d, k, C_init, p, C_out, labels, sse_per_iter, eta_per_iter, iters_done, ws,
                      ws_bytes, stream, nullptr, true);
}

}  // extern "C"

// Appends a replayed iteration's SSE and the flag count so far to the
// histories (one thread).
__global__ void k_record_iteration(const double* __restrict__ sse_slot, const DevCounters* __restrict__ cnt,
                                   double* __restrict__ sse_hist, unsigned long long* __restrict__ flag_hist,
                                   int* hist_len, int cap) {
    const int i = *hist_len;
    if (i < cap) {
        sse_hist[i] = *sse_slot;
        flag_hist[i] = cnt->flagged;
    }
    *hist_len = i + 1;
}

// One iteration of Alg. 3's loop from cur to nxt.  sse_out: the SSE's
// destination; graph: the iteration is being recorded for replay (its SSE and
// flag count go to the slot and are appended by k_record_iteration).
static km_status lloyd_iteration(km_ctx* ctx, const float* X, int64_t n, int d, int k, const km_params* p,
                                 int32_t* labels, const LloydWs& L, const float* cur, float* nxt, double* sse_out,
                                 unsigned long long* flag_out, bool graph, int cap, cudaStream_t st) {
    CK(cudaMemsetAsync(&L.a.cnt->amb_count, 0, 2 * sizeof(int), st));
    km_status s = run_assign(ctx, X, n, cur, k, d, p, labels, L.min_dist, L.a, true, st);
    if (s != KM_OK) return s;
    if (!graph) CK(cudaMemcpyAsync(flag_out, &L.a.cnt->flagged, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    PhaseScope ps(ctx, KM_PHASE_UPDATE, st);
    s = accumulate(ctx, X, n, d, labels, k, L.u, cur, p->low == KM_FP64_DIRECT ? nullptr : L.min_dist, st);
    if (s != KM_OK) return s;
    KL(2, launch_sum_f64(L.min_dist, n, L.a.partials, kSumParts, graph ? L.sse_slot : sse_out, st));
    if ((s = finalize(ctx, L.u, n, k, d, cur, p, X, L.min_dist, nxt, L.counts, L.a.cnt, st, true)) != KM_OK) return s;
    if (graph) {
        k_record_iteration<<<1, 1, 0, st>>>(L.sse_slot, L.a.cnt, L.sse_hist, L.flag_hist, L.hist_len, cap);
        ctx->launches++;
        CK(cudaGetLastError());
    }
    return KM_OK;
}

// Records the two iterations C0 -> C1 and C1 -> C0 as CUDA graphs on gs
// (every pointer the same whatever the iteration); false when the stream
// cannot be captured (the caller then launches the iterations directly).
static bool capture_iterations(km_ctx* ctx, const float* X, int64_t n, int d, int k, const km_params* p,
                               int32_t* labels, const LloydWs& L, int cap, cudaStream_t gs, cudaGraphExec_t (&ge)[2],
                               uint64_t (&nk)[2]) {
    ge[0] = ge[1] = nullptr;
    for (int par = 0; par < 2; par++) {
        if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) break;
        const uint64_t l0 = ctx->launches;
        const std::string err0 = ctx->err;
        km_status s = lloyd_iteration(ctx, X, n, d, k, p, labels, L, par ? L.C1 : L.C0, par ? L.C0 : L.C1, nullptr,
                                      nullptr, true, cap, gs);
        nk[par] = ctx->launches - l0;
        ctx->launches = l0;
        cudaGraph_t g = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(gs, &g);
        if (s != KM_OK || ec != cudaSuccess || !g || cudaGraphInstantiate(&ge[par], g, 0) != cudaSuccess) {
            ctx->err = err0;
            if (g) cudaGraphDestroy(g);
            break;
        }
        cudaGraphDestroy(g);
    }
    if (ge[0] && ge[1]) return true;
    for (cudaGraphExec_t& e : ge)
        if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    cudaGetLastError();  // a refused capture leaves nothing behind
    return false;
}

static km_status lloyd_impl(km_ctx* ctx, const float* X, int64_t n, int d, int k, const float* C_init,
                            const km_params* p, float* C_out, int32_t* labels, double* sse_per_iter,
                            double* eta_per_iter, int* iters_done, void* ws, size_t ws_bytes, void* stream,
                            const volatile int* cancel, bool allow_graphs) {
    km_status s = check_common(ctx, X, n, C_init, k, d);
    if (s != KM_OK) return s;
    if ((s = check_params(ctx, p, d, k)) != KM_OK) return s;
    if (!C_out || !labels || !ws) return fail(ctx, KM_EINVAL, "null output or workspace");
    if (p->max_iter < 0) return fail(ctx, KM_EINVAL, "max_iter must be >= 0");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    LloydWs L = carve_lloyd(cv, n, d, k, p->low, p->max_iter);
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemsetAsync(L.a.cnt, 0, sizeof(DevCounters), st));
    CK(cudaMemsetAsync(L.hist_len, 0, sizeof(int), st));
    CK(cudaMemcpyAsync(L.C0, C_init, sizeof(float) * (size_t)k * d, cudaMemcpyDeviceToDevice, st));
    // the quantised data and its norms are computed once (Section 3.2), and with
    // them the largest |x| that fixes the scale of the exact centre sums
    if (is_tc(p->low)) {
        const int fmt = fmt_of(p->low);
        PhaseScope ps(ctx, KM_PHASE_QUANTISE, st);
        CK(cudaMemsetAsync(L.u.absmax, 0, sizeof(unsigned), st));
        KL(1, launch_quantize(X, n, d, fmt, ldq_of(fmt, d), L.a.Xq, L.a.xstat, L.a.xscale, st, L.u.absmax));
    } else {
        KL(1, launch_absmax(X, n * (int64_t)d, L.u.absmax, st));
    }
    float* cur = L.C0;
    float* nxt = L.C1;
    int t = 0;
    // Iterations as replays of two recorded graphs (C0 -> C1, C1 -> C0): one
    // launch per iteration instead of one per kernel.  Phase timing needs the
    // direct launches (its events sit between the kernels).  Recording happens
    // here, in the caller's thread; the serving workers, which run beside the
    // caller's own work, launch directly (a device-wide synchronisation
    // elsewhere in the process fails while any stream is being recorded).
    cudaGraphExec_t ge[2] = {nullptr, nullptr};
    uint64_t nk[2] = {0, 0};
    cudaStream_t gs = st;
    bool graphs = false;
    if (allow_graphs && !ctx->prof && p->max_iter >= 2) {
        const bool legacy = st == nullptr || st == cudaStreamLegacy || st == cudaStreamPerThread;
        if (legacy) {
            if (!ctx->graph_st) CK(cudaStreamCreateWithFlags(&ctx->graph_st, cudaStreamNonBlocking));
            for (cudaEvent_t& e : ctx->graph_ev)
                if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
            gs = ctx->graph_st;
        }
        graphs = capture_iterations(ctx, X, n, d, k, p, labels, L, p->max_iter + 1, gs, ge, nk);
        if (graphs && legacy) {  // the replays follow the caller's earlier work
            CK(cudaEventRecord(ctx->graph_ev[0], st));
            CK(cudaStreamWaitEvent(gs, ctx->graph_ev[0], 0));
        }
        if (!graphs) gs = st;
    }
    auto drop_graphs = [&]() {
        for (cudaGraphExec_t& e : ge)
            if (e) { cudaGraphExecDestroy(e); e = nullptr; }
    };
    for (t = 0; t < p->max_iter; t++) {
        if (graphs) {
            const cudaError_t e = cudaGraphLaunch(ge[t & 1], gs);
            if (e != cudaSuccess) {
                drop_graphs();
                return fail(ctx, KM_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
            }
            ctx->launches += nk[t & 1];
        } else {
            s = lloyd_iteration(ctx, X, n, d, k, p, labels, L, cur, nxt, L.sse_hist + t, L.flag_hist + t, false, 0, st);
            if (s != KM_OK) return s;
        }
        std::swap(cur, nxt);
        if (cancel && *cancel) {
            drop_graphs();
            CK(cudaStreamSynchronize(gs));
            return fail(ctx, KM_ECANCELLED, "cancelled");
        }
        if (p->tau > 0.0) {
            double shift = 0.0;
            cudaError_t e = cudaMemcpyAsync(&shift, L.u.shift, sizeof(double), cudaMemcpyDeviceToHost, gs);
            if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
            if (e != cudaSuccess) {
                drop_graphs();
                return fail(ctx, KM_ECUDA, "shift read-back: %s", cudaGetErrorString(e));
            }
            if (shift < p->tau) { t++; break; }
        }
    }
    drop_graphs();
    if (gs != st) {  // back on the caller's stream
        CK(cudaEventRecord(ctx->graph_ev[1], gs));
        CK(cudaStreamWaitEvent(st, ctx->graph_ev[1], 0));
    }
    CK(cudaMemsetAsync(&L.a.cnt->amb_count, 0, 2 * sizeof(int), st));
    s = run_assign(ctx, X, n, cur, k, d, p, labels, L.min_dist, L.a, true, st);
    if (s != KM_OK) return s;
    if ((s = refine_winners(ctx, X, n, d, cur, p, labels, L.min_dist, st)) != KM_OK) return s;
    KL(2, launch_sum_f64(L.min_dist, n, L.a.partials, kSumParts, L.sse_hist + t, st));
    CK(cudaMemcpyAsync(L.flag_hist + t, &L.a.cnt->flagged, sizeof(unsigned long long), cudaMemcpyDeviceToDevice, st));
    KL(2, launch_sum_f64(L.min_dist, n, L.a.partials, kSumParts, L.a.sse, st));
    CK(cudaMemcpyAsync(C_out, cur, sizeof(float) * (size_t)k * d, cudaMemcpyDeviceToDevice, st));
    ctx->last_cnt = L.a.cnt;
    ctx->last_sse = L.a.sse;
    ctx->last_stream = st;
    ctx->last_pairs = (uint64_t)n * (uint64_t)k * (uint64_t)(t + 1);
    if ((s = sync_status(ctx, L.a.cnt, st)) != KM_OK) return s;
    std::vector<double> sse(t + 1);
    std::vector<unsigned long long> fl(t + 1);
    CK(cudaMemcpy(sse.data(), L.sse_hist, sizeof(double) * (t + 1), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(fl.data(), L.flag_hist, sizeof(unsigned long long) * (t + 1), cudaMemcpyDeviceToHost));
    const double pairs = (double)n * (double)k;
    for (int i = 0; i <= t; i++) {
        if (sse_per_iter) sse_per_iter[i] = sse[i];
        if (eta_per_iter) eta_per_iter[i] = (double)(fl[i] - (i ? fl[i - 1] : 0ull)) / pairs;
    }
    if (iters_done) *iters_done = t;
    return KM_OK;
}

extern "C" {

km_status km_get_stats(km_ctx* ctx, km_stats* out) {
    if (!ctx || !out) return KM_EINVAL;
    if (!ctx->last_cnt) return fail(ctx, KM_EINVAL, "no call to report on");
    km_status s = sync_status(ctx, ctx->last_cnt, ctx->last_stream);
    DevCounters c{};
    CK(cudaMemcpy(&c, ctx->last_cnt, sizeof c, cudaMemcpyDeviceToHost));
    out->pairs = ctx->last_pairs;
    out->flagged = c.flagged;
    out->fp32_evals = c.fp32_evals;
    out->fp64_evals = c.fp64_evals;
    out->ambiguous_rows = c.amb_rows;
    out->overflow_rows = c.ovf_rows;
    out->sse = 0.0;
    if (ctx->last_sse) CK(cudaMemcpy(&out->sse, ctx->last_sse, sizeof(double), cudaMemcpyDeviceToHost));
    return s;
}

km_status km_set_profiling(km_ctx* ctx, int on) {
    if (!ctx) return KM_EINVAL;
    ctx->prof = on != 0;
    return KM_OK;
}

km_status km_get_phase_times(km_ctx* ctx, double* ms, int64_t* counts) {
    if (!ctx || !ms) return KM_EINVAL;
    for (int ph = 0; ph < KM_NUM_PHASES; ph++) {
        double sum = 0.0;
        for (auto& e : ctx->ev[ph]) {
            CK(cudaEventSynchronize(e.second));
            float t = 0.0f;
            CK(cudaEventElapsedTime(&t, e.first, e.second));
            sum += t;
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        ms[ph] = sum;
        if (counts) counts[ph] = (int64_t)ctx->ev[ph].size();
        ctx->ev[ph].clear();
    }
    return KM_OK;
}

km_status km_get_launch_count(const km_ctx* ctx, uint64_t* launches) {
    if (!ctx || !launches) return KM_EINVAL;
    *launches = ctx->launches;
    return KM_OK;
}

km_status km_submit(km_ctx* ctx, const km_job* job, uint64_t* job_id) {
    if (!ctx || !job || !job_id) return KM_EINVAL;
    if (!ctx->serve) return fail(ctx, KM_EINVAL, "context has no serving arena (km_init with arena_bytes > 0)");
    if (!job->X || !job->C_init || job->n < 1 || job->d < 1 || job->k < 1 || job->k > job->n)
        return fail(ctx, KM_EINVAL, "bad job shape");
    if (job->flags & ~KM_JOB_DEVICE_DATA) return fail(ctx, KM_EINVAL, "unknown job flags 0x%x", job->flags);
    if (job->flags & KM_JOB_DEVICE_DATA) {
        for (const void* ptr : {(const void*)job->X, (const void*)job->C_init}) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess || at.type != cudaMemoryTypeDevice ||
                at.device != ctx->device) {
                cudaGetLastError();
                return fail(ctx, KM_EINVAL, "KM_JOB_DEVICE_DATA: X and C_init must be device memory of device %d",
                            ctx->device);
            }
        }
    }
    km_status s = check_params(ctx, &job->p, job->d, job->k);
    if (s != KM_OK) return s;
    return serve_submit(ctx->serve, job, job_id, &ctx->err);
}
km_status km_poll(km_ctx* ctx, uint64_t job_id, km_result* out) {
    if (!ctx || !out) return KM_EINVAL;
    if (!ctx->serve) return fail(ctx, KM_EINVAL, "context has no serving arena");
    return serve_poll(ctx->serve, job_id, out);
}
km_status km_release(km_ctx* ctx, uint64_t job_id) {
    if (!ctx) return KM_EINVAL;
    if (!ctx->serve) return fail(ctx, KM_EINVAL, "context has no serving arena");
    return serve_release(ctx->serve, job_id);
}
km_status km_cancel(km_ctx* ctx, uint64_t job_id) {
    if (!ctx) return KM_EINVAL;
    if (!ctx->serve) return fail(ctx, KM_EINVAL, "context has no serving arena");
    return serve_cancel(ctx->serve, job_id);
}

}  // extern "C"

size_t km_internal_ws_bytes(int64_t n, int d, int k, const km_params* p) {
    Carve a{nullptr};
    carve_lloyd(a, n, d, k, p->low, std::max(0, (int)p->max_iter));
    Carve b{nullptr};
    carve_assign(b, n, d, k, p->low, false);
    b.take<double>((size_t)n);
    return std::max(a.off, b.off) + 256;
}

bool km_internal_groupable(const km_job& job) {
    return job.kind == 0 && job.p.low == KM_FP32_DIRECT && job.d >= 1 && job.d <= GROUP_MAX_D && job.k >= 1 &&
           job.k <= GROUP_MAX_K && job.n >= job.k && job.n <= GROUP_MAX_N && job.p.max_iter >= 0;
}

km_status km_internal_run_batch(km_ctx_view* v, const km_batch_job* jobs, int njobs, const km_params* p,
                                cudaStream_t st, std::string* err) {
    km_ctx ctx;
    ctx.device = v->device;
    ctx.num_sms = v->num_sms;
    if (v->tune) ctx.tune = v->tune;
    km_status s = km_lloyd_run_batch(&ctx, jobs, njobs, p, st);
    if (s == KM_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            if (err) *err = cudaGetErrorString(e);
            return KM_ECUDA;
        }
    } else if (err) {
        *err = ctx.err;
    }
    return s;
}

// Used by the serving engine: one whole Lloyd / assign job on its own stream.
km_status km_internal_run_job(km_ctx_view* v, const float* X, int64_t n, int d, int k, const float* C_init,
                              const km_params* p, int kind, float* C_out, int32_t* labels, void* ws, size_t ws_bytes,
                              cudaStream_t st, double* sse, double* eta, int* iters, std::string* err,
                              const volatile int* cancel) {
    km_ctx ctx;
    ctx.device = v->device;
    ctx.num_sms = v->num_sms;
    if (v->tune) ctx.tune = v->tune;
    km_status s;
    if (kind == 1) {
        s = km_assign(&ctx, X, n, C_init, k, d, p, labels, nullptr, nullptr, ws, ws_bytes, st);
        if (s == KM_OK) {
            km_stats stt{};
            s = km_get_stats(&ctx, &stt);
            *sse = stt.sse;
            *eta = stt.pairs ? (double)stt.flagged / (double)stt.pairs : 0.0;
            *iters = 0;
        }
        if (s == KM_OK && C_out != C_init)
            cudaMemcpyAsync(C_out, C_init, sizeof(float) * (size_t)k * d, cudaMemcpyDeviceToDevice, st);
    } else {
        std::vector<double> sh(p->max_iter + 1), eh(p->max_iter + 1);
        s = lloyd_impl(&ctx, X, n, d, k, C_init, p, C_out, labels, sh.data(), eh.data(), iters, ws, ws_bytes, st,
                       cancel, false);
        if (s == KM_OK) {
            *sse = sh[*iters];
            double fl = 0;
            for (int i = 0; i <= *iters; i++) fl += eh[i];
            *eta = fl / (*iters + 1);
        }
    }
    if (s != KM_OK && err) *err = ctx.err;
    if (s == KM_OK) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            if (err) *err = cudaGetErrorString(e);
            s = KM_ECUDA;
        }
    }
    return s;
}

// ---- km_assign_static: the certified fp32 direct assignment with static scratch ----
// For callers that cannot allocate device memory at assignment time (device
// memory held by another pool, where cudaMalloc fails; loops that must not
// pay for cudaMalloc/cudaFree, which can synchronise the device).  The
// scratch is a file-scope device array: the counters in the first 256 bytes,
// then the list of rows whose fp32 argmin stayed open.  There is one copy per
// device, so calls that overlap in time on one device race on it.
namespace {
constexpr size_t kStaticCntBytes = 256;
static_assert(sizeof(DevCounters) <= kStaticCntBytes, "counters exceed their slot");
constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mu;
void* g_static_addr[kStaticMaxDevices];  // resolved scratch address per device, null until first use
}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticCntBytes + (size_t)KM_STATIC_MAX_ROWS * sizeof(int32_t)];

namespace {
// Failure-path check: one warp waits on an mbarrier that no thread arrives at.
// The wait is the library's bounded one: it runs out after KM_WAIT_CYCLES,
// sets the status word's timeout bit and returns; nothing faults or hangs.
__global__ void k_wait_unsignalled(DevCounters* cnt) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    (void)mbar_wait(&bar, 0, (volatile int*)&abort_flag, &cnt->status);
}
}  // namespace

extern "C" km_status km_seed_pp(km_ctx* ctx, const float* X, int64_t n, int d, int k, const double* u_host, float* C_out,
                     int64_t* idx_host, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!X || !u_host || !C_out || !ws) return fail(ctx, KM_EINVAL, "null argument");
    if (n < 1 || d < 1 || k < 1 || k > n) return fail(ctx, KM_EINVAL, "need 1 <= k <= n and d >= 1");
    if (n > (int64_t)INT32_MAX) return fail(ctx, KM_EINVAL, "n too large");
    if (d > 512) return fail(ctx, KM_EUNSUPPORTED, "d=%d: seeding takes d <= 512", d);
    for (int t = 0; t < k; t++)
        if (!(u_host[t] >= 0.0 && u_host[t] < 1.0)) return fail(ctx, KM_EINVAL, "draw %d outside [0, 1)", t);
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    Carve cv{(char*)ws};
    double* D2 = cv.take<double>((size_t)n);
    double* u = cv.take<double>((size_t)k);
    int64_t* idx = cv.take<int64_t>((size_t)k);
    double* csum = cv.take<double>(seed_chunk_count(n));
    int64_t* clast = cv.take<int64_t>(seed_chunk_count(n));
    if (ws_bytes < cv.off) return fail(ctx, KM_ENOMEM, "workspace too small: %zu < %zu", ws_bytes, cv.off);
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    CK(cudaMemcpyAsync(u, u_host, sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, st));
    int nl = 0;
    CK(launch_seed_pp(X, n, d, k, u, D2, idx, csum, clast, C_out, ctx->num_sms, st, &nl));
    ctx->launches += (uint64_t)nl;
    if (idx_host) CK(cudaMemcpyAsync(idx_host, idx, sizeof(int64_t) * (size_t)k, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return KM_OK;
}

km_status km_selftest_timeout(km_ctx* ctx, void* ws, size_t ws_bytes, void* stream) {
    if (!ctx) return KM_EINVAL;
    if (!ws) return fail(ctx, KM_EINVAL, "null workspace");
    if (!aligned256(ws)) return fail(ctx, KM_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < sizeof(DevCounters)) return fail(ctx, KM_ENOMEM, "workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    CK(cudaSetDevice(ctx->device));
    DevCounters* cnt = reinterpret_cast<DevCounters*>(ws);
    CK(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), st));
    k_wait_unsignalled<<<1, 32, 0, st>>>(cnt);
    CK(cudaGetLastError());
    ctx->launches++;
    return sync_status(ctx, cnt, st);
}

extern "C" km_status km_assign_static(km_ctx* ctx, const float* X, int64_t n, const float* C, int k, int d,
                                      int32_t* labels, double* min_dist, void* stream) {
    km_status s = check_common(ctx, X, n, C, k, d);
    if (s != KM_OK) return s;
    if (!labels || !min_dist) return fail(ctx, KM_EINVAL, "km_assign_static needs labels and min_dist");
    if (n > (int64_t)KM_STATIC_MAX_ROWS)
        return fail(ctx, KM_ENOMEM, "km_assign_static: n=%lld exceeds its static scratch of %d rows (use km_assign)",
                    (long long)n, KM_STATIC_MAX_ROWS);
    km_params p;
    km_default_params(&p);
    p.low = KM_FP32_DIRECT;
    if ((s = check_params(ctx, &p, d, k)) != KM_OK) return s;
    if (ctx->device < 0 || ctx->device >= kStaticMaxDevices)
        return fail(ctx, KM_EUNSUPPORTED, "km_assign_static: device %d out of range", ctx->device);
    CK(cudaSetDevice(ctx->device));
    void* base = nullptr;
    {
        // one-time set-up per device, with that device current
        std::lock_guard<std::mutex> lock(g_static_mu);
        if (!g_static_addr[ctx->device]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_static_scratch);
            if (e != cudaSuccess)
                return fail(ctx, KM_ECUDA, "cudaGetSymbolAddress(static scratch): %s", cudaGetErrorString(e));
            g_static_addr[ctx->device] = ptr;
        }
        base = g_static_addr[ctx->device];
    }
    DevCounters* cnt = reinterpret_cast<DevCounters*>(base);
    int32_t* amb_list = reinterpret_cast<int32_t*>(static_cast<char*>(base) + kStaticCntBytes);
    cudaStream_t st = (cudaStream_t)stream;
    const TestParams tp = make_tp(&p, d);
    // the counters (amb_count above all) must start at zero; the row list is
    // written before it is read
    CK(cudaMemsetAsync(cnt, 0, sizeof(DevCounters), st));
    KL(1, launch_direct_assign(false, X, n, C, k, d, nullptr, nullptr, labels, min_dist, amb_list, cnt, tp.gamma32,
                               ctx->num_sms, st));
    KL(1, launch_rows_full(false, X, C, k, d, amb_list, &cnt->amb_count, labels, min_dist, cnt, tp.gamma32,
                           ctx->num_sms, st));
    // the winners' distances to binary64 accuracy, as km_assign (no scratch)
    KL(1, launch_winner_dist(X, n, d, C, labels, min_dist, ctx->num_sms, st));
    return KM_OK;
}
