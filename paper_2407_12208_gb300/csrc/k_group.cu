// k_group.cu -- grouped Lloyd runs (Alg. 3) of many small jobs in one launch:
// one CTA per job runs the whole loop with its centres, sums and counts in
// shared memory, so a batch of uneven small jobs costs one launch instead of
// about ten per iteration each.  For the FP32 direct path with d <= 8,
// k <= 64, n <= 16384 (the jobs whose every iteration is a few microseconds).
//
// Every value equals km_lloyd_run's for the same job, bit for bit:
//  * labels: the fp32 direct distances certified by Theorem 4.1's interval
//    (the library's gamma), else binary64 in the oracle's order over the
//    centres still open, lowest index on ties -- the exact binary64 argmin
//    either way, whatever kernel forms it;
//  * min_dist: the double-float direct formula of df.cuh (df_small<D>);
//  * centre sums: exact 64-bit fixed point at the scale of max|x| and n;
//    means in binary64 stored fp32; empty clusters (KM_EMPTY_FARTHEST) take
//    the rows of largest min_dist in ascending cluster order, ties to the
//    lowest row;
//  * SSE: the library's fixed reduction (1024 parts, a 256-wide tree per
//    part, then 32 lanes in order and a butterfly), replayed here;
//  * shift: per centre a warp of fma terms and a butterfly, the maximum.
#include <cmath>

#include "common.cuh"
#include "df.cuh"
#include "fixed.cuh"
#include "group.h"

namespace km {

constexpr int GRP_T = 512;        // threads per job
constexpr int GRP_PARTS = 1024;   // parts of the SSE reduction (as in the library's)

struct GroupSmem {
    float Cc[GROUP_MAX_K * 8], Cn[GROUP_MAX_K * 8];
    long long sums[GROUP_MAX_K * 8], cnt[GROUP_MAX_K];
    double parts[GRP_PARTS];
    unsigned amax;
    unsigned long long shift_bits;
    unsigned long long bmd;  // empty-cluster selection: the largest md's bits, then its lowest row
    int brow;
    int empties[GROUP_MAX_K];
    int nempty;
};

// Binary64 direct formula in coordinate order, products and sums rounded
// separately (the oracle's arithmetic).
template <int D>
KM_DEV double grp_direct64(const float (&x)[D], const float* c) {
    double s = 0.0;
#pragma unroll
    for (int l = 0; l < D; l++) {
        const double t = __dsub_rn((double)x[l], (double)c[l]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

template <int D>
KM_DEV float grp_direct32(const float (&x)[D], const float* c) {
    float s = 0.0f;
#pragma unroll
    for (int l = 0; l < D; l++) {
        const float u = x[l] - c[l];
        s = fmaf(u, u, s);
    }
    return s;
}

// Labels and min_dist of every row against the centres in sm.Cc.
template <int D>
KM_DEV void grp_assign(const float* __restrict__ X, int n, int k, const float* Cc, float g,
                       int32_t* __restrict__ labels, double* __restrict__ md) {
    for (int i = threadIdx.x; i < n; i += GRP_T) {
        float x[D];
#pragma unroll
        for (int l = 0; l < D; l++) x[l] = X[(int64_t)i * D + l];
        float b1 = INFINITY, b2 = INFINITY;
        int j1 = 0;
        for (int j = 0; j < k; j++) {
            const float v = grp_direct32<D>(x, Cc + j * D);
            if (v < b1) { b2 = b1; b1 = v; j1 = j; }
            else if (v < b2) b2 = v;
        }
        int lab = j1;
        if (!(b2 * (1.0f - g) > b1 * (1.0f + g))) {  // not certified: binary64 over the open centres
            const float thr = b1 * (1.0f + g);
            double best = INFINITY;
            int arg = 0x7fffffff;
            for (int j = 0; j < k; j++) {
                const float v = grp_direct32<D>(x, Cc + j * D);
                if (!(v * (1.0f - g) <= thr)) continue;
                const double s = grp_direct64<D>(x, Cc + j * D);
                if (s < best) { best = s; arg = j; }
            }
            if (arg < k) lab = arg;  // (non-finite data: no centre qualifies, the fp32 winner stays)
        }
        labels[i] = lab;
        md[i] = df_value(df_small<D>(x, Cc + lab * D));
    }
}

// The library's deterministic sum of md (1024 parts of ceil(n / 1024) rows,
// each a 256-wide halving tree; then lane l of one warp adds parts l, l + 32,
// ... in order and a butterfly).  With n <= 16384 a part holds at most 16
// rows, so only the tree's last four levels add anything but zeros.
KM_DEV double grp_sse(const double* __restrict__ md, int n, double* parts) {
    const int chunk = (n + GRP_PARTS - 1) / GRP_PARTS;
    for (int p = threadIdx.x; p < GRP_PARTS; p += GRP_T) {
        double a[16];
#pragma unroll
        for (int t = 0; t < 16; t++) {
            const int i = p * chunk + t;
            a[t] = (t < chunk && i < n) ? md[i] : 0.0;
        }
#pragma unroll
        for (int st = 8; st > 0; st >>= 1)
#pragma unroll
            for (int t = 0; t < st; t++) a[t] += a[t + st];
        parts[p] = a[0];
    }
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        for (int i = threadIdx.x; i < GRP_PARTS; i += 32) s += parts[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    }
    return s;  // valid in thread 0
}

// The centre update on the labels just made: exact sums and counts, means,
// empty clusters, and the shift from sm.Cc to sm.Cn (returned in thread 0).
template <int D>
KM_DEV double grp_update(const float* __restrict__ X, int n, int k, const int32_t* __restrict__ labels,
                         const double* __restrict__ md, const FixedScale& fx, int S, bool farthest, GroupSmem& sm) {
    for (int e = threadIdx.x; e < k * D; e += GRP_T) sm.sums[e] = 0;
    for (int j = threadIdx.x; j < k; j += GRP_T) sm.cnt[j] = 0;
    if (threadIdx.x == 0) { sm.nempty = 0; sm.shift_bits = 0ull; }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += GRP_T) {
        const int j = labels[i];
#pragma unroll
        for (int l = 0; l < D; l++)
            atomicAdd(reinterpret_cast<unsigned long long*>(&sm.sums[j * D + l]),
                      (unsigned long long)fx(X[(int64_t)i * D + l]));
        atomicAdd(reinterpret_cast<unsigned long long*>(&sm.cnt[j]), 1ull);
    }
    __syncthreads();
    // means in binary64, stored fp32; an empty cluster keeps its centre
    for (int e = threadIdx.x; e < k * D; e += GRP_T) {
        const long long m = sm.cnt[e / D];
        sm.Cn[e] = m > 0 ? (float)(ldexp((double)sm.sums[e], -S) / (double)m) : sm.Cc[e];
    }
    if (threadIdx.x == 0 && farthest)
        for (int j = 0; j < k; j++)
            if (sm.cnt[j] == 0) sm.empties[sm.nempty++] = j;
    __syncthreads();
    // empty clusters in ascending order take the rows of largest min_dist,
    // ties to the lowest row, each row once: pick r is the first row after
    // pick r - 1 in the order (md descending, row ascending) -- the largest
    // md among the rows after it, then the lowest such row
    double pmd = INFINITY;
    int prow = -1;
    for (int r = 0; r < sm.nempty; r++) {
        if (threadIdx.x == 0) { sm.bmd = 0ull; sm.brow = 0x7fffffff; }
        __syncthreads();
        unsigned long long mb = 0ull;
        for (int i = threadIdx.x; i < n; i += GRP_T) {
            const double v = md[i];
            if (v < pmd || (v == pmd && i > prow)) {
                const unsigned long long vb = (unsigned long long)__double_as_longlong(v);  // md >= 0: bits order like values
                mb = vb > mb ? vb : mb;
            }
        }
        atomicMax(&sm.bmd, mb);
        __syncthreads();
        const double bm = __longlong_as_double((long long)sm.bmd);
        int mr = 0x7fffffff;
        for (int i = threadIdx.x; i < n; i += GRP_T) {
            const double v = md[i];
            if (v == bm && (v < pmd || i > prow) && i < mr) mr = i;
        }
        atomicMin(&sm.brow, mr);
        __syncthreads();
        pmd = bm;
        prow = sm.brow;
        if (prow < n)  // (non-finite distances can leave no row to take)
            for (int l = threadIdx.x; l < D; l += GRP_T) sm.Cn[sm.empties[r] * D + l] = X[(int64_t)prow * D + l];
        __syncthreads();
    }
    // shift: per centre, lane l < D adds (c_new - c_old)_l^2 by fma, a butterfly, the square root
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = wid; j < k; j += GRP_T / 32) {
        double s = 0.0;
        if (lane < D) {
            const double df = (double)sm.Cn[j * D + lane] - (double)sm.Cc[j * D + lane];
            s = fma(df, df, s);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) atomicMax(&sm.shift_bits, (unsigned long long)__double_as_longlong(sqrt(s)));
    }
    __syncthreads();
    return __longlong_as_double((long long)sm.shift_bits);
}

// One job per CTA: Alg. 3 from C_init, max_iter iterations or until the shift
// drops below tau, then the final reassignment (km_lloyd_run's sequence).
template <int D>
__global__ void __launch_bounds__(GRP_T) k_group_lloyd(const __grid_constant__ GroupArgs a) {
    __shared__ GroupSmem sm;
    const GroupJob& J = a.job[blockIdx.x];
    const int n = J.n, k = J.k;
    // max |x| fixes the scale of the exact sums (non-negative floats order as their bits)
    if (threadIdx.x == 0) sm.amax = 0u;
    __syncthreads();
    float m = 0.0f;
    for (int64_t e = threadIdx.x; e < (int64_t)n * D; e += GRP_T) m = fmaxf(m, fabsf(J.X[e]));
    atomicMax(&sm.amax, __float_as_uint(m));
    for (int e = threadIdx.x; e < k * D; e += GRP_T) sm.Cc[e] = J.C_init[e];
    __syncthreads();
    const int S = fixed_shift(sm.amax, n);
    const FixedScale fx(S);
    int t = 0;
    for (t = 0; t < a.max_iter; t++) {
        grp_assign<D>(J.X, n, k, sm.Cc, a.gamma32, J.labels, J.md);
        __syncthreads();
        const double sse = grp_sse(J.md, n, sm.parts);
        if (threadIdx.x == 0) J.sse[t] = sse;
        const double shift = grp_update<D>(J.X, n, k, J.labels, J.md, fx, S, a.empty_farthest != 0, sm);
        for (int e = threadIdx.x; e < k * D; e += GRP_T) sm.Cc[e] = sm.Cn[e];
        __syncthreads();
        if (a.tau > 0.0 && shift < a.tau) { t++; break; }
    }
    grp_assign<D>(J.X, n, k, sm.Cc, a.gamma32, J.labels, J.md);
    __syncthreads();
    const double sse = grp_sse(J.md, n, sm.parts);
    if (threadIdx.x == 0) {
        J.sse[t] = sse;
        *J.iters = t;
    }
    for (int e = threadIdx.x; e < k * D; e += GRP_T) J.C_out[e] = sm.Cc[e];
}

cudaError_t launch_group_lloyd(const GroupArgs& a, int njobs, int d, cudaStream_t st) {
    if (njobs < 1) return cudaSuccess;
    if (njobs > GROUP_MAX) return cudaErrorInvalidValue;
    switch (d) {
#define KM_GL(DD) \
    case DD: k_group_lloyd<DD><<<njobs, GRP_T, 0, st>>>(a); break;
        KM_GL(1) KM_GL(2) KM_GL(3) KM_GL(4) KM_GL(5) KM_GL(6) KM_GL(7) KM_GL(8)
#undef KM_GL
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace km
