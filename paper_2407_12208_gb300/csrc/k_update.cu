// k_update.cu -- centre update, Eq. (center), with the accuracy Section 4.4
// asks of it.
//
// Section 4.4 (Lemma 4.4, Theorem 4.5, Corollary 4.7) shows the update needs
// more precision than the distances, increasingly so late in the iteration.
// Here the per-cluster coordinate sums are formed EXACTLY in 64-bit fixed
// point: every coordinate is scaled by 2^S (S chosen from max|x| and n so
// that no partial sum can exceed 2^62) and rounded once to an integer, after
// which integer addition is exact and associative.  The only error is that
// one rounding, <= 2^-(S+1) per coordinate, so |mu^ - mu| <= 2^-(S+1) before
// the final division (binary64) and the fp32 store -- below the binary64
// recursive-summation bound gamma_m a_bar of Lemma 4.4 for the data sizes
// here, and independent of the order in which threads add: results are
// bitwise reproducible run to run and alone or batched.
#include <algorithm>

#include "common.cuh"
#include "df.cuh"
#include "fixed.cuh"
#include "internal.h"

namespace km {

__global__ void k_absmax(const float* __restrict__ X, int64_t count, unsigned* out) {
    float m = 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(X[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

// Row-parallel accumulation for the shapes the bucketed path does not take:
// shared-memory accumulators when k*d fits, else global atomics (integer, so
// the result does not depend on the order of the adds).
template <bool SMEM>
__global__ void k_accumulate(const float* __restrict__ X, int64_t n, int d, const int32_t* __restrict__ labels,
                             int k, const unsigned* __restrict__ amax_bits, int64_t nscale, long long* __restrict__ sums,
                             long long* __restrict__ counts) {
    extern __shared__ long long acc[];
    const FixedScale fx(fixed_shift(*amax_bits, nscale));
    const int64_t kd = (int64_t)k * d;
    if (SMEM) {
        for (int64_t e = threadIdx.x; e < kd + k; e += blockDim.x) acc[e] = 0;
        __syncthreads();
    }
    long long* sacc = SMEM ? acc : sums;
    long long* cacc = SMEM ? acc + kd : counts;
    // rows spread over the warps; within a row the lanes walk the coordinates
    // (for d < 32 a warp covers 32 / d rows at once)
    const int lane = threadIdx.x & 31;
    const int rpw = d < 32 ? 32 / d : 1;  // rows per warp step
    const int sub = lane / (d < 32 ? d : 32), l_in = lane % (d < 32 ? d : 32);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = gw * rpw; r < n; r += nw * rpw) {
        const int64_t i = r + sub;
        if (sub >= rpw || i >= n) continue;
        const int j = labels[i];
        const float* x = X + i * d;
        for (int l = l_in; l < d; l += (d < 32 ? d : 32)) {
            const long long v = fx(x[l]);
            atomicAdd(reinterpret_cast<unsigned long long*>(&sacc[(int64_t)j * d + l]), (unsigned long long)v);
        }
        if (l_in == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&cacc[j]), 1ull);
    }
    if (SMEM) {
        __syncthreads();
        for (int64_t e = threadIdx.x; e < kd; e += blockDim.x)
            if (acc[e]) atomicAdd(reinterpret_cast<unsigned long long*>(&sums[e]), (unsigned long long)acc[e]);
        for (int e = threadIdx.x; e < k; e += blockDim.x)
            if (acc[kd + e]) atomicAdd(reinterpret_cast<unsigned long long*>(&counts[e]), (unsigned long long)acc[kd + e]);
    }
}

// ---- bucketed reduction: rows grouped by label, summed in registers ------
// Integer (fixed-point) addition is order-independent, so the row order
// inside a bucket (set by atomic cursors) does not change any bit of the
// result.
constexpr int SEG_MAX = 512;     // most rows per warp work item (the 32-bit part sums stay exact)
constexpr int SCAT_ROWS = 4096;  // rows per block of the histogram / scatter kernels

// per-label counts (block histogram in shared memory, one global add per label)
__global__ void k_label_hist(const int32_t* __restrict__ labels, int64_t n, int k, int* __restrict__ cnt32) {
    extern __shared__ int h[];
    for (int j = threadIdx.x; j < k; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * SCAT_ROWS, r1 = min(n, r0 + SCAT_ROWS);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) atomicAdd(&h[labels[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x)
        if (h[j]) atomicAdd(&cnt32[j], h[j]);
}

// Exclusive scans (one block of 1024 threads): bucket offsets, cursors, and
// the offsets of each bucket's first work item; counts as int64.
__global__ void k_bucket_scan(const int* __restrict__ cnt32, int k, int seg, int* __restrict__ off,
                              int* __restrict__ cursor, int* __restrict__ item_off, long long* __restrict__ counts) {
    __shared__ int sa[1024], sb[1024];
    const int t = threadIdx.x, T = blockDim.x;
    const int per = (k + T - 1) / T;
    const int j0 = min(k, t * per), j1 = min(k, j0 + per);
    int a = 0, b = 0;
    for (int j = j0; j < j1; j++) {
        a += cnt32[j];
        b += (cnt32[j] + seg - 1) / seg;
    }
    sa[t] = a;
    sb[t] = b;
    __syncthreads();
    for (int st = 1; st < T; st <<= 1) {
        const int va = (t >= st) ? sa[t - st] : 0, vb = (t >= st) ? sb[t - st] : 0;
        __syncthreads();
        sa[t] += va;
        sb[t] += vb;
        __syncthreads();
    }
    int oa = sa[t] - a, ob = sb[t] - b;
    for (int j = j0; j < j1; j++) {
        off[j] = oa;
        cursor[j] = oa;
        item_off[j] = ob;
        counts[j] = cnt32[j];
        oa += cnt32[j];
        ob += (cnt32[j] + seg - 1) / seg;
    }
    if (t == T - 1) {
        off[k] = sa[T - 1];
        item_off[k] = sb[T - 1];
    }
}

// Each block reserves one contiguous range per label (one global atomic per
// label present) and places its rows with shared-memory cursors.
__global__ void k_bucket_scatter(const int32_t* __restrict__ labels, int64_t n, int k, int* __restrict__ cursor,
                                 int32_t* __restrict__ perm) {
    extern __shared__ int sh[];
    int* h = sh;
    int* lc = sh + k;
    for (int j = threadIdx.x; j < k; j += blockDim.x) h[j] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * SCAT_ROWS, r1 = min(n, r0 + SCAT_ROWS);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) atomicAdd(&h[labels[i]], 1);
    __syncthreads();
    for (int j = threadIdx.x; j < k; j += blockDim.x) lc[j] = h[j] ? atomicAdd(&cursor[j], h[j]) : 0;
    __syncthreads();
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) perm[atomicAdd(&lc[labels[i]], 1)] = (int32_t)i;
}

KM_DEV int bucket_of(const int* __restrict__ item_off, int k, int64_t it) {
    int lo = 0, hi = k;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (item_off[mid] <= it) lo = mid; else hi = mid;
    }
    return lo;
}

// One warp per work item (bucket j, rows [c*CHUNK, (c+1)*CHUNK) of it); each
// row is spread over LPR lanes (NV4 float4 each, d % 4 == 0), so a warp reads
// 32 / LPR rows per load; exact sums in registers, folded across the row
// groups of the warp at the end, one atomic add per coordinate per item.
//
// WD: the same pass also gives each row's distance to its own centre c_j (the
// winner's ||x - c||^2, Eq. (dist-direct)) to binary64 accuracy (df.cuh: the
// rows' chunk partials reduced over the row's lanes, eight rows at a time), so
// the assignment's min_dist costs no second read of X.
template <int NV4, int LPR, bool WD>
__global__ void __launch_bounds__(256, (NV4 == 1 && LPR == 32) ? 3 : (NV4 == 4 ? 1 : 2)) k_bucket_sum(const float* __restrict__ X, int64_t n, int d, int k, int seg,
                                                       const int* __restrict__ off,
                             const int* __restrict__ item_off, const int32_t* __restrict__ perm,
                             const unsigned* __restrict__ amax_bits, int64_t nscale, long long* __restrict__ sums,
                             const float* __restrict__ C, double* __restrict__ md) {
    static_assert(LPR == 32 || NV4 == 1, "rows narrower than a warp take one float4 per lane");
    constexpr int G = 32 / LPR;                            // rows per warp load
    // loads in flight per lane: 8 at full-warp rows of one float4 (three blocks
    // per SM), else up to 16
    constexpr int RB = (NV4 == 1 && LPR == 32) ? 8 : ((16 / NV4) < (32 / G) ? 16 / NV4 : 32 / G);
    constexpr int STEP = RB * G;                           // rows per round (divides 32)
    const FixedScale fx(fixed_shift(*amax_bits, nscale));
    const int lane = threadIdx.x & 31, sub = lane / LPR, cl = lane % LPR;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nitems = item_off[k];
    const int d4 = d >> 2;
    for (int64_t it = w0; it < nitems; it += nw) {
        const int j = bucket_of(item_off, k, it);
        const int c = (int)(it - item_off[j]);
        const int r0 = off[j] + c * seg, r1 = min(off[j + 1], r0 + seg);
        // the bucket's centre: this lane's chunks of c_j (WD)
        float4 cj[NV4];
        if (WD) {
#pragma unroll
            for (int u = 0; u < NV4; u++) {
                const int cidx = cl + LPR * u;
                cj[u] = (cidx < d4) ? reinterpret_cast<const float4*>(C + (int64_t)j * d)[cidx]
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        // biased parts of the fixed-point values, summed modulo 2^32 (SEG_MAX rows at most)
        unsigned a2[NV4][4], a1[NV4][4], a0[NV4][4];
#pragma unroll
        for (int u = 0; u < NV4; u++)
#pragma unroll
            for (int t = 0; t < 4; t++) a2[u][t] = a1[u][t] = a0[u][t] = 0u;
        unsigned rounds = 0;
        int64_t next_i = (r0 + lane < r1) ? (int64_t)perm[r0 + lane] : -1;
        for (int base = r0; base < r1; base += 32) {
            // the row indices of 32 rows in one coalesced load, then broadcast;
            // the following 32 rows' indices are loaded now and their data sent
            // to L2 once this round's loads are out
            const int64_t my_i = next_i;
            next_i = (base + 32 + lane < r1) ? (int64_t)perm[base + 32 + lane] : -1;
            bool pf = true;
#pragma unroll 1
            for (int b0 = 0; b0 < 32 && base + b0 < r1; b0 += STEP) {
                rounds++;
                float4 v[RB][NV4];
#pragma unroll
                for (int b = 0; b < RB; b++) {
                    const int64_t i = __shfl_sync(0xffffffffu, my_i, b0 + b * G + sub);
#pragma unroll
                    for (int u = 0; u < NV4; u++) {
                        const int cidx = cl + LPR * u;
                        v[b][u] = (i >= 0 && cidx < d4) ? reinterpret_cast<const float4*>(X + i * d)[cidx]
                                                         : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                if (LPR < 32 && pf) {  // narrow rows (measured: a loss at 512-byte rows)
                    if (next_i >= 0) prefetch_l2_bulk(X + next_i * d, (uint32_t)d * 4u);
                    pf = false;
                }
#pragma unroll
                for (int b = 0; b < RB; b++)
#pragma unroll
                    for (int u = 0; u < NV4; u++) {
                        uint2 q2, q1, q0;
                        fx.split2(make_float2(v[b][u].x, v[b][u].y), q2, q1, q0);
                        a2[u][0] += q2.x; a2[u][1] += q2.y;
                        a1[u][0] += q1.x; a1[u][1] += q1.y;
                        a0[u][0] += q0.x; a0[u][1] += q0.y;
                        fx.split2(make_float2(v[b][u].z, v[b][u].w), q2, q1, q0);
                        a2[u][2] += q2.x; a2[u][3] += q2.y;
                        a1[u][2] += q1.x; a1[u][3] += q1.y;
                        a0[u][2] += q0.x; a0[u][3] += q0.y;
                    }
                if (WD) {
                    // the rows' distances to c_j, RW rows per multi-row butterfly
                    constexpr int RW = RB < 8 ? RB : 8;
#pragma unroll
                    for (int bb = 0; bb < RB; bb += RW) {
                        DF part[RW];
#pragma unroll
                        for (int b = 0; b < RW; b++) part[b] = df_lane<NV4>(v[bb + b], cj);
                        int rs;
                        const DF r = df_rows<RW, LPR>(part, cl, rs);
                        const int64_t i = __shfl_sync(0xffffffffu, my_i, b0 + (bb + rs) * G + sub);
                        if ((cl & (LPR / RW - 1)) == 0 && i >= 0) md[i] = df_value(r);
                    }
                }
            }
        }
        // the row groups' sums of the same coordinates (modulo 2^32 like the sums)
#pragma unroll
        for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
            for (int u = 0; u < NV4; u++)
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    a2[u][t] += __shfl_xor_sync(0xffffffffu, a2[u][t], o);
                    a1[u][t] += __shfl_xor_sync(0xffffffffu, a1[u][t], o);
                    a0[u][t] += __shfl_xor_sync(0xffffffffu, a0[u][t], o);
                }
        // every row slot of every round was split (absent rows and padding as 0.0f)
        const unsigned m = rounds * (unsigned)STEP;
#pragma unroll
        for (int u = 0; u < NV4; u++) {
            const int cidx = cl + LPR * u;
            if (sub == 0 && cidx < d4)
#pragma unroll
                for (int t = 0; t < 4; t++) {
                    const long long acc = FixedScale::combine(a2[u][t], a1[u][t], a0[u][t], m);
                    if (acc)
                        atomicAdd(reinterpret_cast<unsigned long long*>(&sums[(int64_t)j * d + 4 * cidx + t]),
                                  (unsigned long long)acc);
                }
        }
    }
}

// Small d (d <= 16): lanes over rows, each lane sums its rows' d coordinates,
// then a warp reduction.
template <int D>
__global__ void k_bucket_sum_small(const float* __restrict__ X, int64_t n, int k, int seg, const int* __restrict__ off,
                                   const int* __restrict__ item_off, const int32_t* __restrict__ perm,
                                   const unsigned* __restrict__ amax_bits, int64_t nscale, long long* __restrict__ sums) {
    const FixedScale fx(fixed_shift(*amax_bits, nscale));
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int nitems = item_off[k];
    for (int64_t it = w0; it < nitems; it += nw) {
        const int j = bucket_of(item_off, k, it);
        const int c = (int)(it - item_off[j]);
        const int r0 = off[j] + c * seg, r1 = min(off[j + 1], r0 + seg);
        long long acc[D];
#pragma unroll
        for (int l = 0; l < D; l++) acc[l] = 0;
        for (int r = r0 + lane; r < r1; r += 32) {
            const float* x = X + (int64_t)perm[r] * D;
#pragma unroll
            for (int l = 0; l < D; l++) acc[l] += fx(x[l]);
        }
#pragma unroll
        for (int l = 0; l < D; l++) {
            long long v = acc[l];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(&sums[(int64_t)j * D + l]), (unsigned long long)v);
        }
    }
}

// Small d and small k * d: rows in their natural order (one per lane,
// coalesced), each warp keeps the 32-bit parts of every cluster's fixed-point
// sum (and its count) in shared memory.  A segmented inclusive scan over the
// warp's runs of equal labels (five shuffle levels, whatever the labels: an
// image's pixels come in long runs) leaves each run's total in its last
// lane, which adds it with a shared atomic.  Every AS_CHUNK rows the
// accumulators are folded into the global int64 sums.  Integer additions
// throughout: the order does not matter.
// WD: each row's distance to its own centre (binary64 accuracy, df.cuh) from
// the same read of the row, with C staged in shared memory.
constexpr int AS_CHUNK = 1024;   // rows per warp between folds (keeps each 32-bit part sum below 2^31)
constexpr int AS_MAX_KD = 512;   // k * d bound of this path
template <int D, bool WD>
__global__ void __launch_bounds__(256) k_accum_small(const float* __restrict__ X, int64_t n, int k,
                                                     const int32_t* __restrict__ labels,
                                                     const unsigned* __restrict__ amax_bits, int64_t nscale,
                                                     long long* __restrict__ sums, long long* __restrict__ counts,
                                                     const float* __restrict__ C, double* __restrict__ md) {
    extern __shared__ unsigned acc_sm[];  // per warp: 3 * k * D parts, then k counts; then C (WD)
    const FixedScale fx(fixed_shift(*amax_bits, nscale));
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int kd = k * D;
    unsigned* a = acc_sm + (size_t)wib * (3 * kd + k);
    unsigned* cntw = a + 3 * kd;
    // C with rows of 8 floats (zero past D), 16-byte aligned: two vector reads per row
    const size_t coff = (((size_t)(blockDim.x >> 5) * (3 * kd + k)) + 3) & ~(size_t)3;
    float4* Cs = reinterpret_cast<float4*>(acc_sm + coff);
    if (WD) {
        for (int e = threadIdx.x; e < k * 8; e += blockDim.x) {
            const int j = e >> 3, l = e & 7;
            reinterpret_cast<float*>(Cs)[e] = l < D ? C[j * D + l] : 0.0f;
        }
        __syncthreads();
    }
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c0 = w0 * AS_CHUNK; c0 < n; c0 += nw * AS_CHUNK) {
        for (int e = lane; e < 3 * kd + k; e += 32) a[e] = 0u;
        __syncwarp();
        const int64_t c1 = min(n, c0 + AS_CHUNK);
        for (int64_t base = c0; base < c1; base += 32) {
            const int64_t i = base + lane;
            const bool valid = i < c1;
            const int j = valid ? labels[i] : -1;
            float xr[D];
#pragma unroll
            for (int l = 0; l < D; l++) xr[l] = valid ? X[i * D + l] : 0.0f;
            if (WD && valid) md[i] = df_value(df_small4<D>(xr, Cs[2 * j], D > 4 ? Cs[2 * j + 1] : make_float4(0.f, 0.f, 0.f, 0.f)));
            unsigned v[3 * D + 1];  // true (unbiased) parts modulo 2^32, then the row count
#pragma unroll
            for (int l = 0; l < D; l++) {
                unsigned b2 = FixedScale::kBias, b1 = FixedScale::kBias, b0 = FixedScale::kBias;
                if (valid) fx.split(xr[l], b2, b1, b0);
                v[3 * l + 0] = b2 - FixedScale::kBias;
                v[3 * l + 1] = b1 - FixedScale::kBias;
                v[3 * l + 2] = b0 - FixedScale::kBias;
            }
            v[3 * D] = 1u;
            const int jp = __shfl_up_sync(0xffffffffu, j, 1);
            const bool head = lane == 0 || j != jp;
            bool f = head;  // segment flag of the scan
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const bool fu = __shfl_up_sync(0xffffffffu, f, off);
                const bool take = lane >= off && !f;
#pragma unroll
                for (int t = 0; t <= 3 * D; t++) {
                    const unsigned u = __shfl_up_sync(0xffffffffu, v[t], off);
                    if (take) v[t] += u;
                }
                if (take) f = fu;
            }
            const bool next_head = __shfl_down_sync(0xffffffffu, head, 1);
            const bool tail = lane == 31 || next_head;
            if (valid && tail) {
                unsigned* aj = a + 3 * j * D;
#pragma unroll
                for (int t = 0; t < 3 * D; t++) atomicAdd(&aj[t], v[t]);
                atomicAdd(&cntw[j], v[3 * D]);
            }
        }
        __syncwarp();
        for (int e = lane; e < kd; e += 32) {
            const long long s64 = FixedScale::combine(a[3 * e + 0], a[3 * e + 1], a[3 * e + 2], 0u);
            if (s64) atomicAdd(reinterpret_cast<unsigned long long*>(&sums[e]), (unsigned long long)s64);
        }
        for (int jj = lane; jj < k; jj += 32)
            if (cntw[jj]) atomicAdd(reinterpret_cast<unsigned long long*>(&counts[jj]), (unsigned long long)cntw[jj]);
        __syncwarp();
    }
}

// ---- the winner's distance on its own (rows in natural order) ------------
// min_dist[i] = ||x_i - c_label(i)||^2 to binary64 accuracy, by the same
// arithmetic as the fused centre-sum passes above (df.cuh), so an assignment
// alone and an assignment followed by the centre update give the same bits.
// R rows per lane and pass (R <= LPR), G = 32 / LPR rows per load.
template <int NV4, int LPR, bool VEC>
__global__ void __launch_bounds__(256) k_winner_dist(const float* __restrict__ X, int64_t n, int d,
                                                     const float* __restrict__ C, const int32_t* __restrict__ labels,
                                                     double* __restrict__ md) {
    constexpr int G = 32 / LPR;
    constexpr int R = NV4 == 4 ? 2 : 4;  // 4 rows per pass: measured faster than 8 (occupancy)
    constexpr int STEP = R * G;
    static_assert(R <= LPR, "rows per lane exceed the lanes of a row");
    const int lane = threadIdx.x & 31, sub = lane / LPR, cl = lane % LPR;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = (d + 3) >> 2;
    for (int64_t base = w0 * STEP; base < n; base += nw * STEP) {
        const int jl = (lane < STEP && base + lane < n) ? labels[base + lane] : 0;
        float4 xv[R][NV4], cv[R][NV4];
#pragma unroll
        for (int b = 0; b < R; b++) {
            const int64_t row = base + b * G + sub;
            const int j = __shfl_sync(0xffffffffu, jl, b * G + sub);
#pragma unroll
            for (int u = 0; u < NV4; u++) {
                const int cidx = cl + LPR * u;
                const bool ok = row < n && cidx < d4;
                if (VEC) {
                    xv[b][u] = ok ? reinterpret_cast<const float4*>(X + row * d)[cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
                    cv[b][u] = ok ? reinterpret_cast<const float4*>(C + (int64_t)j * d)[cidx]
                                  : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    float xe[4], ce[4];
#pragma unroll
                    for (int t = 0; t < 4; t++) {
                        const int l = 4 * cidx + t;
                        xe[t] = (ok && l < d) ? X[row * d + l] : 0.0f;
                        ce[t] = (ok && l < d) ? C[(int64_t)j * d + l] : 0.0f;
                    }
                    xv[b][u] = make_float4(xe[0], xe[1], xe[2], xe[3]);
                    cv[b][u] = make_float4(ce[0], ce[1], ce[2], ce[3]);
                }
            }
        }
        DF part[R];
#pragma unroll
        for (int b = 0; b < R; b++) part[b] = df_lane<NV4>(xv[b], cv[b]);
        int rs;
        const DF r = df_rows<R, LPR>(part, cl, rs);
        const int64_t row = base + rs * G + sub;
        if ((cl & (LPR / R - 1)) == 0 && row < n) md[row] = df_value(r);
    }
}

// Rows of D <= 8 coordinates: one thread per row.
template <int D>
__global__ void __launch_bounds__(256) k_winner_small(const float* __restrict__ X, int64_t n,
                                                      const float* __restrict__ C, const int32_t* __restrict__ labels,
                                                      double* __restrict__ md) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = labels[i];
        float xr[D];
#pragma unroll
        for (int l = 0; l < D; l++) xr[l] = X[i * D + l];
        md[i] = df_value(df_small<D>(xr, C + (int64_t)j * D));
    }
}

cudaError_t launch_winner_dist(const float* X, int64_t n, int d, const float* C, const int32_t* labels, double* md,
                               int num_sms, cudaStream_t st) {
    if (n < 1) return cudaSuccess;
    if (d <= 8) {
        const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
        switch (d) {
#define KM_WS(DD) \
    case DD: k_winner_small<DD><<<blocks, 256, 0, st>>>(X, n, C, labels, md); break;
            KM_WS(1) KM_WS(2) KM_WS(3) KM_WS(4) KM_WS(5) KM_WS(6) KM_WS(7) KM_WS(8)
#undef KM_WS
        }
        return cudaGetLastError();
    }
    const bool vec = d % 4 == 0 && ((uintptr_t)X % 16) == 0 && ((uintptr_t)C % 16) == 0;
    const int lpr = df_lpr(d), nv4 = df_nv4(d);
    const void* fn = nullptr;
    void (*kern)(const float*, int64_t, int, const float*, const int32_t*, double*) = nullptr;
#define KM_WD(NV, L)                                                          \
    if (nv4 == NV && lpr == L) {                                              \
        if (vec) kern = k_winner_dist<NV, L, true>;                           \
        else kern = k_winner_dist<NV, L, false>;                              \
    }
    KM_WD(1, 8) KM_WD(1, 16) KM_WD(1, 32) KM_WD(2, 32) KM_WD(4, 32)
#undef KM_WD
    if (!kern) return cudaErrorInvalidValue;
    fn = (const void*)kern;
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
    if (e != cudaSuccess) return e;
    const int rows_per_warp_pass = (nv4 == 4 ? 2 : 4) * (32 / lpr);
    const int64_t warps_needed = (n + rows_per_warp_pass - 1) / rows_per_warp_pass;
    const unsigned blocks = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((warps_needed + 7) / 8, (int64_t)num_sms * std::max(per_sm, 1)));
    kern<<<blocks, 256, 0, st>>>(X, n, d, C, labels, md);
    return cudaGetLastError();
}

// mean = sum 2^-S / m in binary64, stored in fp32 (the working precision).
__global__ void k_means(const long long* __restrict__ sums, const long long* __restrict__ counts,
                        const unsigned* __restrict__ amax_bits, int64_t nscale, int k, int d,
                        const float* __restrict__ C_old, float* __restrict__ C_new, int64_t* counts_out) {
    const int S = fixed_shift(*amax_bits, nscale);
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / d);
        const long long m = counts[j];
        if (m > 0) {
            double s = ldexp((double)sums[e], -S);  // int64 -> binary64 rounds once (2^-53 relative)
            C_new[e] = (float)(s / (double)m);
        } else {
            C_new[e] = C_old[e];
        }
        if (e - (int64_t)j * d == 0 && counts_out) counts_out[j] = m;
    }
}

// ---- empty clusters: the rows with the largest min_dist ------------------
// KM_EMPTY_FARTHEST (reading of "automatic empty cluster reinitialisation",
// Section 6.2): the empty clusters, in ascending j, take the rows in
// decreasing order of min_dist, ties to the lowest row index, each row once.
// One cooperative launch over the resident blocks:
//   1. block 0 lists the empty clusters (E of them, ascending) and clears the
//      histograms; every block returns at once when E == 0;
//   2. radix select (eight passes of 8 bits, most significant first) of T,
//      the E-th largest min_dist bit pattern (non-negative doubles order like
//      their bits), and A, the number of rows above it;
//   3. among the rows equal to T, radix select (four passes) of the
//      (E - A)-th smallest row index I;
//   4. the E rows {md > T} + {md == T, index <= I} are collected, ranked by
//      (md desc, index asc) and copied into the clusters in order.
// Work is O(n) per pass whatever E is.  The blocks meet at a grid barrier
// whose every wait is bounded: on timeout the status word's timeout bit is
// set and the kernel winds down.
struct EmptySel {
    unsigned bar_count, bar_gen;  // grid barrier
    int nempty, ncollected;
    unsigned hist[12][256];       // 8 passes on the distance bits, 4 on the row index
};
size_t empty_select_bytes(int k) {
    return ((sizeof(EmptySel) + 255) & ~(size_t)255) + (size_t)k * (sizeof(int) + 16 + sizeof(int));
}

KM_DEV bool grid_barrier(EmptySel* es, unsigned nblocks, unsigned* status) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &es->bar_gen;
        const unsigned g = *vgen;
        __threadfence();
        if (atomicAdd(&es->bar_count, 1u) == nblocks - 1) {
            es->bar_count = 0;
            __threadfence();
            atomicAdd(&es->bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g) {
                __nanosleep(64);
                if (clock64() - t0 > KM_WAIT_CYCLES) {
                    atomicOr(status, KM_DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// From a pass's histogram: the digit holding the rank-th key (1-based) in the
// given direction (descending: from 255 down), the keys before that digit and
// the rank left within it.  Every thread computes the same answer.
KM_DEV void radix_pick(const unsigned* hist, bool descending, unsigned rank, unsigned& digit, unsigned& before) {
    unsigned acc = 0;
    digit = 0;
    before = 0;
    for (int t = 0; t < 256; t++) {
        const int dgt = descending ? 255 - t : t;
        const unsigned c = __ldcg(hist + dgt);  // written by other blocks' atomics
        if (acc + c >= rank) {
            digit = (unsigned)dgt;
            before = acc;
            return;
        }
        acc += c;
    }
}

// fixed_e > 0: no cluster lists; the fixed_e rows of largest min_dist go, in
// that order, to rows_out / vals_out (a shard's candidates for the empty
// clusters of a row-sharded update).
__global__ void __launch_bounds__(256) k_empty_select(const long long* __restrict__ counts, int64_t n, int k, int d,
                                                      const float* __restrict__ X, const double* __restrict__ md,
                                                      float* __restrict__ C_new, EmptySel* es,
                                                      int* __restrict__ empties, unsigned long long* __restrict__ keys,
                                                      int* __restrict__ rows, int* __restrict__ order,
                                                      unsigned* status, int fixed_e, long long* __restrict__ rows_out,
                                                      double* __restrict__ vals_out) {
    __shared__ unsigned sh[256];
    __shared__ int wsum[8];
    __shared__ int any_empty;
    const unsigned nb = gridDim.x;
    const int t = threadIdx.x;
    // 0. no empty cluster (the usual case): every block sees it in the counts
    //    and leaves at once, before any grid barrier
    if (fixed_e <= 0) {
        if (t == 0) any_empty = 0;
        __syncthreads();
        for (int j = t; j < k; j += blockDim.x)
            if (counts[j] == 0) any_empty = 1;
        __syncthreads();
        if (!any_empty) return;
    }
    // 1. the empty clusters in ascending j (block 0), histograms cleared
    if (blockIdx.x == 0) {
        for (int e = t; e < 12 * 256; e += blockDim.x) (&es->hist[0][0])[e] = 0u;
        int base = 0;
        if (fixed_e > 0) base = (int)min((int64_t)fixed_e, n);
        for (int j0 = 0; fixed_e <= 0 && j0 < k; j0 += blockDim.x) {
            const int j = j0 + t;
            const int e = (j < k && counts[j] == 0) ? 1 : 0;
            int incl = e;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, incl, o);
                if ((t & 31) >= o) incl += v;
            }
            if ((t & 31) == 31) wsum[t >> 5] = incl;
            __syncthreads();
            int pre = 0, tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
                pre += (w < (t >> 5)) ? wsum[w] : 0;
                tot += wsum[w];
            }
            if (e) empties[base + pre + incl - 1] = j;
            base += tot;
            __syncthreads();
        }
        if (t == 0) {
            es->nempty = base;
            es->ncollected = 0;
        }
    }
    if (!grid_barrier(es, nb, status)) return;
    const int E = *(volatile int*)&es->nempty;
    if (E == 0) return;
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + t, gstride = (int64_t)nb * blockDim.x;
    const unsigned long long* mdb = reinterpret_cast<const unsigned long long*>(md);
    // 2. T, the E-th largest distance pattern, and A, the rows above it
    unsigned long long prefix = 0, mask = 0;
    unsigned rank = (unsigned)E, above = 0;
    for (int pass = 0; pass < 8; pass++) {
        const int shift = 56 - 8 * pass;
        sh[t] = 0;
        __syncthreads();
        for (int64_t i = gtid; i < n; i += gstride) {
            const unsigned long long key = mdb[i];
            if ((key & mask) == prefix) atomicAdd(&sh[(key >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (sh[t]) atomicAdd(&es->hist[pass][t], sh[t]);
        if (!grid_barrier(es, nb, status)) return;
        unsigned digit, before;
        radix_pick(es->hist[pass], true, rank, digit, before);
        above += before;
        rank -= before;
        prefix |= (unsigned long long)digit << shift;
        mask |= 255ull << shift;
    }
    const unsigned long long T = prefix;
    // 3. among the rows equal to T, the rank-th smallest index I (rank = E - A)
    unsigned iprefix = 0, imask = 0;
    for (int pass = 0; pass < 4; pass++) {
        const int shift = 24 - 8 * pass;
        sh[t] = 0;
        __syncthreads();
        for (int64_t i = gtid; i < n; i += gstride) {
            if (mdb[i] == T && ((unsigned)i & imask) == iprefix) atomicAdd(&sh[((unsigned)i >> shift) & 255u], 1u);
        }
        __syncthreads();
        if (sh[t]) atomicAdd(&es->hist[8 + pass][t], sh[t]);
        if (!grid_barrier(es, nb, status)) return;
        unsigned digit, before;
        radix_pick(es->hist[8 + pass], false, rank, digit, before);
        rank -= before;
        iprefix |= digit << shift;
        imask |= 255u << shift;
    }
    const unsigned I = iprefix;
    // 4. collect the E rows, rank them, fill the clusters
    for (int64_t i = gtid; i < n; i += gstride) {
        const unsigned long long key = mdb[i];
        if (key > T || (key == T && (unsigned)i <= I)) {
            const int s = atomicAdd(&es->ncollected, 1);
            if (s < E) {
                keys[s] = key;
                rows[s] = (int)i;
            }
        }
    }
    if (!grid_barrier(es, nb, status)) return;
    // (the lists were written by other blocks: read through L2)
    for (int64_t s = gtid; s < E; s += gstride) {
        const unsigned long long ks = __ldcg(keys + s);
        const int rs = __ldcg(rows + s);
        int r = 0;
        for (int q = 0; q < E; q++) {
            const unsigned long long kq = __ldcg(keys + q);
            r += (kq > ks || (kq == ks && __ldcg(rows + q) < rs)) ? 1 : 0;
        }
        order[r] = rs;
    }
    if (!grid_barrier(es, nb, status)) return;
    if (fixed_e > 0) {
        for (int64_t r = gtid; r < E; r += gstride) {
            const int row = __ldcg(order + r);
            rows_out[r] = row;
            vals_out[r] = md[row];
        }
        return;
    }
    for (int64_t e = gtid; e < (int64_t)E * d; e += gstride) {
        const int r = (int)(e / d), l = (int)(e - (int64_t)r * d);
        C_new[(int64_t)__ldcg(empties + r) * d + l] = X[(int64_t)__ldcg(order + r) * d + l];
    }
}

// shift = max_j ||c_new_j - c_old_j||: one warp per cluster, coalesced rows,
// the maximum kept as the bit pattern of a non-negative double (ordered like
// an unsigned integer), so the result does not depend on the order.
__global__ void k_shift(int k, int d, const float* __restrict__ C_old, const float* __restrict__ C_new,
                        unsigned long long* __restrict__ shift_bits) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w0; j < k; j += nw) {
        double s = 0.0;
        for (int l = lane; l < d; l += 32) {
            const double df = (double)C_new[j * d + l] - (double)C_old[j * d + l];
            s = fma(df, df, s);
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0) atomicMax(shift_bits, (unsigned long long)__double_as_longlong(sqrt(s)));
    }
}

// Deterministic sum: fixed partition into `nparts` chunks, fixed in-block tree.
__global__ void k_sum_parts(const double* __restrict__ v, int64_t n, double* __restrict__ parts) {
    __shared__ double red[256];
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t b = (int64_t)blockIdx.x * chunk, e = min(n, b + chunk);
    double s = 0.0;
    for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) s += v[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) parts[blockIdx.x] = red[0];
}
// One warp, a fixed order: lane l adds parts l, l + 32, ... in turn, then a
// fixed butterfly (a serial sum over all parts would chain every binary64
// addition's latency).
__global__ void k_sum_final(const double* __restrict__ parts, int nparts, double* out) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int i = lane; i < nparts; i += 32) s += parts[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) *out = s;
}

cudaError_t launch_absmax(const float* X, int64_t count, unsigned* out_bits, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out_bits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    int64_t blocks = min((int64_t)152 * 8, (count + 255) / 256);
    if (blocks < 1) blocks = 1;
    k_absmax<<<(unsigned)blocks, 256, 0, st>>>(X, count, out_bits);
    return cudaGetLastError();
}

cudaError_t launch_accumulate(const float* X, int64_t n, int d, const int32_t* labels, int k,
                              const unsigned* absmax_bits, long long* sums, long long* counts, int* iscratch,
                              int32_t* perm, int num_sms, cudaStream_t st, const float* C_wd, double* md_out,
                              int* nlaunch, int64_t nscale) {
    if (nscale <= 0) nscale = n;  // the fixed-point scale of n rows (or of all shards' rows)
    // md_out: the rows' distances to their centres (C_wd) come out of the same
    // pass over X where the kernel has the row and its centre in hand, else
    // from the standalone kernel first (the same arithmetic either way)
    const bool want_wd = md_out != nullptr && C_wd != nullptr;
    int nl = 0;
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(long long) * (size_t)k * d, st);
    if (e != cudaSuccess) return e;
    if (d <= 8 && (int64_t)k * d <= AS_MAX_KD) {
        // small d: rows in order, per-warp shared accumulators (+ C for the distances)
        e = cudaMemsetAsync(counts, 0, sizeof(long long) * (size_t)k, st);
        if (e != cudaSuccess) return e;
        const size_t sm = (((size_t)8 * (3 * (size_t)k * d + k) + 3) & ~(size_t)3) * sizeof(unsigned) +
                          (want_wd ? (size_t)k * 8 * sizeof(float) : 0);
        const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms * 8, (n + 8 * AS_CHUNK - 1) / (8 * AS_CHUNK)));
        switch (d) {
#define KM_ACC(DD)                                                                                                  \
    case DD:                                                                                                        \
        if (want_wd) {                                                                                              \
            e = allow_max_smem(k_accum_small<DD, true>);                                                            \
            if (e != cudaSuccess) return e;                                                                         \
            k_accum_small<DD, true><<<(unsigned)blocks, 256, sm, st>>>(X, n, k, labels, absmax_bits, nscale, sums, counts,  \
                                                                       C_wd, md_out);                               \
        } else {                                                                                                    \
            e = allow_max_smem(k_accum_small<DD, false>);                                                           \
            if (e != cudaSuccess) return e;                                                                         \
            k_accum_small<DD, false><<<(unsigned)blocks, 256, sm, st>>>(X, n, k, labels, absmax_bits, nscale, sums, counts, \
                                                                        nullptr, nullptr);                          \
        }                                                                                                           \
        break;
            KM_ACC(1) KM_ACC(2) KM_ACC(3) KM_ACC(4) KM_ACC(5) KM_ACC(6) KM_ACC(7) KM_ACC(8)
#undef KM_ACC
        }
        if (nlaunch) *nlaunch = 1;
        return cudaGetLastError();
    }
    const size_t hsm = sizeof(int) * (size_t)k;
    const bool vec = d % 4 == 0 && ((uintptr_t)X % 16) == 0;
    const bool bucket = 2 * hsm <= 200 * 1024 && (d == 1 || d == 2 || d == 3 || d == 5 || (vec && d <= 512));
    // the bucket kernels of rows wider than 5 coordinates read the rows as
    // float4: they can take the distances along when C is aligned as well
    const bool fused = want_wd && bucket && d > 5 && ((uintptr_t)C_wd % 16) == 0;
    if (want_wd && !fused) {
        e = launch_winner_dist(X, n, d, C_wd, labels, md_out, num_sms, st);
        if (e != cudaSuccess) return e;
        nl++;
    }
    if (bucket) {
        int* cnt32 = iscratch;            // k
        int* off = iscratch + k;          // k + 1
        int* cursor = off + k + 1;        // k
        int* item_off = cursor + k;       // k + 1
        e = cudaMemsetAsync(cnt32, 0, sizeof(int) * (size_t)k, st);
        if (e != cudaSuccess) return e;
        const int64_t nblk = (n + SCAT_ROWS - 1) / SCAT_ROWS;
        e = allow_max_smem(k_label_hist);
        if (e != cudaSuccess) return e;
        k_label_hist<<<(unsigned)nblk, 512, hsm, st>>>(labels, n, k, cnt32);
        // persistent grid: every block resident at once (a partial second wave
        // would leave SMs idle), the items strided over the warps; work items of
        // `seg` rows, about four per resident warp (fewer, longer items mean
        // fewer atomic adds per centre coordinate)
        typedef void (*BucketFn)(const float*, int64_t, int, int, int, const int*, const int*, const int32_t*,
                                 const unsigned*, int64_t, long long*, const float*, double*);
        BucketFn bfn = nullptr;
        if (d > 5) {
#define KM_BS(NV, L) (fused ? (BucketFn)k_bucket_sum<NV, L, true> : (BucketFn)k_bucket_sum<NV, L, false>)
            bfn = d <= 32 ? KM_BS(1, 8) : d <= 64 ? KM_BS(1, 16) : d <= 128 ? KM_BS(1, 32) : d <= 256 ? KM_BS(2, 32)
                                                                                                 : KM_BS(4, 32);
#undef KM_BS
        }
        int per_sm = 8;
        if (bfn) {
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)bfn, 256, 0);
            if (e != cudaSuccess) return e;
        }
        const int64_t resident_warps = (int64_t)num_sms * std::max(per_sm, 1) * 8;
        const int seg = (int)std::min<int64_t>(SEG_MAX, std::max<int64_t>(64, n / (resident_warps * 4) / 32 * 32));
        k_bucket_scan<<<1, 1024, 0, st>>>(cnt32, k, seg, off, cursor, item_off, counts);
        e = allow_max_smem(k_bucket_scatter);
        if (e != cudaSuccess) return e;
        k_bucket_scatter<<<(unsigned)nblk, 512, 2 * hsm, st>>>(labels, n, k, cursor, perm);
        const int64_t items = n / seg + k + 1;
        const unsigned blocks =
            (unsigned)std::max<int64_t>(1, std::min<int64_t>((items * 32 + 255) / 256, (int64_t)num_sms * std::max(per_sm, 1)));
        if (d == 1) k_bucket_sum_small<1><<<blocks, 256, 0, st>>>(X, n, k, seg, off, item_off, perm, absmax_bits, nscale, sums);
        else if (d == 2) k_bucket_sum_small<2><<<blocks, 256, 0, st>>>(X, n, k, seg, off, item_off, perm, absmax_bits, nscale, sums);
        else if (d == 3) k_bucket_sum_small<3><<<blocks, 256, 0, st>>>(X, n, k, seg, off, item_off, perm, absmax_bits, nscale, sums);
        else if (d == 5) k_bucket_sum_small<5><<<blocks, 256, 0, st>>>(X, n, k, seg, off, item_off, perm, absmax_bits, nscale, sums);
        else bfn<<<blocks, 256, 0, st>>>(X, n, d, k, seg, off, item_off, perm, absmax_bits, nscale, sums, C_wd, md_out);
        if (nlaunch) *nlaunch = nl + 4;
        return cudaGetLastError();
    }
    e = cudaMemsetAsync(counts, 0, sizeof(long long) * (size_t)k, st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(long long) * ((size_t)k * d + k);
    const int64_t total = n * d;
    if (smem <= 200 * 1024) {
        e = allow_max_smem(k_accumulate<true>);
        if (e != cudaSuccess) return e;
        const int64_t blk = std::min<int64_t>((int64_t)num_sms, (total + 511) / 512);
        k_accumulate<true><<<(unsigned)std::max<int64_t>(blk, 1), 512, smem, st>>>(X, n, d, labels, k, absmax_bits,
                                                                                    nscale, sums, counts);
    } else {
        const int64_t blk = std::min<int64_t>((int64_t)num_sms * 8, (total + 511) / 512);
        k_accumulate<false><<<(unsigned)std::max<int64_t>(blk, 1), 512, 0, st>>>(X, n, d, labels, k, absmax_bits,
                                                                                  nscale, sums, counts);
    }
    if (nlaunch) *nlaunch = nl + 1;
    return cudaGetLastError();
}

cudaError_t launch_finalize(const long long* sums, const long long* counts, const unsigned* absmax_bits,
                            int64_t n, int k, int d, const float* C_old, int empty_policy, const float* X,
                            const double* min_dist, float* C_new, int64_t* counts_out, double* shift,
                            void* esel, unsigned* status, int num_sms, cudaStream_t st, int* nlaunch, int64_t nscale) {
    int nl = 0;
    int64_t kd = (int64_t)k * d;
    int64_t blocks = min((int64_t)1024, (kd + 255) / 256);
    k_means<<<(unsigned)blocks, 256, 0, st>>>(sums, counts, absmax_bits, nscale > 0 ? nscale : n, k, d, C_old, C_new,
                                               counts_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    nl++;
    if (empty_policy == 1 && min_dist != nullptr) {
        EmptySel* es = reinterpret_cast<EmptySel*>(esel);
        char* tail = reinterpret_cast<char*>(esel) + ((sizeof(EmptySel) + 255) & ~(size_t)255);
        int* empties = reinterpret_cast<int*>(tail);
        unsigned long long* keys = reinterpret_cast<unsigned long long*>(empties + k + (k & 1));
        int* rows = reinterpret_cast<int*>(keys + k);
        int* order = rows + k;
        e = cudaMemsetAsync(es, 0, 2 * sizeof(unsigned), st);
        if (e != cudaSuccess) return e;
        // one block per SM: every block resident at once (cooperative launch)
        int per_sm = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_empty_select, 256, 0);
        if (e != cudaSuccess) return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        int fixed_e = 0;
        long long* rows_out = nullptr;
        double* vals_out = nullptr;
        void* args[] = {(void*)&counts, (void*)&n,     (void*)&k,     (void*)&d,      (void*)&X,
                        (void*)&min_dist, (void*)&C_new, (void*)&es,   (void*)&empties, (void*)&keys,
                        (void*)&rows,   (void*)&order, (void*)&status, (void*)&fixed_e, (void*)&rows_out,
                        (void*)&vals_out};
        e = cudaLaunchCooperativeKernel((const void*)k_empty_select, dim3((unsigned)num_sms), dim3(256), args, 0, st);
        if (e != cudaSuccess) return e;
        nl++;
    }
    if (shift) {  // null: the caller does not want the shift
        e = cudaMemsetAsync(shift, 0, sizeof(double), st);
        if (e != cudaSuccess) return e;
        const int64_t sblocks = std::min<int64_t>(((int64_t)k * 32 + 255) / 256, (int64_t)num_sms * 8);
        k_shift<<<(unsigned)std::max<int64_t>(sblocks, 1), 256, 0, st>>>(k, d, C_old, C_new,
                                                                       reinterpret_cast<unsigned long long*>(shift));
        nl++;
    }
    if (nlaunch) *nlaunch = nl;
    return cudaGetLastError();
}

cudaError_t launch_farthest_rows(const double* min_dist, int64_t n, int e, long long* rows_out, double* vals_out,
                                 void* esel, unsigned* status, int num_sms, cudaStream_t st) {
    EmptySel* es = reinterpret_cast<EmptySel*>(esel);
    char* tail = reinterpret_cast<char*>(esel) + ((sizeof(EmptySel) + 255) & ~(size_t)255);
    int* empties = reinterpret_cast<int*>(tail);
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(empties + e + (e & 1));
    int* rows = reinterpret_cast<int*>(keys + e);
    int* order = rows + e;
    cudaError_t err = cudaMemsetAsync(es, 0, 2 * sizeof(unsigned), st);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_empty_select, 256, 0);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long* counts = nullptr;
    int k = e, d = 0;
    const float* X = nullptr;
    float* C_new = nullptr;
    void* args[] = {(void*)&counts, (void*)&n,     (void*)&k,     (void*)&d,  (void*)&X,    (void*)&min_dist,
                    (void*)&C_new,  (void*)&es,    (void*)&empties, (void*)&keys, (void*)&rows, (void*)&order,
                    (void*)&status, (void*)&e,     (void*)&rows_out, (void*)&vals_out};
    return cudaLaunchCooperativeKernel((const void*)k_empty_select, dim3((unsigned)num_sms), dim3(256), args, 0, st);
}

cudaError_t launch_sum_f64(const double* v, int64_t n, double* partials, int nparts, double* out, cudaStream_t st) {
    k_sum_parts<<<nparts, 256, 0, st>>>(v, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_final<<<1, 32, 0, st>>>(partials, nparts, out);
    return cudaGetLastError();
}

}  // namespace km
