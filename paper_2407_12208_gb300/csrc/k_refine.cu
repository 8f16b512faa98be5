// k_refine.cu -- recompute by the direct formula (Section 4.3: from the
// ORIGINAL data, Eq. (fallback-rule-mp)) and certified argmin.
//
// Per row (one warp), from the candidates the screening kernel kept:
//  1. every candidate j has |d^_j - d_j| <= B_ij (the bound behind the
//     reliability test), so only those with d^_j - B_ij <= min_l (d^_l + B_il)
//     can be the nearest centre;
//  2. those are evaluated by Eq. (dist-direct) in fp32 (lanes over the
//     coordinates, shuffle reduction); Theorem 4.1 puts each true value in
//     [v (1 - g), v (1 + g)], g = gamma_{d+2}(2^-24);
//  3. if more than one fp32 interval can still hold the minimum, those
//     candidates are evaluated in binary64 (products and sums rounded
//     separately, coordinates in order: the oracle's own arithmetic) and the
//     smallest wins, lowest index on ties.
// The winner's direct value is min_dist.  Rows whose candidate list
// overflowed are listed for the full-row direct kernel instead.
//
// k_patch_flagged: binary64 direct values for the flagged pairs of the
// distance matrix (Alg. 2's fallback branch).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

// Candidate r of the row (r < cnt0 + cnt1) is held by lane r.
KM_DEV void row_candidates(const TcArgs& a, int64_t row, int lane, int4 i0, int4 i1, int& j, float& lo, float& hi,
                           const float4& xs) {
    const TestParams& tp = a.tp;
    const int cnt0 = i0.x, cnt = i0.x + i1.x;
    const uint32_t c0 = (lane < a.L) ? a.cand[((size_t)row * 2) * a.L + lane] : 0u;
    const uint32_t c1 = (lane < a.L) ? a.cand[((size_t)row * 2 + 1) * a.L + lane] : 0u;
    const uint32_t c1s = __shfl_sync(0xffffffffu, c1, (lane - cnt0) & 31);
    const uint32_t c = (lane < cnt0) ? c0 : c1s;
    j = 0x7fffffff;
    lo = INFINITY;
    hi = INFINITY;
    if (lane < cnt) {
        j = (int)(c >> 16);
        // the entry holds d^ truncated toward zero to 8 significant bits
        const float t = __uint_as_float(c << 16);
        const float dl = t - fabsf(t) * (1.0f / 128.0f);
        const float du = t + fabsf(t) * (1.0f / 128.0f);
        const float a1 = 2.0f * xs.w, a2 = 2.0f * xs.z, a3 = tp.kacc * xs.z;
        const float4 cs = a.cstat[j];
        const float B = (a1 * cs.y + a2 * cs.w + a3 * cs.z + tp.kn * (xs.x + cs.x)) * tp.bsafe;
        lo = dl - B;
        hi = du + B;
    }
}

// Vector path: d % 4 == 0 and d <= 256, each lane holds up to two float4 of x.
template <int NV>
__global__ void __launch_bounds__(256) k_refine_vec(const float* __restrict__ X, const float* __restrict__ C,
                                                    const TcArgs a, int32_t* __restrict__ labels,
                                                    double* __restrict__ min_dist, int32_t* __restrict__ ovf_list) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d = a.d, d4 = d >> 2;
    const TestParams tp = a.tp;
    unsigned long long ev32 = 0, ev64 = 0, amb = 0, ovf_rows = 0;
    for (int64_t row = warp; row < a.n; row += nw) {
        // round 1: everything that does not depend on anything else
        const int4 i0 = a.rowinfo[row * 2], i1 = a.rowinfo[row * 2 + 1];
        const float4 xs = a.xstat[row];
        const float4* x4 = reinterpret_cast<const float4*>(X + row * d);
        float4 xv[NV];
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = lane + 32 * u;
            xv[u] = (c < d4) ? x4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int cnt = i0.x + i1.x;
        if ((i0.y | i1.y) || cnt > 32) {  // overflowed: whole-row direct evaluation elsewhere
            if (lane == 0) {
                int slot = atomicAdd(&a.cnt->ovf_count, 1);
                ovf_list[slot] = (int32_t)row;
                ovf_rows++;
            }
            continue;
        }
        // round 2: the candidates and their column statistics
        int j;
        float lo, hi;
        row_candidates(a, row, lane, i0, i1, j, lo, hi, xs);
        float U = hi;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) U = fminf(U, __shfl_xor_sync(0xffffffffu, U, off));
        const unsigned surv = __ballot_sync(0xffffffffu, lane < cnt && lo <= U);
        const int nsurv = __popc(surv);
        // round 3: fp32 direct values of the survivors, eight centre rows in flight at a time
        float v32 = INFINITY;
        for (unsigned mrem = surv; mrem;) {
            int rs[8];
            float4 cv[8][NV];
            int nb = 0;
#pragma unroll
            for (int b = 0; b < 8; b++) {
                rs[b] = -1;
                if (mrem) {
                    const int r = __ffs(mrem) - 1;
                    mrem &= mrem - 1;
                    rs[b] = r;
                    nb++;
                    const int jr = __shfl_sync(0xffffffffu, j, r);
                    const float4* c4 = reinterpret_cast<const float4*>(C + (int64_t)jr * d);
#pragma unroll
                    for (int u = 0; u < NV; u++) {
                        const int c = lane + 32 * u;
                        cv[b][u] = (c < d4) ? c4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < 8; b++) {
                if (rs[b] < 0) break;
                float sacc = 0.0f;
#pragma unroll
                for (int u = 0; u < NV; u++) {
                    const float t0 = xv[u].x - cv[b][u].x, t1 = xv[u].y - cv[b][u].y;
                    const float t2 = xv[u].z - cv[b][u].z, t3 = xv[u].w - cv[b][u].w;
                    sacc = fmaf(t0, t0, sacc);
                    sacc = fmaf(t1, t1, sacc);
                    sacc = fmaf(t2, t2, sacc);
                    sacc = fmaf(t3, t3, sacc);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, off);
                if (lane == rs[b]) v32 = sacc;
            }
            (void)nb;
        }
        ev32 += (unsigned long long)nsurv;
        int win_j;
        double win_d;
        const bool in = (surv >> lane) & 1u;
        if (nsurv == 1) {
            const int r = __ffs(surv) - 1;
            win_j = __shfl_sync(0xffffffffu, j, r);
            win_d = (double)__shfl_sync(0xffffffffu, v32, r);
        } else {
            amb++;
            const float g = tp.gamma32;
            const float up = in ? v32 * (1.0f + g) : INFINITY;
            float U2 = up;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) U2 = fminf(U2, __shfl_xor_sync(0xffffffffu, U2, off));
            const unsigned s2 = __ballot_sync(0xffffffffu, in && v32 * (1.0f - g) <= U2);
            if (__popc(s2) == 1) {
                const int r = __ffs(s2) - 1;
                win_j = __shfl_sync(0xffffffffu, j, r);
                win_d = (double)__shfl_sync(0xffffffffu, v32, r);
            } else {
                // binary64, the oracle's arithmetic (products and sums rounded separately)
                double v64 = INFINITY;
                int jj = 0x7fffffff;
                if ((s2 >> lane) & 1u) {
                    const float* x = X + row * d;
                    const float* c = C + (int64_t)j * d;
                    double sacc = 0.0;
                    for (int l = 0; l < d; l++) {
                        const double t = __dsub_rn((double)x[l], (double)c[l]);
                        sacc = __dadd_rn(sacc, __dmul_rn(t, t));
                    }
                    v64 = sacc;
                    jj = j;
                }
                ev64 += (unsigned long long)__popc(s2);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, v64, off);
                    const int oj = __shfl_xor_sync(0xffffffffu, jj, off);
                    if (ov < v64 || (ov == v64 && oj < jj)) { v64 = ov; jj = oj; }
                }
                win_j = jj;
                win_d = v64;
            }
        }
        if (lane == 0) {
            labels[row] = win_j;
            min_dist[row] = win_d;
        }
    }
    if (lane == 0) {
        if (ev32) atomicAdd(&a.cnt->fp32_evals, ev32);
        if (ev64) atomicAdd(&a.cnt->fp64_evals, ev64);
        if (amb) atomicAdd(&a.cnt->amb_rows, amb);
        if (ovf_rows) atomicAdd(&a.cnt->ovf_rows, ovf_rows);
    }
}


// Group path: 8 lanes per row, 4 rows per warp (d % 4 == 0, d <= 256): the
// reductions take 3 shuffle levels and serve 4 rows at once.  NV float4 of x
// per lane (x holds d/4 float4: lane l of the group takes l, l+8, ...).
template <int NV>
__global__ void __launch_bounds__(256) k_refine_g8(const float* __restrict__ X, const float* __restrict__ C,
                                                   const TcArgs a, int32_t* __restrict__ labels,
                                                   double* __restrict__ min_dist, int32_t* __restrict__ ovf_list) {
    constexpr int NS = 6;  // candidate slots per lane (48 per row at most)
    const int lane = threadIdx.x & 31, sl = lane & 7, gbase = lane & ~7;
    const unsigned gmask = 0xFFu << gbase;
    const int64_t gid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4 + (lane >> 3);
    const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * 4;
    const int d = a.d, d4 = d >> 2;
    const TestParams tp = a.tp;
    unsigned long long ev32 = 0, ev64 = 0, amb = 0, ovf_rows = 0;
    for (int64_t row = gid; row < a.n; row += ngroups) {
        const int4 i0 = a.rowinfo[row * 2], i1 = a.rowinfo[row * 2 + 1];
        const float4 xs = a.xstat[row];
        const float4* x4 = reinterpret_cast<const float4*>(X + row * d);
        float4 xv[NV];
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = sl + 8 * u;
            xv[u] = (c < d4) ? x4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const int cnt0 = i0.x, cnt = i0.x + i1.x;
        if ((i0.y | i1.y) || cnt > 8 * NS) {  // overflowed: whole-row direct evaluation elsewhere
            if (sl == 0) {
                int slot = atomicAdd(&a.cnt->ovf_count, 1);
                ovf_list[slot] = (int32_t)row;
                ovf_rows++;
            }
            continue;
        }
        const float a1 = 2.0f * xs.w, a2 = 2.0f * xs.z, a3 = tp.kacc * xs.z;
        int jr[NS];
        float lor[NS], hir[NS];
        float myU = INFINITY;
#pragma unroll
        for (int r = 0; r < NS; r++) {
            const int sidx = sl + 8 * r;
            jr[r] = 0x7fffffff;
            lor[r] = INFINITY;
            hir[r] = INFINITY;
            if (sidx < cnt) {
                const uint32_t c = (sidx < cnt0) ? a.cand[((size_t)row * 2) * a.L + sidx]
                                                 : a.cand[((size_t)row * 2 + 1) * a.L + (sidx - cnt0)];
                const int j = (int)(c >> 16);
                // the entry holds d^ truncated toward zero to 8 significant bits
                const float t = __uint_as_float(c << 16);
                const float4 cs = a.cstat[j];
                const float B = (a1 * cs.y + a2 * cs.w + a3 * cs.z + tp.kn * (xs.x + cs.x)) * tp.bsafe;
                jr[r] = j;
                lor[r] = t - fabsf(t) * (1.0f / 128.0f) - B;
                hir[r] = t + fabsf(t) * (1.0f / 128.0f) + B;
                myU = fminf(myU, hir[r]);
            }
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) myU = fminf(myU, __shfl_xor_sync(gmask, myU, off));
        const float U = myU;
        // fp32 direct values of the surviving candidates
        float v32[NS];
        int nsurv = 0;
#pragma unroll
        for (int r = 0; r < NS; r++) {
            v32[r] = INFINITY;
            unsigned b = (__ballot_sync(gmask, lor[r] <= U && jr[r] != 0x7fffffff) >> gbase) & 0xFFu;
            nsurv += __popc(b);
            while (b) {
                const int owner = __ffs(b) - 1;
                b &= b - 1;
                const int j = __shfl_sync(gmask, jr[r], gbase + owner);
                const float4* c4 = reinterpret_cast<const float4*>(C + (int64_t)j * d);
                float acc = 0.0f;
#pragma unroll
                for (int u = 0; u < NV; u++) {
                    const int c = sl + 8 * u;
                    const float4 cv = (c < d4) ? c4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float t0 = xv[u].x - cv.x, t1 = xv[u].y - cv.y, t2 = xv[u].z - cv.z, t3 = xv[u].w - cv.w;
                    acc = fmaf(t0, t0, acc);
                    acc = fmaf(t1, t1, acc);
                    acc = fmaf(t2, t2, acc);
                    acc = fmaf(t3, t3, acc);
                }
#pragma unroll
                for (int off = 4; off > 0; off >>= 1) acc += __shfl_xor_sync(gmask, acc, off);
                if (sl == owner) v32[r] = acc;
            }
        }
        ev32 += (sl == 0) ? (unsigned long long)nsurv : 0ull;
        // certification by Theorem 4.1's intervals, binary64 where still open
        const float g = tp.gamma32;
        float up = INFINITY;
#pragma unroll
        for (int r = 0; r < NS; r++) up = fminf(up, v32[r] * (1.0f + g));
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) up = fminf(up, __shfl_xor_sync(gmask, up, off));
        unsigned s2 = 0;
#pragma unroll
        for (int r = 0; r < NS; r++) s2 |= (v32[r] != INFINITY && v32[r] * (1.0f - g) <= up) ? (1u << r) : 0u;
        int n2 = __popc(s2);
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) n2 += __shfl_xor_sync(gmask, n2, off);
        double best = INFINITY;
        int bj = 0x7fffffff;
        if (n2 == 1) {
            if (s2) {
                const int r = __ffs(s2) - 1;
                float vv = v32[0];
                int jj = jr[0];
#pragma unroll
                for (int q = 1; q < NS; q++)
                    if (q == r) { vv = v32[q]; jj = jr[q]; }
                best = (double)vv;
                bj = jj;
            }
        } else {
            if (sl == 0) amb++;
            const float* x = X + row * d;
#pragma unroll
            for (int r = 0; r < NS; r++) {
                if ((s2 >> r) & 1u) {
                    const float* c = C + (int64_t)jr[r] * d;
                    double sacc = 0.0;
                    for (int l = 0; l < d; l++) {
                        const double t = __dsub_rn((double)x[l], (double)c[l]);
                        sacc = __dadd_rn(sacc, __dmul_rn(t, t));
                    }
                    ev64++;
                    if (sacc < best || (sacc == best && jr[r] < bj)) { best = sacc; bj = jr[r]; }
                }
            }
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(gmask, best, off);
            const int oj = __shfl_xor_sync(gmask, bj, off);
            if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        if (sl == 0) {
            labels[row] = bj;
            min_dist[row] = best;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev32 += __shfl_xor_sync(0xffffffffu, ev32, off);
        ev64 += __shfl_xor_sync(0xffffffffu, ev64, off);
        amb += __shfl_xor_sync(0xffffffffu, amb, off);
        ovf_rows += __shfl_xor_sync(0xffffffffu, ovf_rows, off);
    }
    if (lane == 0) {
        if (ev32) atomicAdd(&a.cnt->fp32_evals, ev32);
        if (ev64) atomicAdd(&a.cnt->fp64_evals, ev64);
        if (amb) atomicAdd(&a.cnt->amb_rows, amb);
        if (ovf_rows) atomicAdd(&a.cnt->ovf_rows, ovf_rows);
    }
}

// General path (any d): warp per row, lanes over the coordinates.
__global__ void k_refine(const float* __restrict__ X, const float* __restrict__ C, const TcArgs a,
                         int32_t* __restrict__ labels, double* __restrict__ min_dist, int32_t* __restrict__ ovf_list) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d = a.d;
    const TestParams tp = a.tp;
    unsigned long long ev32 = 0, ev64 = 0, amb = 0, ovf_rows = 0;
    for (int64_t row = warp; row < a.n; row += nw) {
        const int4 i0 = a.rowinfo[row * 2], i1 = a.rowinfo[row * 2 + 1];
        const int cnt = i0.x + i1.x;
        if ((i0.y | i1.y) || cnt > 32) {
            if (lane == 0) {
                int slot = atomicAdd(&a.cnt->ovf_count, 1);
                ovf_list[slot] = (int32_t)row;
                ovf_rows++;
            }
            continue;
        }
        const float4 xs = a.xstat[row];
        int j;
        float lo, hi;
        row_candidates(a, row, lane, i0, i1, j, lo, hi, xs);
        float U = hi;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) U = fminf(U, __shfl_xor_sync(0xffffffffu, U, off));
        unsigned surv = __ballot_sync(0xffffffffu, lane < cnt && lo <= U);
        const int nsurv = __popc(surv);
        // fp32 direct values of the survivors (warp-cooperative)
        float v32 = INFINITY;
        const float* x = X + row * d;
        for (unsigned m = surv; m; m &= m - 1) {
            const int r = __ffs(m) - 1;
            const int jr = __shfl_sync(0xffffffffu, j, r);
            const float* c = C + (int64_t)jr * d;
            float s = 0.0f;
            for (int l = lane; l < d; l += 32) {
                const float t = x[l] - c[l];
                s = fmaf(t, t, s);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == r) v32 = s;
        }
        ev32 += (unsigned long long)nsurv;
        int win_j;
        double win_d;
        const bool in = (surv >> lane) & 1u;
        if (nsurv == 1) {
            const int r = __ffs(surv) - 1;
            win_j = __shfl_sync(0xffffffffu, j, r);
            win_d = (double)__shfl_sync(0xffffffffu, v32, r);
        } else {
            amb++;
            const float g = tp.gamma32;
            const float up = in ? v32 * (1.0f + g) : INFINITY;
            float U2 = up;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) U2 = fminf(U2, __shfl_xor_sync(0xffffffffu, U2, off));
            const unsigned s2 = __ballot_sync(0xffffffffu, in && v32 * (1.0f - g) <= U2);
            if (__popc(s2) == 1) {
                const int r = __ffs(s2) - 1;
                win_j = __shfl_sync(0xffffffffu, j, r);
                win_d = (double)__shfl_sync(0xffffffffu, v32, r);
            } else {
                double v64 = INFINITY;
                int jj = 0x7fffffff;
                if ((s2 >> lane) & 1u) {
                    const float* c = C + (int64_t)j * d;
                    double s = 0.0;
                    for (int l = 0; l < d; l++) {
                        const double t = __dsub_rn((double)x[l], (double)c[l]);
                        s = __dadd_rn(s, __dmul_rn(t, t));
                    }
                    v64 = s;
                    jj = j;
                }
                ev64 += (unsigned long long)__popc(s2);
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    const double ov = __shfl_xor_sync(0xffffffffu, v64, off);
                    const int oj = __shfl_xor_sync(0xffffffffu, jj, off);
                    if (ov < v64 || (ov == v64 && oj < jj)) { v64 = ov; jj = oj; }
                }
                win_j = jj;
                win_d = v64;
            }
        }
        if (lane == 0) {
            labels[row] = win_j;
            min_dist[row] = win_d;
        }
    }
    if (lane == 0) {
        if (ev32) atomicAdd(&a.cnt->fp32_evals, ev32);
        if (ev64) atomicAdd(&a.cnt->fp64_evals, ev64);
        if (amb) atomicAdd(&a.cnt->amb_rows, amb);
        if (ovf_rows) atomicAdd(&a.cnt->ovf_rows, ovf_rows);
    }
}

__global__ void k_patch_flagged(const float* __restrict__ X, const float* __restrict__ C, int k, int d,
                                const int2* __restrict__ queue, const unsigned long long* __restrict__ qlen,
                                int64_t cap, float* __restrict__ D, DevCounters* cnt) {
    const int64_t len = min((int64_t)*qlen, cap);
    unsigned long long ev = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < len; t += (int64_t)gridDim.x * blockDim.x) {
        const int2 pr = queue[t];
        const float* x = X + (int64_t)pr.x * d;
        const float* c = C + (int64_t)pr.y * d;
        double s = 0.0;
        for (int l = 0; l < d; l++) {
            const double u = __dsub_rn((double)x[l], (double)c[l]);
            s = __dadd_rn(s, __dmul_rn(u, u));
        }
        D[(int64_t)pr.x * k + pr.y] = (float)s;
        ev++;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, off);
    if ((threadIdx.x & 31) == 0 && ev) atomicAdd(&cnt->fp64_evals, ev);
}

cudaError_t launch_refine(const float* X, const float* C, const TcArgs& a, int32_t* labels, double* min_dist,
                          int32_t* ovf_list, int32_t* /*amb_list*/, int num_sms, cudaStream_t st) {
    int64_t warps = std::min<int64_t>(a.n, (int64_t)num_sms * 64);
    int64_t blocks = (warps * 32 + 255) / 256;
    if (blocks < 1) blocks = 1;
    const bool vec = (a.d % 4 == 0) && a.d <= 256 && ((uintptr_t)X % 16 == 0) && ((uintptr_t)C % 16 == 0);
    if (vec && a.d <= 128)
        k_refine_g8<4><<<(unsigned)blocks, 256, 0, st>>>(X, C, a, labels, min_dist, ovf_list);
    else if (vec)
        k_refine_g8<8><<<(unsigned)blocks, 256, 0, st>>>(X, C, a, labels, min_dist, ovf_list);
    else
        k_refine<<<(unsigned)blocks, 256, 0, st>>>(X, C, a, labels, min_dist, ovf_list);
    return cudaGetLastError();
}

cudaError_t launch_patch_flagged(const float* X, const float* C, int k, int d, const int2* queue,
                                 const unsigned long long* qlen, int64_t cap, float* D, DevCounters* cnt, int num_sms,
                                 cudaStream_t st) {
    k_patch_flagged<<<num_sms * 8, 256, 0, st>>>(X, C, k, d, queue, qlen, cap, D, cnt);
    return cudaGetLastError();
}

}  // namespace km
