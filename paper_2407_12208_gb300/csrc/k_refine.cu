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
#include "common.cuh"
#include "internal.h"

namespace km {

__global__ void k_refine(const float* __restrict__ X, const float* __restrict__ C, const TcArgs a,
                         int32_t* __restrict__ labels, double* __restrict__ min_dist, int32_t* __restrict__ ovf_list) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d = a.d;
    const TestParams tp = a.tp;
    unsigned long long ev32 = 0, ev64 = 0, amb = 0, ovf_rows = 0;
    for (int64_t row = warp; row < a.n; row += nw) {
        // the two epilogue groups of the screening kernel each left a list
        const int4 i0 = a.rowinfo[row * 2], i1 = a.rowinfo[row * 2 + 1];
        const int cnt = i0.x + i1.x;
        if ((i0.y | i1.y) || cnt > 32) {  // overflowed: whole-row direct evaluation elsewhere
            if (lane == 0) {
                int slot = atomicAdd(&a.cnt->ovf_count, 1);
                ovf_list[slot] = (int32_t)row;
                ovf_rows++;
            }
            continue;
        }
        const float4 xs = a.xstat[row];
        const float a1 = 2.0f * xs.w, a2 = 2.0f * xs.z, a3 = tp.kacc * xs.z;
        // candidate r lives in lane r
        int j = 0x7fffffff;
        float lo = INFINITY, hi = INFINITY;
        if (lane < cnt) {
            const size_t slot = (lane < i0.x) ? ((size_t)row * 2) * a.L + lane
                                              : ((size_t)row * 2 + 1) * a.L + (lane - i0.x);
            const uint32_t c = a.cand[slot];
            j = (int)(c >> 16);
            // the entry holds d^ truncated toward zero to 8 significant bits
            const float t = __uint_as_float(c << 16);
            const float dl = t - fabsf(t) * (1.0f / 128.0f);
            const float du = t + fabsf(t) * (1.0f / 128.0f);
            const float4 cs = a.cstat[j];
            const float B = (a1 * cs.y + a2 * cs.w + a3 * cs.z + tp.kn * (xs.x + cs.x)) * tp.bsafe;
            lo = dl - B;
            hi = du + B;
        }
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
