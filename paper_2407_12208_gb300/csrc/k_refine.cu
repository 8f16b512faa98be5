// k_refine.cu -- recompute by the direct formula (Section 4.3: from the
// ORIGINAL data, Eq. (fallback-rule-mp)) and certified argmin.
//
// The screening kernel leaves, per row, lists of candidates, from which only
// the j with d^_j <= d^_min + 2 B_max can still be the nearest centre, where
// |d^_j - d_j| <= B_ij is the bound behind the reliability test (so no other
// centre can win).  Those become a flat list of (row, j) pairs, each row's pairs
// contiguous.
//  0. k_cand_select: the pairs from the screening kernel's per-row lists
//     (rowinfo[TC_GROUPS i + g] = (count, overflow, W, d^min) per epilogue group);
//  1. k_pair_eval: Eq. (dist-direct) in fp32 for every pair, 8 lanes per pair
//     and 4 pairs per warp (no per-row bookkeeping on this path);
//  2. k_certify, one thread per row: Theorem 4.1 puts each true value in
//     [v (1 - g), v (1 + g)], g = gamma_{d+2}(2^-24); when exactly one
//     interval can hold the minimum, that centre is the argmin and v is
//     min_dist; otherwise (near-ties) the open candidates are evaluated in
//     binary64 (products and sums rounded separately, coordinates in order:
//     the oracle's own arithmetic), lowest index on ties.  Overflowed rows
//     are listed for the full-row kernel, which evaluates every centre.

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

// fp32 direct values of the candidate pairs.  NV float4 of a row per lane
// (lane l of a pair's 8 takes float4 l, l + 8, ...); NV == 0: scalar loads
// for any d and alignment.  A group of eight lanes takes two pairs per round
// (pi and pi + G, G the number of groups), all their loads issued first.
template <int NV>
KM_DEV float pair_value(const float* __restrict__ X, const float* __restrict__ C, int d, int2 pr, int sl) {
    float acc = 0.0f;
    if (NV > 0) {
        const int d4 = d >> 2;
        const float4* x4 = reinterpret_cast<const float4*>(X + (int64_t)pr.x * d);
        const float4* c4 = reinterpret_cast<const float4*>(C + (int64_t)pr.y * d);
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = sl + 8 * u;
            const float4 xv = (c < d4) ? x4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 cv = (c < d4) ? c4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float t0 = xv.x - cv.x, t1 = xv.y - cv.y, t2 = xv.z - cv.z, t3 = xv.w - cv.w;
            acc = fmaf(t0, t0, acc);
            acc = fmaf(t1, t1, acc);
            acc = fmaf(t2, t2, acc);
            acc = fmaf(t3, t3, acc);
        }
    } else {
        const float* x = X + (int64_t)pr.x * d;
        const float* c = C + (int64_t)pr.y * d;
        for (int l = sl; l < d; l += 8) {
            const float t = x[l] - c[l];
            acc = fmaf(t, t, acc);
        }
    }
    return acc;
}

template <int NV>
__global__ void __launch_bounds__(256) k_pair_eval(const float* __restrict__ X, const float* __restrict__ C, int d,
                                                   const int2* __restrict__ pairs,
                                                   const unsigned long long* __restrict__ npairs, int64_t cap,
                                                   float* __restrict__ v32) {
    const int lane = threadIdx.x & 31, sl = lane & 7, gbase = lane & ~7;
    const unsigned gmask = 0xFFu << gbase;
    const int64_t gid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4 + (lane >> 3);
    const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * 4;
    const int64_t np = min((int64_t)*npairs, cap);
    for (int64_t pi = gid; pi < np; pi += 2 * ngroups) {
        const int64_t pj = pi + ngroups;
        const int2 pa = pairs[pi];
        const int2 pb = pj < np ? pairs[pj] : make_int2(-1, 0);
        // a slot of a row that did not fit is marked row -1 (the group's eight lanes alike)
        float va = pa.x >= 0 ? pair_value<NV>(X, C, d, pa, sl) : 0.0f;
        float vb = pb.x >= 0 ? pair_value<NV>(X, C, d, pb, sl) : 0.0f;
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            va += __shfl_xor_sync(gmask, va, off);
            vb += __shfl_xor_sync(gmask, vb, off);
        }
        if (sl == 0) {
            if (pa.x >= 0) v32[pi] = va;
            if (pb.x >= 0) v32[pj] = vb;
        }
    }
}

// Candidate selection, one thread per row: the quad entries of every epilogue
// group's list inside the window of the row's final d^ minimum (the smallest
// of the groups' minima), each masked column written out as a (row, j) pair,
// contiguous per row, one atomic reservation per block.  Rows whose list
// overflowed, or that no longer fit in the pair buffer, get count -1
// (whole-row recompute).  A row with a single candidate is decided here: the
// window holds every centre that can be the nearest, so that one is; its
// label is written and its count is 0 (no evaluation: every caller refines
// the winner's distance afterwards, to binary64 accuracy).
__global__ void __launch_bounds__(256) k_cand_select(const int4* __restrict__ rowinfo,
                                                     const uint32_t* __restrict__ cand, int64_t n, int ebits,
                                                     int2* __restrict__ pairs, int64_t cap,
                                                     int2* __restrict__ rowpair, int32_t* __restrict__ labels,
                                                     DevCounters* cnt) {
    const int lane = threadIdx.x & 31;
    const uint32_t emask = (1u << ebits) - 1u;
    const float lscale = __uint_as_float((uint32_t)(127 + ebits - 23) << 23);  // 2^(ebits - 23)
    // rounds of blockDim rows per block, the same count in every warp (the
    // reservation synchronises the block)
    for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < n; b0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = b0 + threadIdx.x;
        const bool valid = row < n;
        int c = 0;
        bool full = false;
        int cnt_g[TC_GROUPS];
        float lim = 0.0f;
        // slot s of group g at cand[(g * TC_LIST + s) * n + row]: a warp reads 32 rows side by side
        const uint32_t* c0 = cand + row;
        unsigned msk[TC_GROUPS];  // entries inside the window, per group
        {
            float dmin = INFINITY, W = 0.0f;
#pragma unroll
            for (int g = 0; g < TC_GROUPS; g++) {
                const int4 ig = valid ? rowinfo[row * TC_GROUPS + g] : make_int4(0, 0, 0, __float_as_int(INFINITY));
                full |= ig.y != 0;
                cnt_g[g] = ig.x;
                dmin = fminf(dmin, __int_as_float(ig.w));
                W = __int_as_float(ig.z);
            }
            lim = dmin + W;
        }
        // the first SPEC slots of every list in one round of loads, the rest (rare) after
        constexpr int SPEC = (16 / TC_GROUPS < TC_LIST) ? 16 / TC_GROUPS : TC_LIST;
#pragma unroll
        for (int g = 0; g < TC_GROUPS; g++) {
            const int ng = full ? 0 : cnt_g[g];
            const uint32_t* cg = c0 + (size_t)g * TC_LIST * n;
            uint32_t eg[SPEC];
#pragma unroll
            for (int s = 0; s < SPEC; s++) eg[s] = (s < ng) ? cg[(size_t)s * n] : 0u;
            unsigned m = 0;
#pragma unroll
            for (int s = 0; s < SPEC; s++) {
                const bool in = s < ng && cand_lower(eg[s], emask, lscale) <= lim;
                m |= in ? (1u << s) : 0u;
                c += in ? __popc(entry_mask(eg[s])) : 0;
            }
            for (int s = SPEC; s < ng; s++) {
                const uint32_t e = cg[(size_t)s * n];
                const bool in = cand_lower(e, emask, lscale) <= lim;
                m |= in ? (1u << s) : 0u;
                c += in ? __popc(entry_mask(e)) : 0;
            }
            msk[g] = m;
        }
        const bool single = valid && !full && c == 1;
        if (single) c = 0;  // decided: nothing to evaluate
        // one reservation per block: lane prefix sums, then warp totals through
        // shared memory (every warp of the block takes part in each round)
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += o;
        }
        __shared__ int wtot[8];
        __shared__ unsigned long long bbase;
        const int wib = threadIdx.x >> 5;
        if (lane == 31) wtot[wib] = incl;
        __syncthreads();
        int wpre = 0, btot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            wpre += (w < wib) ? wtot[w] : 0;
            btot += wtot[w];
        }
        if (threadIdx.x == 0) bbase = btot ? atomicAdd(&cnt->npairs, (unsigned long long)btot) : 0ull;
        __syncthreads();
        const int64_t off0 = (int64_t)bbase + wpre + incl - c;
        const bool fits = off0 + c <= cap;
        if (single) {
#pragma unroll
            for (int g = 0; g < TC_GROUPS; g++) {
                if (msk[g]) {
                    const uint32_t e = c0[((size_t)g * TC_LIST + (__ffs(msk[g]) - 1)) * n];
                    labels[row] = 4 * entry_quad(e, emask) + __ffs(entry_mask(e)) - 1;
                }
            }
            rowpair[row] = make_int2(0, 0);
        } else if (valid) {
            if (!full && !fits) {
                // reserved but past the capacity: the part of the range below the
                // capacity is marked empty (row -1), so the evaluation skips it
                for (int64_t t = off0; t < off0 + c && t < cap; t++) pairs[t] = make_int2(-1, 0);
            }
            if (!full && fits) {
                int w = 0;
#pragma unroll
                for (int g = 0; g < TC_GROUPS; g++) {
                    const uint32_t* cg = c0 + (size_t)g * TC_LIST * n;
                    for (unsigned m = msk[g]; m; m &= m - 1) {
                        const uint32_t e = cg[(size_t)(__ffs(m) - 1) * n];
                        const int j0 = 4 * entry_quad(e, emask);
                        for (unsigned b = entry_mask(e); b; b &= b - 1) pairs[off0 + w++] = make_int2((int)row, j0 + __ffs(b) - 1);
                    }
                }
            }
            rowpair[row] = make_int2(fits ? (int)off0 : 0, (full || !fits) ? -1 : c);
        }
    }
}

// Certification, one thread per row, by Theorem 4.1's intervals: the winner's
// fp32 value and index; where more than one interval can hold the minimum,
// those candidates in binary64 (the oracle's arithmetic), lowest index on
// ties.  Rows with count -1 go on full_list for the full-row kernel.
__global__ void __launch_bounds__(256) k_certify(const int2* __restrict__ rowpair, int64_t n,
                                                 const int2* __restrict__ pairs, const float* __restrict__ v32,
                                                 const float* __restrict__ X, const float* __restrict__ C, int d,
                                                 float gamma32, int32_t* __restrict__ labels,
                                                 double* __restrict__ min_dist, int32_t* __restrict__ full_list,
                                                 int32_t* __restrict__ amb_list, DevCounters* cnt) {
    unsigned long long ev32 = 0, amb = 0, ovf_rows = 0;
    const float g = gamma32;
    for (int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; row < n;
         row += (int64_t)gridDim.x * blockDim.x) {
        const int2 rp = rowpair[row];
        if (rp.y == 0) continue;  // a single candidate: labelled by the selection
        if (rp.y < 0) {
            ovf_rows++;
            const int slot = atomicAdd(&cnt->ovf_count, 1);
            full_list[slot] = (int32_t)row;
            continue;
        }
        float up = INFINITY;
        for (int r = 0; r < rp.y; r++) up = fminf(up, v32[rp.x + r] * (1.0f + g));
        int open = 0, bj = 0x7fffffff;
        float bv = INFINITY;
        for (int r = 0; r < rp.y; r++) {
            const float v = v32[rp.x + r];
            if (v * (1.0f - g) <= up) {
                open++;
                const int j = pairs[rp.x + r].y;
                if (v < bv || (v == bv && j < bj)) { bv = v; bj = j; }
            }
        }
        ev32 += (unsigned long long)rp.y;
        if (open == 1) {
            labels[row] = bj;
            min_dist[row] = (double)bv;
            continue;
        }
        amb++;
        const int slot = atomicAdd(&cnt->amb_count, 1);
        amb_list[slot] = (int32_t)row;
    }

#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev32 += __shfl_xor_sync(0xffffffffu, ev32, off);
        amb += __shfl_xor_sync(0xffffffffu, amb, off);
        ovf_rows += __shfl_xor_sync(0xffffffffu, ovf_rows, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ev32) atomicAdd(&cnt->fp32_evals, ev32);
        if (amb) atomicAdd(&cnt->amb_rows, amb);
        if (ovf_rows) atomicAdd(&cnt->ovf_rows, ovf_rows);
    }
}

// Near-tie rows (listed by k_certify): one warp per row.  The candidates
// whose fp32 interval can still hold the minimum are taken AMB_B at a time:
// the warp stages x and their centre rows in shared memory and forms every
// binary64 product (x_l - c_l)^2 in parallel (each is one rounding, whatever
// the order); then one lane per candidate adds its products in coordinate
// order, one rounding per addition: the oracle's sequential sum.  The warp
// then takes the smallest value, lowest index on ties.
constexpr int AMB_B = 4;
__global__ void __launch_bounds__(256) k_amb_fp64(const int32_t* __restrict__ amb_list, const int* __restrict__ amb_count,
                                                  const int2* __restrict__ rowpair, const int2* __restrict__ pairs,
                                                  const float* __restrict__ v32, const float* __restrict__ X,
                                                  const float* __restrict__ C, int d, float gamma32,
                                                  int32_t* __restrict__ labels, double* __restrict__ min_dist,
                                                  DevCounters* cnt) {
    extern __shared__ double amb_sm[];  // per warp: AMB_B x d products
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double* prod = amb_sm + (size_t)wib * AMB_B * d;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int na = *amb_count;
    const float g = gamma32;
    unsigned long long ev64 = 0;
    for (int64_t t = w0; t < na; t += nw) {
        const int64_t row = amb_list[t];
        const int2 rp = rowpair[row];
        float up = INFINITY;
        for (int r = lane; r < rp.y; r += 32) up = fminf(up, v32[rp.x + r] * (1.0f + g));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) up = fminf(up, __shfl_xor_sync(0xffffffffu, up, off));
        const float* x = X + row * d;
        double best = INFINITY;
        int bj = 0x7fffffff;
        // the open candidates, AMB_B per batch (warp-uniform loop over the row's pairs)
        int r = 0;
        while (true) {
            int js[AMB_B] = {};
            int nb = 0;
            for (; r < rp.y && nb < AMB_B; r++)
                if (v32[rp.x + r] * (1.0f - g) <= up) js[nb++] = pairs[rp.x + r].y;
            if (nb == 0) break;
            __syncwarp();
            // lanes over the coordinates (coalesced loads, no index division)
#pragma unroll
            for (int b = 0; b < AMB_B; b++) {
                if (b < nb) {
                    const float* c = C + (int64_t)js[b] * d;
                    for (int l = lane; l < d; l += 32) {
                        const double u = __dsub_rn((double)x[l], (double)c[l]);
                        prod[b * d + l] = __dmul_rn(u, u);
                    }
                }
            }
            __syncwarp();
            if (lane < nb) {
                const double* pp = prod + (size_t)lane * d;
                double sacc = 0.0;
                for (int l = 0; l < d; l++) sacc = __dadd_rn(sacc, pp[l]);
                int j = js[0];
#pragma unroll
                for (int q = 1; q < AMB_B; q++)
                    if (lane == q) j = js[q];
                ev64++;
                if (sacc < best || (sacc == best && j < bj)) { best = sacc; bj = j; }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, off);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, off);
            if (ob < best || (ob == best && oj < bj)) { best = ob; bj = oj; }
        }
        if (lane == 0) {
            labels[row] = bj;
            min_dist[row] = best;
        }
        __syncwarp();
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ev64 += __shfl_xor_sync(0xffffffffu, ev64, off);
    if (lane == 0 && ev64) atomicAdd(&cnt->fp64_evals, ev64);
}

cudaError_t launch_refine(const float* X, const float* C, const TcArgs& a, int32_t* labels, double* min_dist,
                          int32_t* full_list, int32_t* amb_list, int num_sms, cudaStream_t st, int* nlaunch) {
    // persistent grids: the resident blocks only
    int sel_per_sm = 1, cert_per_sm = 1;
    cudaError_t e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sel_per_sm, k_cand_select, 256, 0);
    if (e0 != cudaSuccess) return e0;
    e0 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cert_per_sm, k_certify, 256, 0);
    if (e0 != cudaSuccess) return e0;
    const int64_t rows_blocks = std::max<int64_t>(1, (a.n + 255) / 256);
    const int64_t rb = std::min<int64_t>(rows_blocks, (int64_t)num_sms * std::max(sel_per_sm, 1));
    const int64_t cb = std::min<int64_t>(rows_blocks, (int64_t)num_sms * std::max(cert_per_sm, 1));
    k_cand_select<<<(unsigned)rb, 256, 0, st>>>(a.rowinfo, a.cand, a.n, a.ebits, a.pairs, a.pair_cap, a.rowpair, labels,
                                                a.cnt);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *nlaunch = 4;
    // pair evaluation: a persistent grid of the resident blocks
    const bool vec = (a.d % 4 == 0) && a.d <= 256 && ((uintptr_t)X % 16 == 0) && ((uintptr_t)C % 16 == 0);
    const void* fn = !vec ? (const void*)k_pair_eval<0>
                          : (a.d <= 32 ? (const void*)k_pair_eval<1>
                                       : (a.d <= 128 ? (const void*)k_pair_eval<4> : (const void*)k_pair_eval<8>));
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 256, 0);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)num_sms * (unsigned)std::max(per_sm, 1);
    const unsigned long long* np = &a.cnt->npairs;
    if (!vec) k_pair_eval<0><<<blocks, 256, 0, st>>>(X, C, a.d, a.pairs, np, a.pair_cap, a.v32);
    else if (a.d <= 32) k_pair_eval<1><<<blocks, 256, 0, st>>>(X, C, a.d, a.pairs, np, a.pair_cap, a.v32);
    else if (a.d <= 128) k_pair_eval<4><<<blocks, 256, 0, st>>>(X, C, a.d, a.pairs, np, a.pair_cap, a.v32);
    else k_pair_eval<8><<<blocks, 256, 0, st>>>(X, C, a.d, a.pairs, np, a.pair_cap, a.v32);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_certify<<<(unsigned)cb, 256, 0, st>>>(a.rowpair, a.n, a.pairs, a.v32, X, C, a.d, a.tp.gamma32, labels, min_dist,
                                             full_list, amb_list, a.cnt);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t amb_smem = (size_t)8 * AMB_B * a.d * sizeof(double);  // 8 warps per block
    e = allow_max_smem(k_amb_fp64);
    if (e != cudaSuccess) return e;
    k_amb_fp64<<<(unsigned)num_sms, 256, amb_smem, st>>>(amb_list, &a.cnt->amb_count, a.rowpair, a.pairs, a.v32, X, C,
                                                          a.d, a.tp.gamma32, labels, min_dist, a.cnt);
    return cudaGetLastError();
}

}  // namespace km
