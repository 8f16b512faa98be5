// k_prep.cu -- input quantisation and row statistics (Section 4.3, Alg. 2
// line 1: x~ = fl_l(x)), and the norms the expanded formula reuses
// (Section 3.2: p_i = x_i^T x_i "precomputed and stored").
//
// One warp per row.  Output per row: the quantised row (fp16 / bf16, or
// E4M3 scaled by a power of two), and stat = (p, ||x||, ||x~||, ||x~ - x||):
//   p is ||x||^2 accumulated as an fp32 double-float (error ~2^-44) and then
//   rounded to fp32 -- the same value as binary64 rounded to fp32 except in
//   ties below 2^-44;  ||x~|| and ||x~ - x|| are fp32 sums inflated by
//   (1 + 2^-12), which covers their own rounding (gamma_d(2^-24) < 2^-12 for
//   d <= 4096), so the bound B built from them stays rigorous.  A non-zero
//   row with ||x||^2 < 2^-100 (squares near binary32's underflow) gets
//   infinite ||x~|| and ||x~ - x||: the bound is then infinite and every pair
//   of the row goes to the direct formula, as for a row that overflowed the
//   low format.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

constexpr float kNormInflate = 1.0f + 1.0f / 4096.0f;
constexpr float kTinyNorm2 = 0x1p-100f;  // below this ||x||^2 the fp32 statistics are not trusted

KM_DEV float quant_val(float v, int fmt) {
    if (fmt == 0) return __half2float(__float2half_rn(v));
    if (fmt == 1) return __bfloat162float(__float2bfloat16_rn(v));
    __nv_fp8_storage_t s = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    __half_raw hr = __nv_cvt_fp8_to_halfraw(s, __NV_E4M3);
    return __half2float(__half(hr));
}

// Row scale of E4M3 (the per-row power-of-two scaling read into Section 4.3's
// quantisation): the smallest power of two s with amax / s <= 448 (E4M3's
// largest finite value), so the row maximum lands in (224, 448]; s is kept a
// normal fp32 number (s >= 2^-126, so 1/s is finite and x / s exact), and an
// all-zero row takes s = 1.  Exact for every fp32 amax, subnormals included:
// amax = f 2^e with f in [0.5, 1) (frexpf is exact), and 448 = 0.875 2^9, so
// s = 2^(e - 9) when f <= 0.875, else 2^(e - 8).
KM_DEV float e4m3_row_scale(float amax) {
    if (!(amax > 0.0f)) return 1.0f;
    int e;
    const float f = frexpf(amax, &e);
    const int k = max(f <= 0.875f ? e - 9 : e - 8, -126);
    return __int_as_float((k + 127) << 23);
}

// Largest |a| seen by the block's threads, folded into *out with one atomic
// per block (non-negative floats order like their bit patterns).
KM_DEV void block_absmax(float v, unsigned* out) {
    __shared__ float wmax[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wmax[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) m = fmaxf(m, wmax[i]);
        atomicMax(out, __float_as_uint(m));
    }
}

__global__ void k_quantize(const float* __restrict__ A, int64_t m, int d, int fmt, int ldq, void* Aq,
                           float4* __restrict__ stat, float* __restrict__ rscale, unsigned* __restrict__ absmax_out) {
    float amx = 0.0f;  // largest |a| of this thread's elements (absmax_out)
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < m; i += nw) {
        const float* a = A + i * d;
        float s = 1.0f;
        if (fmt == 2) {
            float amax = 0.0f;
            for (int l = lane; l < d; l += 32) amax = fmaxf(amax, fabsf(a[l]));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            s = e4m3_row_scale(amax);
        }
        const float inv = 1.0f / s;  // exact: s is a power of two
        float ph = 0.0f, pl = 0.0f, q2 = 0.0f, r2 = 0.0f;
        bool nz = false;
        for (int l = lane; l < ldq; l += 32) {
            float v = (l < d) ? a[l] : 0.0f;
            amx = fmaxf(amx, fabsf(v));
            nz |= v != 0.0f;
            float qv = quant_val(v * inv, fmt);  // quantised value of x / s
            if (l < d) {
                df_add_sq(v, ph, pl);
                float qs = qv * s;                // x~ = s fl_l(x / s), exact scaling
                q2 = fmaf(qs, qs, q2);
                float rr = qs - v;                // exact (Sterbenz): qs and v are within a factor 2
                r2 = fmaf(rr, rr, r2);
            }
            if (fmt == 0) {
                reinterpret_cast<__half*>(Aq)[i * ldq + l] = __float2half_rn(qv);
            } else if (fmt == 1) {
                reinterpret_cast<__nv_bfloat16*>(Aq)[i * ldq + l] = __float2bfloat16_rn(qv);
            } else {
                reinterpret_cast<__nv_fp8_storage_t*>(Aq)[i * ldq + l] =
                    __nv_cvt_float_to_fp8(v * inv, __NV_SATFINITE, __NV_E4M3);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            float oh = __shfl_xor_sync(0xffffffffu, ph, off);
            float ol = __shfl_xor_sync(0xffffffffu, pl, off);
            df_add(ph, pl, oh, ol);
            q2 += __shfl_xor_sync(0xffffffffu, q2, off);
            r2 += __shfl_xor_sync(0xffffffffu, r2, off);
        }
        const bool nzr = __any_sync(0xffffffffu, nz);
        if (lane == 0) {
            float p = ph + pl;
            float4 o;
            o.x = p;
            o.y = sqrtf(p) * kNormInflate;
            o.z = sqrtf(q2) * kNormInflate;
            o.w = sqrtf(r2) * kNormInflate;
            // an element that overflowed the low format, or squares near the
            // underflow, make the row unusable for the expanded formula: an
            // infinite bound flags all its pairs
            if (!isfinite(o.z) || (nzr && !(p >= kTinyNorm2))) { o.z = INFINITY; o.w = INFINITY; }
            stat[i] = o;
            if (rscale) rscale[i] = s;
        }
    }
    if (absmax_out) block_absmax(amx, absmax_out);
}


// Group path (d % 4 == 0, padded width <= 256): 8 lanes per row, 4 rows per
// warp, so the row reductions take 3 shuffle levels and serve 4 rows at once.
// Lane l of a row's 8 holds float4 l, l + 8, ... (NV of them).
// Two coordinates (scale 1, 16-bit formats) into the row's running sums, two
// per packed instruction: ||x||^2 as a pair of double-floats (exact product,
// two-sum), ||x~||^2 and ||x~ - x||^2 in fp32.
KM_DEV float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
KM_DEV void row_sums2(float2 x, float2 q, float2& hi, float2& lo, float2& qq, float2& rr) {
    const float2 p = __fmul2_rn(x, x);
    const float2 pe = __ffma2_rn(x, x, neg2(p));
    const float2 s = __fadd2_rn(hi, p);
    const float2 bb = __fadd2_rn(s, neg2(hi));
    const float2 e = __fadd2_rn(__fadd2_rn(hi, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(p, neg2(bb)));
    hi = s;
    lo = __fadd2_rn(lo, __fadd2_rn(e, pe));
    qq = __ffma2_rn(q, q, qq);
    const float2 r = __fadd2_rn(q, neg2(x));  // exact (Sterbenz)
    rr = __ffma2_rn(r, r, rr);
}

template <int NV>
__global__ void k_quantize_g8(const float* __restrict__ A, int64_t m, int d, int fmt, int ldq, void* Aq,
                              float4* __restrict__ stat, float* __restrict__ rscale, unsigned* __restrict__ absmax_out) {
    float amx = 0.0f;  // largest |a| of this thread's elements (absmax_out)
    const int lane = threadIdx.x & 31, sl = lane & 7;
    const unsigned gmask = 0xFFu << (lane & ~7);
    const int64_t gid = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4 + (lane >> 3);
    const int64_t ngroups = (((int64_t)gridDim.x * blockDim.x) >> 5) * 4;
    const int d4 = d >> 2, ldq4 = ldq >> 2;
    // R rows per group and round, all their loads issued first: at least four
    // 16-byte loads in flight per lane
    constexpr int R = NV >= 4 ? 1 : 4 / NV;
    for (int64_t i0 = gid; i0 < m; i0 += ngroups * R) {
        float4 xr[R][NV];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int64_t ir = i0 + (int64_t)r * ngroups;
            const float4* a4 = reinterpret_cast<const float4*>(A + ir * d);
#pragma unroll
            for (int u = 0; u < NV; u++) {
                const int c = sl + 8 * u;
                xr[r][u] = (ir < m && c < d4) ? a4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
        const int64_t i = i0 + (int64_t)r * ngroups;
        if (i >= m) break;  // the same row for the group's eight lanes
        float4 x[NV];
        bool nz = false;
#pragma unroll
        for (int u = 0; u < NV; u++) {
            x[u] = xr[r][u];
            amx = fmaxf(amx, fmaxf(fmaxf(fabsf(x[u].x), fabsf(x[u].y)), fmaxf(fabsf(x[u].z), fabsf(x[u].w))));
            nz |= (x[u].x != 0.0f) | (x[u].y != 0.0f) | (x[u].z != 0.0f) | (x[u].w != 0.0f);
        }
        const bool nzr = (__ballot_sync(gmask, nz) & gmask) != 0u;
        float s = 1.0f;
        if (fmt == 2) {
            float amax = 0.0f;
#pragma unroll
            for (int u = 0; u < NV; u++)
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(x[u].x), fabsf(x[u].y)), fmaxf(fabsf(x[u].z), fabsf(x[u].w))));
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(gmask, amax, off));
            s = e4m3_row_scale(amax);
        }
        const float inv = 1.0f / s;
        float ph = 0.0f, pl = 0.0f, q2 = 0.0f, r2 = 0.0f;
        if (fmt != 2) {
            // 16-bit formats (scale 1): packed arithmetic, two coordinates at a time
            float2 h2 = make_float2(0.f, 0.f), l2 = h2, qq2 = h2, rr2 = h2;
#pragma unroll
            for (int u = 0; u < NV; u++) {
                const int c = sl + 8 * u;
                if (c >= ldq4) continue;
                const float2 a = make_float2(x[u].x, x[u].y), b = make_float2(x[u].z, x[u].w);
                float2 qa, qb;
                uint2 w;
                if (fmt == 0) {
                    const __half2 ha = __float22half2_rn(a), hb = __float22half2_rn(b);
                    qa = __half22float2(ha);
                    qb = __half22float2(hb);
                    w.x = *reinterpret_cast<const uint32_t*>(&ha);
                    w.y = *reinterpret_cast<const uint32_t*>(&hb);
                } else {
                    const __nv_bfloat162 ha = __float22bfloat162_rn(a), hb = __float22bfloat162_rn(b);
                    qa = __bfloat1622float2(ha);
                    qb = __bfloat1622float2(hb);
                    w.x = *reinterpret_cast<const uint32_t*>(&ha);
                    w.y = *reinterpret_cast<const uint32_t*>(&hb);
                }
                reinterpret_cast<uint2*>(Aq)[i * ldq4 + c] = w;
                row_sums2(a, qa, h2, l2, qq2, rr2);
                row_sums2(b, qb, h2, l2, qq2, rr2);
            }
            ph = h2.x;
            pl = l2.x;
            df_add(ph, pl, h2.y, l2.y);
            q2 = qq2.x + qq2.y;
            r2 = rr2.x + rr2.y;
        } else
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = sl + 8 * u;
            if (c >= ldq4) continue;
            const float xv[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
            float qv[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                qv[t] = quant_val(xv[t] * inv, fmt);
                df_add_sq(xv[t], ph, pl);
                const float qs = qv[t] * s;
                q2 = fmaf(qs, qs, q2);
                const float rr = qs - xv[t];
                r2 = fmaf(rr, rr, r2);
            }
            if (fmt == 0) {
                __half2 h0 = __floats2half2_rn(qv[0], qv[1]), h1 = __floats2half2_rn(qv[2], qv[3]);
                uint2 w;
                w.x = *reinterpret_cast<uint32_t*>(&h0);
                w.y = *reinterpret_cast<uint32_t*>(&h1);
                reinterpret_cast<uint2*>(Aq)[i * ldq4 + c] = w;
            } else if (fmt == 1) {
                __nv_bfloat162 h0 = __floats2bfloat162_rn(qv[0], qv[1]), h1 = __floats2bfloat162_rn(qv[2], qv[3]);
                uint2 w;
                w.x = *reinterpret_cast<uint32_t*>(&h0);
                w.y = *reinterpret_cast<uint32_t*>(&h1);
                reinterpret_cast<uint2*>(Aq)[i * ldq4 + c] = w;
            } else {
                uint32_t w = 0;
#pragma unroll
                for (int t = 0; t < 4; t++)
                    w |= (uint32_t)__nv_cvt_float_to_fp8(xv[t] * inv, __NV_SATFINITE, __NV_E4M3) << (8 * t);
                reinterpret_cast<uint32_t*>(Aq)[i * ldq4 + c] = w;
            }
        }
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) {
            float oh = __shfl_xor_sync(gmask, ph, off);
            float ol = __shfl_xor_sync(gmask, pl, off);
            df_add(ph, pl, oh, ol);
            q2 += __shfl_xor_sync(gmask, q2, off);
            r2 += __shfl_xor_sync(gmask, r2, off);
        }
        if (sl == 0) {
            float p = ph + pl;
            float4 o;
            o.x = p;
            o.y = sqrtf(p) * kNormInflate;
            o.z = sqrtf(q2) * kNormInflate;
            o.w = sqrtf(r2) * kNormInflate;
            // an element that overflowed the low format, or squares near the
            // underflow, make the row unusable for the expanded formula: an
            // infinite bound flags all its pairs
            if (!isfinite(o.z) || (nzr && !(p >= kTinyNorm2))) { o.z = INFINITY; o.w = INFINITY; }
            stat[i] = o;
            if (rscale) rscale[i] = s;
        }
        }
    }
    if (absmax_out) block_absmax(amx, absmax_out);
}

// Vector path (d % 4 == 0, d <= 512): one warp per row, each lane holds up to
// four float4 of the row in registers (coalesced 16-byte loads).
template <int NV>
__global__ void k_quantize_vec(const float* __restrict__ A, int64_t m, int d, int fmt, int ldq, void* Aq,
                               float4* __restrict__ stat, float* __restrict__ rscale, unsigned* __restrict__ absmax_out) {
    float amx = 0.0f;  // largest |a| of this thread's elements (absmax_out)
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = d >> 2, ldq4 = ldq >> 2;
    for (int64_t i = warp; i < m; i += nw) {
        const float4* a4 = reinterpret_cast<const float4*>(A + i * d);
        float4 x[NV];
        bool nz = false;
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = lane + 32 * u;
            x[u] = (c < d4) ? a4[c] : make_float4(0.f, 0.f, 0.f, 0.f);
            amx = fmaxf(amx, fmaxf(fmaxf(fabsf(x[u].x), fabsf(x[u].y)), fmaxf(fabsf(x[u].z), fabsf(x[u].w))));
            nz |= (x[u].x != 0.0f) | (x[u].y != 0.0f) | (x[u].z != 0.0f) | (x[u].w != 0.0f);
        }
        const bool nzr = __any_sync(0xffffffffu, nz);
        float s = 1.0f;
        if (fmt == 2) {
            float amax = 0.0f;
#pragma unroll
            for (int u = 0; u < NV; u++)
                amax = fmaxf(amax, fmaxf(fmaxf(fabsf(x[u].x), fabsf(x[u].y)), fmaxf(fabsf(x[u].z), fabsf(x[u].w))));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
            s = e4m3_row_scale(amax);
        }
        const float inv = 1.0f / s;
        float ph = 0.0f, pl = 0.0f, q2 = 0.0f, r2 = 0.0f;
#pragma unroll
        for (int u = 0; u < NV; u++) {
            const int c = lane + 32 * u;
            if (c >= ldq4) continue;
            const float xv[4] = {x[u].x, x[u].y, x[u].z, x[u].w};
            float qv[4];
#pragma unroll
            for (int t = 0; t < 4; t++) {
                qv[t] = quant_val(xv[t] * inv, fmt);
                df_add_sq(xv[t], ph, pl);
                const float qs = qv[t] * s;
                q2 = fmaf(qs, qs, q2);
                const float rr = qs - xv[t];
                r2 = fmaf(rr, rr, r2);
            }
            if (fmt == 0) {
                __half2 h0 = __floats2half2_rn(qv[0], qv[1]), h1 = __floats2half2_rn(qv[2], qv[3]);
                uint2 w;
                w.x = *reinterpret_cast<uint32_t*>(&h0);
                w.y = *reinterpret_cast<uint32_t*>(&h1);
                reinterpret_cast<uint2*>(Aq)[i * ldq4 + c] = w;
            } else if (fmt == 1) {
                __nv_bfloat162 h0 = __floats2bfloat162_rn(qv[0], qv[1]), h1 = __floats2bfloat162_rn(qv[2], qv[3]);
                uint2 w;
                w.x = *reinterpret_cast<uint32_t*>(&h0);
                w.y = *reinterpret_cast<uint32_t*>(&h1);
                reinterpret_cast<uint2*>(Aq)[i * ldq4 + c] = w;
            } else {
                uint32_t w = 0;
#pragma unroll
                for (int t = 0; t < 4; t++)
                    w |= (uint32_t)__nv_cvt_float_to_fp8(xv[t] * inv, __NV_SATFINITE, __NV_E4M3) << (8 * t);
                reinterpret_cast<uint32_t*>(Aq)[i * ldq4 + c] = w;
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            float oh = __shfl_xor_sync(0xffffffffu, ph, off);
            float ol = __shfl_xor_sync(0xffffffffu, pl, off);
            df_add(ph, pl, oh, ol);
            q2 += __shfl_xor_sync(0xffffffffu, q2, off);
            r2 += __shfl_xor_sync(0xffffffffu, r2, off);
        }
        if (lane == 0) {
            float p = ph + pl;
            float4 o;
            o.x = p;
            o.y = sqrtf(p) * kNormInflate;
            o.z = sqrtf(q2) * kNormInflate;
            o.w = sqrtf(r2) * kNormInflate;
            if (!isfinite(o.z) || (nzr && !(p >= kTinyNorm2))) { o.z = INFINITY; o.w = INFINITY; }
            stat[i] = o;
            if (rscale) rscale[i] = s;
        }
    }
    if (absmax_out) block_absmax(amx, absmax_out);
}

__global__ void k_colmax(const float4* __restrict__ cstat, int k, const float* __restrict__ cscale, ColMax* out,
                         float* __restrict__ qpad, float* __restrict__ spad, int kpad) {
    // q_j for the screening kernel, +inf on the padding so padded columns never
    // win; the centres' E4M3 scales (cscale, nullable: 1), 1 on the padding
    for (int j = threadIdx.x; j < kpad; j += blockDim.x) {
        qpad[j] = (j < k) ? cstat[j].x : INFINITY;
        spad[j] = (j < k && cscale) ? cscale[j] : 1.0f;
    }
    __shared__ float red[10][32];
    float a = 0, b = 0, c = 0, q = 0, c2 = 0;
    float an = INFINITY, bn = INFINITY, cn = INFINITY, qn = INFINITY, c2n = INFINITY;
    for (int j = threadIdx.x; j < k; j += blockDim.x) {
        float4 s = cstat[j];
        a = fmaxf(a, s.y);
        b = fmaxf(b, s.w);
        c = fmaxf(c, s.z);
        q = fmaxf(q, s.x);
        c2 = fmaxf(c2, s.z * s.z);
        an = fminf(an, s.y);
        bn = fminf(bn, s.w);
        cn = fminf(cn, s.z);
        qn = fminf(qn, s.x);
        c2n = fminf(c2n, s.z * s.z);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        a = fmaxf(a, __shfl_xor_sync(0xffffffffu, a, off));
        b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, off));
        c = fmaxf(c, __shfl_xor_sync(0xffffffffu, c, off));
        q = fmaxf(q, __shfl_xor_sync(0xffffffffu, q, off));
        c2 = fmaxf(c2, __shfl_xor_sync(0xffffffffu, c2, off));
        an = fminf(an, __shfl_xor_sync(0xffffffffu, an, off));
        bn = fminf(bn, __shfl_xor_sync(0xffffffffu, bn, off));
        cn = fminf(cn, __shfl_xor_sync(0xffffffffu, cn, off));
        qn = fminf(qn, __shfl_xor_sync(0xffffffffu, qn, off));
        c2n = fminf(c2n, __shfl_xor_sync(0xffffffffu, c2n, off));
    }
    const int w = threadIdx.x >> 5, ln = threadIdx.x & 31;
    if (ln == 0) {
        red[0][w] = a; red[1][w] = b; red[2][w] = c; red[3][w] = q; red[4][w] = c2;
        red[5][w] = an; red[6][w] = bn; red[7][w] = cn; red[8][w] = qn; red[9][w] = c2n;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < (int)(blockDim.x / 32); i++) {
            a = fmaxf(a, red[0][i]); b = fmaxf(b, red[1][i]); c = fmaxf(c, red[2][i]);
            q = fmaxf(q, red[3][i]); c2 = fmaxf(c2, red[4][i]);
            an = fminf(an, red[5][i]); bn = fminf(bn, red[6][i]); cn = fminf(cn, red[7][i]);
            qn = fminf(qn, red[8][i]); c2n = fminf(c2n, red[9][i]);
        }
        ColMax o;
        o.nc = a; o.nrc = b; o.ncq = c; o.q = q; o.ncq2 = c2;
        o.pad[0] = o.pad[1] = o.pad[2] = 0.0f;
        o.nc_min = an; o.nrc_min = bn; o.ncq_min = cn; o.q_min = qn; o.ncq2_min = c2n;
        o.pad2[0] = o.pad2[1] = o.pad2[2] = 0.0f;
        *out = o;
    }
}

cudaError_t launch_quantize(const float* A, int64_t m, int d, int fmt, int ldq, void* Aq, float4* stat,
                            float* rscale, cudaStream_t st, unsigned* absmax_out) {
    // one warp per row, enough warps in flight to cover the memory latency
    int64_t blocks = (m * 32 + 255) / 256;
    if (blocks > 152 * 64) blocks = 152 * 64;
    if (blocks < 1) blocks = 1;
    const bool vec = (d % 4 == 0) && (ldq % 4 == 0) && ((uintptr_t)A % 16 == 0) && ((uintptr_t)Aq % 16 == 0);
    const int nv = (ldq / 4 + 31) / 32;
    const int nv8 = (ldq / 4 + 7) / 8;
    if (vec && nv8 <= 8) {
        blocks = std::min<int64_t>(std::max<int64_t>(1, (m * 8 + 255) / 256), (int64_t)152 * 16);
        if (nv8 <= 1)
            k_quantize_g8<1><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
        else if (nv8 <= 2)
            k_quantize_g8<2><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
        else if (nv8 <= 4)
            k_quantize_g8<4><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
        else
            k_quantize_g8<8><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
    } else if (vec && nv <= 4) {
        if (nv == 1)
            k_quantize_vec<1><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
        else if (nv == 2)
            k_quantize_vec<2><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
        else
            k_quantize_vec<4><<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
    } else {
        k_quantize<<<(unsigned)blocks, 256, 0, st>>>(A, m, d, fmt, ldq, Aq, stat, rscale, absmax_out);
    }
    return cudaGetLastError();
}

// ---- candidate-count prediction (the choice of the low format) ----------
// For a sample of rows: the fp32 direct distances to every centre, the row's
// certification window W = 2 B_max of the format (B_max from the row's
// quantisation statistics and the column maxima of the centres' ones, as the
// screening kernel forms it), and the number of centres within W of the
// row's minimum: the candidates the screen keeps for that row.  A row whose
// candidates exceed one epilogue group's list (TC_LIST entries) is counted
// as an overflow.  acc[0] += candidates, acc[1] += overflowing rows.
__global__ void __launch_bounds__(256) k_predict_candidates(const float* __restrict__ X, int64_t n, int d,
                                                            const float* __restrict__ C, int k, int fmt,
                                                            const ColMax* __restrict__ cmx, TestParams tp, int64_t stride,
                                                            int nsample, unsigned long long* acc) {
    extern __shared__ float xs[];
    __shared__ float red[8];
    __shared__ float sh_stat[4];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const ColMax cm = *cmx;
    for (int sidx = blockIdx.x; sidx < nsample; sidx += gridDim.x) {
        const int64_t i = (int64_t)sidx * stride;
        __syncthreads();
        for (int l = t; l < d; l += blockDim.x) xs[l] = X[i * d + l];
        __syncthreads();
        // the row's statistics in the format (warp 0): ||x||^2, ||x~||, ||x~ - x||
        if (w == 0) {
            float amax = 0.0f;
            for (int l = lane; l < d; l += 32) amax = fmaxf(amax, fabsf(xs[l]));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
            const float s = fmt == 2 ? e4m3_row_scale(amax) : 1.0f;
            float p = 0.0f, q2 = 0.0f, r2 = 0.0f;
            for (int l = lane; l < d; l += 32) {
                const float v = xs[l];
                const float qs = quant_val(v / s, fmt) * s;
                p = fmaf(v, v, p);
                q2 = fmaf(qs, qs, q2);
                r2 = fmaf(qs - v, qs - v, r2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                p += __shfl_xor_sync(0xffffffffu, p, o);
                q2 += __shfl_xor_sync(0xffffffffu, q2, o);
                r2 += __shfl_xor_sync(0xffffffffu, r2, o);
            }
            if (lane == 0) {
                sh_stat[0] = p;
                sh_stat[1] = sqrtf(q2) * kNormInflate;
                sh_stat[2] = sqrtf(r2) * kNormInflate;
            }
        }
        // fp32 direct distances: the row minimum first
        float mn = INFINITY;
        for (int j = t; j < k; j += blockDim.x) {
            const float* c = C + (int64_t)j * d;
            float acc2 = 0.0f;
            for (int l = 0; l < d; l++) {
                const float u = xs[l] - c[l];
                acc2 = fmaf(u, u, acc2);
            }
            mn = fminf(mn, acc2);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        if (lane == 0) red[w] = mn;
        __syncthreads();
        mn = red[0];
        for (int q = 1; q < (int)(blockDim.x >> 5); q++) mn = fminf(mn, red[q]);
        const float p = sh_stat[0], nxq = sh_stat[1], nrx = sh_stat[2];
        const float bmax = (2.0f * nrx * cm.nc + 2.0f * nxq * cm.nrc + tp.kacc * nxq * cm.ncq + tp.kn * (p + cm.q)) * tp.bsafe;
        const float lim = mn + 2.0f * bmax * 1.001f;
        unsigned cntc = 0;
        for (int j = t; j < k; j += blockDim.x) {
            const float* c = C + (int64_t)j * d;
            float acc2 = 0.0f;
            for (int l = 0; l < d; l++) {
                const float u = xs[l] - c[l];
                acc2 = fmaf(u, u, acc2);
            }
            cntc += acc2 <= lim ? 1u : 0u;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cntc += __shfl_xor_sync(0xffffffffu, cntc, o);
        __syncthreads();
        if (lane == 0) reinterpret_cast<unsigned*>(red)[w] = cntc;
        __syncthreads();
        if (t == 0) {
            unsigned tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); q++) tot += reinterpret_cast<unsigned*>(red)[q];
            atomicAdd(&acc[0], (unsigned long long)tot);
            if (tot > (unsigned)TC_LIST) atomicAdd(&acc[1], 1ull);
        }
    }
}

cudaError_t launch_predict_candidates(const float* X, int64_t n, int d, const float* C, int k, int fmt,
                                      const ColMax* cmx, const TestParams& tp, int nsample,
                                      unsigned long long* acc, int num_sms, cudaStream_t st) {
    const int64_t stride = std::max<int64_t>(1, n / nsample);
    const int ns = (int)std::min<int64_t>(nsample, (n + stride - 1) / stride);
    const size_t sm = (size_t)d * sizeof(float);
    cudaError_t e = allow_max_smem(k_predict_candidates);
    if (e != cudaSuccess) return e;
    k_predict_candidates<<<(unsigned)std::max(1, std::min(ns, num_sms * 4)), 256, sm, st>>>(X, n, d, C, k, fmt, cmx, tp,
                                                                                           stride, ns, acc);
    return cudaGetLastError();
}

cudaError_t launch_colmax(const float4* cstat, int k, const float* cscale, ColMax* out, float* qpad, float* spad,
                          int kpad, cudaStream_t st) {
    k_colmax<<<1, 1024, 0, st>>>(cstat, k, cscale, out, qpad, spad, kpad);
    return cudaGetLastError();
}

}  // namespace km
