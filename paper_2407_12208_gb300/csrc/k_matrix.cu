// k_matrix.cu -- the distance-matrix modes of Section 6.1 (Tables 6.1, 6.2)
// that are not the tensor-core screen:
//  * Alg. 2 with binary32 as the low precision ("FP32 -> FP64"): every
//    operation of the expanded formula rounded to binary32 in the order Alg. 2
//    states it (row and centre dot products d_xx, d_yy, d_xy by recursive
//    summation of rounded products, d = max(fl(fl(d_xx - 2 d_xy) + d_yy), 0),
//    E = fl(fl(rho c_A gamma) fl(d_xx + d_yy))), the reliability test, and the
//    flagged pairs marked for the fallback;
//  * the direct formula for every pair (Eq. (dist-direct)) in binary64 or
//    binary32, coordinates in order, products and sums rounded separately;
//  * the fallback of Eq. (fallback-rule) for flagged pairs in a chosen
//    precision: binary64, binary32, or the low format itself (the
//    "same-precision" fallback of Section 4.2, every operation rounded to
//    fp16 / bf16).
// No fused multiply-add anywhere: the values equal the CPU oracle's bit for bit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

constexpr int MX_T = 16;  // pairs tile: 16 rows x 16 centres per block

// out[i] = sum_l fl(a_il a_il) by recursive summation in binary32
__global__ void k_rowdot_fp32(const float* __restrict__ A, int64_t m, int d, float* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const float* a = A + i * d;
        float s = 0.0f;
        for (int l = 0; l < d; l++) s = __fadd_rn(s, __fmul_rn(a[l], a[l]));
        out[i] = s;
    }
}

// One 16 x 16 tile of pairs per block, rows and centres staged in shared
// memory (stride d + 1), a thread per pair.  MODE 0: Alg. 2 in binary32;
// 1: direct formula in binary64; 2: direct formula in binary32.
template <int MODE>
__global__ void __launch_bounds__(256) k_matrix(const float* __restrict__ X, int64_t n, const float* __restrict__ C,
                                                int k, int d, const float* __restrict__ dxx,
                                                const float* __restrict__ dyy, int test, float rho, float coef,
                                                float kacc, float kn, float* __restrict__ D,
                                                uint32_t* __restrict__ flag_bits, int2* __restrict__ queue,
                                                int64_t qcap, unsigned long long* __restrict__ qlen,
                                                DevCounters* cnt) {
    extern __shared__ float msh[];
    float* xs = msh;                    // MX_T x (d + 1)
    float* cs = msh + MX_T * (d + 1);   // MX_T x (d + 1)
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t ntr = (n + MX_T - 1) / MX_T, ntc = (k + MX_T - 1) / MX_T;
    unsigned long long nflag = 0;
    for (int64_t tile = blockIdx.x; tile < ntr * ntc; tile += gridDim.x) {
        const int64_t i0 = (tile / ntc) * MX_T, j0 = (tile % ntc) * MX_T;
        __syncthreads();
        for (int e = threadIdx.x; e < MX_T * d; e += blockDim.x) {
            const int r = e / d, l = e - r * d;
            xs[r * (d + 1) + l] = (i0 + r < n) ? X[(i0 + r) * d + l] : 0.0f;
            cs[r * (d + 1) + l] = (j0 + r < k) ? C[(j0 + r) * d + l] : 0.0f;
        }
        __syncthreads();
        const int64_t i = i0 + ty, j = j0 + tx;
        if (i >= n || j >= k) continue;
        const float* x = xs + ty * (d + 1);
        const float* c = cs + tx * (d + 1);
        float out;
        if (MODE == 1) {
            double s = 0.0;
            for (int l = 0; l < d; l++) {
                const double t = __dsub_rn((double)x[l], (double)c[l]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
            out = (float)s;
        } else if (MODE == 2) {
            float s = 0.0f;
            for (int l = 0; l < d; l++) {
                const float t = __fsub_rn(x[l], c[l]);
                s = __fadd_rn(s, __fmul_rn(t, t));
            }
            out = s;
        } else {
            float dxy = 0.0f;
            for (int l = 0; l < d; l++) dxy = __fadd_rn(dxy, __fmul_rn(x[l], c[l]));
            const float a = dxx[i], b = dyy[j];
            float dh = __fadd_rn(__fsub_rn(a, 2.0f * dxy), b);
            if (dh < 0.0f) dh = 0.0f;
            bool fl = false;
            if (test == 1) {
                fl = dh <= __fmul_rn(coef, __fadd_rn(a, b));
            } else if (test == 0) {
                // the tc form of the bound with no quantisation residuals:
                // accumulation and rounding of d^ only
                const float B = kacc * sqrtf(a) * sqrtf(b) * 1.0001f + kn * (a + b);
                fl = dh <= rho * B;
            }
            out = dh;
            if (fl) {
                out = -1.0f;  // replaced by the fallback's value
                nflag++;
                const unsigned long long pos = atomicAdd(qlen, 1ull);
                if ((int64_t)pos < qcap) queue[pos] = make_int2((int)i, (int)j);
                if (flag_bits) {
                    const unsigned long long bit = (unsigned long long)i * k + j;
                    atomicOr(&flag_bits[bit >> 5], 1u << (bit & 31));
                }
            }
        }
        D[i * k + j] = out;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) nflag += __shfl_xor_sync(0xffffffffu, nflag, off);
    if ((threadIdx.x & 31) == 0 && nflag) atomicAdd(&cnt->flagged, nflag);
}

cudaError_t launch_rowdot_fp32(const float* A, int64_t m, int d, float* out, int num_sms, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)num_sms * 8));
    k_rowdot_fp32<<<blocks, 256, 0, st>>>(A, m, d, out);
    return cudaGetLastError();
}

cudaError_t launch_matrix(int mode, const float* X, int64_t n, const float* C, int k, int d, const float* dxx,
                          const float* dyy, int test, float rho, float coef, float kacc, float kn, float* D,
                          uint32_t* flag_bits, int2* queue, int64_t qcap, unsigned long long* qlen, DevCounters* cnt,
                          int num_sms, cudaStream_t st) {
    const size_t sm = (size_t)2 * MX_T * (d + 1) * sizeof(float);
    const int64_t tiles = ((n + MX_T - 1) / MX_T) * ((k + MX_T - 1) / MX_T);
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms * 8));
    cudaError_t e;
#define KM_MX(M)                                                                                                 \
    e = allow_max_smem(k_matrix<M>);                                                                             \
    if (e != cudaSuccess) return e;                                                                              \
    k_matrix<M><<<blocks, 256, sm, st>>>(X, n, C, k, d, dxx, dyy, test, rho, coef, kacc, kn, D, flag_bits, queue, \
                                         qcap, qlen, cnt);
    if (mode == 0) { KM_MX(0) }
    else if (mode == 1) { KM_MX(1) }
    else { KM_MX(2) }
#undef KM_MX
    return cudaGetLastError();
}

// ---- the fallback of flagged pairs ----------------------------------------
// fb 0: binary64; 1: binary32; 2: the low format (fmt 0 fp16, 1 bf16), every
// operation rounded to it, on the inputs rounded to it.
template <int FB, int FMT>
KM_DEV float fallback_value(const float* x, const float* c, int d) {
    if constexpr (FB == 0) {
        double s = 0.0;
        for (int l = 0; l < d; l++) {
            const double u = __dsub_rn((double)x[l], (double)c[l]);
            s = __dadd_rn(s, __dmul_rn(u, u));
        }
        return (float)s;
    } else if constexpr (FB == 1) {
        float s = 0.0f;
        for (int l = 0; l < d; l++) {
            const float t = __fsub_rn(x[l], c[l]);
            s = __fadd_rn(s, __fmul_rn(t, t));
        }
        return s;
    } else if constexpr (FMT == 0) {
        __half s = __float2half_rn(0.0f);
        for (int l = 0; l < d; l++) {
            const __half t = __hsub(__float2half_rn(x[l]), __float2half_rn(c[l]));
            s = __hadd(s, __hmul(t, t));
        }
        return __half2float(s);
    } else {
        __nv_bfloat16 s = __float2bfloat16_rn(0.0f);
        for (int l = 0; l < d; l++) {
            const __nv_bfloat16 t = __hsub(__float2bfloat16_rn(x[l]), __float2bfloat16_rn(c[l]));
            s = __hadd(s, __hmul(t, t));
        }
        return __bfloat162float(s);
    }
}

// Flagged pairs of the distance matrix (marked -1): the fallback's values,
// from the bounded queue, or, when more pairs were flagged than it holds, by
// a scan of D for the marks.
template <int FB, int FMT>
__global__ void k_patch_flagged(const float* __restrict__ X, const float* __restrict__ C, int k, int d,
                                const int2* __restrict__ queue, const unsigned long long* __restrict__ qlen,
                                int64_t cap, float* __restrict__ D, int64_t n, DevCounters* cnt) {
    const int64_t len = (int64_t)*qlen;
    const bool scan = len > cap;
    const int64_t total = scan ? n * (int64_t)k : len;
    unsigned long long ev = 0;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t row, j;
        if (scan) {
            if (!(D[t] < 0.0f)) continue;
            row = t / k;
            j = t - row * k;
        } else {
            const int2 pr = queue[t];
            row = pr.x;
            j = pr.y;
        }
        D[row * k + j] = fallback_value<FB, FMT>(X + row * d, C + j * d, d);
        ev++;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, off);
    if ((threadIdx.x & 31) == 0 && ev) {
        if (FB == 0) atomicAdd(&cnt->fp64_evals, ev);
        else atomicAdd(&cnt->fp32_evals, ev);
    }
}

cudaError_t launch_patch_flagged(int fb, int fmt, const float* X, const float* C, int64_t n, int k, int d,
                                 const int2* queue, const unsigned long long* qlen, int64_t cap, float* D,
                                 DevCounters* cnt, int num_sms, cudaStream_t st) {
    const unsigned blocks = (unsigned)num_sms * 8;
    if (fb == 0) k_patch_flagged<0, 0><<<blocks, 256, 0, st>>>(X, C, k, d, queue, qlen, cap, D, n, cnt);
    else if (fb == 1) k_patch_flagged<1, 0><<<blocks, 256, 0, st>>>(X, C, k, d, queue, qlen, cap, D, n, cnt);
    else if (fmt == 0) k_patch_flagged<2, 0><<<blocks, 256, 0, st>>>(X, C, k, d, queue, qlen, cap, D, n, cnt);
    else k_patch_flagged<2, 1><<<blocks, 256, 0, st>>>(X, C, k, d, queue, qlen, cap, D, n, cnt);
    return cudaGetLastError();
}

}  // namespace km
