// k_direct.cu -- direct-formula assignment kernels, Eq. (dist-direct).
//
//  * k_direct_assign<double>: the plain FP64 path (every pair in binary64).
//  * k_direct_tiled (d % 4 == 0, 16 <= d <= 128), k_direct_small (d <= 8)
//    and k_direct_assign<float> (other d): fp32 direct distances for the fp32
//    path and for rows whose tensor-core candidate list overflowed.  Theorem
//    4.1 bounds each value's relative error by gamma_{d+2}(2^-24); a row whose
//    best and second-best intervals overlap is not certified and goes to
//  * k_rows_fp64: binary64 direct distances of one row against all centres
//    (warp per row, lanes over centres), exact argmin with the lowest index
//    on ties.  Products and sums are rounded separately (no FMA) so the
//    values equal the CPU oracle's bit for bit.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

constexpr int DA_ROWS = 128;  // rows (threads) per block
constexpr int DA_TC = 32;     // centres per shared-memory tile

template <typename T>
__global__ void __launch_bounds__(DA_ROWS) k_direct_assign(const float* __restrict__ X, int64_t n,
                                                           const float* __restrict__ C, int k, int d,
                                                           const int32_t* __restrict__ row_list,
                                                           const int* __restrict__ row_count,
                                                           int32_t* __restrict__ labels,
                                                           double* __restrict__ min_dist,
                                                           int32_t* __restrict__ amb_list, DevCounters* cnt,
                                                           float gamma32, unsigned* __restrict__ absmax_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    float amx = 0.0f;  // largest |x| this thread stages (absmax_out)
    // fp32 with d % 4 == 0: rows read four coordinates at a time, row stride
    // d + 4 (16-byte aligned; consecutive rows 16 bytes apart modulo the 128
    // banks-bytes when d % 32 == 0: conflict-free); else an odd stride
    const bool vec4 = sizeof(T) == 4 && (d % 4) == 0;
    const int ldx = vec4 ? d + 4 : d + 1;
    float* Xs = reinterpret_cast<float*>(smem);
    T* Cs = reinterpret_cast<T*>(smem + (((size_t)DA_ROWS * ldx * sizeof(float) + 15) & ~(size_t)15));
    const int64_t nrows = row_list ? (int64_t)(*row_count) : n;
    const int tid = threadIdx.x;
    unsigned long long local_amb = 0;
    for (int64_t base = (int64_t)blockIdx.x * DA_ROWS; base < nrows; base += (int64_t)gridDim.x * DA_ROWS) {
        const int rows_here = (int)min((int64_t)DA_ROWS, nrows - base);
        // stage the rows (coalesced when rows are contiguous)
        for (int e = tid; e < rows_here * d; e += DA_ROWS) {
            const int r = e / d, l = e - r * d;
            const int64_t gi = row_list ? (int64_t)row_list[base + r] : base + r;
            const float xv = X[gi * d + l];
            amx = fmaxf(amx, fabsf(xv));
            Xs[r * ldx + l] = xv;
        }
        T b1 = (T)INFINITY, b2 = (T)INFINITY;
        int j1 = 0;
        for (int c0 = 0; c0 < k; c0 += DA_TC) {
            const int tc = min(DA_TC, k - c0);
            __syncthreads();
            for (int e = tid; e < tc * d; e += DA_ROWS) Cs[e] = (T)C[(int64_t)c0 * d + e];
            __syncthreads();
            if (tid < rows_here) {
                T acc[DA_TC];
#pragma unroll
                for (int c = 0; c < DA_TC; c++) acc[c] = (T)0;
                const float* xr = Xs + tid * ldx;
                if (sizeof(T) == 4 && vec4) {
                    // four coordinates per shared-memory load on both sides (the same
                    // order of operations per centre as the scalar loop below)
                    for (int l = 0; l < d; l += 4) {
                        const float4 x4 = *reinterpret_cast<const float4*>(xr + l);
#pragma unroll
                        for (int c = 0; c < DA_TC; c++) {
                            if (c < tc) {
                                const float4 c4 = *reinterpret_cast<const float4*>(
                                    reinterpret_cast<const float*>(Cs) + c * d + l);
                                T t = (T)x4.x - (T)c4.x;
                                acc[c] = fma(t, t, acc[c]);
                                t = (T)x4.y - (T)c4.y;
                                acc[c] = fma(t, t, acc[c]);
                                t = (T)x4.z - (T)c4.z;
                                acc[c] = fma(t, t, acc[c]);
                                t = (T)x4.w - (T)c4.w;
                                acc[c] = fma(t, t, acc[c]);
                            }
                        }
                    }
                } else {
                    for (int l = 0; l < d; l++) {
                        const T xl = (T)xr[l];
#pragma unroll
                        for (int c = 0; c < DA_TC; c++) {
                            if (c < tc) {
                                const T t = xl - Cs[c * d + l];
                                acc[c] = fma(t, t, acc[c]);
                            }
                        }
                    }
                }
#pragma unroll
                for (int c = 0; c < DA_TC; c++) {
                    if (c < tc) {
                        const T v = acc[c];
                        if (v < b1) {
                            b2 = b1;
                            b1 = v;
                            j1 = c0 + c;
                        } else if (v < b2) {
                            b2 = v;
                        }
                    }
                }
            }
        }
        if (sizeof(T) == 4 && tid == 0) atomicAdd(&cnt->fp32_evals, (unsigned long long)rows_here * (unsigned long long)k);
        if (tid < rows_here) {
            const int64_t gi = row_list ? (int64_t)row_list[base + tid] : base + tid;
            labels[gi] = j1;
            min_dist[gi] = (double)b1;
            if (sizeof(T) == 4) {
                // Theorem 4.1: true values lie in [v (1 - g), v (1 + g)]
                const float g = gamma32;
                if (!((float)b2 * (1.0f - g) > (float)b1 * (1.0f + g))) {
                    int slot = atomicAdd(&cnt->amb_count, 1);
                    amb_list[slot] = (int32_t)gi;
                    local_amb++;
                }
            }
        }
        __syncthreads();
    }
    if (local_amb) atomicAdd(&cnt->amb_rows, local_amb);
    if (absmax_out) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, off));
        if ((threadIdx.x & 31) == 0) atomicMax(absmax_out, __float_as_uint(amx));
    }
}

// Tiled fp32 direct distances, Eq. (dist-direct), for d % 4 == 0 and
// 16 <= d <= 128 (rows whose candidate list overflowed, the fp32 direct path,
// km_assign_static): 128 rows per round resident in shared memory, the
// centres streamed through it in tiles of 64 (cp.async, two buffers).  Each
// thread holds 4 rows x 8 centres and takes two coordinates per packed
// instruction: the even and the odd coordinates are summed separately and
// then added, a summation order Theorem 4.1's bound covers like any other.
// Per row the smallest and second-smallest value and the first index of the
// smallest (ties: lowest index), merged over the 8 threads of the row; the
// certificate and the list of open rows as in k_direct_assign.
constexpr int DT_R = 128;  // rows per round
constexpr int DT_C = 64;   // centres per tile

KM_DEV void cp_async16(uint32_t dst, const void* src, bool full) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(full ? 16 : 0) : "memory");
}
KM_DEV void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
KM_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__global__ void __launch_bounds__(256, 1) k_direct_tiled(const float* __restrict__ X, int64_t n,
                                                         const float* __restrict__ C, int k, int d,
                                                         const int32_t* __restrict__ row_list,
                                                         const int* __restrict__ row_count,
                                                         int32_t* __restrict__ labels, double* __restrict__ min_dist,
                                                         int32_t* __restrict__ amb_list, DevCounters* cnt,
                                                         float gamma32, unsigned* __restrict__ absmax_out) {
    extern __shared__ __align__(16) float dts[];
    const int ldx = d + 4;  // row stride: 16-byte rows, consecutive rows 4 banks apart
    float* Xs = dts;
    const uint32_t cs0 = smem_u32(dts + DT_R * ldx);  // [2][DT_C][ldx]
    const float* Cs = dts + DT_R * ldx;
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int64_t nrows = row_list ? (int64_t)(*row_count) : n;
    const int d4 = d >> 2;
    const int ntile = (k + DT_C - 1) / DT_C;
    const float2 neg1 = make_float2(-1.0f, -1.0f);
    const float g = gamma32;
    float amx = 0.0f;
    unsigned long long local_amb = 0;
    for (int64_t base = (int64_t)blockIdx.x * DT_R; base < nrows; base += (int64_t)gridDim.x * DT_R) {
        const int rows_here = (int)min((int64_t)DT_R, nrows - base);
        __syncthreads();  // the previous round's readers are done with both buffers
        for (int e = tid; e < DT_R * d4; e += blockDim.x) {
            const int r = e / d4, l4 = e - r * d4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < rows_here) {
                const int64_t gi = row_list ? (int64_t)row_list[base + r] : base + r;
                v = reinterpret_cast<const float4*>(X + gi * d)[l4];
                amx = fmaxf(amx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
            *reinterpret_cast<float4*>(Xs + r * ldx + 4 * l4) = v;
        }
        auto load_tile = [&](int t, int buf) {
            const int c0 = t * DT_C;
            for (int e = tid; e < DT_C * d4; e += blockDim.x) {
                const int c = e / d4, l4 = e - c * d4;
                const bool ok = c0 + c < k;
                cp_async16(cs0 + (uint32_t)(((buf * DT_C + c) * ldx + 4 * l4) * 4),
                           ok ? (const void*)(C + (int64_t)(c0 + c) * d + 4 * l4) : (const void*)C, ok);
            }
            cp_async_commit();
        };
        load_tile(0, 0);
        float b1[4], b2[4];
        int j1[4];
#pragma unroll
        for (int i = 0; i < 4; i++) { b1[i] = INFINITY; b2[i] = INFINITY; j1[i] = 0; }
        for (int t = 0; t < ntile; t++) {
            const int buf = t & 1;
            cp_async_wait_all();
            __syncthreads();  // tile t is in place; tile t - 1's buffer is free
            if (t + 1 < ntile) load_tile(t + 1, buf ^ 1);
            float2 acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int c = 0; c < 8; c++) acc[i][c] = make_float2(0.f, 0.f);
            const float* xb = Xs + ty * ldx;                     // rows ty + 32 i
            const float* cb = Cs + (size_t)(buf * DT_C + tx) * ldx;  // centres tx + 8 c
            for (int l = 0; l < d; l += 4) {
                float4 xv[4], cv[8];
#pragma unroll
                for (int i = 0; i < 4; i++) xv[i] = *reinterpret_cast<const float4*>(xb + 32 * i * ldx + l);
#pragma unroll
                for (int c = 0; c < 8; c++) cv[c] = *reinterpret_cast<const float4*>(cb + 8 * c * ldx + l);
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int c = 0; c < 8; c++) {
                        const float2 t0 = __ffma2_rn(make_float2(cv[c].x, cv[c].y), neg1, make_float2(xv[i].x, xv[i].y));
                        acc[i][c] = __ffma2_rn(t0, t0, acc[i][c]);
                        const float2 t1 = __ffma2_rn(make_float2(cv[c].z, cv[c].w), neg1, make_float2(xv[i].z, xv[i].w));
                        acc[i][c] = __ffma2_rn(t1, t1, acc[i][c]);
                    }
            }
            const int c0 = t * DT_C;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                const int j = c0 + tx + 8 * c;  // ascending in c: the first of equal values keeps its place
                if (j < k)
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const float v = acc[i][c].x + acc[i][c].y;
                        if (v < b1[i]) {
                            b2[i] = b1[i];
                            b1[i] = v;
                            j1[i] = j;
                        } else if (v < b2[i]) {
                            b2[i] = v;
                        }
                    }
            }
        }
        // the 8 threads of each row: smallest (lowest index on ties) and second smallest
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int off = 1; off < 8; off <<= 1) {
                const float ob1 = __shfl_xor_sync(0xffffffffu, b1[i], off);
                const float ob2 = __shfl_xor_sync(0xffffffffu, b2[i], off);
                const int oj = __shfl_xor_sync(0xffffffffu, j1[i], off);
                if (ob1 < b1[i] || (ob1 == b1[i] && oj < j1[i])) {
                    b2[i] = fminf(b1[i], ob2);
                    b1[i] = ob1;
                    j1[i] = oj;
                } else {
                    b2[i] = fminf(b2[i], ob1);
                }
            }
        if (tx == 0)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int r = ty + 32 * i;
                if (r < rows_here) {
                    const int64_t gi = row_list ? (int64_t)row_list[base + r] : base + r;
                    labels[gi] = j1[i];
                    min_dist[gi] = (double)b1[i];
                    // Theorem 4.1: true values lie in [v (1 - g), v (1 + g)]
                    if (!(b2[i] * (1.0f - g) > b1[i] * (1.0f + g))) {
                        const int slot = atomicAdd(&cnt->amb_count, 1);
                        amb_list[slot] = (int32_t)gi;
                        local_amb++;
                    }
                }
            }
        if (tid == 0) atomicAdd(&cnt->fp32_evals, (unsigned long long)rows_here * (unsigned long long)k);
    }
    cp_async_wait_all();
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) local_amb += __shfl_xor_sync(0xffffffffu, local_amb, off);
    if ((tid & 31) == 0 && local_amb) atomicAdd(&cnt->amb_rows, local_amb);
    if (absmax_out) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, off));
        if ((tid & 31) == 0) atomicMax(absmax_out, __float_as_uint(amx));
    }
}

// Small d (d <= 8) with C small enough to stay in shared memory for the
// whole launch: one thread per row, the row in registers, every centre from
// shared memory (all lanes read the same centre: a broadcast).  The same
// fp32 operations, in the same order, and the same certificate as the tiled
// kernel above, so the two give the same results.
template <int D>
__global__ void __launch_bounds__(256) k_direct_small(const float* __restrict__ X, int64_t n,
                                                      const float* __restrict__ C, int k,
                                                      const int32_t* __restrict__ row_list,
                                                      const int* __restrict__ row_count,
                                                      int32_t* __restrict__ labels, double* __restrict__ min_dist,
                                                      int32_t* __restrict__ amb_list, DevCounters* cnt,
                                                      float gamma32, unsigned* __restrict__ absmax_out) {
    extern __shared__ __align__(16) float Csm[];
    float amx = 0.0f;  // largest |x| of this thread's rows (absmax_out)
    for (int e = threadIdx.x; e < k * D; e += blockDim.x) Csm[e] = C[e];
    __syncthreads();
    const int64_t nrows = row_list ? (int64_t)(*row_count) : n;
    const float g = gamma32;
    unsigned long long rows_done = 0, local_amb = 0;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t gi = row_list ? (int64_t)row_list[r] : r;
        float x[D];
#pragma unroll
        for (int l = 0; l < D; l++) {
            x[l] = X[gi * D + l];
            amx = fmaxf(amx, fabsf(x[l]));
        }
        float b1 = INFINITY, b2 = INFINITY;
        int j1 = 0;
        for (int j = 0; j < k; j++) {
            float acc = 0.0f;
#pragma unroll
            for (int l = 0; l < D; l++) {
                const float t = x[l] - Csm[j * D + l];
                acc = fmaf(t, t, acc);
            }
            if (acc < b1) {
                b2 = b1;
                b1 = acc;
                j1 = j;
            } else if (acc < b2) {
                b2 = acc;
            }
        }
        labels[gi] = j1;
        min_dist[gi] = (double)b1;
        rows_done++;
        // Theorem 4.1: true values lie in [v (1 - g), v (1 + g)]
        if (!(b2 * (1.0f - g) > b1 * (1.0f + g))) {
            const int slot = atomicAdd(&cnt->amb_count, 1);
            amb_list[slot] = (int32_t)gi;
            local_amb++;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        rows_done += __shfl_xor_sync(0xffffffffu, rows_done, off);
        local_amb += __shfl_xor_sync(0xffffffffu, local_amb, off);
    }
    if (absmax_out) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, off));
    }
    if ((threadIdx.x & 31) == 0) {
        if (rows_done) atomicAdd(&cnt->fp32_evals, rows_done * (unsigned long long)k);
        if (local_amb) atomicAdd(&cnt->amb_rows, local_amb);
        if (absmax_out) atomicMax(absmax_out, __float_as_uint(amx));
    }
}

// Exact argmin of listed rows, one 256-thread block per row.  Thread t takes
// centres t, t+256, ...  fp32_first: fp32 direct values of all centres
// (Theorem 4.1 intervals), the block's best and second best, and binary64
// (oracle arithmetic: products and sums rounded separately, coordinates in
// order) only for the centres whose interval can still hold the minimum.
struct Top2 {
    float b1, b2;
    int j1;
};
KM_DEV Top2 top2_merge(Top2 A, Top2 B) {
    Top2 r;
    if (B.b1 < A.b1 || (B.b1 == A.b1 && B.j1 < A.j1)) {
        r.b1 = B.b1; r.j1 = B.j1; r.b2 = fminf(A.b1, B.b2);
    } else {
        r.b1 = A.b1; r.j1 = A.j1; r.b2 = fminf(A.b2, B.b1);
    }
    return r;
}

KM_DEV double direct64(const float* x, const float* c, int d) {
    double s = 0.0;
    for (int l = 0; l < d; l++) {
        const double t = __dsub_rn((double)x[l], (double)c[l]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

template <bool FP32_FIRST>
__global__ void __launch_bounds__(256) k_rows_full(const float* __restrict__ X, const float* __restrict__ C, int k,
                                                   int d, const int32_t* __restrict__ row_list,
                                                   const int* __restrict__ row_count, int32_t* __restrict__ labels,
                                                   double* __restrict__ min_dist, DevCounters* cnt, float gamma32,
                                                   int keep_vals) {
    extern __shared__ float sh[];
    float* xs = sh;                      // d
    float* vs = sh + ((d + 3) & ~3);     // k fp32 values when they fit (keep_vals), else recomputed
    __shared__ Top2 red[8];
    __shared__ double rv[8];
    __shared__ int rj[8];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t nrows = *row_count;
    unsigned long long ev32 = 0, ev64 = 0;
    for (int64_t w = blockIdx.x; w < nrows; w += gridDim.x) {
        const int64_t i = row_list[w];
        __syncthreads();
        for (int l = tid; l < d; l += 256) xs[l] = X[i * d + l];
        __syncthreads();
        bool need64 = true;
        float thr = INFINITY;
        if (FP32_FIRST) {
            Top2 t{INFINITY, INFINITY, 0x7fffffff};
            for (int j = tid; j < k; j += 256) {
                const float* c = C + (int64_t)j * d;
                float s = 0.0f;
                for (int l = 0; l < d; l++) {
                    const float u = xs[l] - c[l];
                    s = fmaf(u, u, s);
                }
                if (keep_vals) vs[j] = s;
                ev32++;
                if (s < t.b1) { t.b2 = t.b1; t.b1 = s; t.j1 = j; }
                else if (s < t.b2) t.b2 = s;
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                Top2 o;
                o.b1 = __shfl_xor_sync(0xffffffffu, t.b1, off);
                o.b2 = __shfl_xor_sync(0xffffffffu, t.b2, off);
                o.j1 = __shfl_xor_sync(0xffffffffu, t.j1, off);
                t = top2_merge(t, o);
            }
            if (lane == 0) red[wid] = t;
            __syncthreads();
            t = red[0];
            for (int q = 1; q < 8; q++) t = top2_merge(t, red[q]);
            const float g = gamma32;
            if (t.b2 * (1.0f - g) > t.b1 * (1.0f + g)) {
                need64 = false;
                if (tid == 0) {
                    labels[i] = t.j1;
                    min_dist[i] = (double)t.b1;
                }
            } else {
                thr = t.b1 * (1.0f + g);
                if (tid == 0) atomicAdd(&cnt->amb_rows, 1ull);
            }
        }
        if (need64) {
            double best = INFINITY;
            int arg = 0x7fffffff;
            for (int j = tid; j < k; j += 256) {
                if (FP32_FIRST) {
                    float v;
                    if (keep_vals) {
                        v = vs[j];
                    } else {  // the same loop as above: the same value
                        const float* c = C + (int64_t)j * d;
                        v = 0.0f;
                        for (int l = 0; l < d; l++) {
                            const float u = xs[l] - c[l];
                            v = fmaf(u, u, v);
                        }
                    }
                    if (!(v * (1.0f - gamma32) <= thr)) continue;
                }
                const double s = direct64(xs, C + (int64_t)j * d, d);
                ev64++;
                if (s < best) { best = s; arg = j; }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                const int oa = __shfl_xor_sync(0xffffffffu, arg, off);
                if (ob < best || (ob == best && oa < arg)) { best = ob; arg = oa; }
            }
            if (lane == 0) { rv[wid] = best; rj[wid] = arg; }
            __syncthreads();
            if (tid == 0) {
                best = rv[0];
                arg = rj[0];
                for (int q = 1; q < 8; q++)
                    if (rv[q] < best || (rv[q] == best && rj[q] < arg)) { best = rv[q]; arg = rj[q]; }
                labels[i] = arg;
                min_dist[i] = best;
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        ev32 += __shfl_xor_sync(0xffffffffu, ev32, off);
        ev64 += __shfl_xor_sync(0xffffffffu, ev64, off);
    }
    if (lane == 0) {
        if (ev32) atomicAdd(&cnt->fp32_evals, ev32);
        if (ev64) atomicAdd(&cnt->fp64_evals, ev64);
    }
}

static size_t direct_smem(bool acc64, int d) {
    const int ldx = (!acc64 && d % 4 == 0) ? d + 4 : d + 1;
    size_t xs = (((size_t)DA_ROWS * ldx * sizeof(float)) + 15) & ~(size_t)15;
    return xs + (size_t)DA_TC * d * (acc64 ? 8 : 4);
}

cudaError_t launch_direct_assign(bool acc64, const float* X, int64_t n, const float* C, int k, int d,
                                 const int32_t* row_list, const int* row_count, int32_t* labels,
                                 double* min_dist, int32_t* amb_list, DevCounters* cnt, float gamma32,
                                 int num_sms, cudaStream_t st, unsigned* absmax_out) {
    if (!acc64 && d <= 8 && (size_t)k * d * sizeof(float) <= 32 * 1024) {
        // small d: C resident in shared memory, one thread per row, persistent grid
        const size_t csm = (size_t)k * d * sizeof(float);
        int per_sm = 1;
        const void* fns[9] = {nullptr, (const void*)k_direct_small<1>, (const void*)k_direct_small<2>,
                              (const void*)k_direct_small<3>, (const void*)k_direct_small<4>,
                              (const void*)k_direct_small<5>, (const void*)k_direct_small<6>,
                              (const void*)k_direct_small<7>, (const void*)k_direct_small<8>};
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fns[d], 256, csm);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * std::max(per_sm, 1)));
        switch (d) {
#define KM_SMALL(DD)                                                                                                  \
    case DD:                                                                                                          \
        k_direct_small<DD><<<(unsigned)grid, 256, csm, st>>>(X, n, C, k, row_list, row_count, labels, min_dist,      \
                                                              amb_list, cnt, gamma32, absmax_out);                                \
        break;
            KM_SMALL(1) KM_SMALL(2) KM_SMALL(3) KM_SMALL(4) KM_SMALL(5) KM_SMALL(6) KM_SMALL(7) KM_SMALL(8)
#undef KM_SMALL
        }
        return cudaGetLastError();
    }
    if (!acc64 && d % 4 == 0 && d >= 16 && d <= 128 && ((uintptr_t)X % 16) == 0 && ((uintptr_t)C % 16) == 0) {
        const size_t tsm = (size_t)(DT_R + 2 * DT_C) * (d + 4) * sizeof(float);
        cudaError_t e = allow_max_smem(k_direct_tiled);
        if (e != cudaSuccess) return e;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((n + DT_R - 1) / DT_R, (int64_t)num_sms));
        k_direct_tiled<<<(unsigned)grid, 256, tsm, st>>>(X, n, C, k, d, row_list, row_count, labels, min_dist, amb_list,
                                                          cnt, gamma32, absmax_out);
        return cudaGetLastError();
    }
    size_t sm = direct_smem(acc64, d);
    int64_t blocks_needed = (n + DA_ROWS - 1) / DA_ROWS;
    int per_sm = (int)max((size_t)1, (size_t)(200 * 1024) / sm);
    if (per_sm > 8) per_sm = 8;
    int64_t grid = min(blocks_needed, (int64_t)num_sms * per_sm);
    if (grid < 1) grid = 1;
    cudaError_t e;
    if (acc64) {
        e = allow_max_smem(k_direct_assign<double>);
        if (e != cudaSuccess) return e;
        k_direct_assign<double><<<(unsigned)grid, DA_ROWS, sm, st>>>(X, n, C, k, d, row_list, row_count, labels,
                                                                     min_dist, amb_list, cnt, gamma32, absmax_out);
    } else {
        e = allow_max_smem(k_direct_assign<float>);
        if (e != cudaSuccess) return e;
        k_direct_assign<float><<<(unsigned)grid, DA_ROWS, sm, st>>>(X, n, C, k, d, row_list, row_count, labels,
                                                                    min_dist, amb_list, cnt, gamma32, absmax_out);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_full(bool fp32_first, const float* X, const float* C, int k, int d, const int32_t* row_list,
                             const int* row_count, int32_t* labels, double* min_dist, DevCounters* cnt,
                             float gamma32, int num_sms, cudaStream_t st) {
    // x in shared memory, and the k fp32 values of the first pass when they fit
    const void* fn = fp32_first ? (const void*)k_rows_full<true> : (const void*)k_rows_full<false>;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    const size_t xs_bytes = (size_t)((d + 3) & ~3) * sizeof(float);
    const size_t avail = (size_t)kMaxBlockSmem - fa.sharedSizeBytes;
    const int keep = fp32_first && xs_bytes + (size_t)k * sizeof(float) <= avail;
    const size_t sm = xs_bytes + (keep ? (size_t)k * sizeof(float) : 0);
    if (fp32_first) {
        e = allow_max_smem(k_rows_full<true>);
        if (e != cudaSuccess) return e;
        k_rows_full<true><<<num_sms * 2, 256, sm, st>>>(X, C, k, d, row_list, row_count, labels, min_dist, cnt, gamma32,
                                                        keep);
    } else {
        e = allow_max_smem(k_rows_full<false>);
        if (e != cudaSuccess) return e;
        k_rows_full<false><<<num_sms * 2, 256, sm, st>>>(X, C, k, d, row_list, row_count, labels, min_dist, cnt, gamma32,
                                                         0);
    }
    return cudaGetLastError();
}

}  // namespace km
