// k_direct.cu -- direct-formula assignment kernels, Eq. (dist-direct).
//
//  * k_direct_assign<double>: the plain FP64 path (every pair in binary64).
//  * k_direct_assign<float>:  fp32 direct distances for small d (image pixels)
//    and for rows whose tensor-core candidate list overflowed.  Theorem 4.1
//    bounds each value's relative error by gamma_{d+2}(2^-24); a row whose
//    best and second-best intervals overlap is not certified and goes to
//  * k_rows_fp64: binary64 direct distances of one row against all centres
//    (warp per row, lanes over centres), exact argmin with the lowest index
//    on ties.  Products and sums are rounded separately (no FMA) so the
//    values equal the CPU oracle's bit for bit.
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
                                                           float gamma32) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ldx = d + 1;  // odd row stride: conflict-free per-thread row reads
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
            Xs[r * ldx + l] = X[gi * d + l];
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
}

// Binary64 direct distances of listed rows against all centres; lane j
// handles centres j, j+32, ...; the warp then takes the exact argmin.
__global__ void k_rows_fp64(const float* __restrict__ X, const float* __restrict__ C, int k, int d,
                            const int32_t* __restrict__ row_list, const int* __restrict__ row_count,
                            int32_t* __restrict__ labels, double* __restrict__ min_dist, DevCounters* cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nrows = *row_count;
    unsigned long long evals = 0;
    for (int64_t w = warp; w < nrows; w += nw) {
        const int64_t i = row_list[w];
        const float* x = X + i * d;
        double best = INFINITY;
        int arg = 0x7fffffff;
        for (int j = lane; j < k; j += 32) {
            const float* c = C + (int64_t)j * d;
            double s = 0.0;
            for (int l = 0; l < d; l++) {
                double t = __dsub_rn((double)x[l], (double)c[l]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
            if (s < best) { best = s; arg = j; }
            evals++;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            double ob = __shfl_xor_sync(0xffffffffu, best, off);
            int oa = __shfl_xor_sync(0xffffffffu, arg, off);
            if (ob < best || (ob == best && oa < arg)) { best = ob; arg = oa; }
        }
        if (lane == 0) {
            labels[i] = arg;
            min_dist[i] = best;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) evals += __shfl_xor_sync(0xffffffffu, evals, off);
    if (lane == 0 && evals) atomicAdd(&cnt->fp64_evals, evals);
}

static size_t direct_smem(bool acc64, int d) {
    size_t xs = (((size_t)DA_ROWS * (d + 1) * sizeof(float)) + 15) & ~(size_t)15;
    return xs + (size_t)DA_TC * d * (acc64 ? 8 : 4);
}

cudaError_t launch_direct_assign(bool acc64, const float* X, int64_t n, const float* C, int k, int d,
                                 const int32_t* row_list, const int* row_count, int32_t* labels,
                                 double* min_dist, int32_t* amb_list, DevCounters* cnt, float gamma32,
                                 int num_sms, cudaStream_t st) {
    size_t sm = direct_smem(acc64, d);
    int64_t blocks_needed = (n + DA_ROWS - 1) / DA_ROWS;
    int per_sm = (int)max((size_t)1, (size_t)(200 * 1024) / sm);
    if (per_sm > 8) per_sm = 8;
    int64_t grid = min(blocks_needed, (int64_t)num_sms * per_sm);
    if (grid < 1) grid = 1;
    cudaError_t e;
    if (acc64) {
        e = cudaFuncSetAttribute(k_direct_assign<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_direct_assign<double><<<(unsigned)grid, DA_ROWS, sm, st>>>(X, n, C, k, d, row_list, row_count, labels,
                                                                     min_dist, amb_list, cnt, gamma32);
    } else {
        e = cudaFuncSetAttribute(k_direct_assign<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_direct_assign<float><<<(unsigned)grid, DA_ROWS, sm, st>>>(X, n, C, k, d, row_list, row_count, labels,
                                                                    min_dist, amb_list, cnt, gamma32);
    }
    return cudaGetLastError();
}

cudaError_t launch_rows_fp64(const float* X, const float* C, int k, int d, const int32_t* row_list,
                             const int* row_count, int64_t max_rows, int32_t* labels, double* min_dist,
                             DevCounters* cnt, int num_sms, cudaStream_t st) {
    int64_t warps = max((int64_t)1, min(max_rows, (int64_t)num_sms * 32));
    int64_t blocks = (warps * 32 + 255) / 256;
    k_rows_fp64<<<(unsigned)blocks, 256, 0, st>>>(X, C, k, d, row_list, row_count, labels, min_dist, cnt);
    return cudaGetLastError();
}

}  // namespace km
