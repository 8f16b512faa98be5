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
#include "common.cuh"
#include "internal.h"

namespace km {

// Fixed-point exponent S for n rows with max |x| given as float bits.
KM_DEV int fixed_shift(unsigned amax_bits, int64_t n) {
    float amax = __uint_as_float(amax_bits);
    int E = (amax > 0.0f) ? ilogbf(amax) : -126;  // amax < 2^(E+1)
    int lgn = 0;
    while (((int64_t)1 << lgn) < n) lgn++;
    return 60 - lgn - E;  // |sum| 2^S < 2^(lgn + E + 1 + S) = 2^61
}

__global__ void k_absmax(const float* __restrict__ X, int64_t count, unsigned* out) {
    float m = 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(X[e]));
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative floats order as uints
}

// Flat element loop: thread e handles X[e] (row e / d, coordinate e % d).
// SMEM accumulators when k*d fits, else global atomics.
template <bool SMEM>
__global__ void k_accumulate(const float* __restrict__ X, int64_t n, int d, const int32_t* __restrict__ labels,
                             int k, const unsigned* __restrict__ amax_bits, long long* __restrict__ sums,
                             long long* __restrict__ counts) {
    extern __shared__ long long acc[];
    const int S = fixed_shift(*amax_bits, n);
    const int64_t kd = (int64_t)k * d;
    if (SMEM) {
        for (int64_t e = threadIdx.x; e < kd + k; e += blockDim.x) acc[e] = 0;
        __syncthreads();
    }
    long long* sacc = SMEM ? acc : sums;
    long long* cacc = SMEM ? acc + kd : counts;
    const int64_t total = n * d;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / d;
        const int l = (int)(e - i * d);
        const int j = labels[i];
        const long long v = __float2ll_rn(ldexpf(X[e], S));
        atomicAdd(reinterpret_cast<unsigned long long*>(&sacc[(int64_t)j * d + l]), (unsigned long long)v);
        if (l == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&cacc[j]), 1ull);
    }
    if (SMEM) {
        __syncthreads();
        for (int64_t e = threadIdx.x; e < kd; e += blockDim.x)
            if (acc[e]) atomicAdd(reinterpret_cast<unsigned long long*>(&sums[e]), (unsigned long long)acc[e]);
        for (int e = threadIdx.x; e < k; e += blockDim.x)
            if (acc[kd + e]) atomicAdd(reinterpret_cast<unsigned long long*>(&counts[e]), (unsigned long long)acc[kd + e]);
    }
}

// mean = sum 2^-S / m in binary64, stored in fp32 (the working precision).
__global__ void k_means(const long long* __restrict__ sums, const long long* __restrict__ counts,
                        const unsigned* __restrict__ amax_bits, int64_t n, int k, int d,
                        const float* __restrict__ C_old, float* __restrict__ C_new, int64_t* counts_out) {
    const int S = fixed_shift(*amax_bits, n);
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

// Empty clusters (ascending j) take the not-yet-taken point with the largest
// min_dist (lowest index on ties); then shift = max_j ||c_new - c_old||.
__global__ void k_empty_and_shift(const long long* __restrict__ counts, int64_t n, int k, int d,
                                  int empty_policy, const float* __restrict__ X, const double* __restrict__ min_dist,
                                  const float* __restrict__ C_old, float* __restrict__ C_new, double* shift,
                                  int32_t* __restrict__ taken) {
    __shared__ double rv[1024];
    __shared__ long long ri[1024];
    __shared__ int ntaken;
    const int t = threadIdx.x;
    if (t == 0) ntaken = 0;
    __syncthreads();
    if (empty_policy == 1 && min_dist != nullptr) {
        for (int j = 0; j < k; j++) {
            if (counts[j] != 0) continue;
            double best = -1.0;
            long long arg = -1;
            for (int64_t i = t; i < n; i += blockDim.x) {
                double v = min_dist[i];
                if (v > best) {
                    bool used = false;
                    for (int q = 0; q < ntaken; q++) used |= (taken[q] == (int32_t)i);
                    if (!used) { best = v; arg = i; }
                }
            }
            rv[t] = best;
            ri[t] = arg;
            __syncthreads();
            for (int s = blockDim.x / 2; s > 0; s >>= 1) {
                if (t < s) {
                    double ov = rv[t + s];
                    long long oi = ri[t + s];
                    if (oi >= 0 && (ov > rv[t] || (ov == rv[t] && (ri[t] < 0 || oi < ri[t])))) {
                        rv[t] = ov;
                        ri[t] = oi;
                    }
                }
                __syncthreads();
            }
            const long long a = ri[0];
            if (a >= 0) {
                for (int l = t; l < d; l += blockDim.x) C_new[(int64_t)j * d + l] = X[a * d + l];
                if (t == 0) taken[ntaken++] = (int32_t)a;
            }
            __syncthreads();
        }
    }
    // shift
    double mx = 0.0;
    for (int j = t; j < k; j += blockDim.x) {
        double s = 0.0;
        for (int l = 0; l < d; l++) {
            double df = (double)C_new[(int64_t)j * d + l] - (double)C_old[(int64_t)j * d + l];
            s = fma(df, df, s);
        }
        mx = fmax(mx, sqrt(s));
    }
    rv[t] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (t < s) rv[t] = fmax(rv[t], rv[t + s]);
        __syncthreads();
    }
    if (t == 0) *shift = rv[0];
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
__global__ void k_sum_final(const double* __restrict__ parts, int nparts, double* out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < nparts; i++) s += parts[i];
        *out = s;
    }
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
                              const unsigned* absmax_bits, long long* sums, long long* counts, int num_sms,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(sums, 0, sizeof(long long) * (size_t)k * d, st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(counts, 0, sizeof(long long) * (size_t)k, st);
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(long long) * ((size_t)k * d + k);
    const int64_t total = n * d;
    if (smem <= 200 * 1024) {
        e = cudaFuncSetAttribute(k_accumulate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = (int)max((size_t)1, min((size_t)4, (size_t)(220 * 1024) / (smem + 1024)));
        int64_t blocks = min((int64_t)num_sms * per_sm, (total + 511) / 512);
        if (blocks < 1) blocks = 1;
        k_accumulate<true><<<(unsigned)blocks, 512, smem, st>>>(X, n, d, labels, k, absmax_bits, sums, counts);
    } else {
        int64_t blocks = min((int64_t)num_sms * 8, (total + 511) / 512);
        if (blocks < 1) blocks = 1;
        k_accumulate<false><<<(unsigned)blocks, 512, 0, st>>>(X, n, d, labels, k, absmax_bits, sums, counts);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const long long* sums, const long long* counts, const unsigned* absmax_bits,
                            int64_t n, int k, int d, const float* C_old, int empty_policy, const float* X,
                            const double* min_dist, float* C_new, int64_t* counts_out, double* shift,
                            int32_t* taken_rows, cudaStream_t st) {
    int64_t kd = (int64_t)k * d;
    int64_t blocks = min((int64_t)1024, (kd + 255) / 256);
    k_means<<<(unsigned)blocks, 256, 0, st>>>(sums, counts, absmax_bits, n, k, d, C_old, C_new, counts_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_empty_and_shift<<<1, 1024, 0, st>>>(counts, n, k, d, empty_policy, X, min_dist, C_old, C_new, shift,
                                           taken_rows);
    return cudaGetLastError();
}

cudaError_t launch_sum_f64(const double* v, int64_t n, double* partials, int nparts, double* out, cudaStream_t st) {
    k_sum_parts<<<nparts, 256, 0, st>>>(v, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum_final<<<1, 32, 0, st>>>(partials, nparts, out);
    return cudaGetLastError();
}

}  // namespace km
