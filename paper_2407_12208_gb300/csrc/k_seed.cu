// k_seed.cu -- initial centres by D^2 sampling (k-means++): Section 2 names
// it beside uniformly drawn initial centres and leaves it outside the
// method.  The draws u_t in [0, 1) are inputs.
//   i_0 = min(floor(u_0 n), n - 1);
//   D^2_i = d(x_i, x_{i_0})^2 by the direct formula (Eq. (dist-direct)) to
//   binary64 accuracy (the double-float arithmetic of df.cuh);
//   for t = 1..k-1: T = sum_i D^2_i; i_t = the first row whose prefix sum
//   exceeds u_t T (the last row with D^2 > 0 when rounding leaves none;
//   min(floor(u_t n), n - 1) when T = 0), then D^2_i = min(D^2_i, d(x_i, x_{i_t})^2).
// Per pick: one pass over X (k_seed_dist), the sums of up to 16384 chunks of
// D^2 (k_seed_chunks, all SMs) and one block that finds the chunk holding
// the target and walks it (k_seed_pick).  Every sum is binary64 in an order
// fixed by n alone, so the result does not depend on the launch.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "df.cuh"
#include "internal.h"
#include "seed.h"

namespace km {

// D^2_i = d(x_i, c)^2 (first) or min(D^2_i, d(x_i, c)^2), c = x_{idx[t]}.
// R rows per lane and pass (a multi-row butterfly), G = 32 / LPR rows per load;
// the centre's chunks are loaded once per warp.
template <int NV4, int LPR, bool VEC>
__global__ void __launch_bounds__(256) k_seed_dist(const float* __restrict__ X, int64_t n, int d,
                                                   const int64_t* __restrict__ idx, int t, bool first,
                                                   double* __restrict__ D2) {
    constexpr int G = 32 / LPR;
    constexpr int R = NV4 == 4 ? 2 : 4;  // rows per lane and pass
    constexpr int STEP = R * G;
    static_assert(R <= LPR, "rows per lane exceed the lanes of a row");
    const int lane = threadIdx.x & 31, sub = lane / LPR, cl = lane % LPR;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int d4 = (d + 3) >> 2;
    const float* c = X + idx[t] * d;
    float4 cv[NV4];
#pragma unroll
    for (int u = 0; u < NV4; u++) {
        const int cidx = cl + LPR * u;
        if (VEC) {
            cv[u] = cidx < d4 ? reinterpret_cast<const float4*>(c)[cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        } else {
            float ce[4];
#pragma unroll
            for (int q = 0; q < 4; q++) ce[q] = (4 * cidx + q < d) ? c[4 * cidx + q] : 0.0f;
            cv[u] = make_float4(ce[0], ce[1], ce[2], ce[3]);
        }
    }
    for (int64_t base = w0 * STEP; base < n; base += nw * STEP) {
        float4 xv[R][NV4];
#pragma unroll
        for (int b = 0; b < R; b++) {
            const int64_t row = base + b * G + sub;
#pragma unroll
            for (int u = 0; u < NV4; u++) {
                const int cidx = cl + LPR * u;
                const bool ok = row < n && cidx < d4;
                if (VEC) {
                    xv[b][u] = ok ? reinterpret_cast<const float4*>(X + row * d)[cidx] : make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    float xe[4];
#pragma unroll
                    for (int q = 0; q < 4; q++) {
                        const int l = 4 * cidx + q;
                        xe[q] = (ok && l < d) ? X[row * d + l] : 0.0f;
                    }
                    xv[b][u] = make_float4(xe[0], xe[1], xe[2], xe[3]);
                }
            }
        }
        DF part[R];
#pragma unroll
        for (int b = 0; b < R; b++) {
            // rows past n hold zeros: their chunks are combined and dropped
            float4 cz[NV4];
#pragma unroll
            for (int u = 0; u < NV4; u++) cz[u] = (base + b * G + sub < n) ? cv[u] : make_float4(0.f, 0.f, 0.f, 0.f);
            part[b] = df_lane<NV4>(xv[b], cz);
        }
        int rs;
        const DF r = df_rows<R, LPR>(part, cl, rs);
        const int64_t row = base + rs * G + sub;
        if ((cl & (LPR / R - 1)) == 0 && row < n) {
            const double v = df_value(r);
            D2[row] = first ? v : fmin(D2[row], v);
        }
    }
}

// Rows of D <= 8 coordinates: one thread per row.
template <int D>
__global__ void __launch_bounds__(256) k_seed_small(const float* __restrict__ X, int64_t n,
                                                    const int64_t* __restrict__ idx, int t, bool first,
                                                    double* __restrict__ D2) {
    const float* c = X + idx[t] * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float xr[D];
#pragma unroll
        for (int l = 0; l < D; l++) xr[l] = X[i * D + l];
        const double v = df_value(df_small<D>(xr, c));
        D2[i] = first ? v : fmin(D2[i], v);
    }
}

// Chunk sums of D^2 for the pick (all SMs): NC = ceil(n / ch) chunks of ch
// rows, one warp per chunk; lane l adds rows l, l + 32, ... of the chunk in
// order, then a fixed shuffle tree -- the same sum whatever the launch.  Also
// each chunk's last row with D^2 > 0 (-1: none).
__global__ void __launch_bounds__(256) k_seed_chunks(const double* __restrict__ D2, int64_t n, int64_t ch,
                                                     int64_t nc, double* __restrict__ csum,
                                                     int64_t* __restrict__ clast) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < nc; c += nw) {
        const int64_t lo = c * ch, hi = lo + ch < n ? lo + ch : n;
        double s = 0.0;
        long long last = -1;
        for (int64_t i = lo + lane; i < hi; i += 32) {
            const double v = D2[i];
            s += v;
            if (v > 0.0) last = i;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s += __shfl_xor_sync(0xffffffffu, s, off);
            const long long o = __shfl_xor_sync(0xffffffffu, last, off);
            last = o > last ? o : last;
        }
        if (lane == 0) {
            csum[c] = s;
            clast[c] = last;
        }
    }
}

// The pick of step t (one block of SEED_T threads; t = 0: floor(u_0 n)).
// Thread p holds chunks [p CPT, (p + 1) CPT).  Starting offsets that never
// decrease: each thread adds its chunk sums in order (L_c, total A_p), lane 0
// of each warp adds its 32 threads' totals in order (B_p, total W_w), thread 0
// adds the warp totals in order (O_w, and T), and E_c = O_w + (B_p + L_c) --
// rounding is monotone, so E_0 = 0 <= E_1 <= ... <= T.  The chunk with
// E_c <= u_t T < E_{c+1} walks its rows in order (when rounding leaves none
// of them past the target, its last row with D^2 > 0 is the pick); a target
// at T or above takes the last row with D^2 > 0.
constexpr int SEED_T = 1024;
constexpr int64_t SEED_NC = 16384;  // chunks at most
__global__ void __launch_bounds__(SEED_T) k_seed_pick(const double* __restrict__ D2, int64_t n, int64_t ch,
                                                      int64_t nc, const double* __restrict__ csum,
                                                      const int64_t* __restrict__ clast,
                                                      const double* __restrict__ u, int t,
                                                      int64_t* __restrict__ idx) {
    __shared__ double tb[SEED_T], wtot[SEED_T / 32], wofs[SEED_T / 32 + 1];
    __shared__ long long lastpos;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const double ut = u[t];
    int64_t uniform_pick = (int64_t)floor(ut * (double)n);
    if (uniform_pick > n - 1) uniform_pick = n - 1;
    if (t == 0) {
        if (tid == 0) idx[0] = uniform_pick;
        return;
    }
    const int64_t cpt = (nc + SEED_T - 1) / SEED_T;
    const int64_t c0 = (int64_t)tid * cpt < nc ? (int64_t)tid * cpt : nc;
    const int64_t c1 = c0 + cpt < nc ? c0 + cpt : nc;
    double A = 0.0;
    long long mylast = -1;
    for (int64_t c = c0; c < c1; c++) {
        A += csum[c];
        mylast = clast[c] > mylast ? clast[c] : mylast;
    }
    tb[tid] = A;
    if (tid == 0) lastpos = -1;
    __syncthreads();
    if (mylast >= 0) atomicMax(&lastpos, mylast);
    if (lane == 0) {  // offsets of the warp's threads, in order
        double a = 0.0;
        for (int q = 0; q < 32; q++) {
            const double v = tb[wid * 32 + q];
            tb[wid * 32 + q] = a;
            a += v;
        }
        wtot[wid] = a;
    }
    __syncthreads();
    if (tid == 0) {  // warp offsets, in order
        double a = 0.0;
        for (int w = 0; w < SEED_T / 32; w++) {
            wofs[w] = a;
            a += wtot[w];
        }
        wofs[SEED_T / 32] = a;  // T
    }
    __syncthreads();
    const double T = wofs[SEED_T / 32];
    // a valid row first (the last row with D^2 > 0, or the uniform pick when
    // T is not positive); the chunk holding the target overwrites it
    if (tid == 0) idx[t] = (T > 0.0 && lastpos >= 0) ? (int64_t)lastpos : uniform_pick;
    __syncthreads();
    if (!(T > 0.0)) return;
    const double target = ut * T;
    if (!(target < T)) return;
    const double O = wofs[wid], B = tb[tid];
    // the thread's next thread's first offset, in the same form (its E at L = 0)
    const double Enext = (tid + 1 < SEED_T) ? wofs[(tid + 1) >> 5] + tb[tid + 1] : T;
    if (!(O + B <= target && target < Enext)) return;  // not this thread's chunks
    double L = 0.0;
    for (int64_t c = c0; c < c1; c++) {
        const double E0 = O + (B + L);
        L += csum[c];
        const double E1 = (c + 1 < c1) ? O + (B + L) : Enext;
        if (E0 <= target && target < E1) {  // the chunk: its rows in order
            const int64_t lo = c * ch, hi = lo + ch < n ? lo + ch : n;
            double acc = E0;
            int64_t pick = clast[c];
            // eight rows' loads in flight, then their additions in row order
            for (int64_t i = lo; i < hi; i += 8) {
                double v[8];
#pragma unroll
                for (int q = 0; q < 8; q++) v[q] = (i + q < hi) ? D2[i + q] : 0.0;
                int hit = -1;
#pragma unroll
                for (int q = 0; q < 8; q++) {
                    if (hit < 0 && i + q < hi) {
                        acc += v[q];
                        if (acc > target) hit = q;
                    }
                }
                if (hit >= 0) {
                    pick = i + hit;
                    break;
                }
            }
            if (pick >= 0) idx[t] = pick;
            return;
        }
    }
}

__global__ void k_seed_gather(const float* __restrict__ X, int d, const int64_t* __restrict__ idx, int k,
                              float* __restrict__ C) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)k * d;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e / d;
        C[e] = X[idx[t] * d + (e - t * d)];
    }
}

size_t seed_chunk_count(int64_t n) { return (size_t)(n < SEED_NC ? n : SEED_NC); }

cudaError_t launch_seed_pp(const float* X, int64_t n, int d, int k, const double* u_dev, double* D2, int64_t* idx,
                           double* csum, int64_t* clast, float* C_out, int num_sms, cudaStream_t st, int* nlaunch) {
    *nlaunch = 0;
    const int64_t ncmax = (int64_t)seed_chunk_count(n);
    const int64_t ch = (n + ncmax - 1) / ncmax, nc = (n + ch - 1) / ch;
    const unsigned cb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nc + 7) / 8, (int64_t)num_sms * 8));
    const bool vec = d % 4 == 0 && ((uintptr_t)X % 16) == 0;
    const int lpr = df_lpr(d), nv4 = df_nv4(d);
    void (*kern)(const float*, int64_t, int, const int64_t*, int, bool, double*) = nullptr;
    void (*small)(const float*, int64_t, const int64_t*, int, bool, double*) = nullptr;
    if (d <= 8) {
        switch (d) {
#define KM_SS(DD) \
    case DD: small = k_seed_small<DD>; break;
            KM_SS(1) KM_SS(2) KM_SS(3) KM_SS(4) KM_SS(5) KM_SS(6) KM_SS(7) KM_SS(8)
#undef KM_SS
        }
    } else {
#define KM_SD(NV, L)                                        \
    if (nv4 == NV && lpr == L) {                            \
        if (vec) kern = k_seed_dist<NV, L, true>;           \
        else kern = k_seed_dist<NV, L, false>;              \
    }
        KM_SD(1, 8) KM_SD(1, 16) KM_SD(1, 32) KM_SD(2, 32) KM_SD(4, 32)
#undef KM_SD
        if (!kern) return cudaErrorInvalidValue;
    }
    unsigned blocks;
    if (small) {
        blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8));
    } else {
        int per_sm = 1;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
        if (e != cudaSuccess) return e;
        const int rows_per_warp_pass = (nv4 == 4 ? 2 : 4) * (32 / lpr);
        const int64_t warps_needed = (n + rows_per_warp_pass - 1) / rows_per_warp_pass;
        blocks = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((warps_needed + 7) / 8, (int64_t)num_sms * std::max(per_sm, 1)));
    }
    k_seed_pick<<<1, SEED_T, 0, st>>>(D2, n, ch, nc, csum, clast, u_dev, 0, idx);
    (*nlaunch)++;
    for (int t = 0; t + 1 < k; t++) {
        if (small) small<<<blocks, 256, 0, st>>>(X, n, idx, t, t == 0, D2);
        else kern<<<blocks, 256, 0, st>>>(X, n, d, idx, t, t == 0, D2);
        k_seed_chunks<<<cb, 256, 0, st>>>(D2, n, ch, nc, csum, clast);
        k_seed_pick<<<1, SEED_T, 0, st>>>(D2, n, ch, nc, csum, clast, u_dev, t + 1, idx);
        *nlaunch += 3;
    }
    const unsigned gb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)k * d + 255) / 256, 4096));
    k_seed_gather<<<gb, 256, 0, st>>>(X, d, idx, k, C_out);
    (*nlaunch)++;
    return cudaGetLastError();
}

}  // namespace km
