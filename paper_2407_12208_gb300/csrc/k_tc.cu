// k_tc.cu -- the tensor-core screening kernel: Eq. (dist-blas3)'s cross term
// X~ C~^T on tcgen05 with the expanded formula, the reliability test of
// Section 4.3 and the running argmin fused into the epilogue.  The n x k
// distance matrix is never written to HBM in assign mode.
//
// Persistent CTAs (one per SM, 192 threads):
//   warp 0      TMA producer: a 128-row block of X~ (all of K, 128-byte
//               swizzled atoms) per row block, and BN-row tiles of C~ through
//               an NS-stage ring.
//   warp 1      allocates TMEM (2 x BN fp32 columns) and issues
//               tcgen05.mma (M=128, N=BN) from one elected lane into one of
//               two TMEM accumulators, so the epilogue of tile t overlaps the
//               MMAs of tile t+1.
//   warps 2..5  epilogue: thread = row (TMEM lane).  Per pair:
//               e = q_j - 2 s g (one FMA), chunk minimum, and only when the
//               chunk can hold a candidate or a flagged pair, the slow path:
//               d^ = p + e, the exact reliability test, and a candidate
//               append.  Candidates: every j with d^_j <= d^_min + 2 B_max,
//               the only centres that can be the true argmin.
//
// All waits are bounded (common.cuh); a timeout sets the status word and the
// CTA winds down.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace km {

constexpr int TC_THREADS = 192;
constexpr int TC_BM = 128;
constexpr int SMEM_BUDGET = 225 * 1024;

struct TcLayout {
    int BN, NA, NS, kchunks;
    size_t a_bytes, b_bytes, q_off, scr_off, bar_off, total;
};

__host__ __device__ inline TcLayout tc_layout(int BN, int kchunks, int k) {
    TcLayout L;
    L.BN = BN;
    L.kchunks = kchunks;
    L.a_bytes = (size_t)kchunks * TC_BM * 128;
    L.b_bytes = (size_t)kchunks * BN * 128;
    const int nt = (k + BN - 1) / BN;
    const size_t qbytes = (((size_t)nt * BN * 4) + 1023) & ~(size_t)1023;
    const size_t scr = (size_t)32 * TC_BM * 4;  // per-thread staging of one 32-column chunk
    const size_t fixed = 1024 /*align slack*/ + qbytes + scr + 1024 /*barriers*/;
    L.NA = 2;
    size_t rem = (size_t)SMEM_BUDGET - fixed - 2 * L.a_bytes;
    if ((long long)rem < (long long)(2 * L.b_bytes)) {
        L.NA = 1;
        rem = (size_t)SMEM_BUDGET - fixed - L.a_bytes;
    }
    L.NS = (int)(rem / L.b_bytes);
    if (L.NS > 6) L.NS = 6;
    L.q_off = (size_t)L.NA * L.a_bytes + (size_t)L.NS * L.b_bytes;
    L.scr_off = L.q_off + qbytes;
    L.bar_off = L.scr_off + scr;
    L.total = L.bar_off + 1024 + 1024;
    return L;
}

static int pick_bn(int kchunks, int k) {
    if (k <= 128) return 128;
    TcLayout L = tc_layout(256, kchunks, k);
    return (L.NS >= 2) ? 256 : 128;
}

template <int FMT, int BN, int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmC, const TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const TcLayout L = tc_layout(BN, a.kchunks, a.k);
    unsigned char* sA = smem;
    unsigned char* sB = smem + (size_t)L.NA * L.a_bytes;
    float* qs = reinterpret_cast<float*>(smem + L.q_off);
    float* escr = reinterpret_cast<float*>(smem + L.scr_off);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* a_full = bars;            // [2]
    uint64_t* a_empty = bars + 2;       // [2]
    uint64_t* b_full = bars + 4;        // [6]
    uint64_t* b_empty = bars + 10;      // [6]
    uint64_t* acc_full = bars + 16;     // [2]
    uint64_t* acc_empty = bars + 18;    // [2]
    uint64_t* mma_done = bars + 20;     // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 22);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 23);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nrb = (a.n + TC_BM - 1) / TC_BM;
    const int NT = (a.k + BN - 1) / BN;
    constexpr uint32_t ESIZE = (FMT == 2) ? 1 : 2;
    constexpr int ATOM_ELEMS = 128 / ESIZE;
    unsigned* status = &a.cnt->status;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) { mbar_init(&a_full[i], 1); mbar_init(&a_empty[i], 1); }
        for (int i = 0; i < 6; i++) { mbar_init(&b_full[i], 1); mbar_init(&b_empty[i], 1); }
        for (int i = 0; i < 2; i++) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 4); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * BN);
    if (warp >= 2) {
        // column norms q_j (+inf past k so padded columns never win)
        for (int j = threadIdx.x - 64; j < NT * BN; j += 128) qs[j] = (j < a.k) ? a.cstat[j].x : INFINITY;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            tma_prefetch_desc(&tmX);
            tma_prefetch_desc(&tmC);
            int64_t bload = 0;
            int iter = 0;
            bool ok = true;
            for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, iter++) {
                const int ab = iter % L.NA;
                if (iter >= L.NA) ok = mbar_wait(&a_empty[ab], ((iter / L.NA) - 1) & 1, abort_flag, status);
                if (!ok) break;
                mbar_arrive_expect_tx(&a_full[ab], (uint32_t)L.a_bytes);
                for (int kc = 0; kc < a.kchunks; kc++)
                    tma_load_2d(sA + (size_t)ab * L.a_bytes + (size_t)kc * TC_BM * 128, &tmX, &a_full[ab],
                                kc * ATOM_ELEMS, (int)(rb * TC_BM));
                for (int nt = 0; nt < NT; nt++, bload++) {
                    const int s = (int)(bload % L.NS);
                    if (bload >= L.NS) ok = mbar_wait(&b_empty[s], ((bload / L.NS) - 1) & 1, abort_flag, status);
                    if (!ok) break;
                    mbar_arrive_expect_tx(&b_full[s], (uint32_t)L.b_bytes);
                    for (int kc = 0; kc < a.kchunks; kc++)
                        tma_load_2d(sB + (size_t)s * L.b_bytes + (size_t)kc * BN * 128, &tmC, &b_full[s],
                                    kc * ATOM_ELEMS, nt * BN);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_make(FMT == 0 ? 0u : (FMT == 1 ? 1u : 0u), TC_BM, BN);
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
            int64_t bcons = 0, tcount = 0;
            int iter = 0;
            bool ok = true;
            for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, iter++) {
                const int ab = iter % L.NA;
                ok = mbar_wait(&a_full[ab], (iter / L.NA) & 1, abort_flag, status);
                if (!ok) break;
                for (int nt = 0; nt < NT; nt++, bcons++, tcount++) {
                    const int s = (int)(bcons % L.NS);
                    ok = mbar_wait(&b_full[s], (bcons / L.NS) & 1, abort_flag, status);
                    if (!ok) break;
                    const int accb = (int)(tcount & 1);
                    if (tcount >= 2) ok = mbar_wait(&acc_empty[accb], ((tcount >> 1) - 1) & 1, abort_flag, status);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)(accb * BN);
                    for (int kc = 0; kc < a.kchunks; kc++) {
                        const uint32_t aa = a0 + (uint32_t)(ab * L.a_bytes + (size_t)kc * TC_BM * 128);
                        const uint32_t bb = b0 + (uint32_t)(s * L.b_bytes + (size_t)kc * BN * 128);
#pragma unroll
                        for (int kk = 0; kk < 4; kk++) {
                            const uint64_t ad = sdesc_sw128(aa + kk * 32);
                            const uint64_t bd = sdesc_sw128(bb + kk * 32);
                            if (FMT == 2)
                                mma_f8(dt, ad, bd, idesc, (kc | kk) ? 1u : 0u);
                            else
                                mma_f16(dt, ad, bd, idesc, (kc | kk) ? 1u : 0u);
                        }
                    }
                    mma_commit(&b_empty[s]);
                    mma_commit(&acc_full[accb]);
                }
                if (!ok) break;
                mma_commit(&a_empty[ab]);
            }
            // drain: every issued MMA completes before TMEM is released
            mma_commit(mma_done);
            mbar_wait_drain(mma_done, 0, status);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue
        const int quarter = warp & 3;  // TMEM lanes this warp may access
        const int r_in = quarter * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        const ColMax cm = *a.colmax;
        const TestParams tp = a.tp;
        int64_t tcount = 0;
        unsigned long long nflag_total = 0;
        bool ok = true;
        for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x) {
            const int64_t row = rb * TC_BM + r_in;
            const bool valid = row < a.n;
            float4 xs = make_float4(0.f, 0.f, 0.f, 0.f);
            float rs = 1.0f;
            if (valid) {
                xs = a.xstat[row];
                if (FMT == 2) rs = a.xscale[row];
            }
            const float p = xs.x;
            const float neg2s = -2.0f * rs * cm.cscale;
            // bound B_ij = (a1 ||c_j|| + a2 ||c~_j - c_j|| + a3 ||c~_j|| + kn (p + q_j)) * bsafe
            const float a1 = 2.0f * xs.w, a2 = 2.0f * xs.z, a3 = tp.kacc * xs.z;
            const float bmax = (a1 * cm.nc + a2 * cm.nrc + a3 * cm.ncq + tp.kn * (p + cm.q)) * tp.bsafe;
            float F;  // no pair with d^ > F can be flagged
            if (tp.test == 0) F = tp.rho * bmax;
            else if (tp.test == 1) F = tp.paper_coef * (xs.z * xs.z + cm.ncq2) * 1.0001f;
            else F = -INFINITY;
            const float Fe = (tp.test == 2) ? -INFINITY : F - p + fabsf(F) * 1e-6f;  // in e = d^ - p units
            const float W = 2.0f * bmax * 1.001f + 1e-30f;      // candidate window
            float m = INFINITY;
            int cnt = 0, ovf = 0, nflag = 0;
            int2* crow = a.cand + (size_t)(valid ? row : 0) * a.L;

            for (int nt = 0; nt < NT; nt++, tcount++) {
                const int accb = (int)(tcount & 1);
                ok = mbar_wait(&acc_full[accb], (tcount >> 1) & 1, abort_flag, status);
                if (!ok) break;
                tc_fence_after();
                for (int ch = 0; ch < BN / 32; ch++) {
                    const int col0 = nt * BN + ch * 32;
                    if (col0 >= a.k) break;
                    float v[32];
                    __syncwarp();
                    tmem_ld32(tmem_base + lane_addr + (uint32_t)(accb * BN + ch * 32), v);
                    if (valid) {
                    const float4* q4 = reinterpret_cast<const float4*>(qs + col0);
                    float e[32];
                    float cmin = INFINITY;
#pragma unroll
                    for (int t4 = 0; t4 < 8; t4++) {
                        const float4 qq = q4[t4];
                        e[4 * t4 + 0] = fmaf(v[4 * t4 + 0], neg2s, qq.x);
                        e[4 * t4 + 1] = fmaf(v[4 * t4 + 1], neg2s, qq.y);
                        e[4 * t4 + 2] = fmaf(v[4 * t4 + 2], neg2s, qq.z);
                        e[4 * t4 + 3] = fmaf(v[4 * t4 + 3], neg2s, qq.w);
                    }
                    if (MODE == 0) {
#pragma unroll
                        for (int t = 0; t < 32; t++) cmin = fminf(cmin, e[t]);
                        m = fminf(m, cmin);
                        const float cthr = m + W;
                        const float sthr = fmaxf(cthr, Fe);
                        if (cmin <= sthr) {
                            float* scr = escr + r_in;
#pragma unroll
                            for (int t = 0; t < 32; t++) scr[t * TC_BM] = e[t];
#pragma unroll 1
                            for (int t = 0; t < 32; t++) {
                                const float et = scr[t * TC_BM];
                                if (et <= sthr) {
                                    const int j = col0 + t;
                                    const float dh = p + et;
                                    if (dh <= F) {
                                        bool fl;
                                        if (tp.test == 0) {
                                            const float4 cs = a.cstat[j];
                                            const float B =
                                                (a1 * cs.y + a2 * cs.w + a3 * cs.z + tp.kn * (p + cs.x)) * tp.bsafe;
                                            fl = dh <= tp.rho * B;
                                        } else {
                                            const float4 cs = a.cstat[j];
                                            fl = dh <= tp.paper_coef * (xs.z * xs.z + cs.z * cs.z);
                                        }
                                        nflag += fl ? 1 : 0;
                                    }
                                    if (et <= cthr && !ovf) {
                                        if (cnt == a.L) {
                                            // compact: keep only entries still inside the window
                                            int w = 0;
                                            const float lim = p + cthr;
                                            for (int r2 = 0; r2 < a.L; r2++) {
                                                const int2 c = crow[r2];
                                                if (__int_as_float(c.y) <= lim) crow[w++] = c;
                                            }
                                            cnt = w;
                                        }
                                        if (cnt < a.L) crow[cnt++] = make_int2(j, __float_as_int(dh));
                                        else ovf = 1;
                                    }
                                }
                            }
                        }
                    } else {
                        // distance-matrix mode: Alg. 2's d = max(d^, 0) and its flag, every pair
                        float* drow = a.D + (size_t)row * a.k;
                        float* scr = escr + r_in;
#pragma unroll
                        for (int t = 0; t < 32; t++) scr[t * TC_BM] = e[t];
#pragma unroll 1
                        for (int t = 0; t < 32; t++) {
                            const int j = col0 + t;
                            if (j >= a.k) break;
                            const float dh = fmaxf(p + scr[t * TC_BM], 0.0f);
                            bool fl = false;
                            if (dh <= F) {
                                const float4 cs = a.cstat[j];
                                if (tp.test == 0) {
                                    const float B = (a1 * cs.y + a2 * cs.w + a3 * cs.z + tp.kn * (p + cs.x)) * tp.bsafe;
                                    fl = dh <= tp.rho * B;
                                } else {
                                    fl = dh <= tp.paper_coef * (xs.z * xs.z + cs.z * cs.z);
                                }
                            }
                            drow[j] = dh;
                            if (fl) {
                                nflag++;
                                const unsigned long long pos = atomicAdd(a.flag_queue_len, 1ull);
                                if ((int64_t)pos < a.flag_queue_cap) a.flag_queue[pos] = make_int2((int)row, j);
                                if (a.flag_bits) {
                                    const unsigned long long bit = (unsigned long long)row * a.k + j;
                                    atomicOr(&a.flag_bits[bit >> 5], 1u << (bit & 31));
                                }
                            }
                        }
                    }
                    }  // valid
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[accb]);
            }
            if (!ok) break;
            if (valid && MODE == 0) a.rowinfo[row] = make_int4(cnt, ovf, nflag, __float_as_int(p + m));
            nflag_total += (unsigned long long)nflag;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nflag_total += __shfl_xor_sync(0xffffffffu, nflag_total, off);
        if (lane == 0 && nflag_total) atomicAdd(&a.cnt->flagged, nflag_total);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, 2 * BN);
}

// ----------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

static cudaError_t make_map(CUtensorMap* m, const void* base, int fmt, int64_t rows, int ldq, int box_rows) {
    EncodeTiledFn enc = get_encode();
    if (!enc) return cudaErrorNotSupported;
    const uint32_t esize = (fmt == 2) ? 1 : 2;
    CUtensorMapDataType dt = (fmt == 0)   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                             : (fmt == 1) ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                          : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    cuuint64_t dims[2] = {(cuuint64_t)ldq, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ldq * esize};
    cuuint32_t box[2] = {128u / esize, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(m, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

size_t tc_smem_bytes(int fmt, int d, int k) {
    const int esize = (fmt == 2) ? 1 : 2;
    const int ldq = (fmt == 2) ? ((d + 15) / 16) * 16 : ((d + 7) / 8) * 8;
    const int kchunks = (ldq * esize + 127) / 128;
    const int bn = pick_bn(kchunks, k);
    TcLayout L = tc_layout(bn, kchunks, k);
    if (L.NS < 2) return 0;
    return L.total;
}

template <int FMT, int BN, int MODE>
static cudaError_t launch_one(const CUtensorMap& mx, const CUtensorMap& mc, const TcArgs& a, int num_sms,
                              cudaStream_t st) {
    TcLayout L = tc_layout(BN, a.kchunks, a.k);
    if (L.NS < 2) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_tc<FMT, BN, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.total);
    if (e != cudaSuccess) return e;
    const int64_t nrb = (a.n + TC_BM - 1) / TC_BM;
    const int grid = (int)std::min<int64_t>(nrb, (int64_t)num_sms);
    k_tc<FMT, BN, MODE><<<grid, TC_THREADS, L.total, st>>>(mx, mc, a);
    return cudaGetLastError();
}

template <int FMT, int MODE>
static cudaError_t launch_fmt(const CUtensorMap& mx, const CUtensorMap& mc, const TcArgs& a, int bn, int num_sms,
                              cudaStream_t st) {
    if (bn == 256) return launch_one<FMT, 256, MODE>(mx, mc, a, num_sms, st);
    return launch_one<FMT, 128, MODE>(mx, mc, a, num_sms, st);
}

cudaError_t launch_tc(const void* Xq, const void* Cq, int ldq, const TcArgs& a, int num_sms, cudaStream_t st) {
    const int bn = pick_bn(a.kchunks, a.k);
    CUtensorMap mx, mc;
    cudaError_t e = make_map(&mx, Xq, a.fmt, a.n, ldq, TC_BM);
    if (e != cudaSuccess) return e;
    e = make_map(&mc, Cq, a.fmt, a.k, ldq, bn);
    if (e != cudaSuccess) return e;
    if (a.mode == 0) {
        if (a.fmt == 0) return launch_fmt<0, 0>(mx, mc, a, bn, num_sms, st);
        if (a.fmt == 1) return launch_fmt<1, 0>(mx, mc, a, bn, num_sms, st);
        return launch_fmt<2, 0>(mx, mc, a, bn, num_sms, st);
    }
    if (a.fmt == 0) return launch_fmt<0, 1>(mx, mc, a, bn, num_sms, st);
    if (a.fmt == 1) return launch_fmt<1, 1>(mx, mc, a, bn, num_sms, st);
    return launch_fmt<2, 1>(mx, mc, a, bn, num_sms, st);
}

}  // namespace km
