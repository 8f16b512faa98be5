// k_tc.cu -- the tensor-core screening kernel: Eq. (dist-blas3)'s cross term
// X~ C~^T on tcgen05 with the expanded formula, the reliability test of
// Section 4.3 and the running argmin fused into the epilogue.  The n x k
// distance matrix is never written to HBM in assign mode.
//
// Persistent CTAs (one per SM, 64 + 128 x TC_NG threads):
//   warp 0      TMA producer: a 128-row block of X~ (all of K, 128-byte
//               swizzled atoms) per row block, and 128-row tiles of C~ through
//               an NS-stage ring.
//   warp 1      allocates TMEM (4 accumulators of 128 fp32 columns) and issues
//               tcgen05.mma (M=128, N=128) from one elected lane, so the
//               epilogues of earlier tiles overlap the MMAs of later ones.
//   warps 2..   TC_NG epilogue groups of four warps; group g drains the tiles
//               t with t mod TC_NG == g, and the groups share their running
//               row minima.  Thread = row (TMEM lane).  Per pair e = q_j - 2 s g
//               (one packed FMA per two columns); per quad of columns its
//               minimum; only the quads that can hold a candidate or a flagged
//               pair take the slow path: d^ = p + e, the exact reliability
//               test, and one list entry per quad with candidates (its index,
//               the mask of its candidate columns, its smallest d^).
//               Candidates: every j with d^_j <= d^_min + 2 B_max, the only
//               centres that can be the true argmin.
//
// All waits are bounded (common.cuh); a timeout sets the status word and the
// CTA winds down.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace km {

constexpr int TC_NG = TC_GROUPS;             // epilogue groups of four warps
constexpr int TC_THREADS = 64 + 128 * TC_NG;  // producer warp, MMA warp, epilogue warps
constexpr int TC_BM = 128;
constexpr int TC_L = TC_LIST;  // candidate slots per row and epilogue group
constexpr int SMEM_BUDGET = 227 * 1024;

struct TcLayout {
    int BN, NA, NS, kchunks;
    size_t a_bytes, b_bytes, list_off, stage_off, bar_off, total;
};

// Epilogue variants (TC_SV_*, internal.h): the columns per step (64, or 32
// for C32) and the shared-memory staging of the walked quads: a float4 per
// quad and lane, quad-major, for the step's 16 quads (FULL: 8 KB per warp) or
// 8 quads at a time (HALF, C32: 4352 bytes per warp, which also holds the
// distance-matrix mode's 32 x 33 transposed tile); REG stages nothing (quads
// picked from registers).  Smaller staging leaves room for a second A stage.
__host__ __device__ constexpr int tc_cw(int sv) { return sv == TC_SV_C32 ? 1 : 2; }
__host__ __device__ constexpr size_t tc_stage_warp_bytes(int sv) {
    return sv == TC_SV_REG ? 0 : (sv == TC_SV_FULL ? (size_t)16 * 32 * 16 : (size_t)4352);
}
__host__ __device__ inline TcLayout tc_layout(int BN, int kchunks, int k, int sv) {
    TcLayout L;
    L.BN = BN;
    L.kchunks = kchunks;
    L.a_bytes = (size_t)kchunks * TC_BM * 128;
    L.b_bytes = (size_t)kchunks * BN * 128;
    (void)k;
    const size_t lists = (size_t)TC_NG * (TC_L + 1) * TC_BM * 4   // per-row candidate lists (+1 dummy slot) of every group
                         + (size_t)TC_NG * TC_BM * 8;         // per-row running minimum published by each group
    const size_t stage = (size_t)TC_NG * 4 * tc_stage_warp_bytes(sv);
    const size_t fixed = 1024 /*align slack*/ + lists + stage + 256 /*barriers*/;
    L.NA = 2;
    size_t rem = (size_t)SMEM_BUDGET - fixed - 2 * L.a_bytes;
    if ((long long)rem < (long long)(2 * L.b_bytes)) {
        L.NA = 1;
        rem = (size_t)SMEM_BUDGET - fixed - L.a_bytes;
    }
    L.NS = (int)(rem / L.b_bytes);
    if (L.NS > 6) L.NS = 6;
    L.list_off = (size_t)L.NA * L.a_bytes + (size_t)L.NS * L.b_bytes;
    L.stage_off = L.list_off + lists;
    L.bar_off = L.stage_off + stage;
    L.total = L.bar_off + 256 + 1024;
    return L;
}

static int pick_bn(int kchunks, int k) {
    (void)kchunks;
    (void)k;
    return 128;  // four accumulators: each epilogue group double-buffered
}

// Asynchronous TMEM load (32 lanes x 32 columns) and the matching wait; the
// wait names the destination registers so no read of them is scheduled
// before it.
KM_DEV void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
KM_DEV void tmem_wait_ld(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]),
                   "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]),
                   "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]),
                   "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]),
                   "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])
                 :
                 : "memory");
}

// 32 lanes x 4 consecutive columns, waited for.
KM_DEV void tmem_ld4(uint32_t taddr, uint32_t (&r)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
}

// Reliability test of one pair (rare path, kept out of line so the hot loop
// stays small; scalar arguments, so nothing goes through the stack): tc form
// rho * B(x, c) or Alg. 2's rho c_A gamma^l_{d+2} (||x~||^2 + ||c~||^2).
__device__ __noinline__ bool pair_flagged(int test, float rho, float kn, float bsafe, float paper_coef,
                                          const float4* cstat, int j, float dh, float a1, float a2, float a3, float p,
                                          float nxq) {
    const float4 cs = cstat[j];
    if (test == 0) {
        const float B = (a1 * cs.y + a2 * cs.w + a3 * cs.z + kn * (p + cs.x)) * bsafe;
        return dh <= rho * B;
    }
    return dh <= paper_coef * (nxq * nxq + cs.z * cs.z);
}
#define KM_PAIR_FLAGGED(j, dh) \
    pair_flagged(tp.test, tp.rho, tp.kn, tp.bsafe, tp.paper_coef, a.cstat, (j), (dh), a1, a2, a3, p, xs.z)

// Keep only the list entries still inside the window (slot-major layout):
// all slots are read first (independent loads), then packed with predicated
// stores.
KM_DEV int compact_list(uint32_t* list, int cnt, float lim, uint32_t emask, float lscale) {
    uint32_t c[TC_L];
#pragma unroll
    for (int r = 0; r < TC_L; r++) c[r] = list[r * TC_BM];
    int w = 0;
#pragma unroll
    for (int r = 0; r < TC_L; r++) {
        const bool keep = r < cnt && cand_lower(c[r], emask, lscale) <= lim;
        if (keep) list[w * TC_BM] = c[r];
        w += keep ? 1 : 0;
    }
    return w;
}

// Three-input minimum (one instruction on sm_100 and later; no NaN reaches it).
KM_DEV float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <int FMT, int BN, int MODE, int SV>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmC, const TcArgs a) {
    extern __shared__ unsigned char smem_raw[];
    // 1024-byte aligned base, derived from the shared array by an offset so that
    // every pointer below stays in the shared state space (LDS/STS, not generic)
    const uint32_t sraw = smem_u32(smem_raw);
    unsigned char* smem = smem_raw + (((sraw + 1023u) & ~1023u) - sraw);
    constexpr bool STG = SV != TC_SV_REG;
    constexpr int TC_CW = tc_cw(SV);  // 32-column TMEM chunks per epilogue step
    const TcLayout L = tc_layout(BN, a.kchunks, a.k, SV);
    unsigned char* sA = smem;
    unsigned char* sB = smem + (size_t)L.NA * L.a_bytes;
    // q_j of every tile column (+inf on the padding: padded columns never win),
    // read through the read-only cache: one broadcast load per float4
    const float* __restrict__ qg = a.qpad;
    uint32_t* lists = reinterpret_cast<uint32_t*>(smem + L.list_off);
    float2* mshare = reinterpret_cast<float2*>(smem + L.list_off + (size_t)TC_NG * (TC_L + 1) * TC_BM * 4);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + L.bar_off);
    uint64_t* a_full = bars;            // [2]
    uint64_t* a_empty = bars + 2;       // [2]
    uint64_t* b_full = bars + 4;        // [6]
    uint64_t* b_empty = bars + 10;      // [6]
    uint64_t* acc_full = bars + 16;     // [4]
    uint64_t* acc_empty = bars + 20;    // [4]
    uint64_t* mma_done = bars + 24;     // [1]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 26);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + 27);
    // TMEM holds NBUF accumulators of BN columns (512 columns in all); tile t
    // uses buffer t % NBUF and is drained by epilogue group t % TC_NG, so the
    // groups work on consecutive tiles at once and the MMA fills the buffers
    // ahead of them.
    constexpr int NBUF = 512 / BN;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t nrb = (a.n + TC_BM - 1) / TC_BM;
    const int NT = (a.k + BN - 1) / BN;
    constexpr uint32_t ESIZE = (FMT == 2) ? 1 : 2;
    constexpr int ATOM_ELEMS = 128 / ESIZE;
    unsigned* status = &a.cnt->status;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; i++) { mbar_init(&a_full[i], 1); mbar_init(&a_empty[i], 1); }
        for (int i = 0; i < 6; i++) { mbar_init(&b_full[i], 1); mbar_init(&b_empty[i], 1); }
        for (int i = 0; i < NBUF; i++) { mbar_init(&acc_full[i], 1); mbar_init(&acc_empty[i], 4); }
        mbar_init(mma_done, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 512);
    if (warp >= 2) {
        for (int j = threadIdx.x - 64; j < TC_NG * TC_BM; j += TC_THREADS - 64)
            mshare[j] = make_float2(INFINITY, __int_as_float(-1));
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
            constexpr uint32_t idesc = idesc_make(FMT == 1 ? 1u : 0u, TC_BM, BN);
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
                    const int accb = (int)(tcount % NBUF);
                    if (tcount >= NBUF) ok = mbar_wait(&acc_empty[accb], ((tcount / NBUF) - 1) & 1, abort_flag, status);
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
        // TC_NG groups of four warps; group g drains the tiles t with
        // t mod TC_NG == g, so the groups overlap.
        const int g = (warp - 2) >> 2;
        const int quarter = warp & 3;  // TMEM lanes this warp may access
        const int r_in = quarter * 32 + lane;
        const uint32_t lane_addr = (uint32_t)(quarter * 32) << 16;
        uint32_t* list = lists + (size_t)g * (TC_L + 1) * TC_BM + r_in;  // slot s at list[s * TC_BM]; slot TC_L is a dummy
        const uint32_t lbase = smem_u32(list);                            // the same as a shared address
        const ColMax cm = *a.colmax;
        const TestParams tp = a.tp;
        const uint32_t emask = (1u << a.ebits) - 1u;
        const float lscale = __uint_as_float((uint32_t)(127 + a.ebits - 23) << 23);  // 2^(ebits - 23)
        unsigned long long nflag_total = 0;
        bool ok = true;
        int iter = 0;
        for (int64_t rb = blockIdx.x; rb < nrb && ok; rb += gridDim.x, iter++) {
            const int64_t row = rb * TC_BM + r_in;
            const bool valid = row < a.n;
            float4 xs = make_float4(0.f, 0.f, 0.f, 0.f);
            float rs = 1.0f;
            if (valid) {
                xs = a.xstat[row];
                if (FMT == 2) rs = a.xscale[row];
            }
            const float p = xs.x;
            // e = q_j - 2 s_i s_j g (E4M3: row and column scales, powers of two)
            const float neg2s = -2.0f * rs;
            // bound B_ij = (a1 ||c_j|| + a2 ||c~_j - c_j|| + a3 ||c~_j|| + kn (p + q_j)) * bsafe
            const float a1 = 2.0f * xs.w, a2 = 2.0f * xs.z, a3 = tp.kacc * xs.z;
            const float bmax = (a1 * cm.nc + a2 * cm.nrc + a3 * cm.ncq + tp.kn * (p + cm.q)) * tp.bsafe;
            float F;  // no pair with d^ > F can be flagged
            if (tp.test == 0) F = tp.rho * bmax;
            else if (tp.test == 1) F = tp.paper_coef * (xs.z * xs.z + cm.ncq2) * 1.0001f;
            else F = -INFINITY;
            if (!valid) F = -INFINITY;  // rows past n: no flags, no candidates
            const float Fe = (F == -INFINITY) ? -INFINITY : F - p + fabsf(F) * 1e-6f;  // in e = d^ - p units
            // every pair with d^ <= Fall is flagged whatever its column: the smallest
            // threshold over the centres, less a margin for its fp32 evaluation
            float Fall;
            if (tp.test == 0)
                Fall = tp.rho * (a1 * cm.nc_min + a2 * cm.nrc_min + a3 * cm.ncq_min + tp.kn * (p + cm.q_min)) * tp.bsafe;
            else if (tp.test == 1)
                Fall = tp.paper_coef * (xs.z * xs.z + cm.ncq2_min);
            else
                Fall = -INFINITY;
            Fall = valid ? Fall * (1.0f - 1.0f / 65536.0f) - fabsf(Fall) * 1e-6f : -INFINITY;
            const float W = 2.0f * bmax * 1.001f + 1e-30f;      // candidate window
            float m = INFINITY;
            int cnt = 0, ovf = 0, nflag = 0;

            for (int nt = 0; nt < NT; nt++) {
                const int64_t tc = (int64_t)iter * NT + nt;
                if ((int)(tc % TC_NG) != g) continue;
                const int buf = (int)(tc % NBUF);
                ok = mbar_wait(&acc_full[buf], (uint32_t)((tc / NBUF) & 1), abort_flag, status);
                if (!ok) break;
                tc_fence_after();
                const int nch = min(BN / 32, (a.k - nt * BN + 31) / 32);
                const uint32_t tbase = tmem_base + lane_addr + (uint32_t)(buf * BN);
                if (MODE == 0) {
                    // TC_CW chunks of 32 columns per step (padded columns have q = +inf:
                    // they never qualify)
                    constexpr int NCOL = 32 * TC_CW, NQ = NCOL / 4;
                    const int nchs = ((nch + TC_CW - 1) / TC_CW) * TC_CW;
                    for (int ch = 0; ch < nchs; ch += TC_CW) {
                        const int col0 = nt * BN + ch * 32;
                        uint32_t v[TC_CW][32];
                        __syncwarp();
#pragma unroll
                        for (int c = 0; c < TC_CW; c++) tmem_ld32_async(tbase + (uint32_t)((ch + c) * 32), v[c]);
                        const float4* q4 = reinterpret_cast<const float4*>(qg + col0);
                        float4 qv[NQ];
#pragma unroll
                        for (int t4 = 0; t4 < NQ; t4++) qv[t4] = __ldg(q4 + t4);
                        float4 sv[FMT == 2 ? NQ : 1];
                        if constexpr (FMT == 2) {
                            const float4* s4 = reinterpret_cast<const float4*>(a.spad + col0);
#pragma unroll
                            for (int t4 = 0; t4 < NQ; t4++) sv[t4] = __ldg(s4 + t4);
                        }
                        // the other groups' running minima of this row block (read before the wait)
                        float mo = INFINITY;
#pragma unroll
                        for (int h = 0; h < TC_NG; h++) {
                            const float2 o = mshare[h * TC_BM + r_in];
                            if (h != g && __float_as_int(o.y) == (int)rb) mo = fminf(mo, o.x);
                        }
#pragma unroll
                        for (int c = 0; c < TC_CW; c++) tmem_wait_ld(v[c]);
                        // e = q_j - 2 s g, two columns per packed FMA (each rounded as fmaf)
                        float e[NCOL];
                        const float2 n2 = make_float2(neg2s, neg2s);
#pragma unroll
                        for (int t4 = 0; t4 < NQ; t4++) {
                            const uint32_t* vv = v[t4 / 8];
                            const int o = (t4 & 7) * 4;
                            const float4 qq = qv[t4];
                            float2 g01 = make_float2(__uint_as_float(vv[o + 0]), __uint_as_float(vv[o + 1]));
                            float2 g23 = make_float2(__uint_as_float(vv[o + 2]), __uint_as_float(vv[o + 3]));
                            if constexpr (FMT == 2) {  // s_j g: exact (power-of-two scale)
                                g01 = __fmul2_rn(g01, make_float2(sv[t4].x, sv[t4].y));
                                g23 = __fmul2_rn(g23, make_float2(sv[t4].z, sv[t4].w));
                            }
                            const float2 lo = __ffma2_rn(g01, n2, make_float2(qq.x, qq.y));
                            const float2 hi = __ffma2_rn(g23, n2, make_float2(qq.z, qq.w));
                            e[4 * t4 + 0] = lo.x;
                            e[4 * t4 + 1] = lo.y;
                            e[4 * t4 + 2] = hi.x;
                            e[4 * t4 + 3] = hi.y;
                        }
                        // quad minima (they steer the slow path) and the minimum of the step
                        float qm[NQ];
#pragma unroll
                        for (int qd = 0; qd < NQ; qd++)
                            qm[qd] = fminf(fmin3(e[4 * qd + 0], e[4 * qd + 1], e[4 * qd + 2]), e[4 * qd + 3]);
                        float c4[NQ / 4];
#pragma unroll
                        for (int i = 0; i < NQ / 4; i++) c4[i] = fminf(fmin3(qm[4 * i], qm[4 * i + 1], qm[4 * i + 2]), qm[4 * i + 3]);
                        float cmin = c4[0];
#pragma unroll
                        for (int i = 1; i < NQ / 4; i++) cmin = fminf(cmin, c4[i]);
                        m = fminf(m, cmin);
                        // publish this group's running minimum; the others' (any upper bound
                        // of the row minimum keeps the window a superset of the final one)
                        mshare[g * TC_BM + r_in] = make_float2(m, __int_as_float((int)rb));
                        const float mm = fminf(m, mo);
                        const float cthr = mm + W;
                        const float sthr = valid ? fmaxf(cthr, Fe) : -INFINITY;
                        unsigned qmask = 0;
#pragma unroll
                        for (int qd = 0; qd < NQ; qd++) qmask |= (qm[qd] <= sthr) ? (1u << qd) : 0u;
                        // Slow path: each lane walks its own quads holding a candidate or a
                        // possibly flagged pair (the warp iterates as often as its busiest
                        // lane).  A quad with candidates becomes one list entry: its index,
                        // the mask of its columns inside the window and its smallest d^ (a
                        // lane with nothing to add writes the dummy slot).
                        if (__any_sync(0xffffffffu, qmask)) {
                            if (__any_sync(0xffffffffu, cnt > TC_L - 4 * TC_CW && !ovf)) {
                                // every lane packs its list (dropping entries that left the window)
                                const int cc = compact_list(list, cnt, p + cthr, emask, lscale);
                                if (!ovf) cnt = cc;
                            }
                            __syncwarp();
                            // Possibly flagged pairs (d^ <= F) lie in the qualifying quads:
                            // they are counted in the walk below, value by value (every
                            // d^ <= Fall is flagged whatever its column); a lane whose
                            // whole step lies under Fall counts the step at once.
                            const bool fstep = __any_sync(0xffffffffu, p + cmin <= F);
                            bool fwhole = false;
                            if (fstep && __any_sync(0xffffffffu, p + e[0] <= Fall)) {
                                float cmax = e[0];
#pragma unroll
                                for (int t = 1; t < NCOL; t++) cmax = fmaxf(cmax, e[t]);
                                fwhole = p + cmax <= Fall;  // padded columns hold +inf: never taken
                                nflag += fwhole ? NCOL : 0;
                            }
                            // one quad: its entry, and (FS) its flagged pairs while they are counted
                            // one by one; the walk is compiled twice so that the common walk,
                            // with no pair near its flag threshold, carries no flag arithmetic
                            auto take_quad = [&](auto fs, float x0, float x1, float x2, float x3, int jq, bool act) {
                                constexpr bool FS = decltype(fs)::value;
                                const unsigned mk = (x0 <= cthr ? 1u : 0u) | (x1 <= cthr ? 2u : 0u) |
                                                    (x2 <= cthr ? 4u : 0u) | (x3 <= cthr ? 8u : 0u);
                                const bool pc = act && mk != 0u && !ovf;
                                const bool room = cnt < TC_L;
                                const int slot = (pc && room) ? cnt : TC_L;
                                const float qmn = fminf(fmin3(x0, x1, x2), x3);
                                st_shared_u32(lbase + slot * (TC_BM * 4), quad_entry(jq >> 2, mk, p + qmn, emask));
                                ovf |= (pc && !room);
                                cnt += (pc && room) ? 1 : 0;
                                if constexpr (FS) {
                                    const float xs4[4] = {x0, x1, x2, x3};
#pragma unroll
                                    for (int c = 0; c < 4; c++) {
                                        const float dh = p + xs4[c];
                                        if (act && !fwhole && dh <= F)
                                            nflag += (dh <= Fall || KM_PAIR_FLAGGED(jq + c, dh)) ? 1 : 0;
                                    }
                                }
                            };
                            // A row whose list overflowed takes no more candidates: it walks
                            // its quads only while flagged pairs remain to be counted one by one.
                            const unsigned walk = (ovf && !(fstep && !fwhole)) ? 0u : qmask;
                            auto run_walk = [&](auto fs) {
                                if constexpr (STG) {
                                    // the lane's quads to walk staged in shared memory (quad-major:
                                    // the 32 lanes of a quad side by side, conflict-free both ways),
                                    // then one loop over them: a 16-byte read per quad.  Each lane
                                    // reads back only what it wrote itself.  HALF stages and walks
                                    // the step's two 32-column halves one after the other.
                                    constexpr int NH = SV == TC_SV_HALF ? 2 : 1, QH = NQ / NH;
                                    const uint32_t stg = smem_u32(smem) + (uint32_t)L.stage_off +
                                                         (uint32_t)((warp - 2) * tc_stage_warp_bytes(SV) + lane * 16);
#pragma unroll
                                    for (int hh = 0; hh < NH; hh++) {
                                        unsigned ph = (walk >> (QH * hh)) & ((1u << QH) - 1u);
#pragma unroll
                                        for (int qd = 0; qd < QH; qd++)
                                            if ((ph >> qd) & 1u)
                                                st_shared_v4(stg + qd * 512, e[4 * (QH * hh + qd)], e[4 * (QH * hh + qd) + 1],
                                                             e[4 * (QH * hh + qd) + 2], e[4 * (QH * hh + qd) + 3]);
                                        while (__any_sync(0xffffffffu, ph)) {
                                            const bool act = ph != 0;
                                            const int qd = act ? __ffs(ph) - 1 : 0;
                                            ph &= ph - 1;
                                            const float4 ev = ld_shared_v4(stg + qd * 512);
                                            take_quad(fs, ev.x, ev.y, ev.z, ev.w, col0 + 4 * (QH * hh + qd), act);
                                        }
                                    }
                                } else {
#pragma unroll
                                    for (int half = 0; half < TC_CW; half++) {
                                        unsigned ph = (walk >> (8 * half)) & 0xffu;
                                        const float* eh = e + 32 * half;
                                        while (__any_sync(0xffffffffu, ph)) {
                                            const bool act = ph != 0;
                                            const int qd = act ? __ffs(ph) - 1 : 0;
                                            ph &= ph - 1;
                                            // the quad's values picked from registers by a select tree
                                            const bool b0 = qd & 1, b1 = qd & 2, b2 = qd & 4;
                                            float et[4];
#pragma unroll
                                            for (int c = 0; c < 4; c++) {
                                                const float s0 = b0 ? eh[4 + c] : eh[c], s1 = b0 ? eh[12 + c] : eh[8 + c];
                                                const float s2 = b0 ? eh[20 + c] : eh[16 + c], s3 = b0 ? eh[28 + c] : eh[24 + c];
                                                const float t0 = b1 ? s1 : s0, t1 = b1 ? s3 : s2;
                                                et[c] = b2 ? t1 : t0;
                                            }
                                            take_quad(fs, et[0], et[1], et[2], et[3], col0 + 32 * half + 4 * qd, act);
                                        }
                                    }
                                }
                            };
                            if (fstep) run_walk(std::true_type{});
                            else run_walk(std::false_type{});
                        }
                    }
                } else {
                    // distance-matrix mode: Alg. 2's d = max(d^, 0) and its flag, every
                    // pair; when K fits two 128-byte atoms the warp's 32 rows x 32
                    // columns go through shared memory (lane = row, stride 33:
                    // conflict-free both ways) so that each store writes 32
                    // consecutive columns of one row
                    float* tr = reinterpret_cast<float*>(smem + L.stage_off) + (size_t)(warp - 2) * 32 * 33;
                    const int64_t row_w = rb * TC_BM + quarter * 32;  // the warp's first row
                    for (int ch = 0; ch < nch; ch++) {
                        const int col0 = nt * BN + ch * 32;
                        uint32_t v[32];
                        __syncwarp();
                        tmem_ld32_async(tbase + (uint32_t)(ch * 32), v);
                        tmem_wait_ld(v);
                        const float4* q4 = reinterpret_cast<const float4*>(qg + col0);
                        const float4* s4 = reinterpret_cast<const float4*>(a.spad + col0);
#pragma unroll
                        for (int t4 = 0; t4 < 8; t4++) {
                            const float4 qq = __ldg(q4 + t4);
                            const float4 sc = FMT == 2 ? __ldg(s4 + t4) : make_float4(1.f, 1.f, 1.f, 1.f);
                            const float ev[4] = {fmaf(__uint_as_float(v[4 * t4 + 0]) * sc.x, neg2s, qq.x),
                                                 fmaf(__uint_as_float(v[4 * t4 + 1]) * sc.y, neg2s, qq.y),
                                                 fmaf(__uint_as_float(v[4 * t4 + 2]) * sc.z, neg2s, qq.z),
                                                 fmaf(__uint_as_float(v[4 * t4 + 3]) * sc.w, neg2s, qq.w)};
#pragma unroll
                            for (int c = 0; c < 4; c++) {
                                const int t = 4 * t4 + c;
                                const int j = col0 + t;
                                const float dh = fmaxf(p + ev[c], 0.0f);
                                const bool fl = valid && j < a.k && (dh <= F) && KM_PAIR_FLAGGED(j, dh);
                                if (fl) {
                                    nflag++;
                                    const unsigned long long pos = atomicAdd(a.flag_queue_len, 1ull);
                                    if ((int64_t)pos < a.flag_queue_cap) a.flag_queue[pos] = make_int2((int)row, j);
                                    if (a.flag_bits) {
                                        const unsigned long long bit = (unsigned long long)row * a.k + j;
                                        atomicOr(&a.flag_bits[bit >> 5], 1u << (bit & 31));
                                    }
                                }
                                // a flagged pair is marked -1 until the fallback's value replaces it
                                if constexpr (STG) tr[lane * 33 + t] = fl ? -1.0f : dh;
                                else if (valid && j < a.k) a.D[(size_t)row * a.k + j] = fl ? -1.0f : dh;
                            }
                        }
                        if constexpr (!STG) continue;  // (wide rows: no room to stage)
                        __syncwarp();
                        const int j = col0 + lane;
#pragma unroll 4
                        for (int r = 0; r < 32; r++) {
                            const float val = tr[r * 33 + lane];
                            if (row_w + r < a.n && j < a.k) a.D[(size_t)(row_w + r) * a.k + j] = val;
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[buf]);
            }
            if (!ok) break;
            if (valid && MODE == 0) {
                // the row's list (slot-major: consecutive rows side by side), its
                // window W and this group's d^ minimum
                uint32_t* ccol = a.cand + (size_t)g * TC_L * a.n + row;
                for (int sl = 0; sl < cnt; sl++) ccol[(size_t)sl * a.n] = list[sl * TC_BM];
                a.rowinfo[row * TC_NG + g] = make_int4(cnt, ovf, __float_as_int(W), __float_as_int(p + m));
            }
            nflag_total += (unsigned long long)nflag;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) nflag_total += __shfl_xor_sync(0xffffffffu, nflag_total, off);
        if (lane == 0 && nflag_total) atomicAdd(&a.cnt->flagged, nflag_total);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tmem_dealloc(tmem_base, 512);
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
    TcLayout L = tc_layout(bn, kchunks, k, kchunks <= 2 ? TC_SV_HALF : TC_SV_REG);
    if (L.NS < 2) return 0;
    return L.total;
}

template <int FMT, int BN, int MODE, int SV>
static cudaError_t launch_one(const CUtensorMap& mx, const CUtensorMap& mc, const TcArgs& a, int num_sms,
                              cudaStream_t st) {
    TcLayout L = tc_layout(BN, a.kchunks, a.k, SV);
    if (L.NS < 2) return cudaErrorInvalidConfiguration;
    cudaError_t e = allow_max_smem(k_tc<FMT, BN, MODE, SV>);
    if (e != cudaSuccess) return e;
    const int64_t nrb = (a.n + TC_BM - 1) / TC_BM;
    const int grid = (int)std::min<int64_t>(nrb, (int64_t)num_sms);
    k_tc<FMT, BN, MODE, SV><<<grid, TC_THREADS, L.total, st>>>(mx, mc, a);
    return cudaGetLastError();
}

template <int FMT, int MODE>
static cudaError_t launch_fmt(const CUtensorMap& mx, const CUtensorMap& mc, const TcArgs& a, int bn, int num_sms,
                              cudaStream_t st) {
    (void)bn;  // 128-column tiles: four TMEM accumulators
    // both modes stage the epilogue's values in shared memory when K fits two
    // 128-byte atoms (assign: the candidate walk, in the variant a.variant
    // names; distance matrix: the transposed stores)
    if (a.kchunks > 2) return launch_one<FMT, 128, MODE, TC_SV_REG>(mx, mc, a, num_sms, st);
    if constexpr (MODE == 1) {
        return launch_one<FMT, 128, MODE, TC_SV_HALF>(mx, mc, a, num_sms, st);
    } else {
        if (a.variant == TC_SV_FULL) return launch_one<FMT, 128, MODE, TC_SV_FULL>(mx, mc, a, num_sms, st);
        if (a.variant == TC_SV_C32) return launch_one<FMT, 128, MODE, TC_SV_C32>(mx, mc, a, num_sms, st);
        return launch_one<FMT, 128, MODE, TC_SV_HALF>(mx, mc, a, num_sms, st);
    }
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
