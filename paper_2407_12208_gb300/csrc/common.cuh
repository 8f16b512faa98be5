// common.cuh -- internal helpers of libmpkm (sm_103a): inline-PTX wrappers for
// mbarrier, TMA (cp.async.bulk.tensor) and tcgen05 (TMEM alloc / MMA / ld),
// bounded waits, and the device status word.  Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <cuda.h>
#include <stdint.h>

#define KM_DEV __device__ __forceinline__

// Device status word bits (written with atomicOr, read by the host).
#define KM_DEVERR_TIMEOUT 1u
#define KM_DEVERR_BOUNDS 2u

// Spin budget of every device-side wait: ~2^31 SM cycles (about a second at
// the GB300's clocks).  After it runs out the waiting thread records
// KM_DEVERR_TIMEOUT and the kernel winds down instead of hanging the GPU.
#define KM_WAIT_CYCLES (1ll << 31)

namespace km {

KM_DEV uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory accesses through 32-bit shared addresses (the screen's
// per-lane staging and candidate lists: plain 32-bit address arithmetic).
KM_DEV void st_shared_v4(uint32_t a, float x, float y, float z, float w) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}
KM_DEV float4 ld_shared_v4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
    return v;
}
KM_DEV void st_shared_u32(uint32_t a, uint32_t v) { asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory"); }

// Candidate entry, one per quad of columns (4q .. 4q + 3): the fp32 bit
// pattern of the quad's smallest d^ with its low ebits bits replaced by
// (q << 4) | mask, mask bit c set when column 4q + c is a candidate
// (ebits = qbits + 4 <= 18, q < 2^qbits).  The stored value t is d^
// truncated toward zero to 24 - ebits significant bits, so every candidate
// of the quad has d^ >= t - |t| 2^(ebits - 23).
KM_DEV uint32_t quad_entry(int q, unsigned mask, float dh, uint32_t emask) {
    return (__float_as_uint(dh) & ~emask) | ((uint32_t)q << 4) | mask;
}
KM_DEV int entry_quad(uint32_t e, uint32_t emask) { return (int)((e & emask) >> 4); }
KM_DEV unsigned entry_mask(uint32_t e) { return e & 15u; }
// lscale = 2^(ebits - 23)
KM_DEV float cand_lower(uint32_t e, uint32_t emask, float lscale) {
    const float t = __uint_as_float(e & ~emask);
    return t - fabsf(t) * lscale;
}

// ---------------------------------------------------------------- mbarrier
KM_DEV void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
KM_DEV void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
KM_DEV void mbar_arrive(uint64_t* bar) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar))
                 : "memory");
}
KM_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
KM_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, "
        "p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase with the given parity to complete.  Returns
// false (and flags the abort word and the global status) on timeout, or
// immediately if another thread of the CTA already aborted.
KM_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned* status) {
    if (mbar_try_wait(bar, parity)) return true;
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        __nanosleep(32);  // back off: leave the issue slots to the warps doing work
        if (*abort_flag) return false;
        if (clock64() - t0 > KM_WAIT_CYCLES) {
            *abort_flag = 1;
            atomicOr(status, KM_DEVERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// Bounded wait that ignores the abort word: used to drain in-flight tensor
// ops before TMEM is released, so it must not give up early.
KM_DEV bool mbar_wait_drain(uint64_t* bar, uint32_t parity, unsigned* status) {
    long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > KM_WAIT_CYCLES) {
            atomicOr(status, KM_DEVERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// --------------------------------------------------------------------- TMA
// Asks L2 to fetch `bytes` (a multiple of 16) at the 16-byte aligned
// global address p; no register receives anything.
KM_DEV void prefetch_l2_bulk(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
KM_DEV void tma_prefetch_desc(const void* tmap) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(tmap) : "memory");
}
KM_DEV void tma_load_2d(void* smem_dst, const void* tmap, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
        "%4}], [%2];" ::"r"(smem_u32(smem_dst)),
        "l"(tmap), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// ----------------------------------------------------------------- tcgen05
KM_DEV void tmem_alloc(uint32_t* smem_slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
KM_DEV void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
KM_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
KM_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (fp16/bf16 inputs, fp32 accumulate)
KM_DEV void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// kind::f8f6f4 (e4m3 inputs, fp32 accumulate)
KM_DEV void mma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// Make `bar` track completion of all tcgen05 ops issued so far by this thread.
KM_DEV void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp gets lane
// (base lane + t), columns col..col+31.
KM_DEV void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor for tcgen05 (K-major operand, 128-byte
// swizzle): start address, leading-byte offset (unused for swizzled K-major),
// stride-byte offset = 1024 (8 rows x 128 B), version 1, layout SWIZZLE_128B.
KM_DEV uint64_t sdesc_sw128(uint32_t smem_addr) {
    uint64_t d = 0;
    d |= (uint64_t)((smem_addr & 0x3FFFF) >> 4);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: fp32 accumulate, K-major A and B, M x N tile.
// ab_fmt: kind::f16 -> 0 fp16, 1 bf16; kind::f8f6f4 -> 0 e4m3.
__host__ __device__ constexpr uint32_t idesc_make(uint32_t ab_fmt, int M, int N) {
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// ----------------------------------------------------------- float helpers
// Error-free sum (Knuth's TwoSum): a + b = s + e exactly.
KM_DEV void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}
// Accumulate x*x into the double-float (hi, lo) using an FMA-based exact product.
KM_DEV void df_add_sq(float x, float& hi, float& lo) {
    float p = x * x;
    float pe = __fmaf_rn(x, x, -p);
    float s, e;
    two_sum(hi, p, s, e);
    hi = s;
    lo += e + pe;
}
KM_DEV void df_add(float& hi, float& lo, float bhi, float blo) {
    float s, e;
    two_sum(hi, bhi, s, e);
    hi = s;
    lo += e + blo;
}

}  // namespace km
