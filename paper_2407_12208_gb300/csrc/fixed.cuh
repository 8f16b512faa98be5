// fixed.cuh -- exact fixed-point values for the centre sums (Eq. (center)
// with the accuracy Section 4.4 asks): every coordinate scaled by 2^S and
// rounded once to an integer, after which integer addition is exact in any
// order.  Shared by the centre-update kernels and the grouped Lloyd kernel.
#pragma once
#include "common.cuh"

namespace km {

// Fixed-point exponent S for n rows with max |x| given as float bits.
KM_DEV int fixed_shift(unsigned amax_bits, int64_t n) {
    float amax = __uint_as_float(amax_bits);
    int E = (amax > 0.0f) ? ilogbf(amax) : -126;  // amax < 2^(E+1)
    int lgn = 0;
    while (((int64_t)1 << lgn) < n) lgn++;
    return 60 - lgn - E;  // |sum| 2^S < 2^(lgn + E + 1 + S) = 2^61
}

// v 2^S rounded to the nearest integer, exactly, without 64-bit conversions
// (float-to-int64 conversion runs on the FP64 pipe, which is narrow here).
//  - Scaling: S lies in [-98, 209]; it is split into two power-of-two
//    factors, each a normal float, and both products are exact whenever the
//    result is a normal float (|v 2^S| < 2^61 never overflows); when it is
//    not, |v 2^S| < 2^-126 and the integer is 0 either way.
//  - Rounding: y = v 2^S (|y| < 2^62) is split by round-to-nearest additions
//    of magic constants into y = p2 + p1 + r0, p2 a multiple of 2^40, p1 of
//    2^20, |r0| <= 2^19; every step is exact (each remainder fits in 24 bits),
//    and round(y) = p2 + p1 + round(r0) because p2 + p1 is even.  The three
//    integers p2 / 2^40, p1 / 2^20 and round(r0) are read off the bits of a
//    float in [2^23, 2^24) (Split::bits: value + 0x4B400000, the bias removed
//    once per sum, modulo 2^32).
// Same integers as rounding ldexpf(v, S) with __float2ll_rn.
struct FixedScale {
    float f1, f2;
    KM_DEV explicit FixedScale(int S) {
        const int s1 = S / 2, s2 = S - s1;
        f1 = __int_as_float((s1 + 127) << 23);
        f2 = __int_as_float((s2 + 127) << 23);
    }
    static constexpr unsigned kBias = 0x4B400000u;  // bits of 1.5 * 2^23
    // biased 32-bit parts of round(v 2^S): (b2, b1, b0), value = sum of (b - kBias) 2^(40, 20, 0)
    KM_DEV void split(float v, unsigned& b2, unsigned& b1, unsigned& b0) const {
        const float y = __fmul_rn(__fmul_rn(v, f1), f2);
        const float c40 = 0x1.8p63f;  // ulp 2^40
        const float c20 = 0x1.8p43f;  // ulp 2^20
        const float c0 = 0x1.8p23f;   // ulp 1
        const float p2 = __fsub_rn(__fadd_rn(y, c40), c40);
        const float r = __fsub_rn(y, p2);
        const float p1 = __fsub_rn(__fadd_rn(r, c20), c20);
        const float r0 = __fsub_rn(r, p1);
        b0 = __float_as_uint(__fadd_rn(r0, c0));
        b1 = __float_as_uint(__fmaf_rn(p1, 0x1p-20f, c0));
        b2 = __float_as_uint(__fmaf_rn(p2, 0x1p-40f, c0));
    }
    // split() on two values at once: the same operations, two per packed
    // instruction (each half rounded exactly as its scalar counterpart)
    KM_DEV void split2(float2 v, uint2& b2, uint2& b1, uint2& b0) const {
        const float2 c40 = make_float2(0x1.8p63f, 0x1.8p63f), n40 = make_float2(-0x1.8p63f, -0x1.8p63f);
        const float2 c20 = make_float2(0x1.8p43f, 0x1.8p43f), n20 = make_float2(-0x1.8p43f, -0x1.8p43f);
        const float2 c0 = make_float2(0x1.8p23f, 0x1.8p23f);
        const float2 y = __fmul2_rn(__fmul2_rn(v, make_float2(f1, f1)), make_float2(f2, f2));
        const float2 p2 = __fadd2_rn(__fadd2_rn(y, c40), n40);
        const float2 r = __fadd2_rn(y, make_float2(-p2.x, -p2.y));
        const float2 p1 = __fadd2_rn(__fadd2_rn(r, c20), n20);
        const float2 r0 = __fadd2_rn(r, make_float2(-p1.x, -p1.y));
        const float2 t0 = __fadd2_rn(r0, c0);
        const float2 t1 = __ffma2_rn(p1, make_float2(0x1p-20f, 0x1p-20f), c0);
        const float2 t2 = __ffma2_rn(p2, make_float2(0x1p-40f, 0x1p-40f), c0);
        b0 = make_uint2(__float_as_uint(t0.x), __float_as_uint(t0.y));
        b1 = make_uint2(__float_as_uint(t1.x), __float_as_uint(t1.y));
        b2 = make_uint2(__float_as_uint(t2.x), __float_as_uint(t2.y));
    }
    // sum of m split values -> int64 (the biased parts were added modulo 2^32;
    // each true part sum is below 2^31 in magnitude for m <= 2^10)
    KM_DEV static long long combine(unsigned s2, unsigned s1, unsigned s0, unsigned m) {
        const int t2 = (int)(s2 - m * kBias), t1 = (int)(s1 - m * kBias), t0 = (int)(s0 - m * kBias);
        return (long long)t2 * (1ll << 40) + (long long)t1 * (1ll << 20) + (long long)t0;
    }
    KM_DEV long long operator()(float v) const {
        unsigned b2, b1, b0;
        split(v, b2, b1, b0);
        return combine(b2, b1, b0, 1u);
    }
};

}  // namespace km
