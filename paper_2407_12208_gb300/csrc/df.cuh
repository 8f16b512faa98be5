// df.cuh -- the winner's squared distance ||x - c||^2 (Eq. (dist-direct))
// to binary64 accuracy on the fp32 pipe (GB300's FP64 pipe is too narrow to
// carry one binary64 evaluation per row at HBM speed).
//
// Arithmetic (fixed, so that every kernel computing it gets the same bits):
//  * each coordinate: t = fl(x - c) and its rounding error tl (TwoSum, exact),
//    so x - c = t + tl; t^2 = p + pe exactly (FMA), and the square is kept as
//    (p, q) with q = fl(2 t tl + pe): its error is below 4 u^2 t^2 (u = 2^-24;
//    tl^2 <= u^2 t^2 is dropped);
//  * a chunk of four coordinates (a float4, zero-padded past d): A = sq0 + sq2
//    and B = sq1 + sq3 as double-floats (TwoSum of the leading parts), then
//    df_combine(A, B);
//  * the chunks of a row, chunk index ci = cl + LPR u (lane cl of the LPR
//    lanes of the row, u < NV4): a lane combines its own chunks (u = 0 with 1,
//    2 with 3, then the two), then a butterfly over the LPR lanes with offsets
//    LPR/2, LPR/4, ..., 1;
//  * the result is (double) hi + (double) lo.
// df_combine is commutative and yields a normalised pair (hi = fl(hi + lo)),
// and combining a normalised pair with zero returns it unchanged, so chunks
// that are all padding may be skipped.  All terms are non-negative, so there
// is no cancellation: with at most 4 coordinates per serial chain and a tree of
// depth <= 7 above it, the relative error is below 2^-40 (about 1e-12 / 11).
#pragma once
#include "common.cuh"

namespace km {

struct DF {
    float hi, lo;
};

// a - b on two coordinates at once (sub.rn.f32x2: each half rounded as a
// scalar subtraction)
KM_DEV float2 fsub2(float2 a, float2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a)), "l"(*reinterpret_cast<const unsigned long long*>(&b)));
    return *reinterpret_cast<const float2*>(&r);
}

// x - c as t + tl, and the square as (p, q) with p + q = (x - c)^2 (1 + O(u^2)).
KM_DEV void df_sq_diff(float x, float c, float& p, float& q) {
    const float t = __fsub_rn(x, c);
    const float bb = __fsub_rn(t, x);
    const float tl = __fadd_rn(__fsub_rn(x, __fsub_rn(t, bb)), __fsub_rn(-c, bb));
    p = __fmul_rn(t, t);
    const float pe = __fmaf_rn(t, t, -p);
    q = __fmaf_rn(__fadd_rn(t, t), tl, pe);
}

// Two coordinates at once (two per packed instruction, each half rounded as
// its scalar counterpart above).
KM_DEV void df_sq_diff2(float2 x, float2 c, float2& p, float2& q) {
    const float2 t = fsub2(x, c);
    const float2 bb = fsub2(t, x);
    const float2 u = fsub2(t, bb);
    // (x - u) + (-c - bb) = (x - u) - (c + bb)
    const float2 tl = fsub2(fsub2(x, u), __fadd2_rn(c, bb));
    p = __fmul2_rn(t, t);
    const float2 pe = __ffma2_rn(t, t, make_float2(-p.x, -p.y));
    q = __ffma2_rn(__fadd2_rn(t, t), tl, pe);
}

// (p1, q1) + (p2, q2) without renormalisation: leading parts by TwoSum, the
// error and the trailing parts added in fp32.
KM_DEV DF df_add_raw(float p1, float q1, float p2, float q2) {
    const float s = __fadd_rn(p1, p2);
    const float bb = __fsub_rn(s, p1);
    const float e = __fadd_rn(__fsub_rn(p1, __fsub_rn(s, bb)), __fsub_rn(p2, bb));
    return DF{s, __fadd_rn(e, __fadd_rn(q1, q2))};
}

// Sum of two double-floats, commutative, normalised (FastTwoSum at the end).
KM_DEV DF df_combine(DF a, DF b) {
    DF r = df_add_raw(a.hi, a.lo, b.hi, b.lo);
    const float hi = __fadd_rn(r.hi, r.lo);
    const float lo = __fsub_rn(r.lo, __fsub_rn(hi, r.hi));
    return DF{hi, lo};
}

// One chunk of four coordinates.
KM_DEV DF df_chunk(float4 x, float4 c) {
    float2 p01, q01, p23, q23;
    df_sq_diff2(make_float2(x.x, x.y), make_float2(c.x, c.y), p01, q01);
    df_sq_diff2(make_float2(x.z, x.w), make_float2(c.z, c.w), p23, q23);
    // A = sq0 + sq2 and B = sq1 + sq3 in one packed TwoSum
    const float2 s = __fadd2_rn(p01, p23);
    const float2 bb = fsub2(s, p01);
    const float2 v = fsub2(s, bb);
    const float2 e = __fadd2_rn(fsub2(p01, v), fsub2(p23, bb));
    const float2 lo = __fadd2_rn(e, __fadd2_rn(q01, q23));
    return df_combine(DF{s.x, lo.x}, DF{s.y, lo.y});
}

// A lane's NV4 chunks (u = 0..NV4-1) in the fixed order.
template <int NV4>
KM_DEV DF df_lane(const float4 (&x)[NV4], const float4 (&c)[NV4]) {
    if constexpr (NV4 == 1) {
        return df_chunk(x[0], c[0]);
    } else if constexpr (NV4 == 2) {
        return df_combine(df_chunk(x[0], c[0]), df_chunk(x[1], c[1]));
    } else {
        static_assert(NV4 == 4, "one, two or four chunks per lane");
        return df_combine(df_combine(df_chunk(x[0], c[0]), df_chunk(x[1], c[1])),
                          df_combine(df_chunk(x[2], c[2]), df_chunk(x[3], c[3])));
    }
}

KM_DEV DF df_shfl_xor(DF v, int o) {
    return DF{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
}

// The butterfly over the L lanes of a row (L consecutive lanes starting at a
// multiple of L), offsets L/2, L/4, ..., 1, for R rows at once: v[r] is this
// lane's partial of row r (R <= L, both powers of two).  While a lane still
// holds several rows, each level halves them (lanes with the offset bit set
// keep the upper half and pass the lower half to their partner), so the
// combines per lane are R - 1 + log2(L / R) instead of R log2 L; every row
// still gets the same tree as a one-row butterfly with these offsets.  On
// return the lane holds the complete sum of row `row`; the L / R lanes that
// differ only in their low log2(L / R) bits hold the same row.
template <int R, int L>
KM_DEV DF df_rows(DF (&v)[R], int cl, int& row) {
    int base = 0;
#pragma unroll
    for (int lev = 0; (L >> (lev + 1)) >= 1; lev++) {
        const int o = L >> (lev + 1);
        const int nr = (R >> lev) > 1 ? (R >> lev) : 1;
        if (nr > 1) {
            const int h = nr >> 1;
            const bool up = (cl & o) != 0;
#pragma unroll
            for (int r = 0; r < h; r++) {
                const DF keep = up ? v[r + h] : v[r];
                const DF send = up ? v[r] : v[r + h];
                v[r] = df_combine(keep, df_shfl_xor(send, o));
            }
            base += up ? h : 0;
        } else {
            v[0] = df_combine(v[0], df_shfl_xor(v[0], o));
        }
    }
    row = base;
    return v[0];
}

// binary32 -> binary64 by moving bits (exact for zeros and normal numbers);
// GB300 runs the conversion instruction on its narrow FP64 pipe, so only
// subnormals (and non-finite values) take it.
KM_DEV double f32_to_f64(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xFFu;
    if ((u & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
    if (e == 0u || e == 0xFFu) return (double)f;
    const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hi, (int)(u << 29));
}
KM_DEV double df_value(DF v) { return f32_to_f64(v.hi) + f32_to_f64(v.lo); }

// A whole row of D <= 8 coordinates in one thread: chunk 0 and (D > 4) chunk 1
// combined -- what the butterfly over the eight lanes of such a row gives,
// since the other six lanes' chunks are padding.
// A chunk whose coordinates past the first L are padding (zero in x and c):
// the same value as df_chunk, with the padding's exact zeros left out
// (a square of (0 - 0) is (+0, +0), and adding it changes nothing).
template <int L>
KM_DEV DF df_chunk_live(float4 x, float4 c) {
    if constexpr (L >= 4) {
        return df_chunk(x, c);
    } else {
        float p0, q0, p1 = 0.0f, q1 = 0.0f;
        df_sq_diff(x.x, c.x, p0, q0);
        if constexpr (L >= 2) df_sq_diff(x.y, c.y, p1, q1);
        DF A{p0, q0};
        if constexpr (L == 3) {
            float p2, q2;
            df_sq_diff(x.z, c.z, p2, q2);
            A = df_add_raw(p0, q0, p2, q2);
        }
        return df_combine(A, DF{p1, q1});
    }
}

// The centre as two float4 (the second unused for D <= 4); coordinates past
// D must be zero in both.
template <int D>
KM_DEV DF df_small4(const float (&x)[D], float4 c0, float4 c1) {
    static_assert(D >= 1 && D <= 8, "rows of at most 8 coordinates");
    float xa[8];
#pragma unroll
    for (int l = 0; l < 8; l++) xa[l] = l < D ? x[l] : 0.0f;
    const DF h0 = df_chunk_live<(D < 4 ? D : 4)>(make_float4(xa[0], xa[1], xa[2], xa[3]), c0);
    if constexpr (D <= 4) {
        return h0;
    } else {
        return df_combine(h0, df_chunk_live<D - 4>(make_float4(xa[4], xa[5], xa[6], xa[7]), c1));
    }
}
template <int D>
KM_DEV DF df_small(const float (&x)[D], const float* c) {
    float ca[8];
#pragma unroll
    for (int l = 0; l < 8; l++) ca[l] = l < D ? c[l] : 0.0f;
    return df_small4<D>(x, make_float4(ca[0], ca[1], ca[2], ca[3]), make_float4(ca[4], ca[5], ca[6], ca[7]));
}

// Chunk geometry of a row of d coordinates: d4 = ceil(d / 4) chunks over LPR
// lanes, NV4 chunks per lane (LPR = 8, 16 or 32; the centre-sum kernel uses
// the same split of a row over its lanes).
__host__ __device__ constexpr int df_lpr(int d) { return (d + 3) / 4 <= 8 ? 8 : ((d + 3) / 4 <= 16 ? 16 : 32); }
__host__ __device__ constexpr int df_nv4(int d) { return (d + 3) / 4 <= 32 ? 1 : ((d + 3) / 4 <= 64 ? 2 : 4); }

}  // namespace km
