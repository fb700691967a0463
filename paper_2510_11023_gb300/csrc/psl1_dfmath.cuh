// psl1_dfmath.cuh -- double-float (unevaluated FP32 pair) arithmetic and the
// coefficient families evaluated in it.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so the per-node evaluation of D
// (a rational function of u) and of the polynomial part of f is done on the
// FP32 pipes: ~48-bit significands from error-free transformations (Knuth's
// TwoSum, the FMA-exact product) and Newton-corrected division, with the
// family parameters and node functions taken from double-float copies made
// once (no FP64 operation per node).  cos u and sin u are evaluated in
// double-float too (df_sincos); only the manufactured sources stay FP64.
#pragma once
#include "psl1_device.cuh"

namespace psl1 {

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a + b with the low part left unnormalised (for long accumulations that take
// the hi part exactly and the lo part as a correction)
__device__ __forceinline__ df df_add(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return {s, __fadd_rn(e, __fadd_rn(a.lo, b.lo))};
}

// |e| <= ulp(s)/2 after this (s + e = a + b exactly when |a| >= |b|)
__device__ __forceinline__ df quick_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// normalised a + b
__device__ __forceinline__ df df_addn(df a, df b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    return quick_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
    return quick_two_sum(p, pe);
}

__device__ __forceinline__ df df_mulf(df a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float pe = __fmaf_rn(a.hi, b, -p);
    pe = __fmaf_rn(a.lo, b, pe);
    return quick_two_sum(p, pe);
}

// a / b: FP32 quotient of the leading parts, then two corrections from the
// double-float remainder (long division in base 2^24)
__device__ __forceinline__ df df_div(df a, df b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    df r = df_addn(a, df_neg(df_mulf(b, q1)));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_addn(r, df_neg(df_mulf(b, q2)));
    const float q3 = __fdiv_rn(r.hi, b.hi);
    float s, e;
    two_sum(q1, q2, s, e);
    return quick_two_sum(s, __fadd_rn(e, q3));
}

__device__ __forceinline__ df dpar_df(const InstDev& I, int i) { return {I.dpf[2 * i], I.dpf[2 * i + 1]}; }
__device__ __forceinline__ df fpar_df(const InstDev& I, int i) { return {I.fpf[2 * i], I.fpf[2 * i + 1]}; }

// D = (d0 + d1/(1+u^2) X1 + d2 u + d3 sin(pi x)) X0,  X_i = 1 + a_i sin(2 pi x) + b_i cos(2 pi y)
// (sx1 = sin(pi x), sx2 = sin(2 pi x), cy2 = cos(2 pi y); cy2 = 0 in 1D)
__device__ __forceinline__ df D_eval_df(const InstDev& I, df sx1, df sx2, df cy2, df u)
{
    const df one{1.f, 0.f};
    df X0 = df_addn(one, df_addn(df_mul(dpar_df(I, 4), sx2), df_mul(dpar_df(I, 5), cy2)));
    df v = df_addn(dpar_df(I, 0), df_mul(dpar_df(I, 3), sx1));
    if (I.dpar[1] != 0.0) {
        df X1 = df_addn(one, df_addn(df_mul(dpar_df(I, 6), sx2), df_mul(dpar_df(I, 7), cy2)));
        df w = df_addn(one, df_mul(u, u));
        v = df_addn(v, df_mul(df_div(dpar_df(I, 1), w), X1));
    }
    if (I.dpar[2] != 0.0) v = df_addn(v, df_mul(dpar_df(I, 2), u));
    return df_mul(v, X0);
}

// exact product a b = p + e
__device__ __forceinline__ df two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// 1/n!, n = 0..17, as double-float pairs (hi = nearest float to 1/n!, lo =
// nearest float to the remainder), written out from exact rational arithmetic.
static __constant__ float kInvFact[18][2] = {
    0x1.0000000000000p+0f, 0x0.0p+0f,   // 1/0!
    0x1.0000000000000p+0f, 0x0.0p+0f,   // 1/1!
    0x1.0000000000000p-1f, 0x0.0p+0f,   // 1/2!
    0x1.5555560000000p-3f, -0x1.5555560000000p-28f,   // 1/3!
    0x1.5555560000000p-5f, -0x1.5555560000000p-30f,   // 1/4!
    0x1.1111120000000p-7f, -0x1.ddddde0000000p-32f,   // 1/5!
    0x1.6c16c20000000p-10f, -0x1.27d27e0000000p-35f,   // 1/6!
    0x1.a01a020000000p-13f, -0x1.7f97fa0000000p-39f,   // 1/7!
    0x1.a01a020000000p-16f, -0x1.7f97fa0000000p-42f,   // 1/8!
    0x1.71de3a0000000p-19f, 0x1.55b1cc0000000p-45f,   // 1/9!
    0x1.27e4fc0000000p-22f, -0x1.10ec140000000p-47f,   // 1/10!
    0x1.ae64560000000p-26f, 0x1.fd51380000000p-52f,   // 1/11!
    0x1.1eed8e0000000p-29f, 0x1.ff1b120000000p-54f,   // 1/12!
    0x1.6124620000000p-33f, -0x1.8af25e0000000p-58f,   // 1/13!
    0x1.93974a0000000p-37f, 0x1.180f940000000p-62f,   // 1/14!
    0x1.ae7f3e0000000p-41f, 0x1.ccee080000000p-67f,   // 1/15!
    0x1.ae7f3e0000000p-45f, 0x1.ccee080000000p-71f,   // 1/16!
    0x1.952c780000000p-49f, -0x1.f9ea560000000p-74f,   // 1/17!
};

__device__ __forceinline__ df inv_fact(int n) { return {kInvFact[n][0], kInvFact[n][1]}; }

// sin u and cos u in double-float: Cody-Waite reduction u = n pi/2 + r with a
// three-float split of pi/2 (each product n * part exact by FMA), then the
// Taylor series of sin and cos on |r| <= pi/4, truncated after r^17 / 17! and
// r^16 / 16! (next terms below 1e-17 there), summed by Horner in r^2.
// Valid range: |u| <= 2^20.  There n < 2^20, the products n P1, n P2 are exact
// and n P3 is off by at most n 2^-73, so the reduced argument carries an
// absolute error of about |u| 2^-48 -- the resolution of the double-float
// input itself.  Beyond 2^20 the split no longer covers the product's bits
// (and rintf stops being exact at 2^24); the solution values of this solver
// are O(1) and the coefficient families are evaluated at them.
__device__ __forceinline__ void df_sincos(df u, df& sn, df& cs)
{
    constexpr double PIO2 = 1.5707963267948966;
    constexpr float P1 = (float)PIO2;
    constexpr float P2 = (float)(PIO2 - (double)P1);
    constexpr float P3 = (float)(PIO2 - (double)P1 - (double)P2);
    const float n = rintf(u.hi * 0.636619772f);   // nearest multiple of pi/2
    df r = df_addn(u, df_neg(two_prod(n, P1)));
    r = df_addn(r, df_neg(two_prod(n, P2)));
    r = df_addn(r, df{-__fmul_rn(n, P3), 0.f});
    const df r2 = df_mul(r, r);
    df S = inv_fact(17), C = inv_fact(16);
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        const df a = inv_fact(2 * j + 1), b = inv_fact(2 * j);
        S = df_addn((j & 1) ? df_neg(a) : a, df_mul(r2, S));
        C = df_addn((j & 1) ? df_neg(b) : b, df_mul(r2, C));
    }
    // the j = 8 terms carry sign (+1): r^16/16! and r^17/17!
    S = df_mul(r, S);
    const int q = ((int)n) & 3;
    const df s0 = S, c0 = C;
    sn = q == 0 ? s0 : q == 1 ? c0 : q == 2 ? df_neg(s0) : df_neg(c0);
    cs = q == 0 ? c0 : q == 1 ? df_neg(s0) : q == 2 ? df_neg(c0) : s0;
}

// f = c0 cos u + c1 sin u + c2 u (1 - u) + c3 sin(pi x) e^{-t} in double-float
// (I.f_df: the manufactured sources c4, c5 are absent); emt = e^{-t} as double-float.
__device__ __forceinline__ df f_eval_df(const InstDev& I, df sx1, df emt, df u)
{
    df v{0.f, 0.f};
    if (I.fpar[0] != 0.0 || I.fpar[1] != 0.0) {
        df sn, cs;
        df_sincos(u, sn, cs);
        if (I.fpar[0] != 0.0) v = df_addn(v, df_mul(fpar_df(I, 0), cs));
        if (I.fpar[1] != 0.0) v = df_addn(v, df_mul(fpar_df(I, 1), sn));
    }
    if (I.fpar[2] != 0.0) v = df_addn(v, df_mul(fpar_df(I, 2), df_mul(u, df_addn(df{1.f, 0.f}, df_neg(u)))));
    if (I.fpar[3] != 0.0) v = df_addn(v, df_mul(fpar_df(I, 3), df_mul(sx1, emt)));
    return v;
}

}  // namespace psl1
