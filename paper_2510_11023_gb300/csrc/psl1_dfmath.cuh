// psl1_dfmath.cuh -- double-float (unevaluated FP32 pair) arithmetic and the
// coefficient families evaluated in it.
//
// GB300 issues FP64 at 1/64 of its FP32 rate, so the per-node evaluation of D
// (a rational function of u) and of the polynomial part of f is done on the
// FP32 pipes: ~48-bit significands from error-free transformations (Knuth's
// TwoSum, the FMA-exact product) and Newton-corrected division, with the
// family parameters and node functions taken from double-float copies made
// once (no FP64 operation per node).  Transcendental terms of f (cos u, sin u,
// e^-t, the manufactured sources) stay FP64.
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

// the polynomial family of f (I.f_poly: only c2 u (1 - u) is active)
__device__ __forceinline__ df f_poly_df(const InstDev& I, df u)
{
    return df_mul(fpar_df(I, 2), df_mul(u, df_addn(df{1.f, 0.f}, df_neg(u))));
}

}  // namespace psl1
