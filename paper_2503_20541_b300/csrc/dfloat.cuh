// dfloat.cuh -- two-float ("double-float") arithmetic for the precise-energy evaluation.
//
// A value is the unevaluated sum hi + lo of two FP32 numbers with |lo| <= ulp(hi)/2, about
// 48 significant bits.  The operations are built from error-free transformations: the
// exact rounding error of a sum (Knuth's TwoSum, six operations, any operand order;
// Dekker's FastTwoSum, three, when |a| >= |b|) and of a product (one FMA:
// fma(a, b, -fl(a b)) is exact).  Additions and subtractions here are the _rn intrinsics,
// which the compiler never contracts into an FMA (a contraction would break the exactness
// of the transformations); every product that must stay separate is explicit.
#pragma once

namespace nb {

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF df_make(float hi, float lo = 0.f) { return DF{hi, lo}; }

// s + e = a + b exactly
__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// s + e = a + b exactly, for |a| >= |b| (or a = 0)
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// p + e = a b exactly (barring underflow)
__device__ __forceinline__ DF two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return DF{p, fmaf(a, b, -p)};
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }

// a + b with both parts summed error-free (accurate also when a.hi and b.hi cancel)
__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

// a + b with the low parts added in FP32 (Dekker's addition): error ~2^-46 of |a| + |b|
// rather than of |a + b|; for sums whose operands do not cancel far below their size.
__device__ __forceinline__ DF df_add_fast(DF a, DF b) {
    const DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ DF df_add_f(DF a, float b) {
    const DF s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const DF p = two_prod(a.hi, b.hi);
    return fast_two_sum(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}

__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    const DF p = two_prod(a.hi, b);
    return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}

// Exact scaling by a power of two (barring underflow).
__device__ __forceinline__ DF df_scale(DF a, float pow2) { return DF{__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

// a / b: the FP32 quotient and two correction quotients of the remainder a - q b.
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdiv_rn(a.hi, b.hi);
    DF r = df_add(a, df_neg(df_mul_f(b, q1)));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_add(r, df_neg(df_mul_f(b, q2)));
    const float q3 = __fdiv_rn(r.hi, b.hi);
    return df_add_f(fast_two_sum(q1, q2), q3);
}

// sqrt(a), a > 0: the FP32 root s and one correction (a - s^2) / (2 s), the residual formed
// exactly (s^2 as a two-product; a.hi - fl(s^2) is exact because s^2 is within an ulp or
// two of a.hi).
__device__ __forceinline__ DF df_sqrt(DF a) {
    const float s = __fsqrt_rn(a.hi);
    const DF p = two_prod(s, s);
    const float res = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return fast_two_sum(s, __fdiv_rn(res, __fmul_rn(2.f, s)));
}

// 1/sqrt(a), a > 0: the hardware estimate y (within ~2 ulp) and one Newton step y (1 + e/2),
// e = 1 - a y^2 formed in two-float (y^2 as a two-product); the step leaves 1.5 e0^2 of an
// estimate off by e0 (below 2.5e-13 at 2 ulp, ~2e-14 when correctly rounded).  No division
// or square root.
__device__ __forceinline__ DF df_rsqrt(DF a) {
    const float y = rsqrtf(a.hi);
    const DF m = df_mul(a, two_prod(y, y));
    const DF e = df_add_f(df_neg(m), 1.f);
    return fast_two_sum(y, __fmul_rn(__fmul_rn(y, e.hi), 0.5f));
}

__device__ __forceinline__ double df_to_double(DF a) { return (double)a.hi + (double)a.lo; }

// Sum of a two-float value over the 32 lanes of a warp in a fixed butterfly; every lane
// ends with the same result (two_sum is exact whatever the operand order, so a + b and
// b + a give the same pair).
__device__ __forceinline__ DF warp_sum_df(DF a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DF b{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
        a = df_add(a, b);
    }
    return a;
}

}  // namespace nb
