// erfc.cuh -- complementary error function of the Ewald direct-space pair term (Sec. 2.1.2:
// ke q_i q_j erfc(alpha r)/r), written for the pair kernel's force-only form so that the
// Gaussian of the force, exp(-(alpha r)^2), and erfc share one exponential and no division.
// Its error (a few ulp) is far inside the force tolerance; the energy sums, which cancel
// ~1000-fold, are evaluated with CUDA's erfcf, whose residual error is smoother.
//
//   erfc(x) = exp(-x^2) erfcx(x),   x >= 0,
//   erfcx(x) = t P(2t - 1),         t = 1 / (1 + x/2) in (0, 1],
//
// P a degree-12 polynomial fitted to erfcx(x)/t over the whole half-line (relative error of
// the fit 1.7e-8 with its coefficients rounded to FP32, mean 4e-9; the coefficients and the
// fit are produced by csrc/erfc_fit.py, a Chebyshev least-squares fit with Lawson-style
// reweighting against scipy's erfcx, rounded to FP32 one coefficient at a time).  exp(-x^2) is
// evaluated as 2^y with y = -x^2 log2(e) carried as an unevaluated sum y + y_lo: x^2 is split
// exactly by an FMA two-product and log2(e) is a two-float constant, the hardware 2^y
// approximation (ex2.approx) takes y, and the factor 2^{y_lo} is applied to first order.
// Without the split, the rounding of x^2 log2(e) alone (|y| ~ 12 at alpha r_c = 2.9) would
// cost ~10 ulp.  t comes from the hardware reciprocal approximation and one Newton-Raphson
// step on 1 + x/2 held as a two-float sum.  Accuracy against the FP64 erfc is checked on
// the device through nb_erfc_eval (tests/test_gpu_erfc.py).
#pragma once

namespace nb {

constexpr float kLog2e = 1.44269502f;         // log2(e) rounded to FP32
constexpr float kLog2eLo = 1.92596299e-08f;   // log2(e) - kLog2e
constexpr float kLn2f = 0.693147182f;

__device__ __forceinline__ float ex2_approx(float y) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(y));
    return r;
}

__device__ __forceinline__ float rcp_approx(float d) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d));
    return r;
}

// exp(-x^2) for x >= 0 to a few ulp (0 once it underflows below the normal range).
__device__ __forceinline__ float exp_neg_sq(float x) {
    const float s = x * x;
    const float s_lo = fmaf(x, x, -s);  // x^2 = s + s_lo exactly
    const float y = -s * kLog2e;
    // -(s + s_lo)(kLog2e + kLog2eLo) - y, dropping the product of the two small parts
    const float y_lo = fmaf(-s, kLog2e, -y) - fmaf(s, kLog2eLo, s_lo * kLog2e);
    const float e = ex2_approx(y);
    return fmaf(e, y_lo * kLn2f, e);
}

// erfc(x) for x >= 0, given E = exp_neg_sq(x).
__device__ __forceinline__ float erfc_with_exp(float x, float E) {
    const float d = fmaf(0.5f, x, 1.f);
    const float d_lo = fmaf(0.5f, x, 1.f - d);  // 1 + x/2 = d + d_lo (exact while d <= 2)
    float t = rcp_approx(d);
    t = fmaf(t, fmaf(-d, t, 1.f) - d_lo * t, t);  // Newton-Raphson step toward 1/(d + d_lo)
    const float u = fmaf(2.f, t, -1.f);
    float p = -6.332287285e-06f;
    p = fmaf(p, u, -1.558731014e-06f);
    p = fmaf(p, u, 6.042340829e-05f);
    p = fmaf(p, u, -3.231707524e-05f);
    p = fmaf(p, u, -3.187433758e-04f);
    p = fmaf(p, u, 4.263879964e-04f);
    p = fmaf(p, u, 1.538239885e-03f);
    p = fmaf(p, u, -3.241579747e-03f);
    p = fmaf(p, u, -1.075335592e-02f);
    p = fmaf(p, u, 1.822133549e-02f);
    p = fmaf(p, u, 1.397358030e-01f);
    p = fmaf(p, u, 3.435803354e-01f);
    p = fmaf(p, u, 5.107913613e-01f);
    return E * (t * p);
}

}  // namespace nb
