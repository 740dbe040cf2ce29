// lj.cuh -- Lennard-Jones pair terms (Sec. 2.1.2, Eq. lj) shared by the pair kernels
// and the all-pairs comparison kernel: eps_ij = sqrt(eps_i) sqrt(eps_j) (carried exactly
// as a two-product), sigma_ij = (sigma_i + sigma_j)/2, optional switch
// S(x) = 1 - 6x^5 + 15x^4 - 10x^3, x = (r - r_s)/(r_c - r_s) on [r_s, r_c].
#pragma once
#include "common.cuh"

namespace nb {

// Electrostatics of the pair kernels (a template argument): none, Ewald direct space
// ke q q erfc(alpha r)/r, or the reaction field ke q q (1/r + k r^2 - c) of Eq. RFA.
constexpr int kCoulNone = 0;
constexpr int kCoulEwald = 1;
constexpr int kCoulRF = 2;

// System constants the pair math needs, held in registers for the whole block.
struct PairK {
    float rc2, alpha, ke, rs, inv_sw;
    float krf, crf;        // reaction field k_RFA, c_RFA (rounded to FP32)
    float krf_lo, crf_lo;  // their rounding errors (the energy uses hi + lo)
    int sw;                // LJ switch on
};

__device__ __forceinline__ PairK pair_k(const SysDev& S) {
    PairK K;
    K.rc2 = S.rc2;
    K.alpha = S.alpha;
    K.ke = S.ke;
    K.krf = S.krf;
    K.crf = S.crf;
    K.krf_lo = S.krf_lo;
    K.crf_lo = S.crf_lo;
    K.rs = S.rs;
    K.inv_sw = S.inv_sw;
    K.sw = S.has_switch;
    return K;
}

// 1/r^2 from rinv = rsqrtf(r2).  (1/r)^2 carries the few-ulp error of the hardware
// reciprocal square root twice, which the 6th and 12th powers of LJ multiply; one
// Newton-Raphson step for the reciprocal of r2, y + y (1 - r2 y) with the residual formed by
// an FMA, brings it to about one ulp of 1/r^2 at three instructions (a correctly rounded
// division costs several times that).
__device__ __forceinline__ float recip_r2(float r2, float rinv) {
    const float y = rinv * rinv;
    return fmaf(y, fmaf(-r2, y, 1.f), y);
}

// (sigma/r)^2 with sigma^2 carried as an FMA two-product hi + lo: every pair of two given
// atom types would otherwise share the same rounding of sigma^2, a bias that the
// 6th/12th powers amplify and that does not average out over the pairs.
__device__ __forceinline__ float sig2_over_r2(float sig, float r2inv) {
    float hi = sig * sig;
    float lo = fmaf(sig, sig, -hi);
    return fmaf(lo, r2inv, hi * r2inv);
}

// LJ per unit eps (u, f = -u'/r) with the optional switch; r2inv = 1/r^2.
__device__ __forceinline__ void lj_unit(float sig, float r2inv, float rinv, float r2, const PairK& K,
                                        float& u, float& f) {
    float s2 = sig2_over_r2(sig, r2inv);
    float s6 = s2 * s2 * s2;
    u = 4.f * (s6 * s6 - s6);
    f = 24.f * (2.f * s6 * s6 - s6) * r2inv;
    if (K.sw) {
        // x = 0 below r_s gives S = 1, S' = 0 exactly: no branch on r
        float r = r2 * rinv;
        float x = fmaxf(0.f, (r - K.rs) * K.inv_sw);
        float x2 = x * x, x3 = x2 * x;
        float sw = 1.f + x3 * (-10.f + x * (15.f - 6.f * x));
        float dsw = x2 * (-30.f + x * (60.f - 30.f * x)) * K.inv_sw;  // dS/dr
        f = f * sw - u * dsw * rinv;
        u *= sw;
    }
}

}  // namespace nb
