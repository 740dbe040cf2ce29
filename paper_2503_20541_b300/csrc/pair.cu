// pair.cu -- fused nonbonded pair kernel and its force vector-Jacobian product.
//
// Forces (Sec. 2.1.2): for every list pair with r < r_c under the minimum image
//   Lennard-Jones, Eq. (lj), eps_ij = sqrt(eps_i) sqrt(eps_j), sigma_ij = (sigma_i + sigma_j)/2,
//     optionally multiplied by the switch S(x) = 1 - 6x^5 + 15x^4 - 10x^3 on [r_s, r_c];
//   Ewald direct space ke q_i q_j erfc(alpha r)/r;
// and, for each of the atom's excluded partners (any distance), the exclusion
// correction -ke q_i q_j erf(alpha r)/r (the reciprocal sum still contains the
// pair).  A pair force is F_i = f(r) d with d = mi(x_i - x_j), f = -U'/r.
//
// Work decomposition: P lanes per atom i (P = 4..32) stride over i's full
// neighbour list (both directions of every pair are listed), i's data stays in
// registers, partial sums are reduced with warp shuffles in a fixed tree.  No
// atomics: the force on i is written once, converted to int64 fixed point.
// Every FP32 summation order is fixed by the list, so results are bitwise
// reproducible.
#include "common.cuh"

namespace nb {

__device__ __forceinline__ void pair_vec(const float4& a, const float4& b, int per, float L0, float L1, float L2,
                                         float h0, float h1, float h2, float& dx, float& dy, float& dz) {
    if (per) {
        dx = mi_pair(a.x, b.x, L0, h0);
        dy = mi_pair(a.y, b.y, L1, h1);
        dz = mi_pair(a.z, b.z, L2, h2);
    } else {
        dx = a.x - b.x;
        dy = a.y - b.y;
        dz = a.z - b.z;
    }
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
__device__ __forceinline__ void lj_unit(float sig, float r2inv, float rinv, float r2, const SysDev& S,
                                        float& u, float& f) {
    float s2 = sig2_over_r2(sig, r2inv);
    float s6 = s2 * s2 * s2;
    u = 4.f * (s6 * s6 - s6);
    f = 24.f * (2.f * s6 * s6 - s6) * r2inv;
    if (S.has_switch) {
        float r = r2 * rinv;
        if (r > S.rs) {
            float x = (r - S.rs) * S.inv_sw;
            float x2 = x * x, x3 = x2 * x;
            float sw = 1.f + x3 * (-10.f + x * (15.f - 6.f * x));
            float dsw = x2 * (-30.f + x * (60.f - 30.f * x)) * S.inv_sw;  // dS/dr
            f = f * sw - u * dsw * rinv;
            u *= sw;
        }
    }
}

template <int P, bool LJ, bool COUL>
__global__ void __launch_bounds__(256) k_pair(int N, int cap, const float4* __restrict__ xs,
                                               const float2* __restrict__ ps, const int* __restrict__ sid,
                                               const SysDev* __restrict__ sys, const int* __restrict__ nbr,
                                               const int* __restrict__ cnt, const int* __restrict__ perm,
                                               const int* __restrict__ iperm, const int* __restrict__ ex_off,
                                               const int* __restrict__ ex_idx, long long* __restrict__ ffix,
                                               float4* __restrict__ e_atom, float scale, unsigned* flags) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt / P, lane = gt % P;
    bool valid = i < N;
    int ii = valid ? i : N - 1;
    const SysDev& S = sys[sid[ii]];
    const float4 xi = xs[ii];
    const float2 pi = ps[ii];
    const int c = valid ? cnt[ii] : 0;
    const int* row = nbr + (size_t)ii * cap;
    const float L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const float h0 = S.halfL[0], h1 = S.halfL[1], h2 = S.halfL[2];
    const int per = S.periodic;
    const float rc2 = S.rc2;
    const float qke = S.ke * xi.w;
    const float alpha = S.alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    for (int k = lane; k < c; k += P) {
        int j = __ldg(row + k);
        float4 xj = xs[j];
        float dx, dy, dz;
        pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
        float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (r2 < rc2) {
            float rinv = rsqrtf(r2);
            float r2inv = __frcp_rn(r2);  // correctly rounded: LJ raises it to the 6th power
            float fr = 0.f;
            if (LJ && pi.y != 0.f) {
                float2 pj = ps[j];
                float eps = pi.y * pj.y;                // eps_ij = eps + eps_lo exactly
                float eps_lo = fmaf(pi.y, pj.y, -eps);
                float u, f;
                lj_unit(0.5f * (pi.x + pj.x), r2inv, rinv, r2, S, u, f);
                elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
                fr = fmaf(eps_lo, f, eps * f);
            }
            if (COUL) {
                float r = r2 * rinv;
                float qq = qke * xj.w;
                float ar = alpha * r;
                float ec = erfcf(ar);
                float gau = gau_c * __expf(-ar * ar);
                edir = fmaf(qq * ec, rinv, edir);
                fr = fmaf(qq * fmaf(ec, rinv, gau), r2inv, fr);
            }
            fx = fmaf(fr, dx, fx);
            fy = fmaf(fr, dy, fy);
            fz = fmaf(fr, dz, fz);
        }
    }
    if (COUL && alpha > 0.f) {
        // exclusion correction for i's excluded partners (at any distance)
        int oi = valid ? perm[ii] : 0;
        int e0 = valid ? ex_off[oi] : 0;
        int ne = valid ? ex_off[oi + 1] - e0 : 0;
        for (int e = lane; e < ne; e += P) {
            int j = iperm[ex_idx[e0 + e]];
            float4 xj = xs[j];
            float dx, dy, dz;
            pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float rinv = rsqrtf(r2);
            float r2inv = rinv * rinv;
            float r = r2 * rinv;
            float qq = qke * xj.w;
            float ar = alpha * r;
            float ef = erff(ar);
            float gau = gau_c * __expf(-ar * ar);
            eex = fmaf(-qq * ef, rinv, eex);
            float fr = qq * (gau - ef * rinv) * r2inv;
            fx = fmaf(fr, dx, fx);
            fy = fmaf(fr, dy, fy);
            fz = fmaf(fr, dz, fz);
        }
    }
    fx = group_sum<P>(fx);
    fy = group_sum<P>(fy);
    fz = group_sum<P>(fz);
    elj = group_sum<P>(elj);
    edir = group_sum<P>(edir);
    eex = group_sum<P>(eex);
    if (valid && lane == 0) {
        ffix[ii] = to_fix(fx, scale, flags + 1);
        ffix[(size_t)N + ii] = to_fix(fy, scale, flags + 1);
        ffix[2 * (size_t)N + ii] = to_fix(fz, scale, flags + 1);
        e_atom[ii] = make_float4(0.5f * elj, 0.5f * edir, 0.5f * eex, 0.f);
    }
}

// Warp-per-atom variant (used when 32 lanes serve one atom): the cut-off test runs on
// 32 list entries at a time and the pairs inside r_c are appended, in list order, to a
// per-warp queue in shared memory; the interaction math then runs on full warps of
// queued pairs, so lanes are not idle on pairs between r_c and r_nl.  Atoms with
// eps_i = 0 skip the LJ term as a whole warp.  The summation order is fixed by the list
// and the ballot order, so results stay bitwise reproducible.
constexpr int kQWarps = 8;

template <bool LJ, bool COUL>
__device__ __forceinline__ void pair_heavy(const float4& q, int j, const float4& xi, const float2& pi, bool do_lj,
                                           const SysDev& S, const float4* __restrict__ xs,
                                           const float2* __restrict__ ps, float qke, float alpha, float gau_c,
                                           float& fx, float& fy, float& fz, float& elj, float& edir) {
    float r2 = q.w;
    float rinv = rsqrtf(r2);
    float r2inv = __frcp_rn(r2);
    float fr = 0.f;
    if (LJ && do_lj) {
        float2 pj = ps[j];
        float eps = pi.y * pj.y;
        float eps_lo = fmaf(pi.y, pj.y, -eps);
        float u, f;
        lj_unit(0.5f * (pi.x + pj.x), r2inv, rinv, r2, S, u, f);
        elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
        fr = fmaf(eps_lo, f, eps * f);
    }
    if (COUL) {
        float r = r2 * rinv;
        float qq = qke * xs[j].w;
        float ar = alpha * r;
        float ec = erfcf(ar);
        float gau = gau_c * __expf(-ar * ar);
        edir = fmaf(qq * ec, rinv, edir);
        fr = fmaf(qq * fmaf(ec, rinv, gau), r2inv, fr);
    }
    fx = fmaf(fr, q.x, fx);
    fy = fmaf(fr, q.y, fy);
    fz = fmaf(fr, q.z, fz);
}

template <bool LJ, bool COUL>
__global__ void __launch_bounds__(kQWarps * 32) k_pair_q(int N, int cap, const float4* __restrict__ xs,
                                                          const float2* __restrict__ ps, const int* __restrict__ sid,
                                                          const SysDev* __restrict__ sys, const int* __restrict__ nbr,
                                                          const int* __restrict__ cnt, const int* __restrict__ perm,
                                                          const int* __restrict__ iperm,
                                                          const int* __restrict__ ex_off,
                                                          const int* __restrict__ ex_idx,
                                                          long long* __restrict__ ffix,
                                                          float4* __restrict__ e_atom, float scale, unsigned* flags) {
    __shared__ float4 qd[kQWarps][64];
    __shared__ int qj[kQWarps][64];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kQWarps + w;
    if (i >= N) return;  // whole warp
    const SysDev& S = sys[sid[i]];
    const float4 xi = xs[i];
    const float2 pi = ps[i];
    const int c = cnt[i];
    const int* row = nbr + (size_t)i * cap;
    const float L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const float h0 = S.halfL[0], h1 = S.halfL[1], h2 = S.halfL[2];
    const int per = S.periodic;
    const float rc2 = S.rc2;
    const float qke = S.ke * xi.w;
    const float alpha = S.alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    const bool do_lj = pi.y != 0.f;
    const unsigned lt = (1u << lane) - 1u;
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    int nq = 0;
    // software pipeline: list indices are loaded two iterations ahead, positions one ahead
    int jA = lane < c ? __ldg(row + lane) : 0;
    int jB = 32 + lane < c ? __ldg(row + 32 + lane) : 0;
    float4 xA = lane < c ? xs[jA] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int base = 0; base < c; base += 32) {
        const int k = base + lane;
        const int j = jA;
        const float4 xj = xA;
        if (k + 32 < c) xA = xs[jB];
        jA = jB;
        jB = (k + 64 < c) ? __ldg(row + k + 64) : 0;
        bool acc = false;
        float dx = 0.f, dy = 0.f, dz = 0.f, r2 = 0.f;
        if (k < c) {
            pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
            r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            acc = r2 < rc2;
        }
        unsigned bits = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            int pos = nq + __popc(bits & lt);
            qd[w][pos] = make_float4(dx, dy, dz, r2);
            qj[w][pos] = j;
        }
        nq += __popc(bits);
        if (nq >= 32) {
            __syncwarp();
            pair_heavy<LJ, COUL>(qd[w][lane], qj[w][lane], xi, pi, do_lj, S, xs, ps, qke, alpha, gau_c, fx, fy, fz,
                                 elj, edir);
            __syncwarp();
            if (lane < nq - 32) {
                qd[w][lane] = qd[w][lane + 32];
                qj[w][lane] = qj[w][lane + 32];
            }
            nq -= 32;
            __syncwarp();
        }
    }
    __syncwarp();
    if (lane < nq)
        pair_heavy<LJ, COUL>(qd[w][lane], qj[w][lane], xi, pi, do_lj, S, xs, ps, qke, alpha, gau_c, fx, fy, fz, elj,
                             edir);
    if (COUL && alpha > 0.f) {
        int oi = perm[i];
        int e0 = ex_off[oi];
        int ne = ex_off[oi + 1] - e0;
        for (int e = lane; e < ne; e += 32) {
            int j = iperm[ex_idx[e0 + e]];
            float4 xj = xs[j];
            float dx, dy, dz;
            pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float rinv = rsqrtf(r2);
            float r2inv = rinv * rinv;
            float r = r2 * rinv;
            float qq = qke * xj.w;
            float ar = alpha * r;
            float ef = erff(ar);
            float gau = gau_c * __expf(-ar * ar);
            eex = fmaf(-qq * ef, rinv, eex);
            float fr = qq * (gau - ef * rinv) * r2inv;
            fx = fmaf(fr, dx, fx);
            fy = fmaf(fr, dy, fy);
            fz = fmaf(fr, dz, fz);
        }
    }
    fx = group_sum<32>(fx);
    fy = group_sum<32>(fy);
    fz = group_sum<32>(fz);
    elj = group_sum<32>(elj);
    edir = group_sum<32>(edir);
    eex = group_sum<32>(eex);
    if (lane == 0) {
        ffix[i] = to_fix(fx, scale, flags + 1);
        ffix[(size_t)N + i] = to_fix(fy, scale, flags + 1);
        ffix[2 * (size_t)N + i] = to_fix(fz, scale, flags + 1);
        e_atom[i] = make_float4(0.5f * elj, 0.5f * edir, 0.5f * eex, 0.f);
    }
}

// Force VJP.  For each directed pair (i, j) with u = lam_i - lam_j and du = d.u:
//   gx_i += f u + (f'/r) du d           (J (lam_i - lam_j), J = f I + (f'/r) d d^T)
//   gq_i += ke q_j (f / qq) du,  gsig_i += 1/2 (df/dsigma_ij) du,  ge_i += sqrt(eps_j) (f/eps) du
// and the forces F_i as in k_pair.  The exclusion correction contributes the same way.
template <int P, bool LJ, bool COUL>
__global__ void __launch_bounds__(256) k_vjp(int N, int cap, const float4* __restrict__ xs,
                                              const float2* __restrict__ ps, const int* __restrict__ sid,
                                              const SysDev* __restrict__ sys, const int* __restrict__ nbr,
                                              const int* __restrict__ cnt, const int* __restrict__ perm,
                                              const int* __restrict__ iperm, const int* __restrict__ ex_off,
                                              const int* __restrict__ ex_idx, const float4* __restrict__ lam,
                                              float4* __restrict__ gx_s, float2* __restrict__ gp_s,
                                              long long* __restrict__ ffix, float4* __restrict__ e_atom,
                                              float scale, unsigned* flags) {
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt / P, lane = gt % P;
    bool valid = i < N;
    int ii = valid ? i : N - 1;
    const SysDev& S = sys[sid[ii]];
    const float4 xi = xs[ii];
    const float2 pi = ps[ii];
    const float4 li = lam[ii];
    const int c = valid ? cnt[ii] : 0;
    const int* row = nbr + (size_t)ii * cap;
    const float L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const float h0 = S.halfL[0], h1 = S.halfL[1], h2 = S.halfL[2];
    const int per = S.periodic;
    const float rc2 = S.rc2;
    const float alpha = S.alpha, a2 = alpha * alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f, gq = 0.f, gs = 0.f, ge = 0.f;
    for (int k = lane; k < c; k += P) {
        int j = __ldg(row + k);
        float4 xj = xs[j];
        float dx, dy, dz;
        pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
        float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        if (r2 < rc2) {
            float4 lj4 = lam[j];
            float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
            float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
            float rinv = rsqrtf(r2);
            float r2inv = __frcp_rn(r2);
            float fr = 0.f, fpr = 0.f;  // f and f'/r
            if (LJ) {
                float2 pj = ps[j];
                float eps = pi.y * pj.y;
                float sig = 0.5f * (pi.x + pj.x);
                float s2 = sig2_over_r2(sig, r2inv);
                float s6 = s2 * s2 * s2, s12 = s6 * s6;
                float u = 4.f * (s12 - s6);                       // per unit eps
                float f = 24.f * (2.f * s12 - s6) * r2inv;
                float fp = -24.f * (28.f * s12 - 8.f * s6) * r2inv * r2inv;
                float sinv = sig > 0.f ? 1.f / sig : 0.f;
                float us = 4.f * (12.f * s12 - 6.f * s6) * sinv;           // du/dsigma
                float fs = 24.f * (24.f * s12 - 6.f * s6) * r2inv * sinv;  // df/dsigma
                if (S.has_switch) {
                    float r = r2 * rinv;
                    if (r > S.rs) {
                        float x = (r - S.rs) * S.inv_sw;
                        float x2 = x * x, x3 = x2 * x;
                        float sw = 1.f + x3 * (-10.f + x * (15.f - 6.f * x));
                        float d1 = x2 * (-30.f + x * (60.f - 30.f * x)) * S.inv_sw;
                        float d2 = x * (-60.f + x * (180.f - 120.f * x)) * S.inv_sw * S.inv_sw;
                        fp = fp * sw + 2.f * f * d1 * rinv - u * (d2 - d1 * rinv) * r2inv;
                        fs = fs * sw - us * d1 * rinv;
                        f = f * sw - u * d1 * rinv;
                        u *= sw;
                    }
                }
                float eps_lo = fmaf(pi.y, pj.y, -eps);
                elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
                fr = fmaf(eps_lo, f, eps * f);
                fpr = eps * fp;
                ge = fmaf(pj.y * f, du, ge);
                gs = fmaf(0.5f * eps * fs, du, gs);
            }
            if (COUL) {
                float r = r2 * rinv;
                float qq = S.ke * xi.w * xj.w;
                float ar = alpha * r;
                float ec = erfcf(ar);
                float gau = gau_c * __expf(-ar * ar);
                float fcu = fmaf(ec, rinv, gau) * r2inv;  // f per unit qq
                edir = fmaf(qq * ec, rinv, edir);
                fr = fmaf(qq, fcu, fr);
                fpr = fmaf(-qq * r2inv, fmaf(3.f, fcu, 2.f * a2 * gau), fpr);
                gq = fmaf(S.ke * xj.w * fcu, du, gq);
            }
            float k2 = fpr * du;
            gx = fmaf(fr, ux, fmaf(k2, dx, gx));
            gy = fmaf(fr, uy, fmaf(k2, dy, gy));
            gz = fmaf(fr, uz, fmaf(k2, dz, gz));
            fx = fmaf(fr, dx, fx);
            fy = fmaf(fr, dy, fy);
            fz = fmaf(fr, dz, fz);
        }
    }
    if (COUL && alpha > 0.f) {
        int oi = valid ? perm[ii] : 0;
        int e0 = valid ? ex_off[oi] : 0;
        int ne = valid ? ex_off[oi + 1] - e0 : 0;
        for (int e = lane; e < ne; e += P) {
            int j = iperm[ex_idx[e0 + e]];
            float4 xj = xs[j];
            float dx, dy, dz;
            pair_vec(xi, xj, per, L0, L1, L2, h0, h1, h2, dx, dy, dz);
            float4 lj4 = lam[j];
            float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
            float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
            float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            float rinv = rsqrtf(r2);
            float r2inv = rinv * rinv;
            float r = r2 * rinv;
            float qq = S.ke * xi.w * xj.w;
            float ar = alpha * r;
            float ef = erff(ar);
            float gau = gau_c * __expf(-ar * ar);
            float fxu = (gau - ef * rinv) * r2inv;  // f per unit qq
            eex = fmaf(-qq * ef, rinv, eex);
            float fr = qq * fxu;
            float fpr = -qq * r2inv * fmaf(3.f, fxu, 2.f * a2 * gau);
            gq = fmaf(S.ke * xj.w * fxu, du, gq);
            float k2 = fpr * du;
            gx = fmaf(fr, ux, fmaf(k2, dx, gx));
            gy = fmaf(fr, uy, fmaf(k2, dy, gy));
            gz = fmaf(fr, uz, fmaf(k2, dz, gz));
            fx = fmaf(fr, dx, fx);
            fy = fmaf(fr, dy, fy);
            fz = fmaf(fr, dz, fz);
        }
    }
    fx = group_sum<P>(fx);
    fy = group_sum<P>(fy);
    fz = group_sum<P>(fz);
    gx = group_sum<P>(gx);
    gy = group_sum<P>(gy);
    gz = group_sum<P>(gz);
    gq = group_sum<P>(gq);
    gs = group_sum<P>(gs);
    ge = group_sum<P>(ge);
    elj = group_sum<P>(elj);
    edir = group_sum<P>(edir);
    eex = group_sum<P>(eex);
    if (valid && lane == 0) {
        ffix[ii] = to_fix(fx, scale, flags + 1);
        ffix[(size_t)N + ii] = to_fix(fy, scale, flags + 1);
        ffix[2 * (size_t)N + ii] = to_fix(fz, scale, flags + 1);
        e_atom[ii] = make_float4(0.5f * elj, 0.5f * edir, 0.5f * eex, 0.f);
        gx_s[ii] = make_float4(gx, gy, gz, gq);
        gp_s[ii] = make_float2(gs, ge);
    }
}

template <int P, bool LJ, bool COUL>
static void pair_p(nb_handle* h, cudaStream_t st) {
    int N = h->n_atoms;
    if (P == 32) {
        k_pair_q<LJ, COUL><<<cdiv(N, kQWarps), kQWarps * 32, 0, st>>>(
            N, h->cap, h->xs, h->ps, h->sid, h->sys, h->nbr, h->nbr_cnt, h->perm, h->iperm, h->ex_off, h->ex_idx,
            h->ffix, h->e_atom, h->fscale, h->flags);
        return;
    }
    k_pair<P, LJ, COUL><<<cdiv((long long)N * P, 256), 256, 0, st>>>(
        N, h->cap, h->xs, h->ps, h->sid, h->sys, h->nbr, h->nbr_cnt, h->perm, h->iperm, h->ex_off, h->ex_idx,
        h->ffix, h->e_atom, h->fscale, h->flags);
}

template <int P, bool LJ, bool COUL>
static void vjp_p(nb_handle* h, cudaStream_t st) {
    int N = h->n_atoms;
    k_vjp<P, LJ, COUL><<<cdiv((long long)N * P, 256), 256, 0, st>>>(
        N, h->cap, h->xs, h->ps, h->sid, h->sys, h->nbr, h->nbr_cnt, h->perm, h->iperm, h->ex_off, h->ex_idx,
        h->lam, h->gx_s, h->gp_s, h->ffix, h->e_atom, h->fscale, h->flags);
}

template <bool LJ, bool COUL>
static void pair_dispatch(nb_handle* h, cudaStream_t st, bool vjp) {
    switch (h->lanes) {
        case 4: vjp ? vjp_p<4, LJ, COUL>(h, st) : pair_p<4, LJ, COUL>(h, st); break;
        case 8: vjp ? vjp_p<8, LJ, COUL>(h, st) : pair_p<8, LJ, COUL>(h, st); break;
        case 16: vjp ? vjp_p<16, LJ, COUL>(h, st) : pair_p<16, LJ, COUL>(h, st); break;
        default: vjp ? vjp_p<32, LJ, COUL>(h, st) : pair_p<32, LJ, COUL>(h, st); break;
    }
}

static void dispatch(nb_handle* h, int terms, cudaStream_t st, bool vjp) {
    bool lj = (terms & NB_TERM_LJ) != 0;
    bool coul = (terms & NB_TERM_COUL) != 0;
    if (lj && coul) pair_dispatch<true, true>(h, st, vjp);
    else if (lj) pair_dispatch<true, false>(h, st, vjp);
    else if (coul) pair_dispatch<false, true>(h, st, vjp);
    else pair_dispatch<false, false>(h, st, vjp);
}

void launch_pair(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, false); }
void launch_vjp(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, true); }

}  // namespace nb
