// langevin.cu -- Langevin dynamics with rigid three-site water (Sec. 2.2.1: the MD loop's
// position and velocity constraint steps, SETTLE, and the Langevin integrator).
//
// One step of the Langevin "middle" scheme in leapfrog variables (velocities at half
// steps), from x_n, v_{n-1/2} and F(x_n):
//   v += dt w F;  constrain v at x_n
//   x' = x_n + dt/2 v;  v = c1 v + c2 sqrt(kT w) xi  (c1 = exp(-gamma dt), c2 = sqrt(1 - c1^2))
//   x'' = x' + dt/2 v;  x_{n+1} = SETTLE(x_n, x'');  v += (x_{n+1} - x'') / dt
// is one kernel with one thread per constraint group (a water molecule or a free atom).
// The constraint algebra runs in FP64: SETTLE (Miyamoto and Kollman) in closed form for
// the positions, the 3x3 linear system of the bond-length rates for the velocities.
#include <math.h>

#include "common.cuh"

namespace nb {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 d3(float4 a) { return {a.x, a.y, a.z}; }
__device__ __forceinline__ D3 operator-(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 operator+(D3 a, D3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 operator*(double s, D3 a) { return {s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 unit(D3 a) { return (1.0 / sqrt(dot(a, a))) * a; }

// SETTLE: the positions (a3, b3, c3) of the rigid molecule (O, H, H; |OH| = d_oh,
// |HH| = d_hh) that solve the SHAKE equations for old positions (a0, b0, c0) and
// unconstrained new ones (a1, b1, c1).  The corrections lie in the old plane, so every
// atom keeps its coordinate along the old normal n0 (taken about the new centre of
// mass); those three coordinates fix two tilt angles phi and psi of the canonical
// triangle, and the in-plane rotation theta follows from the corrections exerting no
// torque about the old positions.  Returns false when no such rigid placement exists
// (a step far too large).
__device__ bool settle(D3 a0, D3 b0, D3 c0, D3 a1, D3 b1, D3 c1, double mo, double mh, double d_oh, double d_hh,
                       D3& a3, D3& b3, D3& c3) {
    const double M = mo + 2.0 * mh;
    const double rc = 0.5 * d_hh;
    const double h = sqrt(d_oh * d_oh - rc * rc);  // O to the H-H midpoint
    const double ra = 2.0 * mh * h / M;            // centre of mass to O
    const double rb = h - ra;                      // centre of mass to the H-H midpoint
    const D3 com = (1.0 / M) * (mo * a1 + mh * (b1 + c1));
    const D3 pa = a1 - com, pb = b1 - com, pc = c1 - com;
    const D3 ob = b0 - a0, oc = c0 - a0;
    const D3 n0 = unit(cross(ob, oc));   // Z: normal of the old plane
    const D3 n1 = unit(cross(pa, n0));   // X: perpendicular to the new O direction
    const D3 n2 = cross(n0, n1);         // Y: the new O projects onto +Y
    const double za = dot(pa, n0);
    const double xb1 = dot(pb, n1), yb1 = dot(pb, n2), zb = dot(pb, n0);
    const double xc1 = dot(pc, n1), yc1 = dot(pc, n2), zc = dot(pc, n0);
    const double xb0 = dot(ob, n1), yb0 = dot(ob, n2), xc0 = dot(oc, n1), yc0 = dot(oc, n2);
    const double sphi = za / ra;
    if (!(fabs(sphi) < 1.0)) return false;
    const double cphi = sqrt(1.0 - sphi * sphi);
    const double spsi = (zb - zc) / (2.0 * rc * cphi);
    if (!(fabs(spsi) < 1.0)) return false;
    const double cpsi = sqrt(1.0 - spsi * spsi);
    // the tilted canonical triangle before the in-plane rotation (A on +Y, B at -X)
    const double ya2 = ra * cphi;
    const double xb2 = -rc * cpsi;
    const double yb2 = -rb * cphi - rc * spsi * sphi;
    const double yc2 = -rb * cphi + rc * spsi * sphi;
    // zero torque about the old positions: al sin(theta) + be cos(theta) = ga
    const double al = xb2 * (xb0 - xc0) + yb0 * yb2 + yc0 * yc2;
    const double be = xb2 * (yc0 - yb0) + xb0 * yb2 + xc0 * yc2;
    const double ga = xb0 * yb1 - xb1 * yb0 + xc0 * yc1 - xc1 * yc0;
    const double r2 = al * al + be * be;
    const double disc = r2 - ga * ga;
    if (!(disc >= 0.0) || !(r2 > 0.0)) return false;
    const double sth = (al * ga - be * sqrt(disc)) / r2;  // the root near theta = 0
    const double cth = sqrt(fmax(0.0, 1.0 - sth * sth));
    const double xa3 = -ya2 * sth, ya3 = ya2 * cth;
    const double xb3 = xb2 * cth - yb2 * sth, yb3 = xb2 * sth + yb2 * cth;
    const double xc3 = -xb2 * cth - yc2 * sth, yc3 = -xb2 * sth + yc2 * cth;
    a3 = com + xa3 * n1 + ya3 * n2 + za * n0;
    b3 = com + xb3 * n1 + yb3 * n2 + zb * n0;
    c3 = com + xc3 * n1 + yc3 * n2 + zc * n0;
    return true;
}

// Velocities of the molecule at (a, b, c) projected so that the three bond lengths have
// zero rate: v_i += w_i sum_k mu_k g_k (sign by bond end), g_k = r_i - r_j, with the 3x3
// system g_k . (v_i - v_j) = 0 solved by Cramer's rule.
__device__ void rattle(D3 a, D3 b, D3 c, double wo, double wh, D3& va, D3& vb, D3& vc) {
    const D3 g0 = a - b, g1 = a - c, g2 = b - c;  // bonds (O,H1), (O,H2), (H1,H2)
    // A_kl = d/dmu_l [g_k . (v_i - v_j)]
    const double A00 = (wo + wh) * dot(g0, g0), A01 = wo * dot(g0, g1), A02 = -wh * dot(g0, g2);
    const double A10 = wo * dot(g1, g0), A11 = (wo + wh) * dot(g1, g1), A12 = wh * dot(g1, g2);
    const double A20 = -wh * dot(g2, g0), A21 = wh * dot(g2, g1), A22 = 2.0 * wh * dot(g2, g2);
    const double r0 = -dot(g0, va - vb), r1 = -dot(g1, va - vc), r2 = -dot(g2, vb - vc);
    const double det = A00 * (A11 * A22 - A12 * A21) - A01 * (A10 * A22 - A12 * A20) + A02 * (A10 * A21 - A11 * A20);
    const double inv = 1.0 / det;
    const double m0 = inv * (r0 * (A11 * A22 - A12 * A21) - A01 * (r1 * A22 - A12 * r2) + A02 * (r1 * A21 - A11 * r2));
    const double m1 = inv * (A00 * (r1 * A22 - A12 * r2) - r0 * (A10 * A22 - A12 * A20) + A02 * (A10 * r2 - r1 * A20));
    const double m2 = inv * (A00 * (A11 * r2 - r1 * A21) - A01 * (A10 * r2 - r1 * A20) + r0 * (A10 * A21 - A11 * A20));
    va = va + (wo * m0) * g0 + (wo * m1) * g1;
    vb = vb + (-wh * m0) * g0 + (wh * m2) * g2;
    vc = vc + (-wh * m1) * g1 + (-wh * m2) * g2;
}

__device__ __forceinline__ float3 force_of(const long long* __restrict__ ffix, int N, int k, float finv) {
    return make_float3(__ll2float_rn(ffix[k]) * finv, __ll2float_rn(ffix[(size_t)N + k]) * finv,
                       __ll2float_rn(ffix[2 * (size_t)N + k]) * finv);
}

// One Langevin middle step of a constraint group of NA atoms (module header).
template <int NA>
__device__ __forceinline__ unsigned langevin_group(const int (&id)[3], float4* __restrict__ xq, float4* __restrict__ v,
                                               double h, double c1, double c2, const long long* ffix,
                                               const int* __restrict__ iperm, int N, float finv, double kT,
                                               const float* __restrict__ xi, double d_oh, double d_hh,
                                               float* __restrict__ ke_atom, unsigned* __restrict__ err,
                                               const SysDev& S, const LoadNext& ln) {
    float4 xo[NA], vo[NA];
    D3 x0[NA], vv[NA], x2[NA], x3[NA];
    double w[NA];
    unsigned need = 0u;  // bit 0: rebuild requested, bit 1: prune requested
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = id[a];
        xo[a] = xq[i];
        vo[a] = v[i];
        w[a] = vo[a].w;
        const float3 F = force_of(ffix, N, iperm[i], finv);
        x0[a] = d3(xo[a]);
        vv[a] = d3(vo[a]) + (h * w[a]) * D3{F.x, F.y, F.z};
    }
    if constexpr (NA == 3) rattle(x0[0], x0[1], x0[2], w[0], w[1], vv[0], vv[1], vv[2]);
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = id[a];
        const D3 x1 = x0[a] + (0.5 * h) * vv[a];
        const double sd = w[a] > 0.0 ? c2 * sqrt(kT * w[a]) : 0.0;
        const D3 z = {xi[3 * (size_t)i], xi[3 * (size_t)i + 1], xi[3 * (size_t)i + 2]};
        vv[a] = c1 * vv[a] + sd * z;
        x2[a] = x1 + (0.5 * h) * vv[a];
        x3[a] = x2[a];
    }
    if constexpr (NA == 3) {
        if (!settle(x0[0], x0[1], x0[2], x2[0], x2[1], x2[2], 1.0 / w[0], 1.0 / w[1], d_oh, d_hh, x3[0], x3[1],
                    x3[2]))
            atomicOr(err, NB_DEVERR_NONFINITE);
#pragma unroll
        for (int a = 0; a < NA; ++a) vv[a] = vv[a] + (1.0 / h) * (x3[a] - x2[a]);
    }
#pragma unroll
    for (int a = 0; a < NA; ++a) {
        const int i = id[a];
        const D3 v0 = d3(vo[a]);
        const double k0 = w[a] > 0.0 ? 0.5 * dot(v0, v0) / w[a] : 0.0;
        const double k1 = w[a] > 0.0 ? 0.5 * dot(vv[a], vv[a]) / w[a] : 0.0;
        ke_atom[i] = (float)(0.5 * (k0 + k1));
        const float4 xn = make_float4((float)x3[a].x, (float)x3[a].y, (float)x3[a].z, xo[a].w);
        xq[i] = xn;
        v[i] = make_float4((float)vv[a].x, (float)vv[a].y, (float)vv[a].z, vo[a].w);
        if (ln.xs) {  // the next evaluation's load (see LoadNext)
            const int k = iperm[i];
            ln.ffix[k] = 0;
            ln.ffix[(size_t)N + k] = 0;
            ln.ffix[2 * (size_t)N + k] = 0;
            bool pr = false;
            if (load_atom(xn, S, ln.xref[i], ln.xsb, ln.xs, k, ln.x_prune, ln.x_prune ? &pr : nullptr)) need |= 1u;
            if (pr) need |= 2u;
        }
    }
    return need;
}

// One Langevin middle step of every constraint group.  groups[g] = (O, H1, H2, 3) for a
// water molecule or (atom, -, -, 1) for a free atom.
__global__ void k_langevin(int n_groups, const int4* __restrict__ groups, float4* __restrict__ xq,
                           float4* __restrict__ v, const float* __restrict__ dt, const float* __restrict__ gamma,
                           const int* __restrict__ sid, const SysDev* __restrict__ sys, const long long* ffix,
                           const int* __restrict__ iperm, int N, float finv, double kT, const float* __restrict__ xi,
                           double d_oh, double d_hh, float* __restrict__ ke_atom, unsigned* __restrict__ err,
                           LoadNext ln) {
    pdl_wait();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    if (g == 0 && ln.xs) ln.flags[NB_FLAG_FRESH] = 0u;  // new positions: the list is no longer fresh
    const int4 G = groups[g];
    const int id[3] = {G.x, G.y, G.z};
    const int s = sid[G.x];
    const double h = dt[s];
    const double c1 = exp(-(double)gamma[s] * h);
    const double c2 = sqrt(fmax(0.0, 1.0 - c1 * c1));
    const SysDev& S = sys[s];
    const unsigned need = G.w == 3
                          ? langevin_group<3>(id, xq, v, h, c1, c2, ffix, iperm, N, finv, kT, xi, d_oh, d_hh, ke_atom,
                                              err, S, ln)
                          : langevin_group<1>(id, xq, v, h, c1, c2, ffix, iperm, N, finv, kT, xi, d_oh, d_hh, ke_atom,
                                              err, S, ln);
    const unsigned act = __activemask();  // threads past n_groups returned above
    if (__any_sync(act, (need & 1u) != 0u) && (threadIdx.x & 31) == __ffs(act) - 1) atomicOr(&ln.flags[0], 1u);
    if (ln.x_prune) request_prune(act, (need & 2u) != 0u, s, ln.prune_sys, ln.flags);
}

// K = |v|^2 / (2 w) per atom (the last state of a run).
__global__ void k_kinetic(int N, const float4* __restrict__ v, float* __restrict__ ke_atom) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 u = v[i];
    ke_atom[i] = u.w > 0.f ? 0.5f * (u.x * u.x + u.y * u.y + u.z * u.z) / u.w : 0.f;
}

// SETTLE of the molecules alone: x constrained relative to x_ref; v (if given) += the
// correction / dt.
__global__ void k_settle(int n_groups, const int4* __restrict__ groups, const float4* __restrict__ x_ref,
                         float4* __restrict__ x, float4* __restrict__ v, const float* __restrict__ inv_mass, float dt,
                         double d_oh, double d_hh, unsigned* __restrict__ err) {
    pdl_wait();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const int4 G = groups[g];
    if (G.w != 3) return;
    const int id[3] = {G.x, G.y, G.z};
    D3 r0[3], r1[3], r3[3];
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r0[a] = d3(x_ref[id[a]]);
        r1[a] = d3(x[id[a]]);
        w[a] = inv_mass[id[a]];
    }
    if (!settle(r0[0], r0[1], r0[2], r1[0], r1[1], r1[2], 1.0 / w[0], 1.0 / w[1], d_oh, d_hh, r3[0], r3[1], r3[2])) {
        atomicOr(err, NB_DEVERR_NONFINITE);
        return;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float4 p = x[id[a]];
        x[id[a]] = make_float4((float)r3[a].x, (float)r3[a].y, (float)r3[a].z, p.w);
        if (v) {
            float4 u = v[id[a]];
            const D3 du = (1.0 / dt) * (r3[a] - r1[a]);
            u.x = (float)(u.x + du.x);
            u.y = (float)(u.y + du.y);
            u.z = (float)(u.z + du.z);
            v[id[a]] = u;
        }
    }
}

__global__ void k_rattle(int n_groups, const int4* __restrict__ groups, const float4* __restrict__ x,
                         float4* __restrict__ v) {
    pdl_wait();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_groups) return;
    const int4 G = groups[g];
    if (G.w != 3) return;
    const int id[3] = {G.x, G.y, G.z};
    D3 r[3], u[3];
    double w[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        r[a] = d3(x[id[a]]);
        const float4 q = v[id[a]];
        u[a] = d3(q);
        w[a] = q.w;
    }
    rattle(r[0], r[1], r[2], w[0], w[1], u[0], u[1], u[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float4 q = v[id[a]];
        v[id[a]] = make_float4((float)u[a].x, (float)u[a].y, (float)u[a].z, q.w);
    }
}

void launch_langevin(nb_handle* h, float4* xq, float4* v, const float* dt, const float* gamma, double kT,
                     const float* xi, cudaStream_t st, bool load_next) {
    LoadNext ln;
    if (load_next) {
        ln.xref = h->xref;
        ln.xsb = h->xsb;
        ln.xs = h->xs;
        ln.ffix = h->ffix;
        ln.flags = h->flags;
        ln.x_prune = h->x_prune;
        ln.prune_sys = h->prune_sys;
    }
    launch_pdl(k_langevin, cdiv(h->n_groups, 128), 128, 0, st, h->n_groups, h->groups, xq, v, dt, gamma, h->sid, h->sys,
                                                       h->ffix, h->iperm, h->n_atoms, h->finv, kT, xi, h->d_oh,
                                                       h->d_hh, h->ke_atom, h->flags + 1, ln);
}

void launch_kinetic(nb_handle* h, const float4* v, cudaStream_t st) {
    launch_pdl(k_kinetic, cdiv(h->n_atoms, 256), 256, 0, st, h->n_atoms, v, h->ke_atom);
}

void launch_settle(nb_handle* h, const float4* x_ref, float4* x, float4* v, const float* inv_mass, float dt,
                   cudaStream_t st) {
    launch_pdl(k_settle, cdiv(h->n_groups, 128), 128, 0, st, h->n_groups, h->groups, x_ref, x, v, inv_mass, dt, h->d_oh,
                                                     h->d_hh, h->flags + 1);
}

void launch_rattle(nb_handle* h, const float4* x, float4* v, cudaStream_t st) {
    launch_pdl(k_rattle, cdiv(h->n_groups, 128), 128, 0, st, h->n_groups, h->groups, x, v);
}

}  // namespace nb
