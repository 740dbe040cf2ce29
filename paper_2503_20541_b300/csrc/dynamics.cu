// dynamics.cu -- energy reduction, velocity Verlet, HMC and the HMC adjoint.
//
// Velocity Verlet (Sec. 2.2.1, steps 1, 2, 4, 5) is run as one fused kernel per
// step: it completes the previous step's second half kick with the new forces,
// records the kinetic energy at the integer step, applies the next first half
// kick and drifts the positions.  All per-system reductions (energies, kinetic
// energy, HMC jump, dt gradient) sum in FP64 in a fixed order (energies: per-block
// partials of 1024 atoms, then one warp per system), so they are deterministic.
#include "reduce.cuh"

namespace nb {

__device__ __forceinline__ double block_sum(double v, double* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    __syncthreads();
    return t;  // valid in thread 0
}

// Energy reduction in one launch (reduce.cuh): each thread sums its atoms of the block's tile.
__global__ void __launch_bounds__(kRedThreads) k_reduce_energy(
    int n_sys, const int* __restrict__ blk_sys, const int* __restrict__ blk_off, const SysDev* __restrict__ sys,
    const float4* __restrict__ e_atom, const float4* __restrict__ e_lo, const float4* __restrict__ xs,
    const float* __restrict__ ke_atom, int with_kin, double* __restrict__ part, const double* __restrict__ e_pme_blk,
    const int* __restrict__ pme_blk_off, int terms, unsigned* __restrict__ ticket, double* __restrict__ dst,
    StepStat ss) {
    pdl_wait();
    int a0, a1;
    red_tile_range(blk_sys, blk_off, sys, a0, a1);
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = a0 + threadIdx.x; k < a1; k += kRedThreads) {
        const float4 e = e_atom[k];
        const float q = xs[k].w;
        v[0] += e.x;
        v[1] += e.y;
        v[2] += e.z;
        if (e_lo) {  // precise energies: the two-float records' low parts
            const float4 l = e_lo[k];
            v[0] += l.x;
            v[1] += l.y;
            v[2] += l.z;
        }
        v[3] += (double)q * q;
        if (with_kin) v[4] += ke_atom[k];
        // a system owns the same index range in both orders: its jump sum reads
        // caller-order entries over that range
        if (ss.jump) v[5] += ss.jump[k];
    }
    energy_reduce_finish(v, n_sys, blk_off, sys, with_kin, part, e_pme_blk, pme_blk_off, terms, ticket, dst, ss);
}

__global__ void k_finalize(int N, const long long* __restrict__ ffix, const int* __restrict__ iperm, float finv,
                           float* __restrict__ f_out) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = iperm[i];
    f_out[3 * (size_t)i] = __ll2float_rn(ffix[k]) * finv;
    f_out[3 * (size_t)i + 1] = __ll2float_rn(ffix[(size_t)N + k]) * finv;
    f_out[3 * (size_t)i + 2] = __ll2float_rn(ffix[2 * (size_t)N + k]) * finv;
}

__device__ __forceinline__ float3 load_force(const long long* __restrict__ ffix, int N, int k, float finv) {
    return make_float3(__ll2float_rn(ffix[k]) * finv, __ll2float_rn(ffix[(size_t)N + k]) * finv,
                       __ll2float_rn(ffix[2 * (size_t)N + k]) * finv);
}

// v <- v + c_pre dt w F ; record KE ; [store x, v] ; v <- v + c_post dt w F ; [store v] ; x <- x + dt v
// (ffix is read here and, with the next step's load, zeroed through ln.ffix: not restrict)
__global__ void k_integrate(int N, float4* __restrict__ xq, float4* __restrict__ v, const float* __restrict__ w_ovr,
                            const float* __restrict__ dt, const int* __restrict__ sid,
                            const long long* ffix, const int* __restrict__ iperm, float finv,
                            float c_pre, float c_post, int drift, float* __restrict__ ke_atom,
                            float4* __restrict__ ck_x, float4* __restrict__ ck_v, float4* __restrict__ ck_p,
                            const SysDev* __restrict__ sys, StepObs ob, LoadNext ln) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int si = sid[i];
    float h = dt[si];
    float3 F = load_force(ffix, N, iperm[i], finv);
    float4 vi = v[i];
    float w = w_ovr ? w_ovr[i] : vi.w;
    float4 x = xq[i];
    float a = c_pre * h * w;
    vi.x = fmaf(a, F.x, vi.x);
    vi.y = fmaf(a, F.y, vi.y);
    vi.z = fmaf(a, F.z, vi.z);
    ke_atom[i] = (w > 0.f) ? 0.5f * (vi.x * vi.x + vi.y * vi.y + vi.z * vi.z) / w : 0.f;
    if (ck_x) ck_x[i] = x;
    if (ck_v) ck_v[i] = make_float4(vi.x, vi.y, vi.z, w);
    if (ob.x0) {
        const SysDev& S = sys[si];
        const float4 b0 = ob.x0[i];
        float dx = x.x - b0.x, dy = x.y - b0.y, dz = x.z - b0.z;
        if (S.periodic) {
            dx = mi_any(dx, S.L[0], S.invL[0]);
            dy = mi_any(dy, S.L[1], S.invL[1]);
            dz = mi_any(dz, S.L[2], S.invL[2]);
        }
        ob.jump[i] = (double)dx * dx + (double)dy * dy + (double)dz * dz;
        if (ob.l_prop[si] == ob.step) ob.x_prop[i] = x;
    }
    float b = c_post * h * w;
    vi.x = fmaf(b, F.x, vi.x);
    vi.y = fmaf(b, F.y, vi.y);
    vi.z = fmaf(b, F.z, vi.z);
    if (ck_p) ck_p[i] = make_float4(vi.x, vi.y, vi.z, w);
    if (drift) {
        x.x = fmaf(h, vi.x, x.x);
        x.y = fmaf(h, vi.y, x.y);
        x.z = fmaf(h, vi.z, x.z);
        xq[i] = x;
    }
    v[i] = vi;
    if (ln.xs) {
        if (i == 0) ln.flags[NB_FLAG_FRESH] = 0u;
        const int k = iperm[i];
        ln.ffix[k] = 0;
        ln.ffix[(size_t)N + k] = 0;
        ln.ffix[2 * (size_t)N + k] = 0;
        bool pr = false;
        const bool need = load_atom(x, sys[si], ln.xref[i], ln.xsb, ln.xs, k, ln.x_prune, ln.x_prune ? &pr : nullptr);
        const unsigned act = __activemask();  // threads past N returned above
        const bool lead = (threadIdx.x & 31) == __ffs(act) - 1;
        if (__any_sync(act, need) && lead) atomicOr(&ln.flags[0], 1u);
        if (ln.x_prune) request_prune(act, pr, si, ln.prune_sys, ln.flags);
    }
}

// ------------------------------------------------------------------ HMC

__global__ void k_hmc_init(int N, const float* __restrict__ w, const float* __restrict__ xi, double kT,
                           float4* __restrict__ v, float* __restrict__ ke_atom) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float wi = w[i];
    float s = sqrtf((float)kT * wi);
    float vx = s * xi[3 * (size_t)i], vy = s * xi[3 * (size_t)i + 1], vz = s * xi[3 * (size_t)i + 2];
    v[i] = make_float4(vx, vy, vz, wi);
    ke_atom[i] = (wi > 0.f) ? 0.5f * (vx * vx + vy * vy + vz * vz) / wi : 0.f;
}

__global__ void k_hmc_jump(int N, const float4* __restrict__ x1, const float4* __restrict__ x0,
                           const int* __restrict__ sid, const SysDev* __restrict__ sys, double* __restrict__ jump) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const SysDev& S = sys[sid[i]];
    float4 a = x1[i], b = x0[i];
    float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    if (S.periodic) {
        dx = mi_any(dx, S.L[0], S.invL[0]);
        dy = mi_any(dy, S.L[1], S.invL[1]);
        dz = mi_any(dz, S.L[2], S.invL[2]);
    }
    jump[i] = (double)dx * dx + (double)dy * dy + (double)dz * dz;
}

__global__ void __launch_bounds__(kRedThreads) k_hmc_accept(const SysDev* __restrict__ sys,
                                                             const double* __restrict__ jump,
                                                             const double* __restrict__ e0,
                                                             const double* __restrict__ e1, double kT,
                                                             const double* __restrict__ u, double* __restrict__ stats) {
    pdl_wait();
    __shared__ double sm[kRedThreads / 32];
    int s = blockIdx.x;
    const SysDev& S = sys[s];
    double j = 0.0;
    for (int k = S.atom_off + threadIdx.x; k < S.atom_off + S.n_atoms; k += kRedThreads) j += jump[k];
    j = block_sum(j, sm);
    if (threadIdx.x == 0) {
        double H0 = 0.0, H1 = 0.0;
        for (int c = 0; c < NB_NE; ++c) {
            H0 += e0[(size_t)s * NB_NE + c];
            H1 += e1[(size_t)s * NB_NE + c];
        }
        double dH = H1 - H0;
        double a = (dH <= 0.0) ? 1.0 : exp(-dH / kT);
        if (!(dH == dH)) a = 0.0;  // NaN energy: reject
        double acc = (u[s] < a) ? 1.0 : 0.0;
        double* o = stats + (size_t)s * 4;
        o[0] = dH;
        o[1] = a;
        o[2] = j;
        o[3] = acc;
    }
}

__global__ void k_hmc_restore(int N, float4* __restrict__ x_out, const float4* __restrict__ x0,
                              const int* __restrict__ sid, const double* __restrict__ stats) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    if (stats[(size_t)sid[i] * 4 + 3] == 0.0) x_out[i] = x0[i];
}

// The proposal of each system is the state after l_prop[s] steps (Sec. 4: the length is
// drawn from the discretised folded normal): its statistics are that step's, and the
// Metropolis test u[s] < alpha decides.  A length outside [1, n_leap] is reported and
// the system keeps x0.
__global__ void k_hmc_pick(int n_sys, const int* __restrict__ l_prop, int n_leap,
                           const double* __restrict__ step_stats, const double* __restrict__ u,
                           double* __restrict__ stats, unsigned* __restrict__ err) {
    pdl_wait();
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sys) return;
    const int l = l_prop[s];
    double* o = stats + (size_t)s * 4;
    if (l < 1 || l > n_leap) {
        atomicOr(err, NB_DEVERR_ARG);
        o[0] = 0.0;
        o[1] = 0.0;
        o[2] = 0.0;
        o[3] = 0.0;
        return;
    }
    const double* q = step_stats + ((size_t)(l - 1) * n_sys + s) * 3;
    o[0] = q[0];
    o[1] = q[1];
    o[2] = q[2];
    o[3] = (u[s] < q[1]) ? 1.0 : 0.0;
}

// ------------------------------------------------------------- HMC adjoint
//
// Reverse sweep over the states l = L..1 of the trajectory.  Entering state l, xbar is
// the cotangent of x_l and vbar that of the half-step velocity v_{l+1/2} (zero at l = L).
// A loss term at state l (acceptance probability alpha_l of H_l = U(x_l) + K(v_l), the
// squared jump |mi(x_l - x_0)|^2) adds
//   c_v = dHbar v_l / w                     to the cotangent of v_l,
//   2 gj mi(x_l - x_0) - dHbar F_l          to xbar,
//   -dHbar |v_l|^2 / (2 w^2)                to wbar (K = |v|^2 / 2w at fixed v),
// with dHbar = ga dalpha/ddH = -ga alpha / kT where alpha < 1.  The two half kicks
// around v_l, v_{l+1/2} = v_l + (dt/2) w F_l and v_l = v_{l-1/2} + (dt/2) w F_l, then
// pass u = 2 vbar + c_v through F: the force VJP takes lam = (dt/2) w u, and the step and
// inverse mass collect (1/2) w F.u and (dt/2) F.u.  The cotangent of v_{l-1/2} is
// vbar + c_v; the drift x_l = x_{l-1} + dt v_{l-1/2} then adds dt xbar to it and
// v_{l-1/2}.xbar to the step's cotangent.

__device__ __forceinline__ float inject_dhbar(const Inject& inj, int s, double kT) {
    if (!inj.ga) return 0.f;
    const double a = inj.alpha[(size_t)s * inj.a_stride];
    return (a < 1.0) ? (float)(-inj.ga[s] * a / kT) : 0.f;
}

// lam (slot order) = (dt/2) w (2 vbar + c_v)
__global__ void k_bwd_lambda(int N, const float4* __restrict__ vbar, const float4* __restrict__ v_state,
                             const float* __restrict__ w, const float* __restrict__ dt, const int* __restrict__ sid,
                             const int* __restrict__ iperm, Inject inj, double kT, float4* __restrict__ lam) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int s = sid[i];
    const float wi = w[i];
    const float c = 0.5f * dt[s] * wi;
    const float4 b = vbar[i];
    float ux = 2.f * b.x, uy = 2.f * b.y, uz = 2.f * b.z;
    const float d = inject_dhbar(inj, s, kT);
    if (d != 0.f && wi > 0.f) {
        const float4 v = v_state[i];
        const float fb = d / wi;
        ux = fmaf(fb, v.x, ux);
        uy = fmaf(fb, v.y, uy);
        uz = fmaf(fb, v.z, uz);
    }
    lam[iperm[i]] = make_float4(c * ux, c * uy, c * uz, 0.f);
}

// One state of the reverse sweep, after the VJP kernels wrote gx_s = (dF/dx)^T lam.
__global__ void k_bwd_adjoint(int N, const float4* __restrict__ gx_s, const long long* __restrict__ ffix,
                              const int* __restrict__ iperm, float finv, const float* __restrict__ w,
                              const float* __restrict__ dt, const int* __restrict__ sid,
                              const SysDev* __restrict__ sys, Inject inj, double kT,
                              const float4* __restrict__ x_state, const float4* __restrict__ v_state,
                              const float4* __restrict__ x0, const float4* __restrict__ p_prev,
                              float4* __restrict__ xbar, float4* __restrict__ vbar, float* __restrict__ wbar,
                              double* __restrict__ hbar) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int s = sid[i];
    const int k = iperm[i];
    const float h = dt[s];
    const float wi = w[i];
    const float3 F = load_force(ffix, N, k, finv);
    const float4 g = gx_s[k];
    float4 xb = xbar[i], vb = vbar[i];
    float ux = 2.f * vb.x, uy = 2.f * vb.y, uz = 2.f * vb.z;
    xb.x += g.x;
    xb.y += g.y;
    xb.z += g.z;
    float wb = 0.f;
    if (inj.ga) {
        const float d = inject_dhbar(inj, s, kT);
        const float gj = 2.f * (float)inj.gj[s];
        const SysDev& S = sys[s];
        const float4 p = x_state[i], q = x0[i];
        float dx = p.x - q.x, dy = p.y - q.y, dz = p.z - q.z;
        if (S.periodic) {
            dx = mi_any(dx, S.L[0], S.invL[0]);
            dy = mi_any(dy, S.L[1], S.invL[1]);
            dz = mi_any(dz, S.L[2], S.invL[2]);
        }
        xb.x += gj * dx - d * F.x;
        xb.y += gj * dy - d * F.y;
        xb.z += gj * dz - d * F.z;
        if (d != 0.f && wi > 0.f) {
            const float4 v = v_state[i];
            const float fb = d / wi;
            const float cx = fb * v.x, cy = fb * v.y, cz = fb * v.z;
            ux += cx;
            uy += cy;
            uz += cz;
            vb.x += cx;
            vb.y += cy;
            vb.z += cz;
            wb = -d * 0.5f * (v.x * v.x + v.y * v.y + v.z * v.z) / (wi * wi);
        }
    }
    const float fu = F.x * ux + F.y * uy + F.z * uz;
    double hb = (double)(0.5f * wi * fu);
    wbar[i] += wb + 0.5f * h * fu;
    const float4 pv = p_prev[i];
    hb += (double)(pv.x * xb.x + pv.y * xb.y + pv.z * xb.z);
    vb.x = fmaf(h, xb.x, vb.x);
    vb.y = fmaf(h, xb.y, vb.y);
    vb.z = fmaf(h, xb.z, vb.z);
    xbar[i] = xb;
    vbar[i] = vb;
    hbar[i] += hb;
}

// State 0: first half kick of step 0 and the Maxwell-Boltzmann draw v0 = sqrt(kT w) xi.
// (K_0 = kT/2 sum xi^2 depends on neither w nor dt.)
__global__ void k_bwd_final(int N, const long long* __restrict__ ffix, const int* __restrict__ iperm, float finv,
                            const float* __restrict__ w, const float* __restrict__ dt, const int* __restrict__ sid,
                            const float* __restrict__ xi, double kT, const float4* __restrict__ vbar,
                            float* __restrict__ wbar, double* __restrict__ hbar) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int s = sid[i];
    float h = dt[s];
    float wi = w[i];
    float3 F = load_force(ffix, N, iperm[i], finv);
    float4 vb = vbar[i];
    float fv = F.x * vb.x + F.y * vb.y + F.z * vb.z;
    hbar[i] += (double)(0.5f * wi * fv);
    float wb = 0.5f * h * fv;
    if (wi > 0.f) {
        float s0 = sqrtf((float)kT * wi);
        float v0x = s0 * xi[3 * (size_t)i], v0y = s0 * xi[3 * (size_t)i + 1], v0z = s0 * xi[3 * (size_t)i + 2];
        wb += (vb.x * v0x + vb.y * v0y + vb.z * v0z) / (2.f * wi);
    }
    wbar[i] += wb;
}

__global__ void __launch_bounds__(kRedThreads) k_bwd_reduce_h(const SysDev* __restrict__ sys,
                                                               const double* __restrict__ hbar,
                                                               double* __restrict__ g_dt) {
    pdl_wait();
    __shared__ double sm[kRedThreads / 32];
    int s = blockIdx.x;
    const SysDev& S = sys[s];
    double t = 0.0;
    for (int k = S.atom_off + threadIdx.x; k < S.atom_off + S.n_atoms; k += kRedThreads) t += hbar[k];
    t = block_sum(t, sm);
    if (threadIdx.x == 0) g_dt[s] += t;
}

// ------------------------------------------------------------------ launchers

void launch_reduce_energy(nb_handle* h, int terms, int with_kin, double* dst, cudaStream_t st, const StepStat& ss,
                          bool precise) {
    launch_pdl(k_reduce_energy, h->n_red_blocks, kRedThreads, 0, st, h->n_sys, h->red_blk_sys, h->red_blk_off, h->sys,
                                                            h->e_atom, precise ? (const float4*)h->e_lo : nullptr,
                                                            h->xs, h->ke_atom, with_kin, h->red_part,
                                                            h->e_pme_blk, h->conv_blk_off, terms, h->red_ticket, dst,
                                                            ss);
}

void launch_finalize_forces(nb_handle* h, float* f_out, cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_finalize, cdiv(N, 256), 256, 0, st, N, h->ffix, h->iperm, h->finv, f_out);
}

void launch_integrate(nb_handle* h, float4* xq, float4* v, const float* w_ovr, const float* dt, float c_pre,
                      float c_post, int drift, float4* ck_x, float4* ck_v, float4* ck_p, cudaStream_t st,
                      const StepObs& ob, bool load_next) {
    int N = h->n_atoms;
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
    launch_pdl(k_integrate, cdiv(N, 256), 256, 0, st, N, xq, v, w_ovr, dt, h->sid, h->ffix, h->iperm, h->finv, c_pre, c_post,
                                              drift, h->ke_atom, ck_x, ck_v, ck_p, h->sys, ob, ln);
}

void launch_hmc_init(nb_handle* h, const float* w, const float* xi, double kT, cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_hmc_init, cdiv(N, 256), 256, 0, st, N, w, xi, kT, h->vwork, h->ke_atom);
}

void launch_hmc_finish(nb_handle* h, float4* x_out, const float4* x0, double kT, const double* u, double* stats,
                       cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_hmc_jump, cdiv(N, 256), 256, 0, st, N, x_out, x0, h->sid, h->sys, h->jump_atom);
    launch_pdl(k_hmc_accept, h->n_sys, kRedThreads, 0, st, h->sys, h->jump_atom, h->e0, h->e1, kT, u, stats);
    launch_pdl(k_hmc_restore, cdiv(N, 256), 256, 0, st, N, x_out, x0, h->sid, stats);
}

void launch_hmc_pick(nb_handle* h, float4* x_out, const float4* x0, const int* l_prop, int n_leap,
                     const double* step_stats, const double* u, double* stats, cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_hmc_pick, cdiv(h->n_sys, 128), 128, 0, st, h->n_sys, l_prop, n_leap, step_stats, u, stats, h->flags + 1);
    launch_pdl(k_hmc_restore, cdiv(N, 256), 256, 0, st, N, x_out, x0, h->sid, stats);
}

void launch_bwd_lambda(nb_handle* h, const float* w, const float* dt, const float4* v_state, const Inject& inj,
                       double kT, cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_bwd_lambda, cdiv(N, 256), 256, 0, st, N, h->vbar, v_state, w, dt, h->sid, h->iperm, inj, kT, h->lam);
}

void launch_bwd_adjoint(nb_handle* h, const float* w, const float* dt, const float4* x_state, const float4* v_state,
                        const float4* x0, const Inject& inj, double kT, const float4* p_prev, float* wbar,
                        cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_bwd_adjoint, cdiv(N, 256), 256, 0, st, N, h->gx_s, h->ffix, h->iperm, h->finv, w, dt, h->sid, h->sys, inj,
                                                kT, x_state, v_state, x0, p_prev, h->xbar, h->vbar, wbar,
                                                h->hbar_atom);
}

void launch_bwd_final(nb_handle* h, const float* w, const float* dt, const float* xi, double kT, float* wbar,
                      double* g_dt, cudaStream_t st) {
    int N = h->n_atoms;
    launch_pdl(k_bwd_final, cdiv(N, 256), 256, 0, st, N, h->ffix, h->iperm, h->finv, w, dt, h->sid, xi, kT, h->vbar, wbar,
                                              h->hbar_atom);
    launch_pdl(k_bwd_reduce_h, h->n_sys, kRedThreads, 0, st, h->sys, h->hbar_atom, g_dt);
}

}  // namespace nb
