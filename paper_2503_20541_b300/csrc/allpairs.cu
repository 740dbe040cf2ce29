// allpairs.cu -- O(N^2) all-pairs Lennard-Jones forces, the comparison baseline of the
// linear cell-list path (Sec. 3 compares the neighbour-list path against all-pairs
// evaluation): every pair (i, j != i) of a system under the minimum image, no list.
//
// One thread per atom i (caller order) walks all atoms of its system in tiles of
// kApTile staged in shared memory, in a fixed order, so the FP32 sums are reproducible.
// The force goes to the int64 fixed-point slot array and the half energy to the
// per-atom energy array, so the handle's finalisation and FP64 reduction apply.
#include "common.cuh"
#include "lj.cuh"

namespace nb {

constexpr int kApTile = 128;

__global__ void __launch_bounds__(kApTile) k_allpairs_lj(int N, int a0, int n, const SysDev* __restrict__ sysp,
                                                         const float4* __restrict__ xq,
                                                         const float2* __restrict__ params,
                                                         const int* __restrict__ iperm,
                                                         long long* __restrict__ ffix, float4* __restrict__ e_atom,
                                                         float scale, unsigned* flags) {
    __shared__ float4 tx[kApTile];
    __shared__ float2 tp[kApTile];
    const SysDev& S = *sysp;
    const PairK K = pair_k(S);
    const float L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const float i0 = S.invL[0], i1 = S.invL[1], i2 = S.invL[2];
    const bool per = S.periodic != 0;
    const int ii = blockIdx.x * kApTile + threadIdx.x;
    const bool valid = ii < n;
    const int i = a0 + (valid ? ii : 0);
    const float4 xi = xq[i];
    const float2 pi = params[i];
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f;
    for (int j0 = 0; j0 < n; j0 += kApTile) {
        __syncthreads();
        if (j0 + threadIdx.x < n) {
            tx[threadIdx.x] = xq[a0 + j0 + threadIdx.x];
            tp[threadIdx.x] = params[a0 + j0 + threadIdx.x];
        }
        __syncthreads();
        const int m = min(kApTile, n - j0);
        for (int jj = 0; jj < m; ++jj) {
            const float4 xj = tx[jj];
            float dx = xi.x - xj.x, dy = xi.y - xj.y, dz = xi.z - xj.z;
            if (per) {
                dx = mi_any(dx, L0, i0);
                dy = mi_any(dy, L1, i1);
                dz = mi_any(dz, L2, i2);
            }
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < K.rc2 && j0 + jj != ii) {
                const float2 pj = tp[jj];
                const float rinv = rsqrtf(r2);
                const float r2inv = recip_r2(r2, rinv);
                const float eps = pi.y * pj.y;
                const float eps_lo = fmaf(pi.y, pj.y, -eps);
                float u, f;
                lj_unit(0.5f * (pi.x + pj.x), r2inv, rinv, r2, K, u, f);
                elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
                const float fr = fmaf(eps_lo, f, eps * f);
                fx = fmaf(fr, dx, fx);
                fy = fmaf(fr, dy, fy);
                fz = fmaf(fr, dz, fz);
            }
        }
    }
    if (valid) {
        const int k = iperm[i];
        ffix[k] = to_fix(fx, scale, flags + 1);
        ffix[(size_t)N + k] = to_fix(fy, scale, flags + 1);
        ffix[2 * (size_t)N + k] = to_fix(fz, scale, flags + 1);
        e_atom[k] = make_float4(0.5f * elj, 0.f, 0.f, 0.f);
    }
}

void launch_allpairs_lj(nb_handle* h, const float4* xq, cudaStream_t st) {
    for (int s = 0; s < h->n_sys; ++s) {
        const SysDev& D = h->sys_h[s];
        if (D.n_atoms == 0) continue;
        k_allpairs_lj<<<cdiv(D.n_atoms, kApTile), kApTile, 0, st>>>(h->n_atoms, D.atom_off, D.n_atoms, h->sys + s, xq,
                                                                     h->params, h->iperm, h->ffix, h->e_atom,
                                                                     h->fscale, h->flags);
    }
}

}  // namespace nb
