// reduce.cuh -- the per-system FP64 energy reduction shared by k_reduce_energy
// (dynamics.cu) and the force-evaluation epilogue k_epilogue (pair.cu).
//
// Each block sums the atoms of one tile of one system (red_tile atoms, slot order; the
// tile depends only on the system's size, so a system sums in the same order batched or
// alone) into six FP64 partials and stores them; the last block to finish (a ticket counter
// behind a fence) adds, per system and in block order, the partials and the PME block
// energies, one warp per (system, component), and one thread per system writes the results.
// Every order is fixed, so the energies are bitwise reproducible; the last block resets the
// counter, so the kernels replay in a graph.
#pragma once
#include "common.cuh"

namespace nb {

constexpr int kRedThreads = 256;
constexpr int kRedComp = 6;  // LJ, direct, exclusion, q^2, kinetic, jump

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sums of v[0..7] over the warp, transposed: lanes exchange half of their values at each of
// the first three steps (xor 16, 8, 4), so 9 additions replace 8 separate trees of 5.  Lane
// l ends with the sum of component (l >> 2) & 7.
__device__ __forceinline__ double warp_sum8_d(const double v[8]) {
    const int lane = threadIdx.x & 31;
    double w[4], u[2];
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const double keep = h4 ? v[4 + j] : v[j], give = h4 ? v[j] : v[4 + j];
        w[j] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const double keep = h3 ? w[2 + j] : w[j], give = h3 ? w[j] : w[2 + j];
        u[j] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
    }
    const double keep = h2 ? u[1] : u[0], give = h2 ? u[0] : u[1];
    double t = keep + __shfl_xor_sync(0xffffffffu, give, 4);
    t += __shfl_xor_sync(0xffffffffu, t, 2);
    t += __shfl_xor_sync(0xffffffffu, t, 1);
    return t;
}

// Atoms [a0, a1) of block b's tile (its system s = blk_sys[b]).
__device__ __forceinline__ void red_tile_range(const int* __restrict__ blk_sys, const int* __restrict__ blk_off,
                                               const SysDev* __restrict__ sys, int& a0, int& a1) {
    const int b = blockIdx.x;
    const int s = blk_sys[b];
    const SysDev& S = sys[s];
    a0 = S.atom_off + (b - blk_off[s]) * S.red_tile;
    a1 = min(a0 + S.red_tile, S.atom_off + S.n_atoms);
}

// The rest of the reduction once each thread holds, in v[0..5], its sums over its atoms of
// the block's tile (LJ, direct, exclusion and kinetic energies, sum q^2, jump).  Called by
// every thread of a kRedThreads block.
__device__ __forceinline__ void energy_reduce_finish(const double (&v)[8], int n_sys, const int* __restrict__ blk_off,
                                                     const SysDev* __restrict__ sys, int with_kin,
                                                     double* __restrict__ part, const double* __restrict__ e_pme_blk,
                                                     const int* __restrict__ pme_blk_off, int terms,
                                                     unsigned* __restrict__ ticket, double* __restrict__ dst,
                                                     const StepStat& ss) {
    constexpr int kW = kRedThreads / 32;
    constexpr int kC = kRedComp;
    __shared__ double sm[kW][kC];
    __shared__ bool last;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    {
        const int b = blockIdx.x;
        const double t = warp_sum8_d(v);
        const int c = lane >> 2;
        if ((lane & 3) == 0 && c < kC) sm[w][c] = t;
        __syncthreads();
        if (threadIdx.x < kC) {
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < kW; ++k) acc += sm[k][threadIdx.x];
            part[(size_t)b * kC + threadIdx.x] = acc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            last = atomicAdd(ticket, 1u) == gridDim.x - 1;
        }
        __syncthreads();
    }
    if (!last) return;
    __threadfence();
    // per (system, component): component kC is the reciprocal energy from the PME blocks;
    // the totals go to part[] past the block partials
    double* tot = part + (size_t)gridDim.x * kC;
    for (int sc = w; sc < n_sys * (kC + 1); sc += kW) {
        const int s = sc / (kC + 1), c = sc % (kC + 1);
        double acc = 0.0;
        if (c < kC) {
            for (int b = blk_off[s] + lane; b < blk_off[s + 1]; b += 32) acc += __ldcg(part + (size_t)b * kC + c);
        } else if ((terms & NB_TERM_PME) && sys[s].pme && pme_blk_off) {
            for (int b = pme_blk_off[s] + lane; b < pme_blk_off[s + 1]; b += 32) acc += e_pme_blk[b];
        }
        acc = warp_sum_d(acc);
        if (lane == 0) tot[sc] = acc;
    }
    __syncthreads();
    for (int s = threadIdx.x; s < n_sys; s += kRedThreads) {
        const SysDev& S = sys[s];
        const double* acc = tot + (size_t)s * (kC + 1);
        const bool coul = (terms & NB_TERM_COUL) != 0;
        double e[NB_NE];
        e[NB_E_LJ] = (terms & NB_TERM_LJ) ? acc[0] : 0.0;
        e[NB_E_DIR] = coul ? acc[1] : 0.0;
        e[NB_E_EXCL] = coul ? acc[2] : 0.0;
        e[NB_E_SELF] = coul ? S.self_coef * acc[3] : 0.0;
        e[NB_E_REC] = acc[kC];
        e[NB_E_KIN] = with_kin ? acc[4] : 0.0;
        double* o = dst + (size_t)s * NB_NE;
#pragma unroll
        for (int c = 0; c < NB_NE; ++c) o[c] = e[c];
        if (ss.sstat) {
            double H0 = 0.0, H1 = 0.0;
            for (int c = 0; c < NB_NE; ++c) {
                H0 += ss.e_ref[(size_t)s * NB_NE + c];
                H1 += e[c];
            }
            const double dH = H1 - H0;
            double a = (dH <= 0.0) ? 1.0 : exp(-dH / ss.kT);
            if (!(dH == dH)) a = 0.0;  // NaN energy: never accepted
            double* q = ss.sstat + (size_t)s * 3;
            q[0] = dH;
            q[1] = a;
            q[2] = acc[5];
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

}  // namespace nb
