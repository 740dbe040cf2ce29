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
// Work decomposition: one block per cell (the cell tile of cell.cuh) stages the
// positions, charges and LJ parameters of the cell's stencil in shared memory with the
// build's images applied; one warp per atom of the cell walks its full neighbour list
// (both directions of every pair are listed; entries are 16-bit stencil indices), tests
// r < r_c on 32 entries at a time and appends the pairs inside r_c to a per-warp queue,
// and the interaction math runs on full warps of queued pairs.  i's data stays in
// registers, partial sums are reduced with warp shuffles in a fixed tree, and the force
// on i is added once, as int64 fixed point, to the zeroed force array (the PME gather
// adds its part concurrently; integer addition makes the order irrelevant).  Every
// FP32 summation order is fixed by the list, so results are bitwise reproducible.
#include "cell.cuh"
#include "lj.cuh"

namespace nb {

constexpr int kPairWarps = 8;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kVjpWarps = 8;
constexpr int kVjpThreads = kVjpWarps * 32;
constexpr int kQueue = 64;  // per-warp queue of pairs inside r_c

// Exclusion partners of slot i: count and the slot of partner e (from the per-slot
// table when it holds all of them, else from the CSR).
struct ExclView {
    int ew;  // table width (0: no exclusions in the handle)
    const int* slot;
    const int* cnt;
    const int* perm;
    const int* iperm;
    const int* off;
    const int* idx;
    __device__ __forceinline__ int count(int i) const { return ew ? cnt[i] : 0; }
    __device__ __forceinline__ int partner(int i, int e) const {
        if (e < ew) return slot[(size_t)i * ew + e];
        return iperm[idx[off[perm[i]] + e]];
    }
};

// Stage the candidates of stencil tile [t0, t1): positions (image applied, q in .w), LJ
// parameters, optionally cotangents, and per-pair image flags.
__device__ __forceinline__ void stage_pair_tile(const CellCtx& C, const BuildRun* runs, int nr, int t0, int t1,
                                                int nthreads, const float4* __restrict__ xs,
                                                const float2* __restrict__ ps, const float4* __restrict__ lam,
                                                float4* cand, float2* par, float4* lamc, unsigned char* cflag) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = nthreads >> 5;
    for (int r = w; r < nr; r += nw) {
        const int sm0 = runs[r].sm0, slot0 = runs[r].slot0;
        const int a = max(sm0, t0), b = min(sm0 + runs[r].n, t1);
        for (int k = a + lane; k < b; k += 32) {
            const int j = slot0 + (k - sm0);
            cp_async16(&cand[k - t0], &xs[j]);
            cp_async8(&par[k - t0], &ps[j]);
            if (lamc) cp_async16(&lamc[k - t0], &lam[j]);
        }
    }
    cp_async_wait_all();
    for (int r = w; r < nr; r += nw) {
        const BuildRun R = runs[r];
        const int a = max(R.sm0, t0), b = min(R.sm0 + R.n, t1);
        for (int k = a + lane; k < b; k += 32) {
            const float4 p = cand[k - t0];
            cand[k - t0] = make_float4(p.x + R.s[0], p.y + R.s[1], p.z + R.s[2], p.w);
            if (C.gen) cflag[k - t0] = (unsigned char)R.flags;
        }
    }
}

// Difference x_i - x_j of atom i (frame-shifted coordinates a, raw coordinates xr) and
// staged candidate cj.
template <bool GEN>
__device__ __forceinline__ void cell_diff(const CellCtx& C, float ax, float ay, float az, const float4& xr,
                                          const float4& cj, int fl, float& dx, float& dy, float& dz) {
    if (GEN) {
        dx = gen_diff(xr.x, cj.x, fl, 1, C.fold[0], C.L[0], C.hL[0]);
        dy = gen_diff(xr.y, cj.y, fl, 2, C.fold[1], C.L[1], C.hL[1]);
        dz = gen_diff(xr.z, cj.z, fl, 4, C.fold[2], C.L[2], C.hL[2]);
    } else {
        dx = ax - cj.x;
        dy = ay - cj.y;
        dz = az - cj.z;
    }
}

__device__ __forceinline__ void pair_vec(const float4& a, const float4& b, int per, const CellCtx& C, float& dx,
                                         float& dy, float& dz) {
    if (per) {
        dx = mi_pair(a.x, b.x, C.L[0], C.hL[0]);
        dy = mi_pair(a.y, b.y, C.L[1], C.hL[1]);
        dz = mi_pair(a.z, b.z, C.L[2], C.hL[2]);
    } else {
        dx = a.x - b.x;
        dy = a.y - b.y;
        dz = a.z - b.z;
    }
}

// One queued pair of the force kernel: (dx, dy, dz, q_j) and stencil index lq (r^2 is
// recomputed with the operations of the cut-off test, so it is the same value).
template <bool LJ, int COUL>
__device__ __forceinline__ void pair_heavy(const float4& q, int lq, const float2& pi, bool do_lj, const PairK& K,
                                           const float4* cand, const float2* par, float qke, float qke_lo,
                                           float alpha, float gau_c, float& fx, float& fy, float& fz, float& elj,
                                           float& edir) {
    const float r2 = fmaf(q.z, q.z, fmaf(q.y, q.y, q.x * q.x));
    const float rinv = rsqrtf(r2);
    float fr = 0.f;
    if (LJ && do_lj) {
        const float2 pj = par[lq];
        const float r2inv = __frcp_rn(r2);  // correctly rounded: LJ raises it to the 6th power
        const float eps = pi.y * pj.y;      // eps_ij = eps + eps_lo exactly
        const float eps_lo = fmaf(pi.y, pj.y, -eps);
        float u, f;
        lj_unit(0.5f * (pi.x + pj.x), r2inv, rinv, r2, K, u, f);
        elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
        fr = fmaf(eps_lo, f, eps * f);
    }
    if (COUL == kCoulEwald && K.ke != 0.f) {  // block-uniform: uncharged systems of a mixed batch skip it
        const float r = r2 * rinv;
        const float qq = qke * q.w;
        const float ar = alpha * r;
        const float ec = erfcf(ar);
        const float gau = gau_c * __expf(-ar * ar);
        // the energy is summed per unit ke q_i (q_j erfc(alpha r)/r) and scaled once per
        // atom: ke q_i q_j, rounded alike for every pair of two atom types, would make its
        // rounding add linearly over a sum that cancels ~10^3-fold
        edir = fmaf(q.w * ec, rinv, edir);
        fr = fmaf(qq * fmaf(ec, rinv, gau), rinv * rinv, fr);
    }
    if (COUL == kCoulRF && K.ke != 0.f) {  // Eq. RFA: qq (1/r + k r^2 - c), f = qq (1/r^3 - 2k)
        // The pair energies of water cancel ~10^4-fold in the sum, so a rounding shared by
        // many pairs would dominate its error: ke q_i q_j (two charge values, every pair of a
        // type pair rounded alike) is carried as hi + lo, and so are k and c.
        const float qj_ = q.w;
        const float qq = qke * qj_;
        const float qq_lo = fmaf(qke_lo, qj_, fmaf(qke, qj_, -qq));
        const float u = fmaf(K.krf, r2, rinv - K.crf) + fmaf(K.krf_lo, r2, -K.crf_lo);
        edir = fmaf(qq, u, fmaf(qq_lo, u, edir));
        fr = fmaf(qq, fmaf(rinv * rinv, rinv, -2.f * K.krf), fr);
    }
    fx = fmaf(fr, q.x, fx);
    fy = fmaf(fr, q.y, fy);
    fz = fmaf(fr, q.z, fz);
}

// Predicated shared-memory stores of a queue entry: the append stays inside the round's
// basic block (no branch around it), so consecutive rounds interleave.
__device__ __forceinline__ void sts_q_if(float4* qd, int* qj, float4 v, int j, bool ok) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(qd);
    const unsigned b = (unsigned)__cvta_generic_to_shared(qj);
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.u32 q, %6, 0;\n @q st.shared.v4.f32 [%0], {%2, %3, %4, %5};\n"
        " @q st.shared.u32 [%1], %7;\n}\n" ::"r"(a),
        "r"(b), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"((unsigned)ok), "r"(j)
        : "memory");
}

// Stencil index of slot j (-1 when j is outside the cell's stencil), found by all lanes
// of the warp testing the runs (uniform j).
__device__ __forceinline__ int stencil_index(const BuildRun* runs, int nr, int j) {
    const int lane = threadIdx.x & 31;
    int li = -1;
    for (int r0 = 0; r0 < nr; r0 += 32) {
        const int r = r0 + lane;
        bool hit = false;
        int k = 0;
        if (r < nr) {
            const BuildRun& R = runs[r];
            hit = j >= R.slot0 && j < R.slot0 + R.n;
            k = R.sm0 + (j - R.slot0);
        }
        const unsigned b = __ballot_sync(0xffffffffu, hit);
        if (b) {
            li = __shfl_sync(0xffffffffu, k, __ffs(b) - 1);
            break;
        }
    }
    return li;
}

// Header of an atom: everything its list walk needs first, loaded one atom ahead.
struct AtomHdr {
    float4 xr;   // position (frame of the last build) and charge
    float2 pi;   // sigma, sqrt(eps)
    int c;       // list length
    uint2 g;     // this lane's four entries of the first 128-entry list group
    uint2 g2;    // ... and of the second (rows of at least 256 entries)
    int ej;      // lane q < table width: slot of exclusion partner q (-1: none)
    int ne;      // number of exclusion partners
};

__device__ __forceinline__ AtomHdr load_hdr(int i, const float4* __restrict__ xs, const float2* __restrict__ ps,
                                            const unsigned short* __restrict__ nbr, const int* __restrict__ cnt,
                                            int cap, const ExclView& X, bool want_excl) {
    const int lane = threadIdx.x & 31;
    AtomHdr H;
    H.xr = xs[i];
    H.pi = ps[i];
    H.c = cnt[i];
    const uint2* row2 = reinterpret_cast<const uint2*>(nbr + (size_t)i * cap);
    // rows hold a multiple of 128 entries, so whole 128-entry groups stay inside the row
    H.g = row2[lane];
    H.g2 = cap >= 256 ? row2[32 + lane] : make_uint2(0u, 0u);  // used only when c > 128
    H.ne = (want_excl && X.ew) ? X.cnt[i] : 0;
    H.ej = (want_excl && lane < X.ew) ? X.slot[(size_t)i * X.ew + lane] : -1;
    return H;
}

// Forces and half energies of atom i over stencil tile [t0, t1) (one warp).
template <bool LJ, int COUL, bool GEN, bool MULTI>
__device__ __forceinline__ void pair_atom(const CellCtx& C, const PairK& K, int N, int i, const AtomHdr& H, int t0,
                                          int t1, bool last, const BuildRun* runs, int nr,
                                          const float4* cand, const float2* par, const unsigned char* cflag,
                                          float4* qd, int* qj, const float4* __restrict__ xs,
                                          const unsigned short* __restrict__ nbr, int cap, const ExclView& X,
                                          long long* __restrict__ ffix, float4* __restrict__ e_atom,
                                          float4* __restrict__ pscr, float scale, unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const float4 xr = H.xr;
    const float ax = xr.x + C.fs[0], ay = xr.y + C.fs[1], az = xr.z + C.fs[2];
    const float2 pi = H.pi;
    const int c = H.c;
    const uint2* row2 = reinterpret_cast<const uint2*>(nbr + (size_t)i * cap);
    const float rc2 = K.rc2;
    const float qke = K.ke * xr.w;
    const float qke_lo = COUL == kCoulRF ? fmaf(K.ke, xr.w, -qke) : 0.f;  // ke q_i = qke + qke_lo exactly
    const float alpha = K.alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    const bool do_lj = pi.y != 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    // pairs inside r_c wait in a 64-entry ring and are evaluated 32 at a time
    int head = 0, nq = 0;
    // the list is read in groups of 128 entries: lane l holds entries 4l..4l+3 of a group
    // (one 8-byte load); groups are loaded two ahead of the one being tested
    uint2 ga = H.g, gb = H.g2;
    for (int g0 = 0; g0 < c; g0 += 128) {
        const uint2 gc = ga;
        ga = gb;
        if (g0 + 256 < c) gb = row2[(g0 + 256) / 4 + lane];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = g0 + 4 * lane + t;
            const unsigned wv = t < 2 ? gc.x : gc.y;
            const int li = (t & 1) ? (int)(wv >> 16) : (int)(wv & 0xffffu);
            const bool in = k < c && (!MULTI || (li >= t0 && li < t1));
            const int lk = in ? li - t0 : 0;  // entries outside the tile read candidate 0, unused
            const float4 cj = cand[lk];
            float dx, dy, dz;
            cell_diff<GEN>(C, ax, ay, az, xr, cj, GEN ? cflag[lk] : 0, dx, dy, dz);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const bool acc = in && r2 < rc2;
            const unsigned bits = __ballot_sync(0xffffffffu, acc);
            const int pos = (head + nq + __popc(bits & lt)) & (kQueue - 1);
            sts_q_if(qd + pos, qj + pos, make_float4(dx, dy, dz, cj.w), lk, acc);
            nq += __popc(bits);
            if (nq >= 32) {
                __syncwarp();
                const int pos = (head + lane) & (kQueue - 1);
                const float4 q = qd[pos];
                const int lq = qj[pos];
                __syncwarp();
                pair_heavy<LJ, COUL>(q, lq, pi, do_lj, K, cand, par, qke, qke_lo, alpha, gau_c, fx, fy, fz, elj,
                                     edir);
                head = (head + 32) & (kQueue - 1);
                nq -= 32;
            }
        }
    }
    __syncwarp();
    if (lane < nq) {
        const int pos = (head + lane) & (kQueue - 1);
        pair_heavy<LJ, COUL>(qd[pos], qj[pos], pi, do_lj, K, cand, par, qke, qke_lo, alpha, gau_c, fx, fy, fz, elj,
                             edir);
    }
    __syncwarp();
    if (COUL == kCoulEwald && last && alpha > 0.f && H.ne > 0) {
        // exclusion correction for i's excluded partners (at any distance); a partner in
        // the staged stencil is read from shared memory with its image, others from xs
        const int ne = H.ne;
        int lk = -1;
        const int nin = min(ne, X.ew);
        for (int q = 0; q < nin; ++q) {
            const int jq = __shfl_sync(0xffffffffu, H.ej, q);
            const int k = stencil_index(runs, nr, jq);
            if (lane == q) lk = k;
        }
        for (int e = lane; e < ne; e += 32) {
            float dx, dy, dz, qj_;
            if (e < 32 && lk >= t0 && lk < t1) {
                const float4 cj = cand[lk - t0];
                cell_diff<GEN>(C, ax, ay, az, xr, cj, GEN ? cflag[lk - t0] : 0, dx, dy, dz);
                qj_ = cj.w;
            } else {
                const int j = e < 32 && e < X.ew ? H.ej : X.partner(i, e);
                const float4 xj = xs[j];
                pair_vec(xr, xj, C.per, C, dx, dy, dz);
                qj_ = xj.w;
            }
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rinv = rsqrtf(r2);
            const float r2inv = rinv * rinv;
            const float r = r2 * rinv;
            const float qq = qke * qj_;
            const float ar = alpha * r;
            const float ef = erff(ar);
            const float gau = gau_c * __expf(-ar * ar);
            eex = fmaf(-qj_ * ef, rinv, eex);  // per unit ke q_i, as edir
            const float fr = qq * (gau - ef * rinv) * r2inv;
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
        if (MULTI) {  // stencil in several tiles: partial sums carried in tile order
            float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
            if (t0 > 0) {
                a = pscr[3 * (size_t)i];
                b = pscr[3 * (size_t)i + 1];
            }
            fx += a.x;
            fy += a.y;
            fz += a.z;
            elj += a.w;
            edir += b.x;
            eex += b.y;
            if (!last) {
                pscr[3 * (size_t)i] = make_float4(fx, fy, fz, elj);
                pscr[3 * (size_t)i + 1] = make_float4(edir, eex, 0.f, 0.f);
            }
        }
        if (last) {
            // added (ffix is zeroed per evaluation): the PME gather adds concurrently
            red_add(ffix + i, to_fix(fx, scale, flags + 1));
            red_add(ffix + (size_t)N + i, to_fix(fy, scale, flags + 1));
            red_add(ffix + 2 * (size_t)N + i, to_fix(fz, scale, flags + 1));
            if (COUL == kCoulEwald) {  // ke q_i = qke + (ke q_i - qke) exactly: one rounding per atom
                const float lo = fmaf(K.ke, xr.w, -qke);
                edir = fmaf(qke, edir, lo * edir);
                eex = fmaf(qke, eex, lo * eex);
            }
            e_atom[i] = make_float4(0.5f * elj, 0.5f * edir, 0.5f * eex, 0.f);
        }
    }
}

template <bool LJ, int COUL>
__global__ void __launch_bounds__(kPairThreads) k_pair_cell(
    int N, int cap, int tile, const int* __restrict__ cell_sys, const SysDev* __restrict__ sys,
    const int* __restrict__ start, const float4* __restrict__ xs, const float2* __restrict__ ps,
    const unsigned short* __restrict__ nbr, const int* __restrict__ cnt, ExclView X, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float4* __restrict__ pscr, float scale, unsigned* flags, int split) {
    pdl_wait();
    // `split` blocks share a cell: block `part` takes atoms i0 + part*kPairWarps + w + stride*m
    const int c = blockIdx.x / split, part = blockIdx.x % split;
    const int stride = kPairWarps * split;
    const SysDev& S = sys[cell_sys[c]];
    const CellCtx C = cell_ctx(c, S, start);
    const PairK K = pair_k(S);
    const int ib = C.i0 + part * kPairWarps + (threadIdx.x >> 5);
    if (C.i0 + part * kPairWarps >= C.i1) return;
    __shared__ BuildRun runs[kMaxRuns];
    __shared__ int n_runs, n_cand;
    __shared__ float4 qd_all[kPairWarps][kQueue];
    __shared__ int qj_all[kPairWarps][kQueue];
    extern __shared__ float4 smem[];
    float4* cand = smem;
    float2* par = reinterpret_cast<float2*>(cand + tile);
    unsigned char* cflag = reinterpret_cast<unsigned char*>(par + tile);
    const int w = threadIdx.x >> 5;
    const bool want_excl = COUL == kCoulEwald && K.alpha > 0.f;
    // the first atom's header is loaded while the stencil is staged
    AtomHdr hn;
    if (ib < C.i1) hn = load_hdr(ib, xs, ps, nbr, cnt, cap, X, want_excl);
    if (w == 0) cell_runs(C, S, start, runs, &n_runs, &n_cand, flags);
    __syncthreads();
    const int nr = n_runs, total = n_cand;
    if (total > 65536) return;  // the build has flagged the overflow
    const bool multi = total > tile;
    for (int t0 = 0; t0 < total; t0 += tile) {
        const int t1 = min(total, t0 + tile);
        stage_pair_tile(C, runs, nr, t0, t1, kPairThreads, xs, ps, nullptr, cand, par, nullptr, cflag);
        __syncthreads();
        const bool last = t1 == total;
        if (t0 > 0 && ib < C.i1) hn = load_hdr(ib, xs, ps, nbr, cnt, cap, X, want_excl);
        for (int i = ib; i < C.i1; i += stride) {
            const AtomHdr H = hn;
            if (i + stride < C.i1) hn = load_hdr(i + stride, xs, ps, nbr, cnt, cap, X, want_excl);
#define NB_PAIR_ARGS C, K, N, i, H, t0, t1, last, runs, nr, cand, par, cflag, qd_all[w], qj_all[w], xs, nbr, cap, X, \
                     ffix, e_atom, pscr, scale, flags
            if (multi) {
                if (C.gen) pair_atom<LJ, COUL, true, true>(NB_PAIR_ARGS);
                else pair_atom<LJ, COUL, false, true>(NB_PAIR_ARGS);
            } else {
                if (C.gen) pair_atom<LJ, COUL, true, false>(NB_PAIR_ARGS);
                else pair_atom<LJ, COUL, false, false>(NB_PAIR_ARGS);
            }
#undef NB_PAIR_ARGS
        }
        if (!last) __syncthreads();
    }
}

// Force VJP.  For each directed pair (i, j) with u = lam_i - lam_j and du = d.u:
//   gx_i += f u + (f'/r) du d           (J (lam_i - lam_j), J = f I + (f'/r) d d^T)
//   gq_i += ke q_j (f / qq) du,  gsig_i += 1/2 (df/dsigma_ij) du,  ge_i += sqrt(eps_j) (f/eps) du
// and the forces F_i as in k_pair_cell.  The exclusion correction contributes the same way.
struct VjpAcc {
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f, gq = 0.f, gs = 0.f, ge = 0.f;
};

template <bool LJ, int COUL>
__device__ __forceinline__ void vjp_heavy(const float4& q, const float4& lj4, const float2& pj,
                                          const float4& li, const float2& pi, float qi, const PairK& K,
                                          float alpha, float a2, float gau_c, VjpAcc& A) {
    // q = (dx, dy, dz, q_j); r^2 with the operations of the cut-off test (the same value)
    const float dx = q.x, dy = q.y, dz = q.z, r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
    const float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
    const float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
    const float rinv = rsqrtf(r2);
    const float r2inv = __frcp_rn(r2);
    float fr = 0.f, fpr = 0.f;  // f and f'/r
    if (LJ) {
        const float eps = pi.y * pj.y;
        const float sig = 0.5f * (pi.x + pj.x);
        const float s2 = sig2_over_r2(sig, r2inv);
        const float s6 = s2 * s2 * s2, s12 = s6 * s6;
        float u = 4.f * (s12 - s6);  // per unit eps
        float f = 24.f * (2.f * s12 - s6) * r2inv;
        float fp = -24.f * (28.f * s12 - 8.f * s6) * r2inv * r2inv;
        const float sinv = sig > 0.f ? 1.f / sig : 0.f;
        const float us = 4.f * (12.f * s12 - 6.f * s6) * sinv;           // du/dsigma
        float fs = 24.f * (24.f * s12 - 6.f * s6) * r2inv * sinv;        // df/dsigma
        if (K.sw) {
            const float r = r2 * rinv;
            const float x = fmaxf(0.f, (r - K.rs) * K.inv_sw);  // S = 1, S' = S'' = 0 below r_s
            const float x2 = x * x, x3 = x2 * x;
            const float sw = 1.f + x3 * (-10.f + x * (15.f - 6.f * x));
            const float d1 = x2 * (-30.f + x * (60.f - 30.f * x)) * K.inv_sw;
            const float d2 = x * (-60.f + x * (180.f - 120.f * x)) * K.inv_sw * K.inv_sw;
            fp = fp * sw + 2.f * f * d1 * rinv - u * (d2 - d1 * rinv) * r2inv;
            fs = fs * sw - us * d1 * rinv;
            f = f * sw - u * d1 * rinv;
            u *= sw;
        }
        const float eps_lo = fmaf(pi.y, pj.y, -eps);
        A.elj = fmaf(eps, u, fmaf(eps_lo, u, A.elj));
        fr = fmaf(eps_lo, f, eps * f);
        fpr = eps * fp;
        A.ge = fmaf(pj.y * f, du, A.ge);
        A.gs = fmaf(0.5f * eps * fs, du, A.gs);
    }
    if (COUL == kCoulEwald && K.ke != 0.f) {  // block-uniform: uncharged systems of a mixed batch skip it
        const float r = r2 * rinv;
        const float qq = K.ke * qi * q.w;
        const float ar = alpha * r;
        const float ec = erfcf(ar);
        const float gau = gau_c * __expf(-ar * ar);
        const float fcu = fmaf(ec, rinv, gau) * r2inv;  // f per unit qq
        A.edir = fmaf(q.w * ec, rinv, A.edir);          // per unit ke q_i, as in the force kernel
        fr = fmaf(qq, fcu, fr);
        fpr = fmaf(-qq * r2inv, fmaf(3.f, fcu, 2.f * a2 * gau), fpr);
        A.gq = fmaf(K.ke * q.w * fcu, du, A.gq);
    }
    if (COUL == kCoulRF && K.ke != 0.f) {  // Eq. RFA: f = qq (r^-3 - 2k), f'/r = -3 qq r^-5
        const float qke = K.ke * qi;
        const float qq = qke * q.w;
        // energy with ke q_i q_j, k and c as double-float pairs, as in the force kernel
        const float qq_lo = fmaf(fmaf(K.ke, qi, -qke), q.w, fmaf(qke, q.w, -qq));
        const float r3inv = r2inv * rinv;
        const float fcu = r3inv - 2.f * K.krf;
        const float u = fmaf(K.krf, r2, rinv - K.crf) + fmaf(K.krf_lo, r2, -K.crf_lo);
        A.edir = fmaf(qq, u, fmaf(qq_lo, u, A.edir));
        fr = fmaf(qq, fcu, fr);
        fpr = fmaf(-3.f * qq, r3inv * r2inv, fpr);
        A.gq = fmaf(K.ke * q.w * fcu, du, A.gq);
    }
    const float k2 = fpr * du;
    A.gx = fmaf(fr, ux, fmaf(k2, dx, A.gx));
    A.gy = fmaf(fr, uy, fmaf(k2, dy, A.gy));
    A.gz = fmaf(fr, uz, fmaf(k2, dz, A.gz));
    A.fx = fmaf(fr, dx, A.fx);
    A.fy = fmaf(fr, dy, A.fy);
    A.fz = fmaf(fr, dz, A.fz);
}

template <bool LJ, int COUL, bool GEN, bool MULTI>
__device__ __forceinline__ void vjp_atom(const CellCtx& C, const PairK& K, int N, int i, const AtomHdr& H, int t0,
                                         int t1, bool last, const BuildRun* runs, int nr, const float4* cand,
                                         const float2* par, const float4* lamc, const unsigned char* cflag,
                                         float4* qd, int* qj, const float4* __restrict__ xs,
                                         const float4* __restrict__ lam, const unsigned short* __restrict__ nbr,
                                         int cap, const ExclView& X, float4* __restrict__ gx_s,
                                         float2* __restrict__ gp_s, long long* __restrict__ ffix,
                                         float4* __restrict__ e_atom, float4* __restrict__ pscr, float scale,
                                         unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    const float4 xr = H.xr;
    const float ax = xr.x + C.fs[0], ay = xr.y + C.fs[1], az = xr.z + C.fs[2];
    const float2 pi = H.pi;
    const float4 li = lam[i];
    const int c = H.c;
    const uint2* row2 = reinterpret_cast<const uint2*>(nbr + (size_t)i * cap);
    const float rc2 = K.rc2;
    const float alpha = K.alpha, a2 = alpha * alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    VjpAcc A;
    int head = 0, nq = 0;
    // the list is read in groups of 128 entries: lane l holds entries 4l..4l+3 of a group
    // (one 8-byte load); groups are loaded two ahead of the one being tested
    uint2 ga = H.g, gb = H.g2;
    for (int g0 = 0; g0 < c; g0 += 128) {
        const uint2 gc = ga;
        ga = gb;
        if (g0 + 256 < c) gb = row2[(g0 + 256) / 4 + lane];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int k = g0 + 4 * lane + t;
            const unsigned wv = t < 2 ? gc.x : gc.y;
            const int le = (t & 1) ? (int)(wv >> 16) : (int)(wv & 0xffffu);
            const bool in = k < c && (!MULTI || (le >= t0 && le < t1));
            const int lk = in ? le - t0 : 0;
            const float4 cj = cand[lk];
            float dx, dy, dz;
            cell_diff<GEN>(C, ax, ay, az, xr, cj, GEN ? cflag[lk] : 0, dx, dy, dz);
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const bool acc = in && r2 < rc2;
            const unsigned bits = __ballot_sync(0xffffffffu, acc);
            const int pos = (head + nq + __popc(bits & lt)) & (kQueue - 1);
            sts_q_if(qd + pos, qj + pos, make_float4(dx, dy, dz, cj.w), lk, acc);
            nq += __popc(bits);
            if (nq >= 32) {
                __syncwarp();
                const int p = (head + lane) & (kQueue - 1);
                const float4 q = qd[p];
                const int lq = qj[p];
                __syncwarp();
                vjp_heavy<LJ, COUL>(q, lamc[lq], par[lq], li, pi, xr.w, K, alpha, a2, gau_c, A);
                head = (head + 32) & (kQueue - 1);
                nq -= 32;
            }
        }
    }
    __syncwarp();
    if (lane < nq) {
        const int p = (head + lane) & (kQueue - 1);
        const int lq = qj[p];
        vjp_heavy<LJ, COUL>(qd[p], lamc[lq], par[lq], li, pi, xr.w, K, alpha, a2, gau_c, A);
    }
    __syncwarp();
    if (COUL == kCoulEwald && last && alpha > 0.f && H.ne > 0) {
        const int ne = H.ne;
        int lk = -1;
        const int nin = min(ne, X.ew);
        for (int q = 0; q < nin; ++q) {
            const int jq = __shfl_sync(0xffffffffu, H.ej, q);
            const int k = stencil_index(runs, nr, jq);
            if (lane == q) lk = k;
        }
        for (int e = lane; e < ne; e += 32) {
            float dx, dy, dz;
            float4 xj, lj4;
            if (e < 32 && lk >= t0 && lk < t1) {
                xj = cand[lk - t0];
                lj4 = lamc[lk - t0];
                cell_diff<GEN>(C, ax, ay, az, xr, xj, GEN ? cflag[lk - t0] : 0, dx, dy, dz);
            } else {
                const int j = e < 32 && e < X.ew ? H.ej : X.partner(i, e);
                xj = xs[j];
                lj4 = lam[j];
                pair_vec(xr, xj, C.per, C, dx, dy, dz);
            }
            const float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
            const float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            const float rinv = rsqrtf(r2);
            const float r2inv = rinv * rinv;
            const float r = r2 * rinv;
            const float qq = K.ke * xr.w * xj.w;
            const float ar = alpha * r;
            const float ef = erff(ar);
            const float gau = gau_c * __expf(-ar * ar);
            const float fxu = (gau - ef * rinv) * r2inv;  // f per unit qq
            A.eex = fmaf(-xj.w * ef, rinv, A.eex);  // per unit ke q_i
            const float fr = qq * fxu;
            const float fpr = -qq * r2inv * fmaf(3.f, fxu, 2.f * a2 * gau);
            A.gq = fmaf(K.ke * xj.w * fxu, du, A.gq);
            const float k2 = fpr * du;
            A.gx = fmaf(fr, ux, fmaf(k2, dx, A.gx));
            A.gy = fmaf(fr, uy, fmaf(k2, dy, A.gy));
            A.gz = fmaf(fr, uz, fmaf(k2, dz, A.gz));
            A.fx = fmaf(fr, dx, A.fx);
            A.fy = fmaf(fr, dy, A.fy);
            A.fz = fmaf(fr, dz, A.fz);
        }
    }
    float v[12] = {A.fx, A.fy, A.fz, A.elj, A.edir, A.eex, A.gx, A.gy, A.gz, A.gq, A.gs, A.ge};
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = group_sum<32>(v[q]);
    if (lane == 0) {
        if (MULTI) {  // partial sums carried in tile order (12 scratch floats per atom)
            float4* sp = pscr + 3 * (size_t)i;
            if (t0 > 0) {
                const float4 a = sp[0], b = sp[1], g = sp[2];
                v[0] += a.x; v[1] += a.y; v[2] += a.z; v[3] += a.w;
                v[4] += b.x; v[5] += b.y; v[6] += b.z; v[7] += b.w;
                v[8] += g.x; v[9] += g.y; v[10] += g.z; v[11] += g.w;
            }
            if (!last) {
                sp[0] = make_float4(v[0], v[1], v[2], v[3]);
                sp[1] = make_float4(v[4], v[5], v[6], v[7]);
                sp[2] = make_float4(v[8], v[9], v[10], v[11]);
            }
        }
        if (last) {
            ffix[i] = to_fix(v[0], scale, flags + 1);
            ffix[(size_t)N + i] = to_fix(v[1], scale, flags + 1);
            ffix[2 * (size_t)N + i] = to_fix(v[2], scale, flags + 1);
            if (COUL == kCoulEwald) {  // ke q_i as hi + lo, as in the force kernel
                const float qke = K.ke * xr.w, lo = fmaf(K.ke, xr.w, -qke);
                v[4] = fmaf(qke, v[4], lo * v[4]);
                v[5] = fmaf(qke, v[5], lo * v[5]);
            }
            e_atom[i] = make_float4(0.5f * v[3], 0.5f * v[4], 0.5f * v[5], 0.f);
            gx_s[i] = make_float4(v[6], v[7], v[8], v[9]);
            gp_s[i] = make_float2(v[10], v[11]);
        }
    }
}

template <bool LJ, int COUL>
// LJ-only instantiations are register-bound (small stencils): capped at 64 registers so
// that four blocks share an SM; with Coulomb (larger staged stencils) two.
__global__ void __launch_bounds__(kVjpThreads, COUL ? 2 : 4) k_vjp_cell(
    int N, int cap, int tile, const int* __restrict__ cell_sys, const SysDev* __restrict__ sys,
    const int* __restrict__ start, const float4* __restrict__ xs, const float2* __restrict__ ps,
    const float4* __restrict__ lam, const unsigned short* __restrict__ nbr, const int* __restrict__ cnt,
    ExclView X, float4* __restrict__ gx_s, float2* __restrict__ gp_s, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float4* __restrict__ pscr, float scale, unsigned* flags, int split) {
    pdl_wait();
    // `split` blocks share a cell, as in k_pair_cell
    const int c = blockIdx.x / split, part = blockIdx.x % split;
    const int stride = kVjpWarps * split;
    const SysDev& S = sys[cell_sys[c]];
    const CellCtx C = cell_ctx(c, S, start);
    const int ib = C.i0 + part * kVjpWarps + (threadIdx.x >> 5);
    if (C.i0 + part * kVjpWarps >= C.i1) return;
    const PairK K = pair_k(S);
    __shared__ BuildRun runs[kMaxRuns];
    __shared__ int n_runs, n_cand;
    __shared__ float4 qd_all[kVjpWarps][kQueue];
    __shared__ int qj_all[kVjpWarps][kQueue];
    extern __shared__ float4 smem[];
    float4* cand = smem;
    float4* lamc = cand + tile;
    float2* par = reinterpret_cast<float2*>(lamc + tile);
    unsigned char* cflag = reinterpret_cast<unsigned char*>(par + tile);
    const int w = threadIdx.x >> 5;
    const bool want_excl = COUL == kCoulEwald && K.alpha > 0.f;
    AtomHdr hn;
    if (ib < C.i1) hn = load_hdr(ib, xs, ps, nbr, cnt, cap, X, want_excl);
    if (w == 0) cell_runs(C, S, start, runs, &n_runs, &n_cand, flags);
    __syncthreads();
    const int nr = n_runs, total = n_cand;
    if (total > 65536) return;
    const bool multi = total > tile;
    for (int t0 = 0; t0 < total; t0 += tile) {
        const int t1 = min(total, t0 + tile);
        stage_pair_tile(C, runs, nr, t0, t1, kVjpThreads, xs, ps, lam, cand, par, lamc, cflag);
        __syncthreads();
        const bool last = t1 == total;
        if (t0 > 0 && ib < C.i1) hn = load_hdr(ib, xs, ps, nbr, cnt, cap, X, want_excl);
        for (int i = ib; i < C.i1; i += stride) {
            const AtomHdr H = hn;
            if (i + stride < C.i1) hn = load_hdr(i + stride, xs, ps, nbr, cnt, cap, X, want_excl);
#define NB_VJP_ARGS C, K, N, i, H, t0, t1, last, runs, nr, cand, par, lamc, cflag, qd_all[w], qj_all[w], xs, lam, nbr, \
                    cap, X, gx_s, gp_s, ffix, e_atom, pscr, scale, flags
            if (multi) {
                if (C.gen) vjp_atom<LJ, COUL, true, true>(NB_VJP_ARGS);
                else vjp_atom<LJ, COUL, false, true>(NB_VJP_ARGS);
            } else {
                if (C.gen) vjp_atom<LJ, COUL, true, false>(NB_VJP_ARGS);
                else vjp_atom<LJ, COUL, false, false>(NB_VJP_ARGS);
            }
#undef NB_VJP_ARGS
        }
        if (!last) __syncthreads();
    }
}

static size_t pair_smem(const nb_handle* h) {
    return (size_t)h->tile * (sizeof(float4) + sizeof(float2) + (h->build_gen ? 1 : 0));
}
static size_t vjp_smem(const nb_handle* h) {
    return (size_t)h->tile * (2 * sizeof(float4) + sizeof(float2) + (h->build_gen ? 1 : 0));
}

static ExclView excl_view(const nb_handle* h) {
    ExclView X;
    X.ew = h->excl_w;
    X.slot = h->ex_slot;
    X.cnt = h->ex_cnt;
    X.perm = h->perm;
    X.iperm = h->iperm;
    X.off = h->ex_off;
    X.idx = h->ex_idx;
    return X;
}

template <bool LJ, int COUL>
static void pair_launch(nb_handle* h, cudaStream_t st, bool vjp) {
    const ExclView X = excl_view(h);
    if (vjp)
        launch_pdl(k_vjp_cell<LJ, COUL>, h->n_cells * h->split_pair, kVjpThreads, vjp_smem(h), st,
            h->n_atoms, h->cap, h->tile, h->cell_sys, h->sys, h->cell_start, h->xs, h->ps, h->lam, h->nbr,
            h->nbr_cnt, X, h->gx_s, h->gp_s, h->ffix, h->e_atom, h->pscr, h->fscale, h->flags, h->split_pair);
    else
        launch_pdl(k_pair_cell<LJ, COUL>, h->n_cells * h->split_pair, kPairThreads, pair_smem(h), st,
            h->n_atoms, h->cap, h->tile, h->cell_sys, h->sys, h->cell_start, h->xs, h->ps, h->nbr, h->nbr_cnt, X,
            h->ffix, h->e_atom, h->pscr, h->fscale, h->flags, h->split_pair);
}

static void dispatch(nb_handle* h, int terms, cudaStream_t st, bool vjp) {
    bool lj = (terms & NB_TERM_LJ) != 0;
    bool coul = (terms & NB_TERM_COUL) != 0 && h->any_coul;  // uncharged systems: LJ-only kernels
    const bool rf = h->coul_kind == kCoulRF;
    if (!lj && !coul) {
        // no real-space term (PME alone): no list walk, only the per-atom outputs the
        // kernels would have written as zeros (forces stay as the load zeroed them)
        const size_t N = (size_t)h->n_atoms;
        cudaMemsetAsync(h->e_atom, 0, sizeof(float4) * N, st);
        if (vjp) {
            cudaMemsetAsync(h->gx_s, 0, sizeof(float4) * N, st);
            cudaMemsetAsync(h->gp_s, 0, sizeof(float2) * N, st);
        }
        return;
    }
    if (lj && coul && rf) pair_launch<true, kCoulRF>(h, st, vjp);
    else if (lj && coul) pair_launch<true, kCoulEwald>(h, st, vjp);
    else if (lj) pair_launch<true, kCoulNone>(h, st, vjp);
    else if (coul && rf) pair_launch<false, kCoulRF>(h, st, vjp);
    else pair_launch<false, kCoulEwald>(h, st, vjp);
}

void launch_pair(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, false); }
void launch_vjp(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, true); }

// The dynamic shared-memory limit of a kernel is process-wide, so it is raised once to
// what the device allows (less the kernel's static shared memory) rather than to one
// handle's need; each launch still asks only for its own tile.
template <class F>
static cudaError_t allow_max_smem(F kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

template <bool LJ, int COUL>
static cudaError_t set_smem() {
    cudaError_t e = allow_max_smem(k_pair_cell<LJ, COUL>);
    if (e != cudaSuccess) return e;
    return allow_max_smem(k_vjp_cell<LJ, COUL>);
}

cudaError_t pair_setup(nb_handle* h) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    // static shared memory of the VJP kernel: queues and runs (~23 KB)
    if ((long long)vjp_smem(h) + 24 * 1024 > optin) return cudaErrorInvalidValue;
    h->split_pair = pick_split(h, kPairWarps, 1);
    e = set_smem<true, kCoulEwald>();
    if (e == cudaSuccess) e = set_smem<true, kCoulRF>();
    if (e == cudaSuccess) e = set_smem<true, kCoulNone>();
    if (e == cudaSuccess) e = set_smem<false, kCoulEwald>();
    if (e == cudaSuccess) e = set_smem<false, kCoulRF>();
    return e;
}

}  // namespace nb
