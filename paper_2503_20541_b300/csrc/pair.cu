// pair.cu -- fused nonbonded pair kernel and its force vector-Jacobian product.
//
// Forces (Sec. 2.1.2): for every list pair with r < r_c under the minimum image
//   Lennard-Jones, Eq. (lj), eps_ij = sqrt(eps_i) sqrt(eps_j), sigma_ij = (sigma_i + sigma_j)/2,
//     optionally multiplied by the switch S(x) = 1 - 6x^5 + 15x^4 - 10x^3 on [r_s, r_c];
//   Ewald direct space ke q_i q_j erfc(alpha r)/r;
// and, for each of the atom's excluded partners (any distance), the exclusion
// correction -ke q_i q_j erf(alpha r)/r (the reciprocal sum still contains the
// pair; k_excl, one thread per atom).  A pair force is F_i = f(r) d with d = mi(x_i - x_j),
// f = -U'/r.
//
// Work decomposition: one warp per atom walks its full neighbour list (both directions of
// every pair are listed).  An entry is the partner's slot with a 6-bit image code (written
// by the list build, which decided the periodic image of the pair), and the partner's
// position, charge and LJ parameters are gathered straight from the slot-ordered arrays
// through L1: a block's warps take consecutive atoms of the slot order (atoms of one cell
// and its neighbours), so their partners overlap and mostly hit L1 after the first touch.
// No stencil is staged and blocks are not tied to cells.  A row holds the pairs that were
// inside r_c at the build at its front and the others at its back.  The front part is
// evaluated in place, 32 entries per round: while the positions are still those of the
// build (the "fresh" flag the build sets and every load clears) every front entry is
// inside r_c by the build's own test (the same difference and pair_r2), and otherwise the
// few that have left r_c are masked.  The back part is tested and the pairs that have
// come inside r_c are queued and evaluated 32 at a time.  i's data stays in registers,
// partial sums are reduced with warp shuffles in a fixed tree, and the force on i is added
// once, as int64 fixed point, to the zeroed force array (the PME gather and the exclusion
// correction add their parts concurrently or later; integer addition makes the order
// irrelevant).  Every FP32 summation order is fixed by the list, so results are bitwise
// reproducible.
#include "cell.cuh"
#include "erfc.cuh"
#include "lj.cuh"
#include "reduce.cuh"
#include "dfloat.cuh"
#include "erfc_df.cuh"

namespace nb {

constexpr int kPairWarps = 8;
constexpr int kPairThreads = kPairWarps * 32;
constexpr int kVjpWarps = 8;
constexpr int kVjpThreads = kVjpWarps * 32;
constexpr int kQueue = 64;        // per-warp queue of back-part pairs inside r_c
constexpr int kAtomsPerWarp = 2;  // atoms of a block's range per warp (header prefetch); 4 on large handles

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

// Per-atom context of the pair kernels: the atom, its row lengths and its system's constants.
struct AtomHdr {
    float4 xr;     // position (frame of the last build) and charge
    float2 pi;     // sigma, sqrt(eps)
    int nin;       // entries at the front of the row (inside r_c at the build)
    int nout;      // entries at the back of the row
    bool wrap;     // some entry of the row may carry an image code or fold an axis
    int sys;       // system index
    unsigned e0, e1, e2, e3;  // front entries lane, 32 + lane, 64 + lane, 96 + lane (0 past the end)
};

__device__ __forceinline__ AtomHdr load_hdr(int i, const int* __restrict__ sid, const float4* __restrict__ xs,
                                            const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
                                            const int* __restrict__ cnt, const int* __restrict__ cnt_out, int cap) {
    const int lane = threadIdx.x & 31;
    AtomHdr H;
    H.xr = xs[i];
    H.pi = ps[i];
    H.nin = cnt[i];
    const int o = cnt_out[i];
    H.nout = o & kOutCountMask;
    H.wrap = (o & kOutWrapBit) != 0;
    H.sys = sid[i];  // a system owns the same index range in slot and caller order
    const unsigned* row = nbr + (size_t)i * cap;
    H.e0 = lane < H.nin ? row[lane] : 0u;
    H.e1 = 32 + lane < H.nin ? row[32 + lane] : 0u;
    H.e2 = 64 + lane < H.nin ? row[64 + lane] : 0u;
    H.e3 = 96 + lane < H.nin ? row[96 + lane] : 0u;
    return H;
}

__device__ __forceinline__ int img_mode(const AtomHdr& H, const PairGeo& G) {
    if (G.fold[0] || G.fold[1] || G.fold[2]) return kImgFold;
    return H.wrap ? kImgCode : kImgPlain;
}

// One pair of the force kernel: (dx, dy, dz, q_j) and partner slot lq (r^2 is recomputed
// with the operations of the cut-off test, so it is the same value).  A lane with
// on == false contributes nothing: its coupling constants are zeroed and its r^2 set to
// r_c^2, so its arithmetic stays finite.  EN: the energies are wanted.  Without them the
// pair is evaluated for its force alone: erfc from the fitted form of erfc.cuh sharing its
// exponential with the Gaussian (a few ulp, far inside the force tolerance; the energy sums
// cancel ~1000-fold and need CUDA's erfcf), and 1/r^2 as (1/r)^2.
template <bool LJ, int COUL, bool EN>
__device__ __forceinline__ void pair_heavy(const float4& q, int lq, bool on, const float2& pi, bool do_lj,
                                           const PairK& K, const float2* __restrict__ par, float qke, float qke_lo,
                                           float alpha, float gau_c, float& fx, float& fy, float& fz, float& elj,
                                           float& edir) {
    const float r2 = on ? pair_r2(q.x, q.y, q.z) : K.rc2;
    const float rinv = rsqrtf(r2);
    float fr = 0.f;
    if (LJ && do_lj) {
        const float2 pj = par[lq];
        // refined for the energy: LJ raises it to the 6th power
        const float r2inv = EN ? recip_r2(r2, rinv) : rinv * rinv;
        const float ej = on ? pj.y : 0.f;
        const float eps = pi.y * ej;         // eps_ij = eps + eps_lo exactly
        const float eps_lo = fmaf(pi.y, ej, -eps);
        float u, f;
        lj_unit(0.5f * (pi.x + pj.x), r2inv, rinv, r2, K, u, f);
        if (EN) elj = fmaf(eps, u, fmaf(eps_lo, u, elj));
        fr = fmaf(eps_lo, f, eps * f);
    }
    const float qj_ = on ? q.w : 0.f;
    if (COUL == kCoulEwald && K.ke != 0.f) {  // block-uniform: uncharged systems of a mixed batch skip it
        const float r = r2 * rinv;
        const float qq = qke * qj_;
        const float ar = alpha * r;
        float ec, gau;
        if (EN) {
            ec = erfcf(ar);
            gau = gau_c * __expf(-ar * ar);
            // the energy is summed per unit ke q_i (q_j erfc(alpha r)/r) and scaled once per
            // atom: ke q_i q_j, rounded alike for every pair of two atom types, would make its
            // rounding add linearly over a sum that cancels ~10^3-fold
            edir = fmaf(qj_ * ec, rinv, edir);
        } else {
            const float E = exp_neg_sq(ar);
            ec = erfc_with_exp(ar, E);
            gau = gau_c * E;
        }
        fr = fmaf(qq * fmaf(ec, rinv, gau), rinv * rinv, fr);
    }
    if (COUL == kCoulRF && K.ke != 0.f) {  // Eq. RFA: qq (1/r + k r^2 - c), f = qq (1/r^3 - 2k)
        // The pair energies of water cancel ~10^4-fold in the sum, so a rounding shared by
        // many pairs would dominate its error: ke q_i q_j (two charge values, every pair of a
        // type pair rounded alike) is carried as hi + lo, and so are k and c.
        const float qq = qke * qj_;
        if (EN) {
            const float qq_lo = fmaf(qke_lo, qj_, fmaf(qke, qj_, -qq));
            const float u = fmaf(K.krf, r2, rinv - K.crf) + fmaf(K.krf_lo, r2, -K.crf_lo);
            edir = fmaf(qq, u, fmaf(qq_lo, u, edir));
        }
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

// The back part of a row (pairs outside r_c at the build, stored in reverse from the end
// of the row): tested, and the ones now inside r_c queued and evaluated 32 at a time.
template <int IMG, class Heavy>
__device__ __forceinline__ void walk_back(const float4& xr, const PairGeo& G, const unsigned* __restrict__ brow,
                                          int nout, float rc2, const float4* __restrict__ xs, float4* qd, int* qj,
                                          Heavy& heavy) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    int head = 0, nq = 0;
    // entries two rounds ahead, the partner's position one round ahead
    unsigned b0 = lane < nout ? brow[lane] : 0u, b1 = 32 + lane < nout ? brow[32 + lane] : 0u;
    float4 g = xs[b0 & kEntrySlotMask];
    for (int e0 = 0; e0 < nout; e0 += 32) {
        const unsigned ent = b0;
        const float4 cj = g;
        b0 = b1;
        const int en = e0 + 64 + lane;
        b1 = en < nout ? brow[en] : 0u;
        if (e0 + 32 + lane < nout) g = xs[b0 & kEntrySlotMask];
        const bool in = e0 + lane < nout;
        const int j = in ? (int)(ent & kEntrySlotMask) : 0;
        float dx, dy, dz;
        entry_diff<IMG>(xr, cj, ent >> kEntrySlotBits, G, dx, dy, dz);
        const bool acc = in && pair_r2(dx, dy, dz) < rc2;
        const unsigned bits = __ballot_sync(0xffffffffu, acc);
        if (bits) {  // warp-uniform: most back rounds accept nothing
            const int pos = (head + nq + __popc(bits & lt)) & (kQueue - 1);
            sts_q_if(qd + pos, qj + pos, make_float4(dx, dy, dz, cj.w), j, acc);
            nq += __popc(bits);
            if (nq >= 32) {
                __syncwarp();
                const int p = (head + lane) & (kQueue - 1);
                const float4 q = qd[p];
                const int lq = qj[p];
                __syncwarp();
                heavy(q, lq, true);
                head = (head + 32) & (kQueue - 1);
                nq -= 32;
            }
        }
    }
    __syncwarp();
    if (nq > 0) {  // warp-uniform
        const int p = (head + lane) & (kQueue - 1);
        const bool on = lane < nq;
        // lanes past the queue's end hold stale or never written entries: replaced by zeros
        const float4 q = on ? qd[p] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int lq = on ? qj[p] : 0;
        __syncwarp();
        heavy(q, lq, on);
    }
    __syncwarp();
}

// The list walk of one atom (one warp): heavy(q, j, on) is called for every round of 32
// pairs, q = (x_i - x_j, q_j), j the partner's slot, `on` whether the lane's pair is inside
// r_c.  Front entries go in place, the lane taking entry e0 + lane of each round; with
// fresh lists their test is the build's own, so they are all on.  Entries are loaded four
// rounds ahead (the first four with the atom's header, one atom ahead) and the partner's
// position one round ahead.
template <int IMG, class Heavy>
__device__ __forceinline__ void walk_list(const AtomHdr& H, const PairGeo& G, const unsigned* __restrict__ row,
                                          int cap, bool fresh, bool skip_back, float rc2, const float4* __restrict__ xs,
                                          float4* qd,
                                          int* qj, Heavy& heavy) {
    const int lane = threadIdx.x & 31;
    const int nin = H.nin;
    const float4 xr = H.xr;
    unsigned p0 = H.e0, p1 = H.e1, p2 = H.e2, p3 = H.e3;
    float4 g = xs[lane < nin ? (int)(p0 & kEntrySlotMask) : 0];
    for (int e0 = 0; e0 < nin; e0 += 32) {
        const unsigned ent = p0;
        const float4 cj = g;
        p0 = p1;
        p1 = p2;
        p2 = p3;
        const int en = e0 + 128 + lane;
        p3 = en < nin ? row[en] : 0u;
        if (e0 + 32 + lane < nin) g = xs[p0 & kEntrySlotMask];
        const bool in = e0 + lane < nin;
        float dx, dy, dz;
        entry_diff<IMG>(xr, cj, ent >> kEntrySlotBits, G, dx, dy, dz);
        const bool on = in && (fresh || pair_r2(dx, dy, dz) < rc2);
        heavy(make_float4(dx, dy, dz, cj.w), in ? (int)(ent & kEntrySlotMask) : 0, on);
    }
    if (!fresh && !skip_back && H.nout > 0)
        walk_back<IMG>(xr, G, row + (cap - H.nout), H.nout, rc2, xs, qd, qj, heavy);
}

// Atoms of block b: [b * per_block, min(N, (b + 1) * per_block)), warp w taking atoms
// w, w + warps, ... of the range.
struct AtomRange {
    int i0, i1, step;
};
__device__ __forceinline__ AtomRange block_atoms(int N, int per_block, int warps) {
    AtomRange R;
    const int b0 = blockIdx.x * per_block;
    R.i0 = b0 + (threadIdx.x >> 5);
    R.i1 = min(N, b0 + per_block);
    R.step = warps;
    return R;
}

// Forces and (EN) half energies of atom i (one warp).
template <bool LJ, int COUL, bool EN, int IMG>
__device__ __forceinline__ void pair_atom(int N, int i, const AtomHdr& H, const SysDev& S, bool fresh, bool pruned,
                                          const float4* __restrict__ xs, const float2* __restrict__ ps,
                                          const unsigned* __restrict__ nbr, int cap, float4* qd, int* qj,
                                          long long* __restrict__ ffix, float4* __restrict__ e_atom, float scale,
                                          unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const PairK K = pair_k(S);
    const PairGeo G = pair_geo(S);
    const float4 xr = H.xr;
    const float2 pi = H.pi;
    const float qke = K.ke * xr.w;
    const float qke_lo = COUL == kCoulRF ? fmaf(K.ke, xr.w, -qke) : 0.f;  // ke q_i = qke + qke_lo exactly
    const float alpha = K.alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    const bool do_lj = pi.y != 0.f;
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f;
    auto heavy = [&](const float4& q, int j, bool on) {
        pair_heavy<LJ, COUL, EN>(q, j, on, pi, do_lj, K, ps, qke, qke_lo, alpha, gau_c, fx, fy, fz, elj, edir);
    };
    walk_list<IMG>(H, G, nbr + (size_t)i * cap, cap, fresh, pruned && S.rin2 > 0.f, K.rc2, xs, qd, qj, heavy);
    if (!EN) {  // lane 8k holds the warp sum of force component k; no energy record
        float v[4] = {fx, fy, fz, 0.f};
        const float sum = warp_sum_transposed<4>(v);
        const int k = lane >> 3;
        if ((lane & 7) == 0 && k < 3) red_add(ffix + (size_t)k * N + i, to_fix(sum, scale, flags + 1));
        return;
    }
    if (COUL == kCoulNone) {  // lane 8k holds the warp sum of value k: fx, fy, fz, elj
        float v[4] = {fx, fy, fz, elj};
        const float sum = warp_sum_transposed<4>(v);
        const int k = lane >> 3;
        if ((lane & 7) == 0 && k < 3) red_add(ffix + (size_t)k * N + i, to_fix(sum, scale, flags + 1));
        else if (lane == 24) e_atom[i] = make_float4(0.5f * sum, 0.f, 0.f, 0.f);  // no exclusion pass
        return;
    }
    // lane 4k holds the warp sum of value k: fx, fy, fz, elj, edir
    float v[8] = {fx, fy, fz, elj, edir, 0.f, 0.f, 0.f};
    const float sum = warp_sum_transposed<8>(v);
    const int k = lane >> 2;
    if ((lane & 3) == 0 && k < 3) {
        // added (ffix is zeroed per evaluation): the PME gather adds concurrently
        red_add(ffix + (size_t)k * N + i, to_fix(sum, scale, flags + 1));
    } else if (lane == 12) {
        reinterpret_cast<float*>(e_atom + i)[0] = 0.5f * sum;
    } else if (lane == 16) {
        float ed = sum;
        if (COUL == kCoulEwald) {  // ke q_i = qke + (ke q_i - qke) exactly: one rounding per atom
            const float lo = fmaf(K.ke, xr.w, -qke);
            ed = fmaf(qke, ed, lo * ed);
        }
        reinterpret_cast<float*>(e_atom + i)[1] = 0.5f * ed;
    } else if (lane == 20) {
        // .z (exclusion correction) is written by k_excl
        reinterpret_cast<float2*>(e_atom + i)[1] = make_float2(0.f, 0.f);
    }
}

// 64 registers, four blocks (32 warps) per SM: the walk is latency-bound and the few
// spilled values are cheaper than the lost occupancy (water 24k: 64.7 -> 63.0 us fresh,
// 106.8 -> 99.6 us with the list reused, against 80 registers and three blocks).
// The two-atoms-per-warp pass of an LJ-only block (defined with k_pair2 below).
template <bool LJ, bool EN>
__device__ __forceinline__ void pair2_block(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
    const int* __restrict__ cnt, const int* __restrict__ cnt_out, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys);

// MIXED: the handle holds both charged and uncharged systems; a block whose atoms all belong
// to one uncharged system runs the two-atoms-per-warp pass (bitwise the same results).
template <bool LJ, int COUL, bool EN, bool MIXED>
__global__ void __launch_bounds__(kPairThreads, 4) k_pair(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
    const int* __restrict__ cnt, const int* __restrict__ cnt_out, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys) {
    pdl_wait();
    if (MIXED) {
        const int b0 = blockIdx.x * per_block, i1 = min(N, b0 + per_block);
        if (b0 < i1) {
            const int s0 = sid[b0];
            if (s0 == sid[i1 - 1] && sys[s0].ke == 0.f) {
                pair2_block<LJ, EN>(N, per_block, cap, sid, sys, xs, ps, nbr, cnt, cnt_out, ffix, e_atom, scale,
                                    flags, prune_sys);
                return;
            }
        }
    }
    __shared__ float4 qd_all[kPairWarps][kQueue];
    __shared__ int qj_all[kPairWarps][kQueue];
    const int w = threadIdx.x >> 5;
    const AtomRange R = block_atoms(N, per_block, kPairWarps);
    if (R.i0 >= R.i1) return;
    const bool fresh = flags[NB_FLAG_FRESH] != 0u;  // positions are those of the list build
    AtomHdr hn = load_hdr(R.i0, sid, xs, ps, nbr, cnt, cnt_out, cap);
    for (int i = R.i0; i < R.i1; i += R.step) {
        const AtomHdr H = hn;
        if (i + R.step < R.i1) hn = load_hdr(i + R.step, sid, xs, ps, nbr, cnt, cnt_out, cap);
        const SysDev& S = sys[H.sys];
        const int mode = img_mode(H, pair_geo(S));
        // the system's back parts hold no pair within r_c (dynamic list pruning)
        const bool pruned = !fresh && prune_sys && (prune_sys[H.sys] & kPruned) != 0u;
#define NB_PAIR_ARGS N, i, H, S, fresh, pruned, xs, ps, nbr, cap, qd_all[w], qj_all[w], ffix, e_atom, scale, flags
        if (mode == kImgPlain) pair_atom<LJ, COUL, EN, kImgPlain>(NB_PAIR_ARGS);
        else if (mode == kImgCode) pair_atom<LJ, COUL, EN, kImgCode>(NB_PAIR_ARGS);
        else pair_atom<LJ, COUL, EN, kImgFold>(NB_PAIR_ARGS);
#undef NB_PAIR_ARGS
    }
}

// ---- Two atoms per warp (LJ-only kernels) ---------------------------------------------
// With few pairs per atom (an LJ fluid: ~54 inside r_c, 1.7 rounds of 32) a warp per atom
// spends much of its time on the per-atom part (header, system constants, reduction).
// k_pair2 gives each half-warp (group g = lane / 16) one atom and lets each lane stand for
// two lanes of the warp-per-atom kernel: lane l' of a group does, for every round of 32
// entries, what lanes l' (set A) and l' + 16 (set B) of k_pair do, in the same order and
// with the same operations; the back part's queue receives the same entries in the same
// order; and the reduction's first level, lane l + lane l ^ 16 in k_pair, is the lane's own
// A + B (addition commutes), the other levels (8, 4, 2, 1) pairing the same lanes.  So
// every atom's forces and energies are bitwise those of k_pair, whichever kernel a handle
// runs (a batched handle with charged systems runs k_pair for its LJ systems too).

// Per-atom context of a group: as AtomHdr, with the first two rounds' entries of both sets
// (row positions l', 16 + l', 32 + l', 48 + l').
struct AtomHdr2 {
    float4 xr;
    float2 pi;
    int nin, nout;
    bool wrap;
    int sys;
    unsigned a0, b0, a1, b1;
};

__device__ __forceinline__ AtomHdr2 load_hdr2(int i, bool valid, const int* __restrict__ sid,
                                              const float4* __restrict__ xs, const float2* __restrict__ ps,
                                              const unsigned* __restrict__ nbr, const int* __restrict__ cnt,
                                              const int* __restrict__ cnt_out, int cap) {
    const int l = threadIdx.x & 15;
    AtomHdr2 H;
    H.xr = xs[i];
    H.pi = ps[i];
    H.nin = valid ? cnt[i] : 0;
    const int o = valid ? cnt_out[i] : 0;
    H.nout = o & kOutCountMask;
    H.wrap = (o & kOutWrapBit) != 0;
    H.sys = sid[i];
    const unsigned* row = nbr + (size_t)i * cap;
    H.a0 = l < H.nin ? row[l] : 0u;
    H.b0 = 16 + l < H.nin ? row[16 + l] : 0u;
    H.a1 = 32 + l < H.nin ? row[32 + l] : 0u;
    H.b1 = 48 + l < H.nin ? row[48 + l] : 0u;
    return H;
}

// The front of the group's row, two rounds of entries ahead and the partners' positions one
// round ahead; rounds past the group's own count are skipped (the other group may have more).
template <int IMG, class HeavyA, class HeavyB>
__device__ __forceinline__ void walk_front2(const AtomHdr2& H, const PairGeo& G, const unsigned* __restrict__ row,
                                            int nin_max, bool fresh, float rc2, const float4* __restrict__ xs,
                                            HeavyA& heavyA, HeavyB& heavyB) {
    const int l = threadIdx.x & 15;
    const int nin = H.nin;
    unsigned pa0 = H.a0, pb0 = H.b0, pa1 = H.a1, pb1 = H.b1;
    float4 ga = xs[l < nin ? (int)(pa0 & kEntrySlotMask) : 0];
    float4 gb = xs[16 + l < nin ? (int)(pb0 & kEntrySlotMask) : 0];
    for (int e0 = 0; e0 < nin_max; e0 += 32) {
        const unsigned ea = pa0, eb = pb0;
        const float4 ca = ga, cb = gb;
        pa0 = pa1;
        pb0 = pb1;
        pa1 = e0 + 64 + l < nin ? row[e0 + 64 + l] : 0u;
        pb1 = e0 + 80 + l < nin ? row[e0 + 80 + l] : 0u;
        if (e0 + 32 + l < nin) ga = xs[pa0 & kEntrySlotMask];
        if (e0 + 48 + l < nin) gb = xs[pb0 & kEntrySlotMask];
        if (e0 < nin) {
            const bool ina = e0 + l < nin, inb = e0 + 16 + l < nin;
            float dx, dy, dz;
            entry_diff<IMG>(H.xr, ca, ea >> kEntrySlotBits, G, dx, dy, dz);
            bool on = ina && (fresh || pair_r2(dx, dy, dz) < rc2);
            heavyA(make_float4(dx, dy, dz, ca.w), ina ? (int)(ea & kEntrySlotMask) : 0, on);
            entry_diff<IMG>(H.xr, cb, eb >> kEntrySlotBits, G, dx, dy, dz);
            on = inb && (fresh || pair_r2(dx, dy, dz) < rc2);
            heavyB(make_float4(dx, dy, dz, cb.w), inb ? (int)(eb & kEntrySlotMask) : 0, on);
        }
    }
}

// The back of the group's row (kept lists that are not pruned): the entries now inside r_c
// are queued in the order k_pair queues them (set A's half of each round of 32, then set
// B's) and evaluated 32 at a time, set A taking queue positions head + l' and set B
// head + 16 + l'.  Each group has its own queue; ballots and barriers are warp-wide.
template <int IMG, class HeavyA, class HeavyB>
__device__ __forceinline__ void walk_back2(const AtomHdr2& H, const PairGeo& G, const unsigned* __restrict__ brow,
                                           int nout, int nout_max, float rc2, const float4* __restrict__ xs,
                                           float4* qd, int* qj, HeavyA& heavyA, HeavyB& heavyB) {
    const int lane = threadIdx.x & 31, l = lane & 15, sh = lane & 16;
    const unsigned lta = (1u << l) - 1u, ltb = (1u << (l + 16)) - 1u;
    int head = 0, nq = 0;
    unsigned ba0 = l < nout ? brow[l] : 0u, bb0 = 16 + l < nout ? brow[16 + l] : 0u;
    unsigned ba1 = 32 + l < nout ? brow[32 + l] : 0u, bb1 = 48 + l < nout ? brow[48 + l] : 0u;
    float4 ga = xs[ba0 & kEntrySlotMask], gb = xs[bb0 & kEntrySlotMask];
    for (int e0 = 0; e0 < nout_max; e0 += 32) {
        const unsigned ea = ba0, eb = bb0;
        const float4 ca = ga, cb = gb;
        ba0 = ba1;
        bb0 = bb1;
        ba1 = e0 + 64 + l < nout ? brow[e0 + 64 + l] : 0u;
        bb1 = e0 + 80 + l < nout ? brow[e0 + 80 + l] : 0u;
        if (e0 + 32 + l < nout) ga = xs[ba0 & kEntrySlotMask];
        if (e0 + 48 + l < nout) gb = xs[bb0 & kEntrySlotMask];
        const bool ina = e0 + l < nout, inb = e0 + 16 + l < nout;
        float ax, ay, az, bx, by, bz;
        entry_diff<IMG>(H.xr, ca, ea >> kEntrySlotBits, G, ax, ay, az);
        entry_diff<IMG>(H.xr, cb, eb >> kEntrySlotBits, G, bx, by, bz);
        const bool acca = ina && pair_r2(ax, ay, az) < rc2;
        const bool accb = inb && pair_r2(bx, by, bz) < rc2;
        const unsigned wa = __ballot_sync(0xffffffffu, acca), wb = __ballot_sync(0xffffffffu, accb);
        // the group's round as k_pair's warp sees it: set A in bits 0-15, set B in 16-31
        const unsigned bits = ((wa >> sh) & 0xffffu) | (((wb >> sh) & 0xffffu) << 16);
        if (__any_sync(0xffffffffu, bits != 0u)) {
            const int pa = (head + nq + __popc(bits & lta)) & (kQueue - 1);
            const int pb = (head + nq + __popc(bits & ltb)) & (kQueue - 1);
            sts_q_if(qd + pa, qj + pa, make_float4(ax, ay, az, ca.w), ina ? (int)(ea & kEntrySlotMask) : 0, acca);
            sts_q_if(qd + pb, qj + pb, make_float4(bx, by, bz, cb.w), inb ? (int)(eb & kEntrySlotMask) : 0, accb);
            nq += __popc(bits);
            const bool flush = nq >= 32;
            if (__any_sync(0xffffffffu, flush)) {
                __syncwarp();
                float4 qa = make_float4(0.f, 0.f, 0.f, 0.f), qb = qa;
                int ja = 0, jb = 0;
                if (flush) {
                    const int p0 = (head + l) & (kQueue - 1), p1 = (head + 16 + l) & (kQueue - 1);
                    qa = qd[p0];
                    ja = qj[p0];
                    qb = qd[p1];
                    jb = qj[p1];
                }
                __syncwarp();
                if (flush) {
                    heavyA(qa, ja, true);
                    heavyB(qb, jb, true);
                    head = (head + 32) & (kQueue - 1);
                    nq -= 32;
                }
            }
        }
    }
    __syncwarp();
    if (__any_sync(0xffffffffu, nq > 0)) {
        const bool ona = l < nq, onb = 16 + l < nq;
        const int p0 = (head + l) & (kQueue - 1), p1 = (head + 16 + l) & (kQueue - 1);
        // positions past the queue's end hold stale or never written entries: zeros instead
        const float4 qa = ona ? qd[p0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 qb = onb ? qd[p1] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int ja = ona ? qj[p0] : 0, jb = onb ? qj[p1] : 0;
        __syncwarp();
        if (nq > 0) {
            heavyA(qa, ja, ona);
            heavyB(qb, jb, onb);
        }
    }
    __syncwarp();
}

// Sums of v[0..NV) over the 16 lanes of a group, transposed as warp_sum_transposed does it
// from its second level on (xor 8, 4, ...): group lane (16 / NV) k ends with the sum of
// value k.  The caller has already formed the first level (its sets A + B).
template <int NV>
__device__ __forceinline__ float group_sum_transposed(float (&v)[NV]) {
    const int lane = threadIdx.x & 31;
    int n = NV, o = 8;
#pragma unroll
    for (int lev = 0; (1 << lev) < NV; ++lev) {
        n >>= 1;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < NV / 2; ++k) {
            if (k < n) {
                const float keep = upper ? v[n + k] : v[k];
                const float give = upper ? v[k] : v[n + k];
                v[k] = keep + __shfl_xor_sync(0xffffffffu, give, o);
            }
        }
        o >>= 1;
    }
    float r = v[0];
#pragma unroll
    for (; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// Forces and (EN) half LJ energy of the group's atom i (LJ only; valid: the group has an
// atom).  Sets A and B accumulate as lanes l' and l' + 16 of k_pair.
template <bool LJ, bool EN, int IMG>
__device__ __forceinline__ void pair_atom2(int N, int i, bool valid, const AtomHdr2& H, const PairK& K,
                                           const PairGeo& G, bool fresh, bool skip_back, int nin_max, int nout_max,
                                           const float4* __restrict__ xs, const float2* __restrict__ ps,
                                           const unsigned* __restrict__ nbr, int cap, float4* qd, int* qj,
                                           long long* __restrict__ ffix, float4* __restrict__ e_atom, float scale,
                                           unsigned* flags) {
    const int l = threadIdx.x & 15;
    const float2 pi = H.pi;
    const bool do_lj = pi.y != 0.f;
    float fxa = 0.f, fya = 0.f, fza = 0.f, ea = 0.f, da = 0.f;
    float fxb = 0.f, fyb = 0.f, fzb = 0.f, eb = 0.f, db = 0.f;
    auto heavy_a = [&](const float4& q, int j, bool on) {
        pair_heavy<LJ, kCoulNone, EN>(q, j, on, pi, do_lj, K, ps, 0.f, 0.f, 0.f, 0.f, fxa, fya, fza, ea, da);
    };
    auto heavy_b = [&](const float4& q, int j, bool on) {
        pair_heavy<LJ, kCoulNone, EN>(q, j, on, pi, do_lj, K, ps, 0.f, 0.f, 0.f, 0.f, fxb, fyb, fzb, eb, db);
    };
    const unsigned* row = nbr + (size_t)i * cap;
    walk_front2<IMG>(H, G, row, nin_max, fresh, K.rc2, xs, heavy_a, heavy_b);
    const int nout = (!fresh && !skip_back) ? H.nout : 0;
    walk_back2<IMG>(H, G, row + (cap - nout), nout, nout_max, K.rc2, xs, qd, qj, heavy_a, heavy_b);
    // lane 4k of the group holds the sum of value k: fx, fy, fz, elj
    float v[4] = {fxa + fxb, fya + fyb, fza + fzb, EN ? ea + eb : 0.f};
    const float sum = group_sum_transposed<4>(v);
    const int k = l >> 2;
    if (!valid || (l & 3) != 0) return;
    if (k < 3) red_add(ffix + (size_t)k * N + i, to_fix(sum, scale, flags + 1));
    else if (EN) e_atom[i] = make_float4(0.5f * sum, 0.f, 0.f, 0.f);  // no exclusion pass
}

// LJ-only pair kernel, two atoms per warp (one per group), the atom ranges of k_pair's
// blocks.  Results bitwise those of k_pair<LJ, kCoulNone, EN>.
template <bool LJ, bool EN>
__device__ __forceinline__ void pair2_block(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
    const int* __restrict__ cnt, const int* __restrict__ cnt_out, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys) {
    __shared__ float4 qd_all[kPairWarps][2][kQueue];
    __shared__ int qj_all[kPairWarps][2][kQueue];
    const int w = threadIdx.x >> 5, grp = (threadIdx.x >> 4) & 1;
    const int b0 = blockIdx.x * per_block;
    const int i1 = min(N, b0 + per_block);
    const bool fresh = flags[NB_FLAG_FRESH] != 0u;
    for (int base = b0 + 2 * w; base < i1; base += 2 * kPairWarps) {
        const int i = base + grp;
        const bool valid = i < i1;
        const AtomHdr2 H = load_hdr2(valid ? i : base, valid, sid, xs, ps, nbr, cnt, cnt_out, cap);
        const SysDev& S = sys[H.sys];
        const PairK K = pair_k(S);
        const PairGeo G = pair_geo(S);
        const bool pruned = !fresh && prune_sys && (prune_sys[H.sys] & kPruned) != 0u;
        const bool skip_back = pruned && S.rin2 > 0.f;
        const int nout = (!fresh && !skip_back) ? H.nout : 0;
        const int nin_max = max(H.nin, __shfl_xor_sync(0xffffffffu, H.nin, 16));
        const int nout_max = max(nout, __shfl_xor_sync(0xffffffffu, nout, 16));
        // the more general image mode of the two atoms (on a row without image codes, or an
        // axis that is not folded, the general forms reduce to the plain difference)
        int mode = (G.fold[0] || G.fold[1] || G.fold[2]) ? kImgFold : (H.wrap ? kImgCode : kImgPlain);
        mode = max(mode, __shfl_xor_sync(0xffffffffu, mode, 16));
        float4* qd = qd_all[w][grp];
        int* qj = qj_all[w][grp];
#define NB_PAIR2_ARGS N, i, valid, H, K, G, fresh, skip_back, nin_max, nout_max, xs, ps, nbr, cap, qd, qj, ffix, e_atom, \
                      scale, flags
        if (mode == kImgPlain) pair_atom2<LJ, EN, kImgPlain>(NB_PAIR2_ARGS);
        else if (mode == kImgCode) pair_atom2<LJ, EN, kImgCode>(NB_PAIR2_ARGS);
        else pair_atom2<LJ, EN, kImgFold>(NB_PAIR2_ARGS);
#undef NB_PAIR2_ARGS
    }
}

template <bool LJ, bool EN>
__global__ void __launch_bounds__(kPairThreads, 4) k_pair2(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
    const int* __restrict__ cnt, const int* __restrict__ cnt_out, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys) {
    pdl_wait();
    pair2_block<LJ, EN>(N, per_block, cap, sid, sys, xs, ps, nbr, cnt, cnt_out, ffix, e_atom, scale, flags, prune_sys);
}

// Force VJP.  For each directed pair (i, j) with u = lam_i - lam_j and du = d.u:
//   gx_i += f u + (f'/r) du d           (J (lam_i - lam_j), J = f I + (f'/r) d d^T)
//   gq_i += ke q_j (f / qq) du,  gsig_i += 1/2 (df/dsigma_ij) du,  ge_i += sqrt(eps_j) (f/eps) du
// and the forces F_i as in k_pair_cell.  The exclusion correction contributes the same way.
struct VjpAcc {
    float fx = 0.f, fy = 0.f, fz = 0.f, elj = 0.f, edir = 0.f, eex = 0.f;
    float gx = 0.f, gy = 0.f, gz = 0.f, gq = 0.f, gs = 0.f, ge = 0.f;
};

// One pair of the VJP kernel, q = (dx, dy, dz, q_j); r^2 with the operations of the cut-off
// test (the same value).  A lane with on == false contributes nothing (its couplings are
// zeroed and its r^2 set to r_c^2), as in pair_heavy.
template <bool LJ, int COUL>
__device__ __forceinline__ void vjp_heavy(const float4& q, const float4& lj4, float2 pj, bool on,
                                          const float4& li, const float2& pi, float qi, const PairK& K,
                                          float alpha, float a2, float gau_c, VjpAcc& A) {
    const float dx = q.x, dy = q.y, dz = q.z, r2 = on ? pair_r2(dx, dy, dz) : K.rc2;
    pj.y = on ? pj.y : 0.f;
    const float qj_ = on ? q.w : 0.f;
    const float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
    const float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
    const float rinv = rsqrtf(r2);
    const float r2inv = recip_r2(r2, rinv);
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
        const float qq = K.ke * qi * qj_;
        const float ar = alpha * r;
        const float ec = erfcf(ar);
        const float gau = gau_c * __expf(-ar * ar);
        const float fcu = fmaf(ec, rinv, gau) * r2inv;  // f per unit qq
        A.edir = fmaf(qj_ * ec, rinv, A.edir);          // per unit ke q_i, as in the force kernel
        fr = fmaf(qq, fcu, fr);
        fpr = fmaf(-qq * r2inv, fmaf(3.f, fcu, 2.f * a2 * gau), fpr);
        A.gq = fmaf(K.ke * qj_ * fcu, du, A.gq);
    }
    if (COUL == kCoulRF && K.ke != 0.f) {  // Eq. RFA: f = qq (r^-3 - 2k), f'/r = -3 qq r^-5
        const float qke = K.ke * qi;
        const float qq = qke * qj_;
        // energy with ke q_i q_j, k and c as double-float pairs, as in the force kernel
        const float qq_lo = fmaf(fmaf(K.ke, qi, -qke), qj_, fmaf(qke, qj_, -qq));
        const float r3inv = r2inv * rinv;
        const float fcu = r3inv - 2.f * K.krf;
        const float u = fmaf(K.krf, r2, rinv - K.crf) + fmaf(K.krf_lo, r2, -K.crf_lo);
        A.edir = fmaf(qq, u, fmaf(qq_lo, u, A.edir));
        fr = fmaf(qq, fcu, fr);
        fpr = fmaf(-3.f * qq, r3inv * r2inv, fpr);
        A.gq = fmaf(K.ke * qj_ * fcu, du, A.gq);
    }
    const float k2 = fpr * du;
    A.gx = fmaf(fr, ux, fmaf(k2, dx, A.gx));
    A.gy = fmaf(fr, uy, fmaf(k2, dy, A.gy));
    A.gz = fmaf(fr, uz, fmaf(k2, dz, A.gz));
    A.fx = fmaf(fr, dx, A.fx);
    A.fy = fmaf(fr, dy, A.fy);
    A.fz = fmaf(fr, dz, A.fz);
}

template <bool LJ, int COUL, int IMG>
__device__ __forceinline__ void vjp_atom(int N, int i, const AtomHdr& H, const SysDev& S, bool fresh, bool pruned,
                                         const float4* __restrict__ xs, const float2* __restrict__ ps,
                                         const float4* __restrict__ lam, const unsigned* __restrict__ nbr, int cap,
                                         float4* qd, int* qj, float4* __restrict__ gx_s, float2* __restrict__ gp_s,
                                         long long* __restrict__ ffix, float4* __restrict__ e_atom, float scale,
                                         unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const PairK K = pair_k(S);
    const PairGeo G = pair_geo(S);
    const float4 xr = H.xr;
    const float2 pi = H.pi;
    const float4 li = lam[i];
    const float alpha = K.alpha, a2 = alpha * alpha;
    const float gau_c = 2.f * alpha * kInvSqrtPi;
    VjpAcc A;
    auto heavy = [&](const float4& q, int j, bool on) {
        vjp_heavy<LJ, COUL>(q, lam[j], ps[j], on, li, pi, xr.w, K, alpha, a2, gau_c, A);
    };
    walk_list<IMG>(H, G, nbr + (size_t)i * cap, cap, fresh, pruned && S.rin2 > 0.f, K.rc2, xs, qd, qj, heavy);
    // lane 2k holds the warp sum of value k
    float v[16] = {A.fx, A.fy, A.fz, A.elj, A.edir, A.gx, A.gy, A.gz, A.gq, A.gs, A.ge, 0.f, 0.f, 0.f, 0.f, 0.f};
    float sum = warp_sum_transposed<16>(v);
    const int k = lane >> 1;
    if (COUL == kCoulEwald && k == 4) {  // ke q_i as hi + lo, as in the force kernel
        const float qke = K.ke * xr.w, lo = fmaf(K.ke, xr.w, -qke);
        sum = fmaf(qke, sum, lo * sum);
    }
    // the fixed-point forces by lanes 0, 2, 4 in parallel; the other sums go to lane 0 (one
    // shuffle each), which writes the atom's energy and gradient records
    if ((lane & 1) == 0 && k < 3) ffix[(size_t)k * N + i] = to_fix(sum, scale, flags + 1);
    float w[11];
#pragma unroll
    for (int q = 3; q < 11; ++q) w[q] = __shfl_sync(0xffffffffu, sum, 2 * q);
    if (lane == 0) {
        e_atom[i] = make_float4(0.5f * w[3], 0.5f * w[4], 0.f, 0.f);
        gx_s[i] = make_float4(w[5], w[6], w[7], w[8]);
        gp_s[i] = make_float2(w[9], w[10]);
    }
}

template <bool LJ, int COUL>
// LJ-only instantiations are register-bound: capped at 64 registers so that four blocks
// share an SM; with Coulomb two.
__global__ void __launch_bounds__(kVjpThreads, COUL ? 2 : 4) k_vjp(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const float4* __restrict__ lam,
    const unsigned* __restrict__ nbr, const int* __restrict__ cnt, const int* __restrict__ cnt_out,
    float4* __restrict__ gx_s, float2* __restrict__ gp_s, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys) {
    pdl_wait();
    __shared__ float4 qd_all[kVjpWarps][kQueue];
    __shared__ int qj_all[kVjpWarps][kQueue];
    const int w = threadIdx.x >> 5;
    const AtomRange R = block_atoms(N, per_block, kVjpWarps);
    if (R.i0 >= R.i1) return;
    const bool fresh = flags[NB_FLAG_FRESH] != 0u;
    AtomHdr hn = load_hdr(R.i0, sid, xs, ps, nbr, cnt, cnt_out, cap);
    for (int i = R.i0; i < R.i1; i += R.step) {
        const AtomHdr H = hn;
        if (i + R.step < R.i1) hn = load_hdr(i + R.step, sid, xs, ps, nbr, cnt, cnt_out, cap);
        const SysDev& S = sys[H.sys];
        const int mode = img_mode(H, pair_geo(S));
        const bool pruned = !fresh && prune_sys && (prune_sys[H.sys] & kPruned) != 0u;
#define NB_VJP_ARGS N, i, H, S, fresh, pruned, xs, ps, lam, nbr, cap, qd_all[w], qj_all[w], gx_s, gp_s, ffix, e_atom, scale, \
                    flags
        if (mode == kImgPlain) vjp_atom<LJ, COUL, kImgPlain>(NB_VJP_ARGS);
        else if (mode == kImgCode) vjp_atom<LJ, COUL, kImgCode>(NB_VJP_ARGS);
        else vjp_atom<LJ, COUL, kImgFold>(NB_VJP_ARGS);
#undef NB_VJP_ARGS
    }
}

// Force VJP of an LJ-only handle, two atoms per warp as in k_pair2: lane l' of group g does
// what lanes l' and l' + 16 of k_vjp do for the group's atom (sets A and B), and the
// reduction's first level is A + B, so the results are bitwise those of k_vjp.
template <int IMG>
__device__ __forceinline__ void vjp_atom2(int N, int i, bool valid, const AtomHdr2& H, const PairK& K,
                                          const PairGeo& G, bool fresh, bool skip_back, int nin_max, int nout_max,
                                          const float4* __restrict__ xs, const float2* __restrict__ ps,
                                          const float4* __restrict__ lam, const unsigned* __restrict__ nbr, int cap,
                                          float4* qd, int* qj, float4* __restrict__ gx_s, float2* __restrict__ gp_s,
                                          long long* __restrict__ ffix, float4* __restrict__ e_atom, float scale,
                                          unsigned* flags) {
    const int lane = threadIdx.x & 31, l = lane & 15;
    const float2 pi = H.pi;
    const float4 li = lam[i];
    VjpAcc A, B;
    auto heavy_a = [&](const float4& q, int j, bool on) {
        vjp_heavy<true, kCoulNone>(q, lam[j], ps[j], on, li, pi, H.xr.w, K, 0.f, 0.f, 0.f, A);
    };
    auto heavy_b = [&](const float4& q, int j, bool on) {
        vjp_heavy<true, kCoulNone>(q, lam[j], ps[j], on, li, pi, H.xr.w, K, 0.f, 0.f, 0.f, B);
    };
    const unsigned* row = nbr + (size_t)i * cap;
    walk_front2<IMG>(H, G, row, nin_max, fresh, K.rc2, xs, heavy_a, heavy_b);
    const int nout = (!fresh && !skip_back) ? H.nout : 0;
    walk_back2<IMG>(H, G, row + (cap - nout), nout, nout_max, K.rc2, xs, qd, qj, heavy_a, heavy_b);
    // group lane k holds the sum of value k
    float v[16] = {A.fx + B.fx, A.fy + B.fy, A.fz + B.fz, A.elj + B.elj, A.edir + B.edir, A.gx + B.gx,
                   A.gy + B.gy, A.gz + B.gz, A.gq + B.gq, A.gs + B.gs, A.ge + B.ge, 0.f, 0.f, 0.f, 0.f, 0.f};
    const float sum = group_sum_transposed<16>(v);
    if (valid && l < 3) ffix[(size_t)l * N + i] = to_fix(sum, scale, flags + 1);
    float w[11];
#pragma unroll
    for (int q = 3; q < 11; ++q) w[q] = __shfl_sync(0xffffffffu, sum, (lane & 16) + q);
    if (valid && l == 0) {
        e_atom[i] = make_float4(0.5f * w[3], 0.5f * w[4], 0.f, 0.f);
        gx_s[i] = make_float4(w[5], w[6], w[7], w[8]);
        gp_s[i] = make_float2(w[9], w[10]);
    }
}

template <bool LJ>
__global__ void __launch_bounds__(kVjpThreads, 3) k_vjp2(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const float4* __restrict__ lam,
    const unsigned* __restrict__ nbr, const int* __restrict__ cnt, const int* __restrict__ cnt_out,
    float4* __restrict__ gx_s, float2* __restrict__ gp_s, long long* __restrict__ ffix,
    float4* __restrict__ e_atom, float scale, unsigned* flags, const unsigned* __restrict__ prune_sys) {
    pdl_wait();
    __shared__ float4 qd_all[kVjpWarps][2][kQueue];
    __shared__ int qj_all[kVjpWarps][2][kQueue];
    const int w = threadIdx.x >> 5, grp = (threadIdx.x >> 4) & 1;
    const int b0 = blockIdx.x * per_block;
    const int i1 = min(N, b0 + per_block);
    const bool fresh = flags[NB_FLAG_FRESH] != 0u;
    for (int base = b0 + 2 * w; base < i1; base += 2 * kVjpWarps) {
        const int i = base + grp;
        const bool valid = i < i1;
        const AtomHdr2 H = load_hdr2(valid ? i : base, valid, sid, xs, ps, nbr, cnt, cnt_out, cap);
        const SysDev& S = sys[H.sys];
        const PairK K = pair_k(S);
        const PairGeo G = pair_geo(S);
        const bool pruned = !fresh && prune_sys && (prune_sys[H.sys] & kPruned) != 0u;
        const bool skip_back = pruned && S.rin2 > 0.f;
        const int nout = (!fresh && !skip_back) ? H.nout : 0;
        const int nin_max = max(H.nin, __shfl_xor_sync(0xffffffffu, H.nin, 16));
        const int nout_max = max(nout, __shfl_xor_sync(0xffffffffu, nout, 16));
        int mode = (G.fold[0] || G.fold[1] || G.fold[2]) ? kImgFold : (H.wrap ? kImgCode : kImgPlain);
        mode = max(mode, __shfl_xor_sync(0xffffffffu, mode, 16));
        float4* qd = qd_all[w][grp];
        int* qj = qj_all[w][grp];
#define NB_VJP2_ARGS N, valid ? i : base, valid, H, K, G, fresh, skip_back, nin_max, nout_max, xs, ps, lam, nbr, cap, \
                     qd, qj, gx_s, gp_s, ffix, e_atom, scale, flags
        if (mode == kImgPlain) vjp_atom2<kImgPlain>(NB_VJP2_ARGS);
        else if (mode == kImgCode) vjp_atom2<kImgCode>(NB_VJP2_ARGS);
        else vjp_atom2<kImgFold>(NB_VJP2_ARGS);
#undef NB_VJP2_ARGS
    }
}

// Exclusion correction (Ewald): for each excluded partner j of atom i (at any distance; the
// reciprocal sum still contains the pair), -ke q_i q_j erf(alpha r)/r and its force, one
// thread per atom (slot order), launched after the pair (or VJP) kernel.  The partners are
// few (two per water atom), so a warp per atom in the pair kernel left most lanes idle and
// held its block at a barrier.  The difference is the minimum image of the two positions
// in the frame of the last build.  The force is added as fixed point (ffix is an integer
// sum, so the order against the pair kernel's and the PME gather's adds is irrelevant);
// the energy (per unit ke q_i, scaled by ke q_i as hi + lo) goes to e_atom[i].z, which the
// pair kernel wrote as 0.  VJP: J (lam_i - lam_j) and the charge gradient are added to
// gx_s[i].  Systems without Ewald electrostatics (ke = 0 or alpha = 0) are skipped.
// Exclusion correction of slot i (the frame of the last build): force (fx, fy, fz), energy
// per unit ke q_i (eex), and with VJP the J (lam_i - lam_j) and charge-gradient terms.
// Returns false (nothing to add) for atoms without exclusions and systems without Ewald
// electrostatics (ke = 0 or alpha = 0).
template <bool VJP>
__device__ __forceinline__ bool excl_terms(int i, const SysDev& S, const float4* __restrict__ xs,
                                           const float4* __restrict__ lam, const ExclView& X, float& fx, float& fy,
                                           float& fz, float& eex, float& gx, float& gy, float& gz, float& gq) {
    fx = fy = fz = eex = gx = gy = gz = gq = 0.f;
    const int ne = X.count(i);
    if (ne == 0) return false;
    const float alpha = S.alpha, ke = S.ke;
    if (!(alpha > 0.f) || ke == 0.f) return false;
    const float gau_c = 2.f * alpha * kInvSqrtPi, a2 = alpha * alpha;
    const float4 xr = xs[i];
    float4 li = make_float4(0.f, 0.f, 0.f, 0.f);
    if (VJP) li = lam[i];
    const float qke = ke * xr.w;
    for (int e = 0; e < ne; ++e) {
        const int j = X.partner(i, e);
        const float4 xj = xs[j];
        float dx = xr.x - xj.x, dy = xr.y - xj.y, dz = xr.z - xj.z;
        if (S.periodic) {
            dx = mi_pair(xr.x, xj.x, S.L[0], S.halfL[0]);
            dy = mi_pair(xr.y, xj.y, S.L[1], S.halfL[1]);
            dz = mi_pair(xr.z, xj.z, S.L[2], S.halfL[2]);
        }
        const float r2 = pair_r2(dx, dy, dz);
        const float rinv = rsqrtf(r2);
        const float r2inv = rinv * rinv;
        const float r = r2 * rinv;
        const float qq = qke * xj.w;
        const float ar = alpha * r;
        const float ef = erff(ar);
        const float gau = gau_c * __expf(-ar * ar);
        const float fxu = (gau - ef * rinv) * r2inv;  // f per unit qq
        eex = fmaf(-xj.w * ef, rinv, eex);
        const float fr = qq * fxu;
        fx = fmaf(fr, dx, fx);
        fy = fmaf(fr, dy, fy);
        fz = fmaf(fr, dz, fz);
        if (VJP) {
            const float4 lj4 = lam[j];
            const float ux = li.x - lj4.x, uy = li.y - lj4.y, uz = li.z - lj4.z;
            const float du = fmaf(dz, uz, fmaf(dy, uy, dx * ux));
            const float fpr = -qq * r2inv * fmaf(3.f, fxu, 2.f * a2 * gau);
            gq = fmaf(ke * xj.w * fxu, du, gq);
            const float k2 = fpr * du;
            gx = fmaf(fr, ux, fmaf(k2, dx, gx));
            gy = fmaf(fr, uy, fmaf(k2, dy, gy));
            gz = fmaf(fr, uz, fmaf(k2, dz, gz));
        }
    }
    return true;
}

// The atom's exclusion energy record (e_atom .z): half of ke q_i eex, ke q_i carried as
// qke + lo exactly so that only one rounding per atom enters.
__device__ __forceinline__ float excl_energy_half(float ke, float q, float eex) {
    const float qke = ke * q;
    const float lo = fmaf(ke, q, -qke);  // ke q_i = qke + lo exactly
    return 0.5f * fmaf(qke, eex, lo * eex);
}

// ---- Precise energies (NB_ENERGY_PRECISE) ---------------------------------------------
// The pair energies of water cancel 10^3-10^4-fold in their sums (sum |e_ij| over |E|), so
// the FP32 pair energies leave relative errors of a few 1e-6 on small boxes.  The precise
// evaluation recomputes the energies -- not the forces, which the force-only pair kernel
// gives -- in two-float arithmetic from the coordinate differences on: each difference is
// exact (two_sum of the two image-shifted coordinates), r^2, r, 1/r, erfc and the LJ powers
// carry 1e-14 - 1e-12 relative error (1/r by a Newton step on the hardware reciprocal square
// root, no division), the per-atom sums are two-float and scaled once per atom by
// ke q_i as an exact two-product, and the atom's record is split into hi (e_atom) and lo
// (e_lo) parts that the epilogue adds in FP64.  The differences are taken from the caller's
// positions (the slot-ordered frame positions may carry a rounding from the wrap into the
// box), in the periodic image that the FP32 difference of the list entry names.  The pair
// set is the exact one, r < r_c decided on the two-float r^2 against r_c^2 = rc rc (an exact
// two-product), which is the FP64 oracle's: the FP32 test of the force kernel may put a pair
// within its rounding band of r_c on the other side, and in water one such Coulomb pair at
// r_c (ke q_O q_H erfc(alpha r_c)/r_c ~ 2.4e-3 kJ/mol at alpha r_c = 2.88) already moves a
// box's E_dir by ~1e-6 relative.  So the pass walks the whole row (the back part too, except
// where the system's prune has ruled it out: no pair there can be within r_c).

constexpr float kTwoInvSqrtPi = 1.12837916709551257f;  // 2 / sqrt(pi)

// erfc(x) in two-float, x = x.hi + x.lo >= 0: the piecewise interpolant of erfc_df.cuh at
// x.hi (t = x.hi - k H is exact) plus the Taylor terms in d = x.lo to second order,
// d erfc'(x.hi) (1 - x.hi d) with erfc'(x) = -(2/sqrt(pi)) exp(-x^2) and erfc'' = -2x erfc'
// (|d| <= 2^-24 x.hi: the first-order term is ~1e-6 of erfc and needs FP32 accuracy, a few
// ulp; the second ~2 x^2 d^2 relative, 4e-12 at x = 6; the third is below 1e-18).  Past the
// table (erfc < 2.2e-17) the FP32 erfcf.  tab: the table of erfc_df.cuh, or a copy of it
// in shared memory (lanes of a warp read different intervals).
constexpr int kErfcDfTab = kErfcDfIntervals * (kErfcDfDeg + 1);
__device__ __forceinline__ DF erfc_df(DF x, const float2* tab) {
    const float xh = x.hi;
    if (!(xh < kErfcDfH * (float)kErfcDfIntervals)) return DF{erfcf(xh), 0.f};
    const int k = max(0, min((int)(xh * kErfcDfInvH), kErfcDfIntervals - 1));
    const float t = __fsub_rn(xh, __fmul_rn((float)k, kErfcDfH));
    const float2* c = tab + k * (kErfcDfDeg + 1);
    float2 ck = c[kErfcDfDeg];
    DF p{ck.x, ck.y};
#pragma unroll
    for (int m = kErfcDfDeg - 1; m >= 0; --m) {
        ck = c[m];
        // each step's two terms stay within a factor ~20 of the result (the series alternates
        // at most that much on an interval of 0.25): Dekker's addition is enough
        p = df_add_fast(df_mul_f(p, t), DF{ck.x, ck.y});
    }
    // exp(-x^2) with x^2 = sq.hi + sq.lo: the rounding of x^2 alone would be x^2 2^-24 of
    // the exponent (5e-7 relative at x = 3); expf, as __expf's error also grows with x^2
    const DF sq = two_prod(xh, xh);
    const float d1 = -kTwoInvSqrtPi * expf(-sq.hi) * (1.f - sq.lo);
    return df_add_f(p, __fmul_rn(__fmul_rn(x.lo, d1), fmaf(-xh, x.lo, 1.f)));
}

// The exact two-float difference x_i - x_j of the caller's positions oi, oj in the periodic
// image of the FP32 difference d32 (taken in the frame of the list build): the two differ by
// a whole number n of box lengths along each periodic axis (plus FP32 rounding, far below
// L/2), and n L is subtracted as an exact two-product.
__device__ __forceinline__ void caller_diff_df(const float4& oi, const float4& oj, const float d32[3],
                                               const SysDev& S, DF d[3]) {
    const float a[3] = {oi.x, oi.y, oi.z}, b[3] = {oj.x, oj.y, oj.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        d[k] = two_sum(a[k], -b[k]);
        if (S.periodic) {
            const float n = rintf(__fdiv_rn(__fsub_rn(d[k].hi, d32[k]), S.L[k]));
            if (n != 0.f) d[k] = df_add(d[k], two_prod(-n, S.L[k]));
        }
    }
}

// r^2 < r_c^2 on two-float values (both normalised)
__device__ __forceinline__ bool df_less(DF a, DF b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }

__device__ __forceinline__ DF r2_df(const DF d[3]) {
    return df_add(df_add(df_mul(d[0], d[0]), df_mul(d[1], d[1])), df_mul(d[2], d[2]));
}

// LJ energy of one pair per unit eps_ij in two-float: 4 ((s/r)^12 - (s/r)^6), times the
// switch S(x), x = (r - r_s)/(r_c - r_s), above r_s.
__device__ __forceinline__ DF lj_unit_df(float sig_i, float sig_j, DF r2, const SysDev& S) {
    const DF sig = df_scale(two_sum(sig_i, sig_j), 0.5f);
    const DF rinv = df_rsqrt(r2);
    const DF s2 = df_mul(df_mul(sig, sig), df_mul(rinv, rinv));
    const DF s6 = df_mul(df_mul(s2, s2), s2);
    DF u = df_scale(df_add(df_mul(s6, s6), df_neg(s6)), 4.f);
    if (S.has_switch) {
        const DF r = df_mul(r2, rinv);
        const DF x = df_mul(df_add_f(r, -S.rs), DF{S.inv_sw, S.inv_sw_lo});
        if (x.hi > 0.f) {
            // S = 1 + x^3 (-10 + x (15 - 6 x))
            DF p = df_add_f(df_mul_f(x, -6.f), 15.f);
            p = df_add_f(df_mul(p, x), -10.f);
            const DF sw = df_add_f(df_mul(df_mul(df_mul(p, x), x), x), 1.f);
            u = df_mul(u, sw);
        }
    }
    return u;
}

// Ewald direct-space (EWALD) or reaction-field energy of one pair per unit ke q_i, in
// two-float: q_j erfc(alpha r)/r, or q_j (1/r + k r^2 - c) of Eq. RFA.
template <int COUL>
__device__ __forceinline__ DF coul_unit_df(float qj, DF r2, const SysDev& S, const float2* tab) {
    const DF rinv = df_rsqrt(r2);
    const DF r = df_mul(r2, rinv);
    if (COUL == kCoulEwald) return df_mul_f(df_mul(erfc_df(df_mul_f(r, S.alpha), tab), rinv), qj);
    DF u = df_add(rinv, df_mul(DF{S.krf, S.krf_lo}, r2));
    u = df_add(u, DF{-S.crf, -S.crf_lo});
    return df_mul_f(u, qj);
}

// Exclusion-correction energy of slot i in two-float: half of ke q_i sum_e -q_j erf(alpha r)/r
// (erf = 1 - erfc), each excluded pair's difference from the caller's positions (xo, caller
// order; perm: slot -> caller index) in the minimum image that excl_terms takes.
__device__ __forceinline__ DF excl_energy_df(int i, const SysDev& S, const float4* __restrict__ xs, const ExclView& X,
                                             const float4* __restrict__ xo, const int* __restrict__ perm,
                                             const float2* tab) {
    const float4 xr = xs[i];
    const float4 oi = xo[perm[i]];
    const int ne = X.count(i);
    DF sum{0.f, 0.f};
    for (int e = 0; e < ne; ++e) {
        const int j = X.partner(i, e);
        const float4 xj = xs[j];
        float d32[3] = {xr.x - xj.x, xr.y - xj.y, xr.z - xj.z};
        if (S.periodic) {
            d32[0] = mi_pair(xr.x, xj.x, S.L[0], S.halfL[0]);
            d32[1] = mi_pair(xr.y, xj.y, S.L[1], S.halfL[1]);
            d32[2] = mi_pair(xr.z, xj.z, S.L[2], S.halfL[2]);
        }
        DF d[3];
        caller_diff_df(oi, xo[perm[j]], d32, S, d);
        const DF r2 = r2_df(d);
        const DF rinv = df_rsqrt(r2);
        const DF erf = df_add_f(df_neg(erfc_df(df_mul_f(df_mul(r2, rinv), S.alpha), tab)), 1.f);
        sum = df_add(sum, df_mul_f(df_mul(erf, rinv), -xj.w));  // the charges: xs .w = xq .w
    }
    return df_scale(df_mul(two_prod(S.ke, xr.w), sum), 0.5f);
}

// Precise energies of atom i (one warp): lane l takes entries l, l + 32, ... of the row's
// front and, unless the system's prune has ruled it out, its back; the pair is in if its
// two-float r^2 (caller positions) is below r_c^2; each pair's energy and the sums are
// two-float.  The record: half of E_LJ and of E_dir (or E_RF), hi parts in e_atom, lo parts
// in e_lo.
template <bool LJ, int COUL, int IMG>
__device__ __forceinline__ void energy_df_atom(int i, const AtomHdr& H, const SysDev& S, bool skip_back,
                                               const float4* __restrict__ xs, const float4* __restrict__ xo,
                                               const int* __restrict__ perm, const float2* __restrict__ ps,
                                               const unsigned* __restrict__ nbr, int cap, const ExclView& X,
                                               const float2* tab, float4* __restrict__ e_atom,
                                               float4* __restrict__ e_lo) {
    const int lane = threadIdx.x & 31;
    const PairGeo G = pair_geo(S);
    const float4 xr = H.xr;
    const float2 pi = H.pi;
    const bool do_lj = LJ && pi.y != 0.f;
    const bool do_coul = COUL != kCoulNone && S.ke != 0.f;
    const unsigned* row = nbr + (size_t)i * cap;
    const int n_all = H.nin + (skip_back ? 0 : H.nout);
    const float4 oi = xo[perm[i]];
    const DF rc2 = two_prod(S.rc, S.rc);
    DF elj{0.f, 0.f}, eq{0.f, 0.f};
    for (int e = lane; e < n_all; e += 32) {
        const unsigned ent = e < H.nin ? row[e] : row[cap - H.nout + (e - H.nin)];
        const int j = (int)(ent & kEntrySlotMask);
        const float4 cj = xs[j];
        float d32[3];
        entry_diff<IMG>(xr, cj, ent >> kEntrySlotBits, G, d32[0], d32[1], d32[2]);
        // clearly outside r_c: the FP32 r^2 (relative error ~1e-7, plus the rounding of the
        // wrap of caller positions into the frame, ~1e-6 of r_c^2 for positions within a few
        // box lengths) above r_c^2 (1 + 1e-3)
        if (pair_r2(d32[0], d32[1], d32[2]) > S.rc2 * 1.001f) continue;
        DF d[3];
        caller_diff_df(oi, xo[perm[j]], d32, S, d);
        const DF r2 = r2_df(d);
        if (!df_less(r2, rc2)) continue;
        if (do_lj) {
            const float2 pj = ps[j];
            if (pj.y != 0.f) elj = df_add(elj, df_mul(two_prod(pi.y, pj.y), lj_unit_df(pi.x, pj.x, r2, S)));
        }
        if (do_coul) eq = df_add(eq, coul_unit_df<COUL>(cj.w, r2, S, tab));
    }
    elj = warp_sum_df(elj);
    eq = warp_sum_df(eq);
    if (lane == 0) {
        if (COUL != kCoulNone) eq = df_mul(two_prod(S.ke, xr.w), eq);
        // the exclusion correction's energy record (Ewald systems with excluded partners)
        DF ex{0.f, 0.f};
        if (COUL == kCoulEwald && X.count(i) > 0 && S.alpha > 0.f && S.ke != 0.f)
            ex = excl_energy_df(i, S, xs, X, xo, perm, tab);
        e_atom[i] = make_float4(0.5f * elj.hi, 0.5f * eq.hi, ex.hi, 0.f);
        e_lo[i] = make_float4(0.5f * elj.lo, 0.5f * eq.lo, ex.lo, 0.f);
    }
}

// Precise-energy pass (one warp per atom, the pair kernel's atom ranges), launched after the
// force-only pair kernel of the same evaluation.
template <bool LJ, int COUL>
__global__ void __launch_bounds__(kPairThreads) k_energy_df(
    int N, int per_block, int cap, const int* __restrict__ sid, const SysDev* __restrict__ sys,
    const float4* __restrict__ xs, const float2* __restrict__ ps, const unsigned* __restrict__ nbr,
    const int* __restrict__ cnt, const int* __restrict__ cnt_out, float4* __restrict__ e_atom,
    float4* __restrict__ e_lo, const unsigned* __restrict__ flags, const unsigned* __restrict__ prune_sys,
    const float4* __restrict__ xo, const int* __restrict__ perm, ExclView X) {
    // the erfc table in shared memory: the lanes of a warp read ~a dozen different intervals
    __shared__ float2 tab[kErfcDfTab];
    for (int k = threadIdx.x; k < kErfcDfTab; k += blockDim.x) tab[k] = (&g_erfc_df[0][0])[k];
    __syncthreads();
    pdl_wait();
    const AtomRange R = block_atoms(N, per_block, kPairWarps);
    const bool fresh = flags[NB_FLAG_FRESH] != 0u;
    for (int i = R.i0; i < R.i1; i += R.step) {
        const AtomHdr H = load_hdr(i, sid, xs, ps, nbr, cnt, cnt_out, cap);
        const SysDev& S = sys[H.sys];
        // a pruned row's back holds no pair within r_c (its front: all within r_c + the prune skin)
        const bool skip_back = !fresh && prune_sys && (prune_sys[H.sys] & kPruned) != 0u && S.rin2 > 0.f;
        const int mode = img_mode(H, pair_geo(S));
        if (mode == kImgPlain)
            energy_df_atom<LJ, COUL, kImgPlain>(i, H, S, skip_back, xs, xo, perm, ps, nbr, cap, X, tab, e_atom, e_lo);
        else if (mode == kImgCode)
            energy_df_atom<LJ, COUL, kImgCode>(i, H, S, skip_back, xs, xo, perm, ps, nbr, cap, X, tab, e_atom, e_lo);
        else
            energy_df_atom<LJ, COUL, kImgFold>(i, H, S, skip_back, xs, xo, perm, ps, nbr, cap, X, tab, e_atom, e_lo);
    }
}

// Exclusion correction, one thread per atom (slot order), after the pair kernel: the
// force is added as fixed point (ffix is an integer sum, so the order against the pair
// kernel's and the PME gather's adds is irrelevant); the energy (per unit ke q_i, scaled by
// ke q_i as hi + lo) goes to e_atom[i].z, which the pair kernel wrote as 0.  VJP:
// J (lam_i - lam_j) and the charge gradient are added to gx_s[i].
template <bool VJP>
__global__ void k_excl(int N, const int* __restrict__ sid, const SysDev* __restrict__ sys,
                       const float4* __restrict__ xs, const float4* __restrict__ lam, ExclView X,
                       long long* __restrict__ ffix, float4* __restrict__ e_atom, float4* __restrict__ gx_s,
                       float scale, unsigned* flags, int write_energy) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const SysDev& S = sys[sid[i]];  // a system owns the same index range in slot and caller order
    float fx, fy, fz, eex, gx, gy, gz, gq;
    if (!excl_terms<VJP>(i, S, xs, lam, X, fx, fy, fz, eex, gx, gy, gz, gq)) return;
    red_add(ffix + i, to_fix(fx, scale, flags + 1));
    red_add(ffix + (size_t)N + i, to_fix(fy, scale, flags + 1));
    red_add(ffix + 2 * (size_t)N + i, to_fix(fz, scale, flags + 1));
    // (precise energies: the two-float pass has written the record)
    if (write_energy) reinterpret_cast<float*>(e_atom + i)[2] = excl_energy_half(S.ke, xs[i].w, eex);
    if (VJP) {
        float4 g = gx_s[i];
        g.x += gx;
        g.y += gy;
        g.z += gz;
        g.w += gq;
        gx_s[i] = g;
    }
}

// The end of a force evaluation (nonbonded_forces) in one launch, over the tiles of the
// energy reduction (reduce.cuh; blocks of kRedThreads threads, red_tile atoms of one system,
// slot order): per atom, the exclusion correction of k_excl (do_excl), the force output in
// caller order (f_out: the fixed-point sum of the pair kernel, the PME gather and the
// correction, converted as k_finalize does) and, with dst, the energy sums of
// k_reduce_energy, with the correction's energy record taken from registers.  The same
// integers are added and the same FP64 sums formed in the same order as by the three
// separate kernels, so the results are bitwise theirs; two launches fewer on the step's
// critical path.
__global__ void __launch_bounds__(kRedThreads) k_epilogue(
    int N, int n_sys, const int* __restrict__ blk_sys, const int* __restrict__ blk_off,
    const SysDev* __restrict__ sys, const float4* __restrict__ xs, ExclView X, int do_excl,
    const long long* __restrict__ ffix, const int* __restrict__ perm, float scale, float finv,
    float* __restrict__ f_out, const float4* __restrict__ e_atom, const float4* __restrict__ e_lo,
    const float4* __restrict__ xo, double* __restrict__ part,
    const double* __restrict__ e_pme_blk, const int* __restrict__ pme_blk_off, int terms,
    unsigned* __restrict__ ticket, double* __restrict__ dst, unsigned* flags) {
    pdl_wait();
    int a0, a1;
    red_tile_range(blk_sys, blk_off, sys, a0, a1);
    const SysDev& S = sys[blk_sys[blockIdx.x]];
    double v[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int k = a0 + threadIdx.x; k < a1; k += kRedThreads) {
        float fx = 0.f, fy = 0.f, fz = 0.f, ez = 0.f;
        bool has_excl = false;
        if (do_excl) {
            float eex, gx, gy, gz, gq;
            has_excl = excl_terms<false>(k, S, xs, nullptr, X, fx, fy, fz, eex, gx, gy, gz, gq);
            if (has_excl) ez = excl_energy_half(S.ke, xs[k].w, eex);
        }
        if (f_out) {
            long long F0 = ffix[k], F1 = ffix[(size_t)N + k], F2 = ffix[2 * (size_t)N + k];
            if (has_excl) {
                F0 += to_fix(fx, scale, flags + 1);
                F1 += to_fix(fy, scale, flags + 1);
                F2 += to_fix(fz, scale, flags + 1);
            }
            const size_t o = 3 * (size_t)perm[k];
            f_out[o] = __ll2float_rn(F0) * finv;
            f_out[o + 1] = __ll2float_rn(F1) * finv;
            f_out[o + 2] = __ll2float_rn(F2) * finv;
        }
        if (dst) {
            const float4 e = e_atom[k];
            const float q = xs[k].w;
            if (e_lo) {  // precise energies: hi + lo of the pair records, the correction's in two-float
                const float4 l = e_lo[k];
                v[0] += (double)e.x + (double)l.x;
                v[1] += (double)e.y + (double)l.y;
                v[2] += (double)e.z + (double)l.z;  // the two-float pass's exclusion energy
            } else {
                v[0] += e.x;
                v[1] += e.y;
                v[2] += has_excl ? ez : e.z;
            }
            v[3] += (double)q * q;
        }
    }
    if (dst)
        energy_reduce_finish(v, n_sys, blk_off, sys, 0, part, e_pme_blk, pme_blk_off, terms, ticket, dst, StepStat());
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

// Atoms per block of the pair and VJP kernels: kAtomsPerWarp per warp, fewer when the
// handle is too small to give every SM a few blocks; with `wide`, four per warp when the
// grid still holds at least eight waves of four blocks per SM (LJ 256k: pair kernel 136.9 ->
// 128.8 us fresh, 182.2 -> 171.9 us kept; the 24,000-atom water box, at 1.3 waves with four,
// keeps two: 58.2 against 64.9 us).
static int pair_atoms_per_block(const nb_handle* h, int warps, bool wide = false) {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long n = h->n_atoms;
    if (wide && n >= (long long)warps * 4 * 4LL * sms * 8) return warps * 4;
    const long long full = (long long)warps * kAtomsPerWarp;
    if (n >= full * 4LL * sms) return (int)full;
    return warps;
}

template <bool LJ, int COUL>
static void pair_launch(nb_handle* h, cudaStream_t st, bool vjp, bool energy, bool defer_excl, bool precise) {
    const int N = h->n_atoms;
    if (vjp) {
        const int pb = pair_atoms_per_block(h, kVjpWarps);
        if (COUL == kCoulNone && LJ && pb >= 2 * kVjpWarps)  // LJ only: two atoms per warp, bitwise the same
            launch_pdl(k_vjp2<LJ>, cdiv(N, pb), kVjpThreads, 0, st, N, pb, h->cap, h->sid, h->sys, h->xs, h->ps,
                       h->lam, h->nbr, h->nbr_cnt, h->nbr_out, h->gx_s, h->gp_s, h->ffix, h->e_atom, h->fscale,
                       h->flags, (const unsigned*)h->prune_sys);
        else
            launch_pdl(k_vjp<LJ, COUL>, cdiv(N, pb), kVjpThreads, 0, st, N, pb, h->cap, h->sid, h->sys, h->xs,
                       h->ps, h->lam, h->nbr, h->nbr_cnt, h->nbr_out, h->gx_s, h->gp_s, h->ffix, h->e_atom, h->fscale,
                       h->flags, (const unsigned*)h->prune_sys);
    } else {
        const int pb = pair_atoms_per_block(h, kPairWarps, true);
        // LJ only: two atoms per warp, bitwise the same results; not on handles too small to
        // give every SM a few blocks of two atoms per warp (LJ 864: a warp per atom keeps
        // twice the warps busy, 91 against 84 thousand MD steps/s)
        if (COUL == kCoulNone && pb >= 2 * kPairWarps)
            launch_pdl(energy ? k_pair2<LJ, true> : k_pair2<LJ, false>, cdiv(N, pb), kPairThreads, 0, st, N, pb,
                       h->cap, h->sid, h->sys, h->xs, h->ps, h->nbr, h->nbr_cnt, h->nbr_out, h->ffix, h->e_atom,
                       h->fscale, h->flags, (const unsigned*)h->prune_sys);
        else if (LJ && COUL != kCoulNone && h->any_uncharged && pb >= 2 * kPairWarps)
            launch_pdl(energy ? k_pair<LJ, COUL, true, true> : k_pair<LJ, COUL, false, true>, cdiv(N, pb),
                       kPairThreads, 0, st, N, pb, h->cap, h->sid, h->sys, h->xs, h->ps, h->nbr, h->nbr_cnt,
                       h->nbr_out, h->ffix, h->e_atom, h->fscale, h->flags, (const unsigned*)h->prune_sys);
        else
            launch_pdl(energy ? k_pair<LJ, COUL, true, false> : k_pair<LJ, COUL, false, false>, cdiv(N, pb),
                       kPairThreads, 0, st, N, pb, h->cap, h->sid, h->sys, h->xs, h->ps, h->nbr, h->nbr_cnt,
                       h->nbr_out, h->ffix, h->e_atom, h->fscale, h->flags, (const unsigned*)h->prune_sys);
        if (precise)
            launch_pdl(k_energy_df<LJ, COUL>, cdiv(N, pb), kPairThreads, 0, st, N, pb, h->cap, h->sid, h->sys, h->xs,
                       h->ps, h->nbr, h->nbr_cnt, h->nbr_out, h->e_atom, h->e_lo, (const unsigned*)h->flags,
                       (const unsigned*)h->prune_sys, h->xq_in, (const int*)h->perm, excl_view(h));
    }
    if (COUL == kCoulEwald && h->excl_w && !(defer_excl && !vjp)) {
        const ExclView X = excl_view(h);
        if (vjp)
            launch_pdl(k_excl<true>, cdiv(N, 128), 128, 0, st, N, h->sid, h->sys, h->xs, h->lam, X, h->ffix,
                       h->e_atom, h->gx_s, h->fscale, h->flags, 1);
        else
            launch_pdl(k_excl<false>, cdiv(N, 128), 128, 0, st, N, h->sid, h->sys, h->xs, (const float4*)nullptr, X,
                       h->ffix, h->e_atom, (float4*)nullptr, h->fscale, h->flags, precise ? 0 : 1);
    }
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
        if (!vjp && (terms & kTermPrecise)) cudaMemsetAsync(h->e_lo, 0, sizeof(float4) * N, st);
        if (vjp) {
            cudaMemsetAsync(h->gx_s, 0, sizeof(float4) * N, st);
            cudaMemsetAsync(h->gp_s, 0, sizeof(float2) * N, st);
        }
        return;
    }
    // precise energies: the force-only pair kernel, then the two-float energy pass (only
    // where energies are asked for; other evaluations of a precise call run as usual)
    const bool pe = !vjp && (terms & kTermPrecise) != 0 && (terms & kTermEnergy) != 0;
    const bool en = vjp || ((terms & kTermEnergy) != 0 && !pe);
    const bool df = (terms & kTermDeferExcl) != 0;
    if (lj && coul && rf) pair_launch<true, kCoulRF>(h, st, vjp, en, df, pe);
    else if (lj && coul) pair_launch<true, kCoulEwald>(h, st, vjp, en, df, pe);
    else if (lj) pair_launch<true, kCoulNone>(h, st, vjp, en, df, pe);
    else if (coul && rf) pair_launch<false, kCoulRF>(h, st, vjp, en, df, pe);
    else pair_launch<false, kCoulEwald>(h, st, vjp, en, df, pe);
}

// The exclusion correction runs in the epilogue (not after the pair kernel) exactly when
// the pair kernel would have been followed by k_excl: Ewald electrostatics on a handle with
// exclusions and the Coulomb term selected.
bool epilogue_has_excl(const nb_handle* h, int terms) {
    return (terms & NB_TERM_COUL) && h->any_coul && h->coul_kind != kCoulRF && h->excl_w;
}

void launch_epilogue(nb_handle* h, int terms, float* f_out, double* dst, cudaStream_t st, bool precise) {
    const ExclView X = excl_view(h);
    launch_pdl(k_epilogue, h->n_red_blocks, kRedThreads, 0, st, h->n_atoms, h->n_sys, h->red_blk_sys,
               h->red_blk_off, h->sys, h->xs, X, epilogue_has_excl(h, terms) ? 1 : 0, h->ffix, h->perm, h->fscale,
               h->finv, f_out, h->e_atom, (precise && dst) ? h->e_lo : nullptr, h->xq_in, h->red_part, h->e_pme_blk, h->conv_blk_off, terms, h->red_ticket, dst,
               h->flags);
}

void launch_pair(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, false); }
void launch_vjp(nb_handle* h, int terms, cudaStream_t st) { dispatch(h, terms, st, true); }

cudaError_t pair_setup(nb_handle* h) {
    h->split_pair = 1;
    return cudaSuccess;
}

}  // namespace nb

namespace nb {
namespace {
__global__ void k_erfc_eval(int n, const float* __restrict__ x, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = erfc_with_exp(x[i], exp_neg_sq(x[i]));
}
__global__ void k_erfc_df_eval(int n, const float* __restrict__ xh, const float* __restrict__ xl,
                               float* __restrict__ oh, float* __restrict__ ol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DF e = erfc_df(DF{xh[i], xl[i]}, &g_erfc_df[0][0]);
    oh[i] = e.hi;
    ol[i] = e.lo;
}
}  // namespace
}  // namespace nb

extern "C" nb_status nb_erfc_eval(const float* x, float* out, int32_t n, void* stream) {
    if (n < 0 || (n > 0 && (!x || !out))) return NB_ERR_ARG;
    if (n == 0) return NB_OK;
    nb::k_erfc_eval<<<nb::cdiv(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, x, out);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}

extern "C" nb_status nb_erfc_df_eval(const float* x_hi, const float* x_lo, float* out_hi, float* out_lo, int32_t n,
                                     void* stream) {
    if (n < 0 || (n > 0 && (!x_hi || !x_lo || !out_hi || !out_lo))) return NB_ERR_ARG;
    if (n == 0) return NB_OK;
    nb::k_erfc_df_eval<<<nb::cdiv(n, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(n, x_hi, x_lo, out_hi,
                                                                                        out_lo);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ERR_CUDA;
}
