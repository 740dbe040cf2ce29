// cell.cuh -- the cell tile of the list build: one block per cell stages the cell's
// stencil (Sec. 2.1.2 "Neighborlists": the 27-cell, or 125-cell for half-width cells,
// neighbourhood) in shared memory.
//
// The stencil is listed as runs of consecutive cells along x; each run is one contiguous
// slot range (slot order is sorted by cell).  Concatenating the runs gives the cell's
// candidate array; the Verlet list stores, for every atom, its partners' slots together
// with the image code of the run each came from, so that the pair kernels read partners
// from the slot-ordered arrays without a stencil of their own.
//
// Images.  Along an axis with a stencil (nc >= 2 st + 1) the unwrapped cell index of a run
// fixes the image, which is the minimum image of every pair within r_nl.  A run from
// below the first cell (index < 0) is moved down by L: xj - L is exact because xj >= L/2.
// A run from beyond the last cell (index >= nc) is met by moving the atom down instead.
// When nc >= 4 st that is done once for the block: the cell's atoms and all candidates
// that did not wrap are moved down by L, every shift exact since all of them lie above
// L/2; otherwise the shift rides with the candidate as a flag and the atom side is chosen
// per pair.  Axes without a stencil (nc <= 2 st) fold per pair.  Between rebuilds the
// positions stay in the frame of the last build (build position plus minimum-image
// displacement, never re-wrapped), so the images chosen at the build remain those of
// every pair that can come within r_c.
#pragma once
#include <climits>

#include "common.cuh"

namespace nb {

constexpr int kMaxRuns = 64;  // (2*2+1)^2 rows x 2 runs (periodic wrap) at most 50
constexpr float kFar = 1.0e18f;

struct BuildRun {
    int slot0;  // first slot of the run
    int sm0;    // offset of the run in the concatenated candidate array
    int n;      // candidates in the run
    int flags;  // per-pair image: bit d = atom moves down by L on axis d
    float s[3]; // shift added to the candidates' coordinates
    unsigned code;  // the run's image code of a list entry (common.cuh), shifted to its place
};

struct CellCtx {
    int i0, i1;            // slot range of the cell's atoms
    int nc[3], cc[3], st;  // cells per axis, this cell's coordinates, stencil half-width
    bool per;
    bool all[3];           // axis without a stencil: every cell visited once
    bool fold[3];          // per-pair minimum image along this axis
    bool frame[3];         // block frame moved down by L along this axis
    bool gen;              // some axis needs per-pair images
    float L[3], hL[3];
    float fs[3];           // shift of the cell's own atoms
};

__device__ __forceinline__ CellCtx cell_ctx(int c, const SysDev& S, const int* __restrict__ start) {
    CellCtx C;
    C.i0 = start[c];
    C.i1 = start[c + 1];
    C.st = S.stencil;
    C.per = S.periodic != 0;
    const int lc = c - S.cell_off;
    C.nc[0] = S.nc[0];
    C.nc[1] = S.nc[1];
    C.nc[2] = S.nc[2];
    C.cc[0] = lc % C.nc[0];
    C.cc[1] = (lc / C.nc[0]) % C.nc[1];
    C.cc[2] = lc / (C.nc[0] * C.nc[1]);
    bool gen = false;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        C.all[d] = C.nc[d] <= 2 * C.st;
        C.fold[d] = C.per && C.all[d];
        const bool top = C.per && !C.all[d] && C.cc[d] >= C.nc[d] - C.st;
        gen = gen || C.fold[d] || (top && C.nc[d] < 4 * C.st);
        C.frame[d] = top;
        C.L[d] = S.L[d];
        C.hL[d] = S.halfL[d];
    }
    C.gen = gen;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        C.frame[d] = C.frame[d] && !gen;
        C.fs[d] = C.frame[d] ? -C.L[d] : 0.f;
    }
    return C;
}

// Image of a run along one axis with unwrapped cell index u.
__device__ __forceinline__ void run_image(int u, int nc, bool fold, bool frame, float L, int bit, float& s,
                                          int& fl) {
    s = 0.f;
    if (fold || u == INT_MIN) return;
    if (u < 0) s = -L;
    else if (u >= nc) {
        if (!frame) fl |= bit;
    } else if (frame) {
        s = -L;
    }
}

// Image code bits of a run along one axis with unwrapped cell index u: below the first
// cell the partner moves down by L, beyond the last the atom does (folded axes: none).
__device__ __forceinline__ unsigned run_code(int u, int nc, bool fold, int d) {
    if (fold || u == INT_MIN) return 0u;
    if (u < 0) return 2u << (2 * d);
    if (u >= nc) return 1u << (2 * d);
    return 0u;
}

// The stencil runs of the cell, computed by one warp: lane l handles stencil row l (at
// most 25 rows), giving 0-2 runs.  Writes runs[], *n_runs and *n_cand (shared).
__device__ __forceinline__ void cell_runs(const CellCtx& C, const SysDev& S, const int* __restrict__ start,
                                          BuildRun* runs, int* n_runs, int* n_cand, unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const int nc0 = C.nc[0], nc1 = C.nc[1], nc2 = C.nc[2], st = C.st;
    const bool xall = C.all[0], yall = C.all[1], zall = C.all[2];
    const int nz = zall ? nc2 : 2 * st + 1, ny = yall ? nc1 : 2 * st + 1;
    const int nrows = nz * ny;  // <= 32 for stencil <= 2
    int nseg = 0, seg_lo[2] = {0, 0}, seg_hi[2] = {0, 0}, row = 0, yu = INT_MIN, zu = INT_MIN;
    if (lane < nrows) {
        int iz = lane / ny, iy = lane % ny;
        bool ok = true;
        int z = iz, y = iy;
        if (!zall) {
            zu = C.cc[2] + iz - st;
            if (!C.per && (zu < 0 || zu >= nc2)) ok = false;
            z = zu < 0 ? zu + nc2 : (zu >= nc2 ? zu - nc2 : zu);
        }
        if (!yall) {
            yu = C.cc[1] + iy - st;
            if (!C.per && (yu < 0 || yu >= nc1)) ok = false;
            y = yu < 0 ? yu + nc1 : (yu >= nc1 ? yu - nc1 : yu);
        }
        if (ok) {
            row = S.cell_off + (z * nc1 + y) * nc0;
            int lo = xall ? 0 : C.cc[0] - st, hi = xall ? nc0 - 1 : C.cc[0] + st;
            if (!xall && !C.per) {
                lo = max(lo, 0);
                hi = min(hi, nc0 - 1);
            }
            if (xall || (lo >= 0 && hi < nc0)) {
                seg_lo[0] = lo; seg_hi[0] = hi; nseg = 1;
            } else if (lo < 0) {
                seg_lo[0] = lo; seg_hi[0] = -1; seg_lo[1] = 0; seg_hi[1] = hi; nseg = 2;
            } else {
                seg_lo[0] = lo; seg_hi[0] = nc0 - 1; seg_lo[1] = nc0; seg_hi[1] = hi; nseg = 2;
            }
        }
    }
    int slot0[2] = {0, 0}, nn[2] = {0, 0};
    for (int g = 0; g < nseg; ++g) {
        int x0 = seg_lo[g], x1 = seg_hi[g];
        int xw0 = x0 < 0 ? x0 + nc0 : (x0 >= nc0 ? x0 - nc0 : x0);
        slot0[g] = start[row + xw0];
        nn[g] = start[row + xw0 + (x1 - x0) + 1] - slot0[g];
    }
    // exclusive prefix over lanes of run counts and candidate counts
    int myruns = nseg, mycand = nn[0] + nn[1];
    int rpre = myruns, cpre = mycand;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int ra = __shfl_up_sync(0xffffffffu, rpre, o), ca = __shfl_up_sync(0xffffffffu, cpre, o);
        if (lane >= o) {
            rpre += ra;
            cpre += ca;
        }
    }
    int rtot = __shfl_sync(0xffffffffu, rpre, 31), ctot = __shfl_sync(0xffffffffu, cpre, 31);
    rpre -= myruns;
    cpre -= mycand;
    for (int g = 0; g < nseg; ++g) {
        int r = rpre + g;
        if (r >= kMaxRuns) break;
        BuildRun R;
        R.slot0 = slot0[g];
        R.sm0 = cpre + (g ? nn[0] : 0);
        R.n = nn[g];
        R.flags = 0;
        run_image(xall ? INT_MIN : seg_lo[g], nc0, C.fold[0], C.frame[0], C.L[0], 1, R.s[0], R.flags);
        run_image(yu, nc1, C.fold[1], C.frame[1], C.L[1], 2, R.s[1], R.flags);
        run_image(zu, nc2, C.fold[2], C.frame[2], C.L[2], 4, R.s[2], R.flags);
        R.code = (run_code(xall ? INT_MIN : seg_lo[g], nc0, C.fold[0], 0) | run_code(yu, nc1, C.fold[1], 1) |
                  run_code(zu, nc2, C.fold[2], 2)) << kEntrySlotBits;
        runs[r] = R;
    }
    if (lane == 0) {
        *n_runs = min(rtot, kMaxRuns);
        *n_cand = ctot;
        if (rtot > kMaxRuns) atomicOr(&flags[1], NB_DEVERR_LIST_OVERFLOW);
    }
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Slot of candidate k of the stencil (binary search over the runs).
__device__ __forceinline__ int run_of(const BuildRun* runs, int nr, int k) {
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (runs[mid].sm0 <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Squared distance of a pair from its difference vector.  The list build and the pair
// kernels both use this one function (same operations, same order), so a pair that the
// build found inside r_c has, from the same positions, the same r^2 in the pair kernels.
__device__ __forceinline__ float pair_r2(float dx, float dy, float dz) { return fmaf(dz, dz, fmaf(dy, dy, dx * dx)); }

// Per-pair difference for GEN cells: flagged axes move the atom down by L, folded axes
// take the minimum image of the raw coordinates.
__device__ __forceinline__ float gen_diff(float xi, float xj, int fl, int bit, bool fold, float L, float hL) {
    return fold ? mi_pair(xi, xj, L, hL) : ((fl & bit) ? xi - L : xi) - xj;
}

// Periodic geometry of a system as the list entries need it.
struct PairGeo {
    float L[3], hL[3];
    bool fold[3];  // axis with fewer cells than the stencil spans: per-pair minimum image
};

__device__ __forceinline__ PairGeo pair_geo(const SysDev& S) {
    PairGeo G;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        G.L[d] = S.L[d];
        G.hL[d] = S.halfL[d];
        G.fold[d] = S.periodic && S.nc[d] <= 2 * S.stencil;
    }
    return G;
}

// Image handling of an atom's row (warp-uniform): plain differences, image codes, or image
// codes with the minimum image on folded axes (systems with fewer cells than the stencil).
constexpr int kImgPlain = 0;
constexpr int kImgCode = 1;
constexpr int kImgFold = 2;

// x_i - x_j of a list entry: image code bit 2d (x_i moves down by L) and bit 2d + 1 (x_j
// moves down by L), each shift exact (the moved coordinate lies above L/2), or the minimum
// image on folded axes.  The list build computed the same difference for its test.
template <int IMG>
__device__ __forceinline__ void entry_diff(const float4& xr, const float4& cj, unsigned code, const PairGeo& G,
                                           float& dx, float& dy, float& dz) {
    if (IMG == kImgPlain) {
        dx = xr.x - cj.x;
        dy = xr.y - cj.y;
        dz = xr.z - cj.z;
        return;
    }
    const float xi[3] = {xr.x, xr.y, xr.z}, xj[3] = {cj.x, cj.y, cj.z};
    float d[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (IMG == kImgFold && G.fold[k]) {
            d[k] = mi_pair(xi[k], xj[k], G.L[k], G.hL[k]);
        } else {
            const float a = (code >> (2 * k)) & 1u ? xi[k] - G.L[k] : xi[k];
            const float b = (code >> (2 * k + 1)) & 1u ? xj[k] - G.L[k] : xj[k];
            d[k] = a - b;
        }
    }
    dx = d[0];
    dy = d[1];
    dz = d[2];
}


}  // namespace nb
