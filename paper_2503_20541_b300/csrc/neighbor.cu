// neighbor.cu -- cell list + Verlet neighbour list (Sec. 2.1.2 "Neighborlists").
//
// Every evaluation starts with k_load: scatter the caller's positions into slot
// order and test the list's validity (an atom moved more than r_skin/2 since the
// last build).  The rebuild chain (bin -> scan -> scatter -> in-cell sort ->
// Verlet build) is always launched but each kernel returns at once unless the
// device-side rebuild flag is set, so a step never waits on the host and the
// whole sequence can be captured in a CUDA graph.  The last block of the Verlet
// build counts the rebuild and clears the flag.
//
// The sort is a counting sort by (system, cell) followed by a rank sort inside
// each cell on the caller index, so the slot order -- and with it the list and
// every FP32 summation order downstream -- depends only on the positions.
#include "cell.cuh"

namespace nb {

// Positions stay in the frame of the last build: slot k holds its wrapped build
// position plus the minimum-image displacement since the build, never re-wrapped, so the
// stencil images chosen at the build stay valid until the next one.
// It also zeroes the fixed-point force array, into which the pair kernel and the PME
// gather of this evaluation add.
__global__ void k_load(int N, const float4* __restrict__ xq, const int* __restrict__ iperm,
                       const int* __restrict__ sid, const SysDev* __restrict__ sys,
                       const float4* __restrict__ xref, const float4* __restrict__ xsb, float4* __restrict__ xs,
                       long long* __restrict__ ffix, const float4* __restrict__ x_prune,
                       unsigned* __restrict__ prune_sys, unsigned* flags) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) flags[NB_FLAG_FRESH] = 0u;  // the positions may differ from the build's from here on
    bool need = false, pr = false;
    if (i < N) {
        ffix[i] = 0;
        ffix[(size_t)N + i] = 0;
        ffix[2 * (size_t)N + i] = 0;
        need = load_atom(xq[i], sys[sid[i]], xref[i], xsb, xs, iperm[i], x_prune, x_prune ? &pr : nullptr);
    }
    if (__any_sync(0xffffffffu, need) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1u);
    if (x_prune) request_prune(0xffffffffu, pr, i < N ? sid[i] : 0, prune_sys, flags);
}

__device__ __forceinline__ int cell_coord(float w, float scale, int nc) {
    int c = (int)(w * scale);
    return min(max(c, 0), nc - 1);
}

__device__ __forceinline__ void bin_atom(int i, const float4* __restrict__ xq, const int* __restrict__ sid,
                                         const SysDev* __restrict__ sys, int* __restrict__ cellid, int* cell_count,
                                         unsigned* flags) {
    float4 p = xq[i];
    const SysDev& S = sys[sid[i]];
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) {
        atomicOr(&flags[1], NB_DEVERR_NONFINITE);
        p.x = p.y = p.z = 0.f;
    }
    if (S.periodic) {
        p.x = wrap1(p.x, S.L[0], S.invL[0]);
        p.y = wrap1(p.y, S.L[1], S.invL[1]);
        p.z = wrap1(p.z, S.L[2], S.invL[2]);
    }
    int cx = cell_coord(p.x, S.cell_scale[0], S.nc[0]);
    int cy = cell_coord(p.y, S.cell_scale[1], S.nc[1]);
    int cz = cell_coord(p.z, S.cell_scale[2], S.nc[2]);
    int c = S.cell_off + (cz * S.nc[1] + cy) * S.nc[0] + cx;
    cellid[i] = c;
    atomicAdd(&cell_count[c], 1);
}

__device__ __forceinline__ void scan_any_body(int n, const int* count, int* start, int* cursor, int* zero);

// With scan != 0 (a grid of at most kScanTile cells) the last block to finish binning (a
// ticket counter behind a fence, reset by that block) also performs the exclusive scan of
// the cell counts (the work of k_scan_single), one launch fewer in the rebuild chain.
__device__ __forceinline__ void bin_then_scan(int n_cells, int* cell_count, int* start, int* cursor,
                                              unsigned* ticket) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    scan_any_body(n_cells, cell_count, start, cursor, cell_count);
    if (threadIdx.x == 0) *ticket = 0u;
}

__global__ void k_bin(int N, const float4* __restrict__ xq, const int* __restrict__ sid,
                      const SysDev* __restrict__ sys, int* __restrict__ cellid, int* cell_count,
                      int scan, int n_cells, int* start, int* cursor, unsigned* ticket, unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) bin_atom(i, xq, sid, sys, cellid, cell_count, flags);
    if (scan) bin_then_scan(n_cells, cell_count, start, cursor, ticket);
}

// The load of an evaluation whose list is rebuilt in any case (a forced rebuild): the
// validity test and the slot positions of k_load would be discarded by the re-slotting, so
// this kernel only zeroes the fixed-point forces, clears the fresh-list flag and bins the
// atoms (k_bin; with scan != 0 also the scan).  The rebuild request is already set.
__global__ void k_load_bin(int N, const float4* __restrict__ xq, const int* __restrict__ sid,
                           const SysDev* __restrict__ sys, int* __restrict__ cellid, int* cell_count,
                           long long* __restrict__ ffix, int scan, int n_cells, int* start, int* cursor,
                           unsigned* ticket, unsigned* flags) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) flags[NB_FLAG_FRESH] = 0u;
    if (i < N) {
        ffix[i] = 0;
        ffix[(size_t)N + i] = 0;
        ffix[2 * (size_t)N + i] = 0;
        bin_atom(i, xq, sid, sys, cellid, cell_count, flags);
    }
    if (scan) bin_then_scan(n_cells, cell_count, start, cursor, ticket);
}

// Block-wide exclusive scan of one int per thread (1024 threads); returns the block total.
__device__ __forceinline__ int block_exscan(int v, int* total) {
    __shared__ int warp_tot[32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
        int t = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        int s = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_tot[lane] = s - t;
        if (lane == 31) *total = s;
    }
    __syncthreads();
    int r = warp_tot[w] + x - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(1024) k_scan_a(int n, const int* __restrict__ count, int* start,
                                                  int* bsum, const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    __shared__ int tot;
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? count[base + k] : 0;
        s += v[k];
    }
    int pre = block_exscan(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) start[base + k] = pre;
        pre += v[k];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_b(int nb, int n, int* bsum, int* start,
                                                  const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    __shared__ int tot;
    int carry = 0;
    for (int b0 = 0; b0 < nb; b0 += 1024) {
        int idx = b0 + threadIdx.x;
        int v = idx < nb ? bsum[idx] : 0;
        int pre = block_exscan(v, &tot);
        if (idx < nb) bsum[idx] = pre + carry;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) start[n] = carry;
}

__global__ void __launch_bounds__(1024) k_scan_c(int n, int* start, const int* __restrict__ bsum,
                                                  int* count, int* cursor, const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    int off = bsum[blockIdx.x];
    int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        int idx = base + k;
        if (idx < n) {
            start[idx] += off;
            count[idx] = 0;
            cursor[idx] = 0;
        }
    }
}

// All three scan steps in one block of 1024 threads, for grids of at most kScanTile cells.
__device__ __forceinline__ void scan_single_body(int n, int* count, int* start, int* cursor) {
    __shared__ int tot;
    int base = threadIdx.x * kScanItems;
    int v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? count[base + k] : 0;
        s += v[k];
    }
    int pre = block_exscan(s, &tot);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) {
            start[base + k] = pre;
            count[base + k] = 0;
            cursor[base + k] = 0;
        }
        pre += v[k];
    }
    if (threadIdx.x == 0) start[n] = tot;
}

// The same scan by one block of any multiple of 32 threads: thread t takes a contiguous run
// of ceil(n / blockDim) cells.  The counts are read through L2 (they were summed there by
// other blocks' atomics) and zeroed with the cursors.
__device__ __forceinline__ void scan_any_body(int n, const int* count, int* start, int* cursor, int* zero) {
    __shared__ int tot;
    const int per = (n + (int)blockDim.x - 1) / (int)blockDim.x;
    const int b = threadIdx.x * per, e = min(n, b + per);
    int s = 0;
    for (int k = b; k < e; ++k) s += __ldcg(count + k);
    int pre = block_exscan(s, &tot);
    for (int k = b; k < e; ++k) {
        const int c = __ldcg(count + k);
        start[k] = pre;
        zero[k] = 0;
        cursor[k] = 0;
        pre += c;
    }
    if (threadIdx.x == 0) start[n] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_single(int n, int* count, int* start, int* cursor,
                                                       const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    scan_single_body(n, count, start, cursor);
}

__global__ void k_scatter(int N, const int* __restrict__ cellid, const int* __restrict__ start,
                          int* cursor, int* __restrict__ perm_tmp, const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = cellid[i];
    perm_tmp[start[c] + atomicAdd(&cursor[c], 1)] = i;
}

// Atom i at slot `slot`: its permutation entries, reference and slot positions (wrapped
// into the box) and parameters.
__device__ __forceinline__ void place_atom(int i, int slot, const float4* __restrict__ xq,
                                           const float2* __restrict__ params, const int* __restrict__ sid,
                                           const SysDev* __restrict__ sys, int* __restrict__ perm,
                                           int* __restrict__ iperm, float4* __restrict__ xs,
                                           float4* __restrict__ xsb, float2* __restrict__ ps,
                                           float4* __restrict__ xref) {
    perm[slot] = i;
    iperm[i] = slot;
    float4 p = xq[i];
    xref[i] = p;
    const SysDev& S = sys[sid[i]];
    if (!(isfinite(p.x) && isfinite(p.y) && isfinite(p.z))) p.x = p.y = p.z = 0.f;
    if (S.periodic) {
        p.x = wrap1(p.x, S.L[0], S.invL[0]);
        p.y = wrap1(p.y, S.L[1], S.invL[1]);
        p.z = wrap1(p.z, S.L[2], S.invL[2]);
    }
    xs[slot] = p;
    xsb[slot] = p;
    ps[slot] = params[i];
}

// Atoms of cell w (one warp) in caller-index order, and their slot data.
__device__ __forceinline__ void sort_cell(int w, const int* __restrict__ start, const int* __restrict__ perm_tmp,
                                          const float4* __restrict__ xq, const float2* __restrict__ params,
                                          const int* __restrict__ sid, const SysDev* __restrict__ sys,
                                          int* __restrict__ perm, int* __restrict__ iperm, float4* __restrict__ xs,
                                          float4* __restrict__ xsb, float2* __restrict__ ps,
                                          float4* __restrict__ xref) {
    const int lane = threadIdx.x & 31;
    const int b = start[w], m = start[w + 1] - b;
    for (int a = lane; a < m; a += 32) {
        const int i = perm_tmp[b + a];
        int rank = 0;
        for (int t = 0; t < m; ++t) rank += (perm_tmp[b + t] < i);
        place_atom(i, b + rank, xq, params, sid, sys, perm, iperm, xs, xsb, ps, xref);
    }
}

// One warp per cell: order the cell's atoms by caller index and gather slot data.
__global__ void k_cellsort(int n_cells, const int* __restrict__ start, const int* __restrict__ perm_tmp,
                           const float4* __restrict__ xq, const float2* __restrict__ params,
                           const int* __restrict__ sid, const SysDev* __restrict__ sys,
                           int* __restrict__ perm, int* __restrict__ iperm, float4* __restrict__ xs,
                           float4* __restrict__ xsb, float2* __restrict__ ps, float4* __restrict__ xref,
                           const unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (w >= n_cells) return;
    sort_cell(w, start, perm_tmp, xq, params, sid, sys, perm, iperm, xs, xsb, ps, xref);
}


// The whole re-slotting of a small handle (at most kScanTile cells, kSmallSortAtoms
// atoms) in one block of 1024 threads: binning, the scan, the scatter and the in-cell
// sort of k_bin, k_scan_single, k_scatter and k_cellsort, phase after phase behind block
// barriers.  A step that keeps its list then runs one early-exiting kernel instead of four.
__global__ void __launch_bounds__(1024) k_sort_small(int N, int n_cells, const float4* __restrict__ xq,
                                                      const int* __restrict__ sid, const SysDev* __restrict__ sys,
                                                      int* __restrict__ cellid, int* cell_count, int* start,
                                                      int* cursor, int* __restrict__ perm_tmp,
                                                      const float2* __restrict__ params, int* __restrict__ perm,
                                                      int* __restrict__ iperm, float4* __restrict__ xs,
                                                      float4* __restrict__ xsb, float2* __restrict__ ps,
                                                      float4* __restrict__ xref, unsigned* flags) {
    pdl_wait();
    if (flags[0] == 0u) return;
    for (int i = threadIdx.x; i < N; i += blockDim.x) bin_atom(i, xq, sid, sys, cellid, cell_count, flags);
    __syncthreads();
    scan_single_body(n_cells, cell_count, start, cursor);
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int c = cellid[i];
        perm_tmp[start[c] + atomicAdd(&cursor[c], 1)] = i;
    }
    __syncthreads();
    // the in-cell order by caller index, one thread per atom (k_cellsort's result)
    for (int p = threadIdx.x; p < N; p += blockDim.x) {
        const int i = perm_tmp[p];
        const int c = cellid[i];
        const int b = start[c], m = start[c + 1] - b;
        int rank = 0;
        for (int t = 0; t < m; ++t) rank += (perm_tmp[b + t] < i);
        place_atom(i, b + rank, xq, params, sid, sys, perm, iperm, xs, xsb, ps, xref);
    }
}

// Predicated 32-bit store: keeps the list append inside one basic block (no branch
// around it), so the tests of all held atoms interleave.  Nothing in the build reads
// the list back.
__device__ __forceinline__ void st32_if(unsigned* p, unsigned v, bool ok) {
    asm volatile(
        "{\n .reg .pred q;\n setp.ne.u32 q, %2, 0;\n @q st.global.u32 [%0], %1;\n}\n" ::"l"(p), "r"(v),
        "r"((unsigned)ok));
}

// Verlet list build, one block per cell (the cell tile of cell.cuh).  The block stages
// the candidates of the cell's stencil in shared memory (in tiles of `tile` when the
// stencil is larger) with each run's image applied and the candidate's slot in .w.
// Each warp then holds up to kBuildAtoms atoms of the cell in registers; lane l tests
// candidate l of each 32-wide chunk against every held atom and the accepted candidates
// are appended, as 16-bit stencil indices, with a ballot.  The list order is the stencil
// order, which depends only on the positions, and each row is written by one warp.
constexpr int kBuildThreads = 128;
constexpr int kBuildWarps = kBuildThreads / 32;
constexpr int kBuildAtoms = 6;      // atoms per warp held in registers (plain images)
constexpr int kBuildAtomsGen = 3;   // atoms per warp held in registers (per-pair images)
static_assert(kBuildAtoms == 6, "build_tile dispatches group sizes 1..6");

// Tests of one tile against the atoms [m0, m0 + na) of warp w of the cell's W warps (atom
// m of the warp is slot i0 + w + W m; W = kBuildWarps times the blocks per cell), na <= A.  Held atoms beyond na sit far away so that the
// unrolled tests run without branches.  GEN: per-pair image flags and folded axes.
// SLOW: atoms may have more than E exclusions (the rest are read from the CSR).
template <int E, bool SLOW, bool GEN, int A>
__device__ __forceinline__ void build_atoms(const CellCtx& C, int w, int W, int m0, int na, int t0, int nt, bool last,
                                            const float4* cand, const unsigned char* cflag,
                                            const float4* __restrict__ xs, const int* __restrict__ perm,
                                            const int* __restrict__ iperm, const int* __restrict__ ex_off,
                                            const int* __restrict__ ex_idx, const int* __restrict__ ex_slot,
                                            unsigned* __restrict__ nbr, int* __restrict__ nbr_cnt,
                                            int* __restrict__ nbr_out, int cap, float rnl2, float rc2,
                                            bool wrap, unsigned* flags) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    float ax[A], ay[A], az[A];
    int ex[A][E + 1];
    int cin[A], cout[A];
    unsigned* row[A];
    unsigned slow = 0u;
#pragma unroll
    for (int a = 0; a < A; ++a) {
        ax[a] = ay[a] = az[a] = -kFar;
        cin[a] = cout[a] = 0;
        row[a] = nbr;
#pragma unroll
        for (int q = 0; q <= E; ++q) ex[a][q] = -1;
        if (a < na) {
            const int i = C.i0 + w + W * (m0 + a);
            const float4 p = xs[i];
            ax[a] = p.x + C.fs[0];
            ay[a] = p.y + C.fs[1];
            az[a] = p.z + C.fs[2];
            ex[a][0] = i;  // the atom itself
#pragma unroll
            for (int q = 0; q < E; ++q) ex[a][q + 1] = ex_slot[(size_t)i * E + q];
            if (SLOW) {
                const int oi = perm[i];
                if (ex_off[oi + 1] - ex_off[oi] > E) slow |= 1u << a;
            }
            cin[a] = (t0 == 0) ? 0 : nbr_cnt[i];
            cout[a] = (t0 == 0) ? 0 : (nbr_out[i] & kOutCountMask);
            row[a] = nbr + (size_t)i * cap;
        }
    }
    for (int base = 0; base < nt; base += 32) {
        const float4 cj = cand[base + lane];
        const unsigned ent = __float_as_uint(cj.w);  // list entry: slot | image code
        const int j = (int)(ent & kEntrySlotMask);
        int fl = 0;
        if (GEN) fl = cflag[base + lane];
        float r2[A];
#pragma unroll
        for (int a = 0; a < A; ++a) {
            float dx, dy, dz;
            if (GEN) {
                dx = gen_diff(ax[a], cj.x, fl, 1, C.fold[0], C.L[0], C.hL[0]);
                dy = gen_diff(ay[a], cj.y, fl, 2, C.fold[1], C.L[1], C.hL[1]);
                dz = gen_diff(az[a], cj.z, fl, 4, C.fold[2], C.L[2], C.hL[2]);
            } else {
                dx = ax[a] - cj.x;
                dy = ay[a] - cj.y;
                dz = az[a] - cj.z;
            }
            r2[a] = pair_r2(dx, dy, dz);
        }
#pragma unroll
        for (int a = 0; a < A; ++a) {
            bool acc = r2[a] < rnl2;
#pragma unroll
            for (int q = 0; q <= E; ++q) acc = acc && (j != ex[a][q]);
            if (SLOW && ((slow >> a) & 1u) && acc) {
                const int i = C.i0 + w + W * (m0 + a);
                const int oi = perm[i];
                const int e0 = ex_off[oi], e1 = ex_off[oi + 1];
                for (int e = e0 + E; e < e1 && acc; ++e) acc = (iperm[ex_idx[e]] != j);
            }
            // pairs inside r_c at the build go to the front of the row, the others to the
            // back (in reverse order), so that the pair kernels can take the front part
            // without a cut-off test while the positions are those of the build
            const bool inn = acc && r2[a] < rc2;
            const unsigned ba = __ballot_sync(0xffffffffu, acc);
            if (ba == 0u) continue;  // warp-uniform: ~40% of (atom, chunk) pairs accept nothing
            const unsigned bi = __ballot_sync(0xffffffffu, inn);
            const int ni = __popc(bi), no = __popc(ba) - ni;
            // a chunk is written when both parts stay apart inside the row; once a row is
            // full the counts run on past cap and nothing more is written (see below)
            const bool room = cin[a] + cout[a] + ni + no <= cap;
            const int pi = __popc(bi & lt), po = __popc(ba & lt) - pi;
            const int pos = inn ? cin[a] + pi : cap - 1 - (cout[a] + po);
            st32_if(row[a] + pos, ent, acc && room);
            cin[a] += ni;
            cout[a] += no;
        }
    }
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < A; ++a) {
            if (a < na) {
                const int i = C.i0 + w + W * (m0 + a);
                int ci = cin[a], co = cout[a];
                if (last && ci + co > cap) {
                    // the row overflowed: flagged, and left empty, so that the kernels that
                    // read it before the host sees the flag find no unwritten entries
                    atomicOr(&flags[1], NB_DEVERR_LIST_OVERFLOW);
                    ci = 0;
                    co = 0;
                }
                nbr_cnt[i] = ci;  // running counts between tiles, cleared after the last on overflow
                nbr_out[i] = co | (wrap ? kOutWrapBit : 0);
            }
        }
    }
}

template <int E, bool SLOW>
__device__ __forceinline__ void build_tile(const CellCtx& C, int w, int W, int t0, int nt, bool last,
                                           const float4* cand,
                                           const unsigned char* cflag, const float4* __restrict__ xs,
                                           const int* __restrict__ perm, const int* __restrict__ iperm,
                                           const int* __restrict__ ex_off, const int* __restrict__ ex_idx,
                                           const int* __restrict__ ex_slot, unsigned* __restrict__ nbr,
                                           int* __restrict__ nbr_cnt, int* __restrict__ nbr_out, int cap,
                                           float rnl2, float rc2, bool wrap, unsigned* flags) {
    const int n_i = C.i1 - C.i0;
    const int mw = n_i > w ? (n_i - w + W - 1) / W : 0;  // atoms of this warp
    if (mw == 0) return;
    const int A = C.gen ? kBuildAtomsGen : kBuildAtoms;
    const int ng = (mw + A - 1) / A;
    const int gs = (mw + ng - 1) / ng;  // balanced group size <= A
    for (int m0 = 0; m0 < mw; m0 += gs) {
        const int na = min(gs, mw - m0);
#define NB_BUILD_ARGS C, w, W, m0, na, t0, nt, last, cand, cflag, xs, perm, iperm, ex_off, ex_idx, ex_slot, nbr, \
                      nbr_cnt, nbr_out, cap, rnl2, rc2, wrap, flags
        if (C.gen) {
            build_atoms<E, SLOW, true, kBuildAtomsGen>(NB_BUILD_ARGS);
        } else {
            switch (na) {  // warp-uniform: straight-line code for each group size
                case 1: build_atoms<E, SLOW, false, 1>(NB_BUILD_ARGS); break;
                case 2: build_atoms<E, SLOW, false, 2>(NB_BUILD_ARGS); break;
                case 3: build_atoms<E, SLOW, false, 3>(NB_BUILD_ARGS); break;
                case 4: build_atoms<E, SLOW, false, 4>(NB_BUILD_ARGS); break;
                case 5: build_atoms<E, SLOW, false, 5>(NB_BUILD_ARGS); break;
                default: build_atoms<E, SLOW, false, 6>(NB_BUILD_ARGS); break;
            }
        }
#undef NB_BUILD_ARGS
    }
}

template <int E, bool SLOW>
__device__ __forceinline__ void build_cell_body(const CellCtx& C, const SysDev& S, int cap, int tile,
                                                const int* __restrict__ start, const float4* __restrict__ xs,
                                                const int* __restrict__ perm, const int* __restrict__ iperm,
                                                const int* __restrict__ ex_off, const int* __restrict__ ex_idx,
                                                int* __restrict__ ex_slot, int* __restrict__ ex_cnt,
                                                unsigned* __restrict__ nbr, int* __restrict__ nbr_cnt,
                                                int* __restrict__ nbr_out, unsigned* flags, int part, int split);

// ---------------------------------------------------------------- dynamic list pruning
//
// Between builds the rows of the pruning systems (SysDev::rin2 > 0) are re-partitioned at
// the current positions: the entries within r_in = r_c + delta (delta the prune skin) go to
// the front of the row, the others to its back (stored in reverse from the end, as the build
// stores them), each part in the order the entries are met (the old front part, then the old
// back part as stored), so the result depends only on the list and the positions.  While no
// atom has moved more than delta/2 since (the loads compare the positions with x_prune), no
// pair of a back part can come within r_c: its distance was >= r_c + delta and changes by at
// most delta; the pair and VJP kernels then skip the back parts.  The list's pair set, its
// build and its rebuild test are untouched.  A system is re-partitioned on an evaluation that
// keeps the list when it is not pruned yet (the first such evaluation after a build) or a
// load has requested it.  The work runs in the list-build launch that returns at once when
// no rebuild is due (one launch per evaluation in any case): each block takes the atoms of
// its cell, one warp per atom staging the row in the block's shared tile so that the
// partition can be written over it in place; the block that finishes a system's last cell
// (a per-system counter) marks the system pruned.

template <int IMG>
__device__ __forceinline__ void prune_row(const float4& xr, const PairGeo& G, const unsigned* buf, int m, float rin2,
                                          const float4* __restrict__ xs, unsigned* row, int cap, int& ci, int& co) {
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    ci = 0;
    co = 0;
    // four rounds of 32 entries at a time: their partner gathers are in flight together
    for (int b0 = 0; b0 < m; b0 += 128) {  // warp-uniform
        unsigned ent[4];
        float4 cj[4];
        bool inn[4], ok[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int e = b0 + 32 * u + lane;
            ok[u] = e < m;
            ent[u] = ok[u] ? buf[e] : 0u;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) cj[u] = xs[ent[u] & kEntrySlotMask];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            float dx, dy, dz;
            entry_diff<IMG>(xr, cj[u], ent[u] >> kEntrySlotBits, G, dx, dy, dz);
            inn[u] = ok[u] && pair_r2(dx, dy, dz) < rin2;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const unsigned bi = __ballot_sync(0xffffffffu, inn[u]), bo = __ballot_sync(0xffffffffu, ok[u]) & ~bi;
            const int pos = inn[u] ? ci + __popc(bi & lt) : cap - 1 - (co + __popc(bo & lt));
            if (ok[u]) row[pos] = ent[u];
            ci += __popc(bi);
            co += __popc(bo);
        }
    }
}

// The prune of cell c's atoms (block `part` of the cell's `split`), when due for its system.
__device__ __forceinline__ void prune_cell(int c, int part, int split, int cap, const int* __restrict__ cell_sys,
                                           const SysDev* __restrict__ sys, const int* __restrict__ start,
                                           const float4* __restrict__ xs, unsigned* __restrict__ nbr,
                                           int* __restrict__ nbr_cnt, int* __restrict__ nbr_out,
                                           float4* __restrict__ x_prune, unsigned* __restrict__ prune_sys,
                                           unsigned* __restrict__ prune_cnt, unsigned* buf_all) {
    const int s = cell_sys[c];
    const SysDev& S = sys[s];
    if (!(S.rin2 > 0.f)) return;
    const unsigned ps = prune_sys[s];
    if ((ps & kPruned) && !(ps & kPruneReq)) return;  // block-uniform
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned* buf = buf_all + (size_t)w * cap;
    const PairGeo G = pair_geo(S);
    const bool fold = G.fold[0] || G.fold[1] || G.fold[2];
    const int i0 = start[c], i1 = start[c + 1], W = split * kBuildWarps;
    for (int k = i0 + part * kBuildWarps + w; k < i1; k += W) {
        const int nin = nbr_cnt[k], o = nbr_out[k], nout = o & kOutCountMask;
        unsigned* row = nbr + (size_t)k * cap;
        for (int e = lane; e < nin; e += 32) buf[e] = row[e];
        for (int e = lane; e < nout; e += 32) buf[nin + e] = row[cap - nout + e];
        __syncwarp();
        const float4 xr = xs[k];
        int ci, co;
        if (fold) prune_row<kImgFold>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        else if (o & kOutWrapBit) prune_row<kImgCode>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        else prune_row<kImgPlain>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        if (lane == 0) {
            nbr_cnt[k] = ci;
            nbr_out[k] = co | (o & kOutWrapBit);
            x_prune[k] = xr;
        }
        __syncwarp();  // the staging buffer is reused by the warp's next atom
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned blocks = (unsigned)(S.nc[0] * S.nc[1] * S.nc[2] * split);
        if (atomicAdd(&prune_cnt[s], 1u) + 1u == blocks) {
            prune_sys[s] = kPruned;
            prune_cnt[s] = 0u;
        }
    }
}

// Two ways to run the prune, chosen per evaluation.  A force evaluation with PME folds it
// into the build launch (prune_cell, above): one kernel fewer between the build and the pair
// kernel matters there, because the PME kernels on the second stream take the SMs the pair
// kernel would start on (an idle kernel at that place cost the water 24k step 20 us with
// PME, 2 us without).  Elsewhere (dynamics, the VJP) the prune kernel below runs after the
// build launch: at 8 warps per block and a small staging buffer it keeps more warps and more
// L1 per SM than the build's blocks (128 threads, 40 KB tile) and prunes ~2x faster.
// The prune kernel: a few blocks per SM, one warp per atom (grid-stride over the atoms),
// each warp staging its row in its own part of the block's shared buffer.  It returns at
// once unless some system may need a prune (NB_FLAG_PRUNE_ANY) and the list is not fresh;
// the last block to finish (a ticket behind a fence) marks the systems it re-partitioned
// (the same test as the warps', on the same unchanged words) and clears the flag.
constexpr int kPruneWarps = 8;

__device__ __forceinline__ bool prune_due(const SysDev& S, unsigned ps) {
    return S.rin2 > 0.f && (!(ps & kPruned) || (ps & kPruneReq));
}

__global__ void __launch_bounds__(kPruneWarps * 32) k_prune(int N, int cap, const int* __restrict__ sid,
                                                             const SysDev* __restrict__ sys, int n_sys,
                                                             const float4* __restrict__ xs, unsigned* __restrict__ nbr,
                                                             int* __restrict__ nbr_cnt, int* __restrict__ nbr_out,
                                                             float4* __restrict__ x_prune,
                                                             unsigned* __restrict__ prune_sys, unsigned* ticket,
                                                             unsigned* flags) {
    pdl_wait();
    if (flags[NB_FLAG_FRESH] != 0u || flags[NB_FLAG_PRUNE_ANY] == 0u) return;  // grid-uniform
    extern __shared__ unsigned prune_buf[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned* buf = prune_buf + (size_t)w * cap;
    for (int k = blockIdx.x * kPruneWarps + w; k < N; k += gridDim.x * kPruneWarps) {
        const int s = sid[k];  // a system owns the same index range in slot and caller order
        const SysDev& S = sys[s];
        if (!prune_due(S, prune_sys[s])) continue;  // warp-uniform
        const int nin = nbr_cnt[k], o = nbr_out[k], nout = o & kOutCountMask;
        unsigned* row = nbr + (size_t)k * cap;
        for (int e = lane; e < nin; e += 32) buf[e] = row[e];
        for (int e = lane; e < nout; e += 32) buf[nin + e] = row[cap - nout + e];
        __syncwarp();
        const float4 xr = xs[k];
        const PairGeo G = pair_geo(S);
        int ci, co;
        if (G.fold[0] || G.fold[1] || G.fold[2]) prune_row<kImgFold>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        else if (o & kOutWrapBit) prune_row<kImgCode>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        else prune_row<kImgPlain>(xr, G, buf, nin + nout, S.rin2, xs, row, cap, ci, co);
        if (lane == 0) {
            nbr_cnt[k] = ci;
            nbr_out[k] = co | (o & kOutWrapBit);
            x_prune[k] = xr;
        }
        __syncwarp();  // the staging buffer is reused by the warp's next atom
    }
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        for (int s = 0; s < n_sys; ++s)
            if (prune_due(sys[s], prune_sys[s])) prune_sys[s] = kPruned;
        flags[NB_FLAG_PRUNE_ANY] = 0u;
        *ticket = 0u;
    }
}

// Without exclusions (E = 0) 64 registers and eight blocks per SM: LJ 256k 263 -> 248 us per
// build against 96 registers and five; with exclusions the extra blocks cost more than they
// give (water 24k: 108 -> 121 us at 80 registers, 156 us at 64), and a minimum of 0 blocks
// leaves their register count to the compiler.
template <int E, bool SLOW>
__global__ void __launch_bounds__(kBuildThreads, E == 0 ? 8 : 0) k_build_cell(
    int cap, int tile, const int* __restrict__ cell_sys, const SysDev* __restrict__ sys,
    const int* __restrict__ start, const float4* __restrict__ xs, const int* __restrict__ perm,
    const int* __restrict__ iperm, const int* __restrict__ ex_off, const int* __restrict__ ex_idx,
    int* __restrict__ ex_slot, int* __restrict__ ex_cnt, unsigned* __restrict__ nbr,
    int* __restrict__ nbr_cnt, int* __restrict__ nbr_out, unsigned* ticket, unsigned* flags, int split,
    unsigned* __restrict__ prune_sys, int n_sys, float4* __restrict__ x_prune, unsigned* __restrict__ prune_cnt,
    int fold_prune) {
    pdl_wait();
    if (flags[0] == 0u) {
        // the list is kept: with fold_prune, re-partition the cell's rows here when its
        // system's prune is due (else k_prune, launched next, does it)
        if (fold_prune && prune_sys && flags[NB_FLAG_FRESH] == 0u) {
            extern __shared__ float4 prune_tile[];  // the candidate tile, as kBuildWarps rows of cap entries
            prune_cell(blockIdx.x / split, blockIdx.x % split, split, cap, cell_sys, sys, start, xs, nbr, nbr_cnt,
                       nbr_out, x_prune, prune_sys, prune_cnt, reinterpret_cast<unsigned*>(prune_tile));
        }
        return;
    }
    // `split` blocks share a cell, block `part` taking warps part*kBuildWarps.. of its W
    const int c = blockIdx.x / split, part = blockIdx.x % split;
    const SysDev& S = sys[cell_sys[c]];
    const CellCtx C = cell_ctx(c, S, start);
    if (C.i0 + part * kBuildWarps < C.i1)
        build_cell_body<E, SLOW>(C, S, cap, tile, start, xs, perm, iperm, ex_off, ex_idx, ex_slot, ex_cnt, nbr,
                                 nbr_cnt, nbr_out, flags, part, split);
    // the last block to finish counts the rebuild and clears the request
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        unsigned long long* cnt = reinterpret_cast<unsigned long long*>(flags + 2);
        *cnt += 1ull;
        flags[0] = 0u;
        flags[NB_FLAG_FRESH] = 1u;  // slot positions are those of this build until the next load
        flags[NB_FLAG_EXPORT] = 0u;  // the export's stored per-row counts are of the old list
        if (prune_sys) {  // the rows are split at r_c of the build, not pruned: the next
            for (int s = 0; s < n_sys; ++s) prune_sys[s] = 0u;  // evaluation that keeps them prunes
            flags[NB_FLAG_PRUNE_ANY] = 1u;
        }
        *ticket = 0u;
    }
}

template <int E, bool SLOW>
__device__ __forceinline__ void build_cell_body(const CellCtx& C, const SysDev& S, int cap, int tile,
                                                const int* __restrict__ start, const float4* __restrict__ xs,
                                                const int* __restrict__ perm, const int* __restrict__ iperm,
                                                const int* __restrict__ ex_off, const int* __restrict__ ex_idx,
                                                int* __restrict__ ex_slot, int* __restrict__ ex_cnt,
                                                unsigned* __restrict__ nbr, int* __restrict__ nbr_cnt,
                                                int* __restrict__ nbr_out, unsigned* flags, int part, int split) {
    __shared__ BuildRun runs[kMaxRuns];
    __shared__ int n_runs, n_cand;
    // dynamic: `tile` candidates, then `tile` image-flag bytes when any system can need
    // per-pair images
    extern __shared__ float4 cand[];
    unsigned char* cflag = reinterpret_cast<unsigned char*>(cand + tile);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (w == 0) cell_runs(C, S, start, runs, &n_runs, &n_cand, flags);
    __syncthreads();
    const int nr = n_runs, total = n_cand;
    // rows of this cell may hold image codes (or the system folds an axis): the pair kernels
    // then take the per-axis image path for its atoms
    bool wrap = C.gen;
    for (int r = 0; r < nr; ++r) wrap = wrap || runs[r].code != 0u;
    const float rnl2 = S.rnl2, rc2 = S.rc2;
    for (int t0 = 0; t0 < total; t0 += tile) {
        const int t1 = min(total, t0 + tile);
        const int nt = t1 - t0;
        // stage: warp w copies runs w, w + kBuildWarps, ...; lanes over the run's slots.  The
        // copies go straight to shared memory, all in flight at once; each thread then adds
        // the run's image shift and the slot to the entries it copied itself.
        for (int r = w; r < nr; r += kBuildWarps) {
            const int sm0 = runs[r].sm0, slot0 = runs[r].slot0;
            const int a = max(sm0, t0), b = min(sm0 + runs[r].n, t1);
            for (int k = a + lane; k < b; k += 32) cp_async16(&cand[k - t0], &xs[slot0 + (k - sm0)]);
        }
        if (E > 0 && t0 == 0) {
            // exclusion partners of this block's atoms as slots, while the copies are in
            // flight (read by the tests below and by the pair kernels); the block's atoms
            // are i0 + part*kBuildWarps + (a % kBuildWarps) + W (a / kBuildWarps)
            const int W = split * kBuildWarps;
            const int nb = (C.i1 - C.i0 - part * kBuildWarps + W - 1) / W * kBuildWarps;
            for (int idx = threadIdx.x; idx < nb * E; idx += kBuildThreads) {
                const int a = idx / E, q = idx % E;
                const int i = C.i0 + part * kBuildWarps + a % kBuildWarps + W * (a / kBuildWarps);
                if (i >= C.i1) continue;
                const int oi = perm[i];
                const int e0 = ex_off[oi], ne = ex_off[oi + 1] - e0;
                ex_slot[(size_t)i * E + q] = q < ne ? iperm[ex_idx[e0 + q]] : -1;
                if (q == 0) ex_cnt[i] = ne;
            }
        }
        cp_async_wait_all();
        for (int r = w; r < nr; r += kBuildWarps) {
            const BuildRun R = runs[r];
            const int a = max(R.sm0, t0), b = min(R.sm0 + R.n, t1);
            for (int k = a + lane; k < b; k += 32) {
                const float4 p = cand[k - t0];
                cand[k - t0] = make_float4(p.x + R.s[0], p.y + R.s[1], p.z + R.s[2],
                                           __uint_as_float((unsigned)(R.slot0 + (k - R.sm0)) | R.code));
                if (C.gen) cflag[k - t0] = (unsigned char)R.flags;
            }
        }
        const int ntp = (nt + 31) & ~31;
        for (int k = nt + threadIdx.x; k < ntp; k += kBuildThreads) {
            cand[k] = make_float4(kFar, kFar, kFar, __uint_as_float(kEntrySlotMask));  // never accepted
            if (C.gen) cflag[k] = 0;
        }
        __syncthreads();
        const bool last = t1 == total;
        build_tile<E, SLOW>(C, part * kBuildWarps + w, split * kBuildWarps, t0, nt, last, cand, cflag, xs, perm,
                            iperm, ex_off, ex_idx, ex_slot, nbr, nbr_cnt, nbr_out, cap, rnl2, rc2, wrap, flags);
        if (!last) __syncthreads();
    }
}

// Pairs of the list as caller indices (i < j), one warp per atom, eight atoms per block.
// Every unordered pair is listed in both rows; the row whose slot is the smaller one emits
// it, which an entry's slot bits decide without the permutation, and only the emitted
// entries are mapped to caller indices (a random gather each).  Each block takes its output
// range with one counter update; a single counter updated per warp round serialised ~450k
// atomic adds on one address (water 24k: 160 us; now 19 us counting, 29 us writing).  The
// rows' pair counts come from a counting walk, which also stores them (exp_cnt) for a later
// writing call on the same list (NB_FLAG_EXPORT, cleared by every build): the usual
// count-then-write sequence walks each row twice, not three times.  Each walk loads four
// rounds of a row at once (it is latency-bound).  The order of the output is not defined;
// the set is.  out == nullptr: count only.
constexpr int kExportWarps = 8;

__device__ __forceinline__ int export_slot(const unsigned* row, int n, int m, int m_in, int gap) {
    return n < m ? (int)(row[n < m_in ? n : n + gap] & kEntrySlotMask) : -1;
}

__global__ void __launch_bounds__(kExportWarps * 32) k_export_pairs(int N, int cap, const unsigned* __restrict__ nbr,
                                                                    const int* __restrict__ cnt,
                                                                    const int* __restrict__ cnt_out,
                                                                    const int* __restrict__ perm, int2* out,
                                                                    long long max_pairs, unsigned long long* counter,
                                                                    int* __restrict__ exp_cnt, unsigned* flags) {
    __shared__ unsigned wcnt[kExportWarps];
    __shared__ unsigned long long wbase[kExportWarps];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kExportWarps + w;
    // counts stored by an earlier counting call on this list (read before any write below;
    // only a counting call sets the flag, and only after this launch's reads of it)
    const bool stored = out != nullptr && flags[NB_FLAG_EXPORT] != 0u;
    int m_in = 0, m = 0, gap = 0;
    const unsigned* row = nbr;
    if (i < N) {  // no early return: the block meets at barriers
        // entries [0, m_in) and [cap - m_out, cap) of the row, walked as one range
        m_in = cnt[i];
        m = m_in + (cnt_out[i] & kOutCountMask);
        gap = cap - m;
        row = nbr + (size_t)i * cap;
    }
    unsigned c = 0;
    if (stored) {
        c = i < N ? (unsigned)exp_cnt[i] : 0u;
    } else {
        for (int n0 = 0; n0 < m; n0 += 128) {
            int sj[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) sj[k] = export_slot(row, n0 + 32 * k + lane, m, m_in, gap);
#pragma unroll
            for (int k = 0; k < 4; ++k) c += __popc(__ballot_sync(0xffffffffu, sj[k] > i));
        }
        if (lane == 0 && i < N) exp_cnt[i] = (int)c;
    }
    if (lane == 0) wcnt[w] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int k = 0; k < kExportWarps; ++k) t += wcnt[k];
        unsigned long long b = t ? atomicAdd(counter, t) : 0ull;
        for (int k = 0; k < kExportWarps; ++k) {
            wbase[k] = b;
            b += wcnt[k];
        }
    }
    __syncthreads();
    if (!out || m == 0) return;
    const int oi = perm[i];
    unsigned long long base = wbase[w];
    for (int n0 = 0; n0 < m; n0 += 128) {
        int sj[4], oj[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) sj[k] = export_slot(row, n0 + 32 * k + lane, m, m_in, gap);
#pragma unroll
        for (int k = 0; k < 4; ++k) oj[k] = sj[k] > i ? perm[sj[k]] : 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool take = sj[k] > i;
            const unsigned b = __ballot_sync(0xffffffffu, take);
            const unsigned long long pos = base + __popc(b & ((1u << lane) - 1u));
            if (take && (long long)pos < max_pairs) out[pos] = make_int2(min(oi, oj[k]), max(oi, oj[k]));
            base += __popc(b);
        }
    }
}

// Marks the export's per-row counts as those of the current list (after a counting walk).
__global__ void k_export_counted(unsigned* flags) { flags[NB_FLAG_EXPORT] = 1u; }

// The re-slotting of this handle bins in its own kernel (not in the one-block k_sort_small).
static bool bins_separately(const nb_handle* h) { return !(h->n_scan_blocks == 1 && h->n_atoms <= kSmallSortAtoms); }

bool launch_load(nb_handle* h, const float4* xq, cudaStream_t st, bool forced) {
    int N = h->n_atoms;
    if (forced && bins_separately(h)) {
        launch_pdl(k_load_bin, cdiv(N, 256), 256, 0, st, N, xq, h->sid, h->sys, h->cellid, h->cell_count, h->ffix,
                   h->n_scan_blocks == 1 ? 1 : 0, h->n_cells, h->cell_start, h->cell_cursor, h->bin_ticket,
                   h->flags);
        return true;
    }
    launch_pdl(k_load, cdiv(N, 256), 256, 0, st, N, xq, h->iperm, h->sid, h->sys, h->xref, h->xsb, h->xs, h->ffix,
               (const float4*)h->x_prune, h->prune_sys, h->flags);
    return false;
}

size_t build_smem(const nb_handle* h) { return (size_t)h->tile * (sizeof(float4) + (h->build_gen ? 1 : 0)); }

void launch_build(nb_handle* h, cudaStream_t st, bool fold_prune) {
    auto build = h->excl_w == 0   ? k_build_cell<0, false>
                 : h->excl_w == 2 ? k_build_cell<2, false>
                 : h->max_excl <= 4 ? k_build_cell<4, false>
                                    : k_build_cell<4, true>;
    launch_pdl(build, h->n_cells * h->split_build, kBuildThreads, build_smem(h), st,
        h->cap, h->tile, h->cell_sys, h->sys, h->cell_start, h->xs, h->perm, h->iperm, h->ex_off, h->ex_idx,
        h->ex_slot, h->ex_cnt, h->nbr, h->nbr_cnt, h->nbr_out, h->build_ticket, h->flags, h->split_build,
        h->prune_sys, h->n_sys, h->x_prune, h->prune_cnt, fold_prune && h->fold_prune_ok ? 1 : 0);
}

// Dynamic list pruning (k_prune), after the build of every evaluation that uses the list
// (folded: the build launch has done it).
void launch_prune(nb_handle* h, cudaStream_t st, bool folded) {
    if (!h->prune_sys || (folded && h->fold_prune_ok)) return;
    const int N = h->n_atoms;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::min(cdiv(N, kPruneWarps), 4 * sms);
    launch_pdl(k_prune, grid, kPruneWarps * 32, (size_t)kPruneWarps * h->cap * sizeof(unsigned), st, N, h->cap,
               h->sid, h->sys, h->n_sys, h->xs, h->nbr, h->nbr_cnt, h->nbr_out, h->x_prune, h->prune_sys,
               h->prune_ticket, h->flags);
}

// Re-slotting of a rebuild: binning, scan, scatter and in-cell sort (one block for small
// handles); the Verlet list build (launch_build) follows.
void launch_reslot(nb_handle* h, const float4* xq, cudaStream_t st, bool binned) {
    int N = h->n_atoms;
    if (!bins_separately(h)) {
        launch_pdl(k_sort_small, 1, 1024, 0, st, N, h->n_cells, xq, h->sid, h->sys, h->cellid, h->cell_count,
                                         h->cell_start, h->cell_cursor, h->perm_tmp, h->params, h->perm, h->iperm,
                                         h->xs, h->xsb, h->ps, h->xref, h->flags);
        return;
    }
    // a single-block scan runs in the last block of the binning kernel (k_bin or k_load_bin)
    if (!binned)
        launch_pdl(k_bin, cdiv(N, 256), 256, 0, st, N, xq, h->sid, h->sys, h->cellid, h->cell_count,
                   h->n_scan_blocks == 1 ? 1 : 0, h->n_cells, h->cell_start, h->cell_cursor, h->bin_ticket,
                   h->flags);
    if (h->n_scan_blocks != 1) {
        launch_pdl(k_scan_a, h->n_scan_blocks, 1024, 0, st, h->n_cells, h->cell_count, h->cell_start, h->scan_bsum,
                                                    h->flags);
        launch_pdl(k_scan_b, 1, 1024, 0, st, h->n_scan_blocks, h->n_cells, h->scan_bsum, h->cell_start, h->flags);
        launch_pdl(k_scan_c, h->n_scan_blocks, 1024, 0, st, h->n_cells, h->cell_start, h->scan_bsum, h->cell_count,
                                                    h->cell_cursor, h->flags);
    }
    launch_pdl(k_scatter, cdiv(N, 256), 256, 0, st, N, h->cellid, h->cell_start, h->cell_cursor, h->perm_tmp, h->flags);
    launch_pdl(k_cellsort, cdiv((long long)h->n_cells * 32, 256), 256, 0, st,
        h->n_cells, h->cell_start, h->perm_tmp, xq, h->params, h->sid, h->sys, h->perm, h->iperm, h->xs, h->xsb,
        h->ps, h->xref, h->flags);
}


// The dynamic shared-memory limit of a kernel is process-wide, so it is raised once to
// what the device allows (less the kernel's static shared memory) rather than to one
// handle's need; each launch still asks only for its own tile.
template <class K>
static cudaError_t allow_max_smem(K kernel) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    return e;
}

cudaError_t build_setup(nb_handle* h) {
    if (build_smem(h) + 4096 > 227 * 1024) return cudaErrorInvalidValue;
    if (h->prune_sys) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t need = (size_t)kPruneWarps * h->cap * sizeof(unsigned);
        // the build launch can prune when its shared tile holds a row per warp
        h->fold_prune_ok = (size_t)kBuildWarps * h->cap * sizeof(unsigned) <= build_smem(h) ? 1 : 0;
        if (need + 1024 > (size_t)optin) {
            // rows too long to stage: the lists are not pruned
            h->prune_sys = nullptr;
            h->x_prune = nullptr;
        } else {
            cudaError_t e = cudaFuncSetAttribute(k_prune, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need);
            if (e != cudaSuccess) return e;
        }
    }
    h->split_build = pick_split(h, kBuildWarps, 3);  // keep >= 3 atoms per warp for register blocking
    cudaError_t e = allow_max_smem(k_build_cell<0, false>);
    if (e == cudaSuccess) e = allow_max_smem(k_build_cell<2, false>);
    if (e == cudaSuccess) e = allow_max_smem(k_build_cell<4, false>);
    if (e == cudaSuccess) e = allow_max_smem(k_build_cell<4, true>);
    return e;
}

void launch_export_pairs(nb_handle* h, int2* out, long long max_pairs, unsigned long long* counter,
                         cudaStream_t st) {
    const int N = h->n_atoms;
    k_export_pairs<<<cdiv(N, kExportWarps), kExportWarps * 32, 0, st>>>(N, h->cap, h->nbr, h->nbr_cnt, h->nbr_out,
                                                                         h->perm, out, max_pairs, counter,
                                                                         h->exp_cnt, h->flags);
    k_export_counted<<<1, 1, 0, st>>>(h->flags);
}

}  // namespace nb
