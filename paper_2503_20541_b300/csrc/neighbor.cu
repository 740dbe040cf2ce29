// neighbor.cu -- cell list + Verlet neighbour list (Sec. 2.1.2 "Neighborlists").
//
// Every evaluation starts with k_load: scatter the caller's positions into slot
// order and test the list's validity (an atom moved more than r_skin/2 since the
// last build).  The rebuild chain (bin -> scan -> scatter -> in-cell sort ->
// Verlet build) is always launched but each kernel returns at once unless the
// device-side rebuild flag is set, so a step never waits on the host and the
// whole sequence can be captured in a CUDA graph.
//
// The sort is a counting sort by (system, cell) followed by a rank sort inside
// each cell on the caller index, so the slot order -- and with it the list and
// every FP32 summation order downstream -- depends only on the positions.
#include "common.cuh"

namespace nb {

__global__ void k_load(int N, const float4* __restrict__ xq, const int* __restrict__ iperm,
                       const int* __restrict__ sid, const SysDev* __restrict__ sys,
                       const float4* __restrict__ xref, float4* __restrict__ xs, unsigned* flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool need = false;
    if (i < N) {
        float4 p = xq[i];
        const SysDev& S = sys[sid[i]];
        float4 w = p;
        float4 r = xref[i];
        float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        if (S.periodic) {
            w.x = wrap1(p.x, S.L[0], S.invL[0]);
            w.y = wrap1(p.y, S.L[1], S.invL[1]);
            w.z = wrap1(p.z, S.L[2], S.invL[2]);
            dx = mi_any(dx, S.L[0], S.invL[0]);
            dy = mi_any(dy, S.L[1], S.invL[1]);
            dz = mi_any(dz, S.L[2], S.invL[2]);
        }
        xs[iperm[i]] = w;
        float d2 = dx * dx + dy * dy + dz * dz;
        need = !(d2 <= S.disp2);  // NaN (first call, bad input) also requests a rebuild
    }
    if (__any_sync(0xffffffffu, need) && (threadIdx.x & 31) == 0) atomicOr(&flags[0], 1u);
}

__device__ __forceinline__ int cell_coord(float w, float scale, int nc) {
    int c = (int)(w * scale);
    return min(max(c, 0), nc - 1);
}

__global__ void k_bin(int N, const float4* __restrict__ xq, const int* __restrict__ sid,
                      const SysDev* __restrict__ sys, int* __restrict__ cellid, int* cell_count,
                      unsigned* flags) {
    if (flags[0] == 0u) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
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

__global__ void k_scatter(int N, const int* __restrict__ cellid, const int* __restrict__ start,
                          int* cursor, int* __restrict__ perm_tmp, const unsigned* flags) {
    if (flags[0] == 0u) return;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int c = cellid[i];
    perm_tmp[start[c] + atomicAdd(&cursor[c], 1)] = i;
}

// One warp per cell: order the cell's atoms by caller index and gather slot data.
__global__ void k_cellsort(int n_cells, const int* __restrict__ start, const int* __restrict__ perm_tmp,
                           const float4* __restrict__ xq, const float2* __restrict__ params,
                           const int* __restrict__ sid, const SysDev* __restrict__ sys,
                           int* __restrict__ perm, int* __restrict__ iperm, float4* __restrict__ xs,
                           float2* __restrict__ ps, float4* __restrict__ xref, const unsigned* flags) {
    if (flags[0] == 0u) return;
    int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= n_cells) return;
    int b = start[w], m = start[w + 1] - b;
    for (int a = lane; a < m; a += 32) {
        int i = perm_tmp[b + a];
        int rank = 0;
        for (int t = 0; t < m; ++t) rank += (perm_tmp[b + t] < i);
        int slot = b + rank;
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
        ps[slot] = params[i];
    }
}

// Cells visited along one axis: either every cell once (nc <= 2*st) or the
// 2*st+1 cells around c, wrapped (periodic) or clipped (open).
struct AxisRange {
    int lo, hi;    // first range [lo, hi]
    int lo2, hi2;  // second range (wrap), empty if lo2 > hi2
};

__device__ __forceinline__ AxisRange axis_range(int c, int nc, int st, int periodic) {
    AxisRange r;
    r.lo2 = 1;
    r.hi2 = 0;
    if (nc <= 2 * st) {
        r.lo = 0;
        r.hi = nc - 1;
        return r;
    }
    int a = c - st, b = c + st;
    if (!periodic) {
        r.lo = max(a, 0);
        r.hi = min(b, nc - 1);
        return r;
    }
    if (a < 0) {
        r.lo = 0; r.hi = b;
        r.lo2 = a + nc; r.hi2 = nc - 1;
    } else if (b >= nc) {
        r.lo = a; r.hi = nc - 1;
        r.lo2 = 0; r.hi2 = b - nc;
    } else {
        r.lo = a; r.hi = b;
    }
    return r;
}

// Full Verlet list: P lanes per atom split the candidates of each neighbour-cell
// run; accepted candidates are compacted with a ballot, so the list order is the
// fixed visiting order.
template <int P>
__global__ void __launch_bounds__(256) k_build(int N, int cap, const float4* __restrict__ xs,
                                                const int* __restrict__ sid, const SysDev* __restrict__ sys,
                                                const int* __restrict__ start, const int* __restrict__ perm,
                                                const int* __restrict__ ex_off, const int* __restrict__ ex_idx,
                                                int* __restrict__ nbr, int* __restrict__ nbr_cnt,
                                                unsigned* flags) {
    if (flags[0] == 0u) return;
    int gt = blockIdx.x * blockDim.x + threadIdx.x;
    int i = gt / P, lane = gt % P;
    bool valid = i < N;
    int ii = valid ? i : N - 1;
    int wl = threadIdx.x & 31;
    int gbase = (wl / P) * P;
    unsigned gmask = (P == 32) ? 0xffffffffu : (((1u << P) - 1u) << gbase);
    const SysDev& S = sys[sid[ii]];
    float4 xi = xs[ii];
    int cx = cell_coord(xi.x, S.cell_scale[0], S.nc[0]);
    int cy = cell_coord(xi.y, S.cell_scale[1], S.nc[1]);
    int cz = cell_coord(xi.z, S.cell_scale[2], S.nc[2]);
    int oi = perm[ii];
    int e0 = ex_off[oi], ne = ex_off[oi + 1] - e0;
    int exl[kMaxExclInline];
#pragma unroll
    for (int k = 0; k < kMaxExclInline; ++k) exl[k] = (k < ne) ? ex_idx[e0 + k] : -1;
    const float L0 = S.L[0], L1 = S.L[1], L2 = S.L[2];
    const float h0 = S.halfL[0], h1 = S.halfL[1], h2 = S.halfL[2];
    const int per = S.periodic;
    const float rnl2 = S.rnl2;
    int cnt = 0;
    size_t rowbase = (size_t)ii * cap;
    AxisRange rz = axis_range(cz, S.nc[2], S.stencil, per);
    AxisRange ry = axis_range(cy, S.nc[1], S.stencil, per);
    AxisRange rx = axis_range(cx, S.nc[0], S.stencil, per);
    for (int zp = 0; zp < 2; ++zp) {
        int zlo = zp ? rz.lo2 : rz.lo, zhi = zp ? rz.hi2 : rz.hi;
        for (int z = zlo; z <= zhi; ++z) {
            for (int yp = 0; yp < 2; ++yp) {
                int ylo = yp ? ry.lo2 : ry.lo, yhi = yp ? ry.hi2 : ry.hi;
                for (int y = ylo; y <= yhi; ++y) {
                    int row = S.cell_off + (z * S.nc[1] + y) * S.nc[0];
                    for (int xp = 0; xp < 2; ++xp) {
                        int xlo = xp ? rx.lo2 : rx.lo, xhi = xp ? rx.hi2 : rx.hi;
                        if (xlo > xhi) continue;
                        int b = start[row + xlo], e = start[row + xhi + 1];
                        for (int base = b; base < e; base += P) {
                            int j = base + lane;
                            bool acc = false;
                            if (valid && j < e && j != ii) {
                                float4 xj = xs[j];
                                float dx, dy, dz;
                                if (per) {
                                    dx = mi_pair(xi.x, xj.x, L0, h0);
                                    dy = mi_pair(xi.y, xj.y, L1, h1);
                                    dz = mi_pair(xi.z, xj.z, L2, h2);
                                } else {
                                    dx = xi.x - xj.x;
                                    dy = xi.y - xj.y;
                                    dz = xi.z - xj.z;
                                }
                                float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
                                acc = r2 < rnl2;
                                if (acc && ne > 0) {
                                    int oj = perm[j];
#pragma unroll
                                    for (int k = 0; k < kMaxExclInline; ++k) acc = acc && (exl[k] != oj);
                                    for (int k = kMaxExclInline; k < ne; ++k) acc = acc && (ex_idx[e0 + k] != oj);
                                }
                            }
                            unsigned bits = (__ballot_sync(gmask, acc) >> gbase);
                            if (P < 32) bits &= (1u << P) - 1u;
                            if (acc) {
                                int pos = cnt + __popc(bits & ((1u << lane) - 1u));
                                if (pos < cap) nbr[rowbase + pos] = j;
                            }
                            cnt += __popc(bits);
                        }
                    }
                }
            }
        }
    }
    if (valid && lane == 0) {
        nbr_cnt[ii] = min(cnt, cap);
        if (cnt > cap) atomicOr(&flags[1], NB_DEVERR_LIST_OVERFLOW);
    }
}

__global__ void k_clear_rebuild(unsigned* flags) {
    if (flags[0] != 0u) {
        unsigned long long* c = reinterpret_cast<unsigned long long*>(flags + 2);
        *c += 1ull;
        flags[0] = 0u;
    }
}

__global__ void k_export_pairs(int N, int cap, const int* __restrict__ nbr, const int* __restrict__ cnt,
                               const int* __restrict__ perm, int2* out, long long max_pairs,
                               unsigned long long* counter) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    int oi = perm[k];
    int c = cnt[k];
    for (int n = 0; n < c; ++n) {
        int oj = perm[nbr[(size_t)k * cap + n]];
        if (oi < oj) {
            unsigned long long pos = atomicAdd(counter, 1ull);
            if (out && (long long)pos < max_pairs) out[pos] = make_int2(oi, oj);
        }
    }
}

void launch_load(nb_handle* h, const float4* xq, cudaStream_t st) {
    int N = h->n_atoms;
    k_load<<<cdiv(N, 256), 256, 0, st>>>(N, xq, h->iperm, h->sid, h->sys, h->xref, h->xs, h->flags);
}

template <int P>
static void launch_build_p(nb_handle* h, cudaStream_t st) {
    int N = h->n_atoms;
    k_build<P><<<cdiv((long long)N * P, 256), 256, 0, st>>>(N, h->cap, h->xs, h->sid, h->sys, h->cell_start,
                                                            h->perm, h->ex_off, h->ex_idx, h->nbr, h->nbr_cnt,
                                                            h->flags);
}

void launch_rebuild(nb_handle* h, const float4* xq, cudaStream_t st) {
    int N = h->n_atoms;
    k_bin<<<cdiv(N, 256), 256, 0, st>>>(N, xq, h->sid, h->sys, h->cellid, h->cell_count, h->flags);
    k_scan_a<<<h->n_scan_blocks, 1024, 0, st>>>(h->n_cells, h->cell_count, h->cell_start, h->scan_bsum, h->flags);
    k_scan_b<<<1, 1024, 0, st>>>(h->n_scan_blocks, h->n_cells, h->scan_bsum, h->cell_start, h->flags);
    k_scan_c<<<h->n_scan_blocks, 1024, 0, st>>>(h->n_cells, h->cell_start, h->scan_bsum, h->cell_count,
                                                h->cell_cursor, h->flags);
    k_scatter<<<cdiv(N, 256), 256, 0, st>>>(N, h->cellid, h->cell_start, h->cell_cursor, h->perm_tmp, h->flags);
    k_cellsort<<<cdiv((long long)h->n_cells * 32, 256), 256, 0, st>>>(
        h->n_cells, h->cell_start, h->perm_tmp, xq, h->params, h->sid, h->sys, h->perm, h->iperm, h->xs, h->ps,
        h->xref, h->flags);
    switch (h->lanes) {
        case 4: launch_build_p<4>(h, st); break;
        case 8: launch_build_p<8>(h, st); break;
        case 16: launch_build_p<16>(h, st); break;
        default: launch_build_p<32>(h, st); break;
    }
}

void launch_clear_rebuild(nb_handle* h, cudaStream_t st) { k_clear_rebuild<<<1, 1, 0, st>>>(h->flags); }

void launch_export_pairs(nb_handle* h, int2* out, long long max_pairs, unsigned long long* counter,
                         cudaStream_t st) {
    int N = h->n_atoms;
    k_export_pairs<<<cdiv(N, 128), 128, 0, st>>>(N, h->cap, h->nbr, h->nbr_cnt, h->perm, out, max_pairs, counter);
}

}  // namespace nb
