// common.cuh -- internal types and device helpers of libnbcore (sm_103a).
//
// Layout in HBM (N atoms over all systems, "caller order" i, "slot order" k):
//   caller order : xq float4 (x,y,z,q)  [caller-owned], sid int32, params float2
//                  (sigma, sqrt_eps), xref float4 (positions at the last list build),
//                  exclusion CSR.
//   slot order   : atoms sorted by (system, cell, caller index) after each rebuild;
//                  xs float4 (x,y,z,q in the frame of the last build), ps float2, the
//                  full neighbour list nbr[k*cap + n] (uint32: partner slot and periodic
//                  image code) with counts, fixed-point forces
//                  ffix[d*N + k] (int64, 2^force_bits per unit), per-atom half
//                  energies e_atom float4.
//   System s owns the same index range [atom_off, atom_off + n) in both orders.
#pragma once
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/nbcore.h"

namespace nb {

constexpr float kInvSqrtPi = 0.56418958354775628f;
constexpr int kScanItems = 4;
constexpr int kScanTile = 1024 * kScanItems;  // cells per block of the multi-block scan
// Atoms per block of the energy reduction of a system of n atoms: about one block per SM
// for the system alone (FP64 is slow on this part: the work is spread over the SMs), in
// multiples of 128 from 128 to 4096.  A function of the system alone, so that a system
// sums in the same order whether it is batched with others or not.
inline int red_tile(int n) {
    const int t = (n + 147) / 148;
    return std::min(4096, std::max(128, (t + 127) / 128 * 128));
}
constexpr int kSmallSortAtoms = 8192;          // handles re-slotted by one block (k_sort_small)
// Words of the handle's device flag array: [0] rebuild request, [1] error bits, [2..3] rebuild
// count (u64), [NB_FLAG_FRESH] 1 while the slot positions are exactly those of the last list
// build (set by the build, cleared by every load of new positions), [NB_FLAG_EXPORT] 1 while
// exp_cnt holds the pair export's per-atom counts of the current list (set by a counting
// export, cleared by the build).
constexpr int NB_FLAG_FRESH = 4;
constexpr int NB_FLAG_EXPORT = 5;
// Per-system word of dynamic list pruning (nb_handle::prune_sys): kPruned while the system's
// rows are partitioned at the positions of its last prune (x_prune) into the pairs within
// r_c + prune skin (front) and the rest (back), set by the prune kernel; kPruneReq set by a
// load that finds an atom of the system more than half the prune skin from its x_prune
// position.  The build clears both; the prune kernel sets kPruned and clears kPruneReq of the
// systems it re-partitions.  Kept per system, so that a system's prune schedule (and with
// it every summation order) does not depend on the other systems of a batch.
constexpr unsigned kPruned = 1u;
constexpr unsigned kPruneReq = 2u;
// [NB_FLAG_PRUNE_ANY] some system may need a prune: set by the build (the next evaluation
// that keeps the list prunes every pruning system) and by the loads with a request; cleared
// by the prune kernel, which returns at once while it is clear.
constexpr int NB_FLAG_PRUNE_ANY = 6;
// Internal bit of the `terms` passed to launch_pair: the per-atom energies are wanted (an
// evaluation whose energies nobody reduces runs the pair kernel's force-only form).
constexpr int kTermEnergy = 1 << 16;
// Internal bit of the `terms` passed to launch_pair: the exclusion correction is left to the
// evaluation's epilogue (launch_epilogue), which adds it while it writes the forces.
constexpr int kTermDeferExcl = 1 << 17;
// Internal bit of the `terms` passed to launch_pair: precise (two-float) energies; the pair
// kernel runs its force-only form and k_energy_df writes e_atom and e_lo.
constexpr int kTermPrecise = 1 << 18;
constexpr int kFlagWords = 8;
// A neighbour-list entry: the partner's slot in the low kEntrySlotBits bits and, above them,
// the pair's periodic image as 2 bits per axis d: bit 2d, atom i moves down by L; bit 2d + 1,
// partner j moves down by L (each shift exact: the moved coordinate lies above L/2).
constexpr int kEntrySlotBits = 26;
constexpr unsigned kEntrySlotMask = (1u << kEntrySlotBits) - 1u;
// nbr_out[k]: the count of back entries in the low bits; kOutWrapBit set when some entry of
// the row may carry an image code or the system folds an axis (periodic pairs near a face).
constexpr int kOutCountMask = (1 << 30) - 1;
constexpr int kOutWrapBit = 1 << 30;

// Per-system constants, resident in device memory (read through the L1 path).
struct SysDev {
    float L[3], invL[3], halfL[3];
    float cell_scale[3];  // cells per unit length: nc / L
    float rc2, rnl2, disp2;
    float rin2;           // (r_c + prune skin)^2 of dynamic list pruning (0: the system does not prune)
    float prune2;         // (prune skin / 2)^2: a larger displacement since the prune requests the next
    float rs, inv_sw;     // switch start and 1/(r_c - r_s)
    float alpha, ke;
    float beta2;          // alpha^2
    float inv_sw_lo;      // 1/(r_c - r_s) - inv_sw: the constant as a double-float pair (precise energies)
    int nc[3];
    int cell_off;
    int atom_off, n_atoms;
    int periodic, has_switch, has_coul, has_lj;
    int pme;
    int K[3];
    int stencil;          // cell_div: neighbour cells span +-stencil per axis
    long long grid_off;   // real PME mesh offset (elements)
    long long cgrid_off;  // complex half-spectrum offset (elements)
    int red_tile;         // atoms per block of the energy reduction (red_tile(n_atoms))
    double self_coef;     // -ke alpha / sqrt(pi)
    float kl_hi[3], kl_lo[3];  // K_d / L_d as an unevaluated sum hi + lo (double-float)
    float krf, crf;       // reaction field (Eq. RFA): k = (eps_s-1)/((2eps_s+1) r_c^3), c = 3eps_s/((2eps_s+1) r_c)
    float krf_lo, crf_lo; // k - krf and c - crf: the constants as double-float pairs for the energy
    int index;            // the system's index in the handle
    float rc;             // r_c (FP32; r_c^2 = rc rc exactly as a two-float product)
};

// An FFT group: PME systems sharing one mesh shape, meshes at a fixed stride.
struct FftGroup {
    int K[3];
    int count;
    long long grid_off, cgrid_off;
    long long dist_r = 0, dist_c = 0;  // padded mesh strides within the group
    cufftHandle r2c = 0, c2r = 0;
    bool has_r2c = false, has_c2r = false;
};

}  // namespace nb

struct nb_handle {
    int device = 0;
    int n_sys = 0;
    int n_atoms = 0;
    int cap = 0;        // per-atom neighbour capacity (full list)
    int cell_div = 0;   // the handle's option (0: per system, SysDev::stencil)
    int force_bits = 32;
    float fscale = 4294967296.0f, finv = 1.0f / 4294967296.0f;
    double gscale = 4294967296.0;  // PME mesh fixed-point scale
    int n_cells = 0;
    int n_scan_blocks = 0;
    int has_pme = 0;
    int blocks_per_cell = 0;     // option (0: auto)
    int split_build = 1;         // blocks per cell of the list build
    int split_pair = 1;          // blocks per cell of the pair and VJP kernels
    // rigid water (Langevin dynamics): constraint groups covering every atom once,
    // (O, H1, H2, 3) or (atom, -1, -1, 1)
    int n_groups = 0;
    int4* groups = nullptr;
    int n_water = 0;
    double d_oh = 0.0, d_hh = 0.0;
    std::vector<int> sid_host;   // system of each atom (caller order)
    int any_coul = 0;   // some system has ke != 0
    int any_uncharged = 0;  // some system has ke == 0
    int coul_kind = 1;  // electrostatics of the charged systems: 1 Ewald, 2 reaction field
    long long grid_total = 0, cgrid_total = 0;
    int n_conv_blocks = 0;

    std::vector<nb_system_desc> desc;
    std::vector<nb::SysDev> sys_h;
    std::vector<nb::FftGroup> fft;
    std::vector<void*> allocs;

    nb::SysDev* sys = nullptr;
    int* sid = nullptr;          // [N]
    float2* params = nullptr;    // [N] caller order
    int* ex_off = nullptr;       // [N+1]
    int* ex_idx = nullptr;       // [M]
    int max_excl = 0;            // most exclusions of one atom
    int excl_w = 0;              // exclusion slots per atom in ex_slot (0, 2 or 4)
    int* ex_slot = nullptr;      // [N * excl_w] slot order: partners' slots, -1 padded
    int* ex_cnt = nullptr;       // [N] slot order: number of exclusion partners
    int build_gen = 0;           // some system needs per-pair images in the list build
    int* cell_count = nullptr;   // [n_cells]
    int* cell_start = nullptr;   // [n_cells+1]
    int* cell_cursor = nullptr;  // [n_cells]
    int* scan_bsum = nullptr;    // [n_scan_blocks]
    int* cell_sys = nullptr;     // [n_cells] system of each cell
    int* cellid = nullptr;       // [N] caller order
    int* perm_tmp = nullptr;     // [N]
    int* perm = nullptr;         // [N] slot -> caller
    int* iperm = nullptr;        // [N] caller -> slot
    float4* xs = nullptr;        // [N] slot: positions in the frame of the last build
    float4* xsb = nullptr;       // [N] slot: wrapped positions at the last build
    float2* ps = nullptr;        // [N] slot
    float4* xref = nullptr;      // [N] caller
    unsigned* nbr = nullptr;     // [N*cap] list entries (partner slot | image code << kEntrySlotBits)
    int tile = 0;                // candidates per shared-memory tile of the cell kernels
    int* nbr_cnt = nullptr;      // [N] entries at the front of the row (inside r_c at the build)
    int* nbr_out = nullptr;      // [N] entries at the back of the row (outside r_c at the build), | kOutWrapBit
    int* exp_cnt = nullptr;      // [N] pairs each row emits in the pair export (valid per NB_FLAG_EXPORT)
    long long* ffix = nullptr;   // [3N] slot
    float4* e_atom = nullptr;    // [N] slot: half energies (E_lj, E_dir, E_excl, 0) of each atom
    float4* e_lo = nullptr;      // [N] slot: low parts of e_atom .x, .y in a precise-energy evaluation
    const float4* xq_in = nullptr;  // caller-order positions of the current precise-energy evaluation
    unsigned* flags = nullptr;   // [kFlagWords]: rebuild request, error bits, rebuild count, fresh list
    unsigned* build_ticket = nullptr;  // [1] blocks of the list build done (reset by the last)
    unsigned* bin_ticket = nullptr;    // [1] blocks of the binning done (reset by the last, which scans)
    float4* x_prune = nullptr;   // [N] slot: positions (frame of the last build) at the last prune
    unsigned* prune_sys = nullptr;  // [n_sys] kPruned | kPruneReq per system (null: no pruning)
    unsigned* prune_ticket = nullptr;  // [1] blocks of the prune kernel done (reset by the last)
    unsigned* prune_cnt = nullptr;  // [n_sys] blocks of the system done in a prune folded into the build
    int fold_prune_ok = 0;       // the build launch's shared tile can stage a row per warp
    int any_prune = 0;           // some system prunes its list between builds
    double* energy = nullptr;    // [n_sys * NB_NE] scratch
    int n_red_blocks = 0;        // energy reduction: blocks of red_tile atoms, none straddling systems
    int* red_blk_sys = nullptr;  // [n_red_blocks]
    int* red_blk_off = nullptr;  // [n_sys+1] first reduction block of each system
    double* red_part = nullptr;  // [n_red_blocks * 6] per-block FP64 partial sums, then [n_sys * 7] totals
    unsigned* red_ticket = nullptr;  // [1] blocks of the energy reduction done (reset by the last)
    float* ke_atom = nullptr;    // [N] caller
    // PME
    long long* gfix = nullptr;   // [grid_total]
    float* grid = nullptr;       // [grid_total]
    float* grid2 = nullptr;      // [grid_total] second mesh of the reciprocal VJP
    unsigned* lam_max = nullptr; // [1] largest |lam| (float bits) of a VJP call
    float kl_max = 0.f;          // largest K/L over the PME systems
    float2* cgrid = nullptr;     // [cgrid_total]
    float* green = nullptr;      // [cgrid_total] influence function G(m)
    int* conv_blk_sys = nullptr; // [n_conv_blocks]
    int* conv_blk_off = nullptr; // [n_sys+1] first convolve block of each system
    double* e_pme_blk = nullptr; // [n_conv_blocks]
    // dynamics scratch
    float4* vwork = nullptr;     // [N]
    float4* lam = nullptr;       // [N] slot: cotangent for the VJP kernels
    float4* gx_s = nullptr;      // [N] slot: VJP result (x,y,z) and gq (w)
    float2* gp_s = nullptr;      // [N] slot: gsigma, gsqrt_eps
    double* hbar_atom = nullptr; // [N]
    double* jump_atom = nullptr; // [N]
    double* e0 = nullptr;        // [n_sys * NB_NE]
    double* e1 = nullptr;        // [n_sys * NB_NE]
    float4* seg = nullptr;       // [3 * (seg_k + 1) * N] backward segment states
    int seg_k = 0;
    float4* xbar = nullptr;      // [N] caller
    float4* vbar = nullptr;      // [N] caller
    float4* xwork = nullptr;     // [N] caller: backward recomputation positions
    unsigned long long* counter = nullptr;  // pair export counter
    // second stream for the PME chain, forked from and joined to the caller's stream
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_built = nullptr;
    // optional per-stage CUDA-event timing
    int timing = 0;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_stage;           // stage of each recorded (start, stop) pair
    std::vector<cudaEvent_t> ev_used;    // start, stop, start, stop, ...
};

namespace nb {

// ---------------------------------------------------------------- device helpers

__device__ __forceinline__ float wrap1(float x, float L, float invL) {
    float w = x - L * floorf(x * invL);
    if (w >= L) w -= L;
    if (w < 0.f) w = 0.f;
    return w;
}

// Minimum-image difference xi - xj of two coordinates wrapped into [0, L).  When the
// pair straddles the boundary the far coordinate is shifted by L first: that shift is
// exact (Sterbenz), so the only rounding is that of the small final difference (a plain
// (xi - xj) -/+ L rounds an intermediate of magnitude ~L).
__device__ __forceinline__ float mi_pair(float xi, float xj, float L, float hL) {
    float d = xi - xj;
    if (d > hL) d = (xi - L) - xj;
    else if (d < -hL) d = xi - (xj - L);
    return d;
}

// Minimum image of an arbitrary difference.
__device__ __forceinline__ float mi_any(float d, float L, float invL) {
    return d - L * rintf(d * invL);
}

__device__ __forceinline__ long long to_fix(float v, float scale, unsigned* err) {
    float s = v * scale;
    if (!(fabsf(s) < 9.0e18f)) {
        atomicOr(err, NB_DEVERR_FIXEDPOINT);
        return 0;
    }
    return __float2ll_rn(s);
}

// Programmatic dependent launch: the kernels of an evaluation's main chain are launched
// with cudaLaunchAttributeProgrammaticStreamSerialization (launch_pdl), so that a kernel's
// launch overlaps the end of the previous kernel in the stream.  Each of them first waits
// here until that kernel has completed and its writes are visible (without the attribute
// the wait returns at once).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ void red_add(long long* p, long long v) {
    atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

template <int P>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = P / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Warp sums of NV values (NV a power of two, 2..32) by a transposed butterfly: at each of
// the first log2(NV) levels a lane keeps half of its values and sends the other half to
// its partner, so every level moves half as many values as the last; the remaining levels
// are plain pairwise sums.  Returns, in lane l, the warp sum of value l >> (5 - log2 NV)
// (NV - 1 + 5 - log2 NV shuffles instead of 5 NV).  The summation order is fixed.
template <int NV>
__device__ __forceinline__ float warp_sum_transposed(float (&v)[NV]) {
    const int lane = threadIdx.x & 31;
    int n = NV, o = 16;
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

inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ------------------------------------------------------------------ launchers
// neighbor.cu
// the evaluation's load; forced: the list is rebuilt in any case, and the kernel then also
// bins the atoms (and scans the cell counts) when the re-slotting would do that in its own
// kernels, returning true (pass it to launch_reslot as `binned`)
bool launch_load(nb_handle* h, const float4* xq, cudaStream_t st, bool forced = false);
void launch_reslot(nb_handle* h, const float4* xq, cudaStream_t st, bool binned = false);
// fold_prune: the build launch also does the dynamic list pruning when due (launch_prune
// then launches nothing)
void launch_build(nb_handle* h, cudaStream_t st, bool fold_prune = false);
void launch_prune(nb_handle* h, cudaStream_t st, bool folded = false);  // returns at once unless due
cudaError_t build_setup(nb_handle* h);
void launch_export_pairs(nb_handle* h, int2* out, long long max_pairs, unsigned long long* counter,
                         cudaStream_t st);
// pair.cu
void launch_pair(nb_handle* h, int terms, cudaStream_t st);
void launch_vjp(nb_handle* h, int terms, cudaStream_t st);
// exclusion correction (when deferred), force output (f_out, may be null) and energy
// reduction (dst, may be null) of a force evaluation in one launch
void launch_epilogue(nb_handle* h, int terms, float* f_out, double* dst, cudaStream_t st, bool precise = false);
cudaError_t pair_setup(nb_handle* h);
// allpairs.cu
void launch_allpairs_lj(nb_handle* h, const float4* xq, cudaStream_t st);
// pme.cu
cudaError_t pme_setup(nb_handle* h);
int launch_pme(nb_handle* h, cudaStream_t st);  // spread + FFT + convolve + FFT + gather into ffix
int launch_pme_vjp(nb_handle* h, cudaStream_t st);  // launch_pme, then the reciprocal VJP into gx_s
void launch_pme_spread(nb_handle* h, const float4* x, cudaStream_t st);  // x: caller or slot order
int launch_pme_fft(nb_handle* h, int inverse, cudaStream_t st);
void launch_pme_convolve(nb_handle* h, cudaStream_t st);
// adds -q grad into ffix: atom i of x at slot slot_of[i] (x in caller order), or slot i (null)
void launch_pme_gather(nb_handle* h, const float4* x, const int* slot_of, cudaStream_t st);
void launch_pme_spread_only(nb_handle* h, float* grid_out, cudaStream_t st);
void launch_pme_gather_only(nb_handle* h, const float* phi, float* f_out, cudaStream_t st);
// Validity check of one atom at position p (caller index i, slot k): true when it has
// moved more than r_skin/2 from its position at the last build (or the position is not
// finite), which requests a rebuild.  Writes the atom's slot position in the frame of the
// last build (the wrapped position when it requests the rebuild).
__device__ __forceinline__ bool load_atom(float4 p, const SysDev& S, float4 r, const float4* __restrict__ xsb,
                                          float4* __restrict__ xs, int k, const float4* __restrict__ xp = nullptr,
                                          bool* prune = nullptr) {
    float4 w = p;
    float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
    if (S.periodic) {
        dx = mi_any(dx, S.L[0], S.invL[0]);
        dy = mi_any(dy, S.L[1], S.invL[1]);
        dz = mi_any(dz, S.L[2], S.invL[2]);
    }
    float d2 = dx * dx + dy * dy + dz * dz;
    const bool need = !(d2 <= S.disp2);  // NaN (first call, bad input) also requests a rebuild
    if (S.periodic) {
        // an atom that needs the rebuild is wrapped (the rebuild re-slots it anyway;
        // calls that only spread or gather PME charges use it as it is)
        const float4 b = xsb[k];
        w = need ? make_float4(wrap1(p.x, S.L[0], S.invL[0]), wrap1(p.y, S.L[1], S.invL[1]),
                               wrap1(p.z, S.L[2], S.invL[2]), p.w)
                 : make_float4(b.x + dx, b.y + dy, b.z + dz, p.w);
    }
    xs[k] = w;
    if (prune && S.prune2 > 0.f && !need) {
        // displacement since the last prune, both positions in the frame of the last build
        const float4 q = xp[k];
        const float ex = w.x - q.x, ey = w.y - q.y, ez = w.z - q.z;
        *prune = !(ex * ex + ey * ey + ez * ez <= S.prune2);
    }
    return need;
}

// A load's prune request for system s (pr: one of its atoms has moved more than half the
// prune skin since the last prune), one atomic per system among the warp's requesting lanes
// (when a prune falls due, most atoms request it at once).  Called by all lanes of `act`.
__device__ __forceinline__ void request_prune(unsigned act, bool pr, int s, unsigned* prune_sys, unsigned* flags) {
    const unsigned want = __ballot_sync(act, pr);
    if (!want) return;
    const unsigned grp = __match_any_sync(act, pr ? s : -1);
    if (pr && (threadIdx.x & 31) == __ffs(grp & want) - 1) {
        atomicOr(&prune_sys[s], kPruneReq);
        atomicOr(&flags[NB_FLAG_PRUNE_ANY], 1u);
    }
}

// The next evaluation's load, done by the integrator right after the drift: the new
// positions' validity check and slot positions, the zeroing of the fixed-point forces
// (each thread zeroes the slot whose force it has just read) and the clearing of the
// fresh-list flag.  xs == nullptr: none.
struct LoadNext {
    const float4* xref = nullptr;
    const float4* xsb = nullptr;
    float4* xs = nullptr;
    long long* ffix = nullptr;
    unsigned* flags = nullptr;
    const float4* x_prune = nullptr;
    unsigned* prune_sys = nullptr;
};

// Blocks per cell for a cell kernel whose blocks hold `warps` warps and want at least
// `atoms_per_warp` atoms per warp on average: 1 unless the cells are too few to give
// every SM several blocks.
inline int pick_split(const nb_handle* h, int warps, int atoms_per_warp) {
    if (h->blocks_per_cell) return h->blocks_per_cell;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long target = 4LL * sms;
    if (h->n_cells >= target) return 1;
    const int want = (int)std::min<long long>(32, (target + h->n_cells - 1) / h->n_cells);
    const int fill = (int)((double)h->n_atoms / h->n_cells / ((double)warps * atoms_per_warp));
    return std::max(1, std::min(want, fill));
}

// dynamics.cu
// Observables of an HMC trajectory recorded by the integrator at integer step `step`
// (before its drift): the squared minimum-image jump |x - x0|^2 of every atom (FP64,
// caller order) and, for each system s with l_prop[s] == step, its positions as the
// proposal.  x0 == nullptr records nothing.
struct StepObs {
    const float4* x0 = nullptr;
    double* jump = nullptr;
    const int* l_prop = nullptr;
    float4* x_prop = nullptr;
    int step = 0;
};
// Statistics of the state whose energies a reduction sums: with sstat != nullptr, per
// system (dH, alpha, jump) = (H - H_ref, min(1, exp(-dH/kT)), sum of `jump`).
struct StepStat {
    const double* jump = nullptr;
    const double* e_ref = nullptr;
    double kT = 1.0;
    double* sstat = nullptr;
};
// Loss cotangents entering the HMC adjoint at one state l: ga[s] and gj[s] of the
// acceptance probability and squared jump of proposing state l, alpha[s * a_stride] its
// acceptance probability.  ga == nullptr: no loss term at this state.
struct Inject {
    const double* ga = nullptr;
    const double* gj = nullptr;
    const double* alpha = nullptr;
    int a_stride = 0;
};
void launch_reduce_energy(nb_handle* h, int terms, int with_kin, double* dst, cudaStream_t st,
                          const StepStat& ss = StepStat(), bool precise = false);
void launch_finalize_forces(nb_handle* h, float* f_out, cudaStream_t st);
void launch_integrate(nb_handle* h, float4* xq, float4* v, const float* w_override, const float* dt,
                      float c_pre, float c_post, int drift, float4* ck_x, float4* ck_v,
                      float4* ck_p, cudaStream_t st, const StepObs& ob = StepObs(), bool load_next = false);
void launch_hmc_init(nb_handle* h, const float* w, const float* xi, double kT, cudaStream_t st);
void launch_hmc_finish(nb_handle* h, float4* x_out, const float4* x0, double kT, const double* u,
                       double* stats, cudaStream_t st);
void launch_hmc_pick(nb_handle* h, float4* x_out, const float4* x0, const int* l_prop, int n_leap,
                     const double* step_stats, const double* u, double* stats, cudaStream_t st);
void launch_bwd_lambda(nb_handle* h, const float* w, const float* dt, const float4* v_state,
                       const Inject& inj, double kT, cudaStream_t st);
void launch_bwd_adjoint(nb_handle* h, const float* w, const float* dt, const float4* x_state,
                        const float4* v_state, const float4* x0, const Inject& inj, double kT,
                        const float4* p_prev, float* wbar, cudaStream_t st);
void launch_bwd_final(nb_handle* h, const float* w, const float* dt, const float* xi, double kT,
                      float* wbar, double* g_dt, cudaStream_t st);
// langevin.cu
void launch_langevin(nb_handle* h, float4* xq, float4* v, const float* dt, const float* gamma, double kT,
                     const float* xi, cudaStream_t st, bool load_next = false);
void launch_kinetic(nb_handle* h, const float4* v, cudaStream_t st);
void launch_settle(nb_handle* h, const float4* x_ref, float4* x, float4* v, const float* inv_mass, float dt,
                   cudaStream_t st);
void launch_rattle(nb_handle* h, const float4* x, float4* v, cudaStream_t st);

}  // namespace nb
