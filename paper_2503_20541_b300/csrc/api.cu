// api.cu -- handle lifecycle and the C entry points of libnbcore (include/nbcore.h).
//
// Each entry point only enqueues kernels on the caller's stream; the only host
// synchronisations are nl_build (which returns a count), nb_check,
// nb_rebuild_count, nb_timing_read and nb_destroy.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"

using namespace nb;

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

nb_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return NB_OK;
    if (e == cudaErrorMemoryAllocation) return NB_ERR_NOMEM;
    return NB_ERR_CUDA;
}

template <class T>
cudaError_t dalloc(nb_handle* h, T** p, size_t count) {
    if (count == 0) count = 1;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, sizeof(T) * count);
    if (e == cudaSuccess) {
        h->allocs.push_back(q);
        *p = static_cast<T*>(q);
    }
    return e;
}

void free_all(nb_handle* h) {
    cudaDeviceSynchronize();
    for (auto& g : h->fft) {
        if (g.has_r2c) cufftDestroy(g.r2c);
        if (g.has_c2r) cufftDestroy(g.c2r);
    }
    for (void* p : h->allocs) cudaFree(p);
    h->allocs.clear();
}

inline cudaStream_t S(void* st) { return static_cast<cudaStream_t>(st); }

int round_up(long long a, int b) { return (int)(((a + b - 1) / b) * b); }

const float4* F4(const float* p) { return reinterpret_cast<const float4*>(p); }
float4* F4(float* p) { return reinterpret_cast<float4*>(p); }

void request_rebuild(nb_handle* h, cudaStream_t st) { cudaMemsetAsync(h->flags, 0x01, sizeof(unsigned), st); }

// Brackets the kernels of one stage with CUDA events when timing is enabled.
// Stages may nest (the list build inside the rebuild): each remembers its own end event.
struct Stage {
    nb_handle* h;
    cudaStream_t st;
    cudaEvent_t end = nullptr;
    explicit Stage(nb_handle* hh, int stage, cudaStream_t s) : h(hh), st(s) {
        if (!h->timing) return;
        for (int k = 0; k < 2; ++k) {
            cudaEvent_t e;
            if (h->ev_pool.empty()) {
                cudaEventCreate(&e);
            } else {
                e = h->ev_pool.back();
                h->ev_pool.pop_back();
            }
            h->ev_used.push_back(e);
        }
        h->ev_stage.push_back(stage);
        end = h->ev_used.back();
        cudaEventRecord(h->ev_used[h->ev_used.size() - 2], st);
    }
    ~Stage() {
        if (h->timing) cudaEventRecord(end, st);
    }
};

// Validity check, conditional rebuild (device-side flag), flag reset.  loaded: the
// integrator has already done the check (launch_integrate with load_next).
void prepare(nb_handle* h, const float4* xq, bool force, cudaStream_t st, bool loaded = false) {
    bool binned = false;
    {
        Stage sc(h, NB_STAGE_CHECK, st);
        if (force) request_rebuild(h, st);
        if (!loaded) binned = launch_load(h, xq, st, force);
    }
    {
        Stage sc(h, NB_STAGE_REBUILD, st);
        launch_reslot(h, xq, st, binned);
        Stage sb(h, NB_STAGE_BUILD, st);
        launch_build(h, st);
    }
    launch_prune(h, st);
}

// The mesh half of PME (spread, FFT, convolution, inverse FFT) for positions x.
nb_status run_pme_mesh(nb_handle* h, const float4* x, cudaStream_t st) {
    {
        Stage sc(h, NB_STAGE_SPREAD, st);
        launch_pme_spread(h, x, st);
    }
    {
        Stage sc(h, NB_STAGE_FFT, st);
        if (launch_pme_fft(h, 0, st)) return NB_ERR_CUDA;
    }
    {
        Stage sc(h, NB_STAGE_CONVOLVE, st);
        launch_pme_convolve(h, st);
    }
    Stage sc(h, NB_STAGE_FFT, st);
    if (launch_pme_fft(h, 1, st)) return NB_ERR_CUDA;
    return NB_OK;
}

// Full force evaluation into h->ffix (slot order) and the energy partials.  After the
// load, PME runs on the handle's second stream (forked and joined with events; under
// CUDA-graph capture this becomes a fork/join of the graph).  Its mesh half reads the
// caller's positions and charges, not the slot order, so it overlaps the (conditional)
// list rebuild; the gather waits for the rebuild only because it adds into ffix by slot,
// and then overlaps the pair kernel.  Both add per-atom fixed-point forces into ffix
// (zeroed by the load): integer sums, so the result does not depend on which finishes
// first.
// energy: the per-atom energies are reduced afterwards (otherwise the pair kernel runs its
// force-only form and leaves them unwritten).
nb_status eval(nb_handle* h, const float4* xq, int terms, bool force, cudaStream_t st, bool loaded = false,
               bool energy = true) {
    const bool pme = (terms & NB_TERM_PME) && h->has_pme;
    if (terms & kTermPrecise) h->xq_in = xq;  // the two-float energy pass reads the caller's positions
    bool binned = false;
    {
        Stage sc(h, NB_STAGE_CHECK, st);
        if (force) request_rebuild(h, st);
        if (!loaded) binned = launch_load(h, xq, st, force);
    }
    nb_status s = NB_OK;
    if (pme) {
        cudaEventRecord(h->ev_fork, st);
        cudaStreamWaitEvent(h->aux, h->ev_fork, 0);
        s = run_pme_mesh(h, xq, h->aux);
    }
    {
        Stage sc(h, NB_STAGE_REBUILD, st);
        launch_reslot(h, xq, st, binned);
        Stage sb(h, NB_STAGE_BUILD, st);
        launch_build(h, st, pme);  // with PME running alongside, the prune rides in the build launch
    }
    launch_prune(h, st, pme);
    if (pme) {
        cudaEventRecord(h->ev_built, st);
        cudaStreamWaitEvent(h->aux, h->ev_built, 0);
        {
            Stage sc(h, NB_STAGE_GATHER, h->aux);
            launch_pme_gather(h, xq, h->iperm, h->aux);
        }
        cudaEventRecord(h->ev_join, h->aux);
    }
    {
        Stage sc(h, NB_STAGE_PAIR, st);
        launch_pair(h, terms | (energy ? kTermEnergy : 0), st);
    }
    if (pme) cudaStreamWaitEvent(st, h->ev_join, 0);
    return s;
}

nb_status launched() { return from_cuda(cudaGetLastError()); }

__global__ void k_lam_scatter(int N, const float* __restrict__ lam, const int* __restrict__ iperm,
                              float4* __restrict__ out) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[iperm[i]] = make_float4(lam[3 * (size_t)i], lam[3 * (size_t)i + 1], lam[3 * (size_t)i + 2], 0.f);
}

__global__ void k_vjp_out(int N, const float4* __restrict__ gx_s, const float2* __restrict__ gp_s,
                          const int* __restrict__ iperm, float* __restrict__ gx, float* __restrict__ gq,
                          float* __restrict__ gsig, float* __restrict__ geps) {
    pdl_wait();
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int k = iperm[i];
    float4 g = gx_s[k];
    gx[3 * (size_t)i] = g.x;
    gx[3 * (size_t)i + 1] = g.y;
    gx[3 * (size_t)i + 2] = g.z;
    if (gq) gq[i] = g.w;
    float2 p = gp_s[k];
    if (gsig) gsig[i] = p.x;
    if (geps) geps[i] = p.y;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

}  // namespace

extern "C" {

const char* nb_status_str(nb_status s) {
    switch (s) {
        case NB_OK: return "ok";
        case NB_ERR_ARG: return "invalid argument";
        case NB_ERR_BOX_TOO_SMALL: return "periodic box edge smaller than 2 r_nl";
        case NB_ERR_LIST_OVERFLOW: return "neighbour list capacity exceeded";
        case NB_ERR_FIXEDPOINT_OVERFLOW: return "fixed-point force accumulator overflow";
        case NB_ERR_NONFINITE: return "non-finite coordinate";
        case NB_ERR_TIMEOUT: return "device wait timed out";
        case NB_ERR_CUDA: return "CUDA or cuFFT error";
        case NB_ERR_NOMEM: return "device allocation failed";
    }
    return "unknown status";
}

nb_status nb_create(nb_handle** out, const nb_system_desc* sys, int32_t n_systems, const float* sigma,
                    const float* sqrt_eps, const int32_t* excl_off, const int32_t* excl_idx,
                    const nb_options* opt) {
    if (!out) return NB_ERR_ARG;
    *out = nullptr;
    if (!sys || n_systems <= 0 || !sigma || !sqrt_eps) return NB_ERR_ARG;
    long long N = 0;
    int coul_kind = 0;
    for (int s = 0; s < n_systems; ++s) {
        const nb_system_desc& d = sys[s];
        if (d.n_atoms <= 0) return NB_ERR_ARG;
        for (int k = 0; k < 3; ++k)
            if (!finite_pos(d.box[k])) return NB_ERR_ARG;
        if (!finite_pos(d.r_cut) || !(d.r_skin >= 0.0) || !std::isfinite(d.r_skin)) return NB_ERR_ARG;
        if (d.r_switch >= d.r_cut) return NB_ERR_ARG;
        if (!(d.alpha >= 0.0) || !std::isfinite(d.alpha) || !std::isfinite(d.ke)) return NB_ERR_ARG;
        if (d.eps_rf != 0.0) {
            // reaction field: no Ewald splitting, no mesh
            if (!(d.eps_rf >= 1.0) || !std::isfinite(d.eps_rf) || d.alpha != 0.0) return NB_ERR_ARG;
            if (d.pme_grid[0] || d.pme_grid[1] || d.pme_grid[2]) return NB_ERR_ARG;
        }
        if (d.ke != 0.0) {
            const int kind = d.eps_rf != 0.0 ? 2 : 1;
            if (coul_kind != 0 && coul_kind != kind) return NB_ERR_ARG;  // one electrostatics per handle
            coul_kind = kind;
        }
        double rnl = d.r_cut + d.r_skin;
        if (d.periodic)
            for (int k = 0; k < 3; ++k)
                if (d.box[k] < 2.0 * rnl) return NB_ERR_BOX_TOO_SMALL;
        int npme = (d.pme_grid[0] > 0) + (d.pme_grid[1] > 0) + (d.pme_grid[2] > 0);
        if (npme != 0 && npme != 3) return NB_ERR_ARG;
        if (npme == 3) {
            if (!d.periodic || !(d.alpha > 0.0)) return NB_ERR_ARG;
            if (d.pme_order != 4 && d.pme_order != 0) return NB_ERR_ARG;
            for (int k = 0; k < 3; ++k)
                if (d.pme_grid[k] < 4) return NB_ERR_ARG;
        }
        N += d.n_atoms;
    }
    if (N >= (1LL << 31) - 64) return NB_ERR_ARG;
    nb_options o;
    std::memset(&o, 0, sizeof(o));
    if (opt) o = *opt;
    if (o.cell_div != 0 && o.cell_div != 1 && o.cell_div != 2) return NB_ERR_ARG;
    if (o.stencil_tile != 0 && (o.stencil_tile < 256 || o.stencil_tile > 4096 || o.stencil_tile % 64 != 0))
        return NB_ERR_ARG;
    if (o.max_neighbors < 0 || o.force_bits < 0 || o.force_bits > 48 || (o.force_bits > 0 && o.force_bits < 8))
        return NB_ERR_ARG;
    if (o.blocks_per_cell < 0 || o.blocks_per_cell > 32) return NB_ERR_ARG;
    if (!(o.prune_skin == o.prune_skin)) return NB_ERR_ARG;  // NaN

    // exclusions: validate and symmetrise
    std::vector<std::vector<int>> ex((size_t)N);
    std::vector<int> sid_h((size_t)N);
    {
        long long off = 0;
        for (int s = 0; s < n_systems; ++s) {
            for (int a = 0; a < sys[s].n_atoms; ++a) sid_h[(size_t)(off + a)] = s;
            off += sys[s].n_atoms;
        }
    }
    if (excl_off) {
        if (excl_off[0] != 0) return NB_ERR_ARG;
        for (long long i = 0; i < N; ++i) {
            if (excl_off[i + 1] < excl_off[i]) return NB_ERR_ARG;
            for (int e = excl_off[i]; e < excl_off[i + 1]; ++e) {
                if (!excl_idx) return NB_ERR_ARG;
                long long j = excl_idx[e];
                if (j < 0 || j >= N || j == i || sid_h[(size_t)j] != sid_h[(size_t)i]) return NB_ERR_ARG;
                ex[(size_t)i].push_back((int)j);
                ex[(size_t)j].push_back((int)i);
            }
        }
    }
    std::vector<int> ex_off_h((size_t)N + 1, 0), ex_idx_h;
    for (long long i = 0; i < N; ++i) {
        auto& v = ex[(size_t)i];
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        ex_off_h[(size_t)i + 1] = ex_off_h[(size_t)i] + (int)v.size();
        ex_idx_h.insert(ex_idx_h.end(), v.begin(), v.end());
    }
    int max_excl = 0;
    for (long long i = 0; i < N; ++i) max_excl = std::max(max_excl, ex_off_h[(size_t)i + 1] - ex_off_h[(size_t)i]);
    ex.clear();
    ex.shrink_to_fit();

    nb_handle* h = new (std::nothrow) nb_handle();
    if (!h) return NB_ERR_NOMEM;
    h->coul_kind = coul_kind ? coul_kind : 1;
    cudaGetDevice(&h->device);
    h->n_sys = n_systems;
    h->n_atoms = (int)N;
    h->max_excl = max_excl;
    h->desc.assign(sys, sys + n_systems);

    // tuning defaults from the densest system; the list capacity is a multiple of 128
    // entries because the pair kernels read rows in 128-entry groups
    double nb_max = 0.0;
    int n_max = 0;
    // cell size per system: the handle's option for all, or by default cells of edge
    // r_nl/2 for a system with >= 5 of them along every axis and >= 64 atoms per r_nl^3
    // (dense enough for the finer stencil to pay), else cells of edge r_nl
    std::vector<int> cell_div((size_t)n_systems, o.cell_div);
    for (int s = 0; s < n_systems; ++s) {
        const nb_system_desc& d = sys[s];
        double rnl = d.r_cut + d.r_skin;
        double V = d.box[0] * d.box[1] * d.box[2];
        nb_max = std::max(nb_max, d.n_atoms / V * 4.18879020478639 * rnl * rnl * rnl);
        n_max = std::max(n_max, d.n_atoms);
        if (o.cell_div) continue;
        bool fine = d.n_atoms / V * rnl * rnl * rnl >= 64.0;
        for (int k = 0; k < 3; ++k)
            if (std::floor(d.box[k] * 2.0 / rnl) < 5.0) fine = false;
        cell_div[(size_t)s] = fine ? 2 : 1;
    }
    h->cell_div = o.cell_div;
    if (o.max_neighbors > 0) {
        h->cap = std::max(128, round_up(o.max_neighbors, 128));
    } else {
        h->cap = round_up((long long)(1.5 * nb_max + 64.0), 128);
        h->cap = std::max(128, std::min(h->cap, round_up(n_max, 128)));
    }
    h->force_bits = o.force_bits ? o.force_bits : 32;
    h->fscale = std::ldexp(1.0f, h->force_bits);
    h->finv = std::ldexp(1.0f, -h->force_bits);
    h->gscale = std::ldexp(1.0, 32);

    // per-system constants and cell grids
    h->sys_h.resize(n_systems);
    int cell_off = 0, atom_off = 0;
    for (int s = 0; s < n_systems; ++s) {
        const nb_system_desc& d = sys[s];
        SysDev& D = h->sys_h[s];
        std::memset(&D, 0, sizeof(D));
        double rnl = d.r_cut + d.r_skin;
        long long ncells = 1;
        for (int k = 0; k < 3; ++k) {
            D.L[k] = (float)d.box[k];
            D.invL[k] = (float)(1.0 / d.box[k]);
            D.halfL[k] = (float)(0.5 * d.box[k]);
            int nc = std::max(1, (int)std::floor(d.box[k] * cell_div[(size_t)s] / rnl));
            nc = std::min(nc, 1024);
            D.nc[k] = nc;
            D.cell_scale[k] = (float)(nc / d.box[k]);
            ncells *= nc;
        }
        if ((long long)cell_off + ncells >= (1LL << 31) - 1) {
            delete h;
            return NB_ERR_ARG;
        }
        D.index = s;
        D.rc2 = (float)(d.r_cut * d.r_cut);
        D.rc = (float)d.r_cut;
        D.rnl2 = (float)(rnl * rnl);
        D.disp2 = (float)(0.25 * d.r_skin * d.r_skin);
        {
            // inner skin of dynamic list pruning (off: 0)
            double ps = o.prune_skin;
            if (ps == 0.0) ps = d.r_skin >= 0.15 * d.r_cut ? d.r_skin / 3.0 : -1.0;
            const bool on = ps > 0.0 && ps < d.r_skin;
            D.rin2 = on ? (float)((d.r_cut + ps) * (d.r_cut + ps)) : 0.f;
            D.prune2 = on ? (float)(0.25 * ps * ps) : 0.f;
            if (on) h->any_prune = 1;
        }
        D.has_switch = (d.r_switch >= 0.0 && d.r_switch < d.r_cut) ? 1 : 0;
        D.rs = D.has_switch ? (float)d.r_switch : 0.f;
        D.inv_sw = D.has_switch ? (float)(1.0 / (d.r_cut - d.r_switch)) : 0.f;
        D.inv_sw_lo = D.has_switch ? (float)(1.0 / (d.r_cut - d.r_switch) - (double)D.inv_sw) : 0.f;
        D.alpha = (float)d.alpha;
        D.ke = (float)d.ke;
        D.beta2 = (float)(d.alpha * d.alpha);
        D.cell_off = cell_off;
        D.atom_off = atom_off;
        D.n_atoms = d.n_atoms;
        D.periodic = d.periodic ? 1 : 0;
        D.has_coul = d.ke != 0.0;
        if (D.has_coul) h->any_coul = 1;
        else h->any_uncharged = 1;
        D.has_lj = 1;
        D.pme = d.pme_grid[0] > 0;
        for (int k = 0; k < 3; ++k) {
            D.K[k] = D.pme ? d.pme_grid[k] : 0;
            double kl = D.K[k] / d.box[k];
            D.kl_hi[k] = (float)kl;
            D.kl_lo[k] = (float)(kl - (double)D.kl_hi[k]);
        }
        D.stencil = cell_div[(size_t)s];
        D.red_tile = red_tile(D.n_atoms);
        if (D.periodic)
            for (int k = 0; k < 3; ++k)
                if (D.nc[k] < 4 * D.stencil) h->build_gen = 1;  // per-pair images in some cells
        D.self_coef = -d.ke * d.alpha / std::sqrt(3.14159265358979323846);
        if (d.eps_rf != 0.0) {
            const double den = 2.0 * d.eps_rf + 1.0;
            const double k = (d.eps_rf - 1.0) / (den * d.r_cut * d.r_cut * d.r_cut);
            const double c = 3.0 * d.eps_rf / (den * d.r_cut);
            D.krf = (float)k;
            D.crf = (float)c;
            D.krf_lo = (float)(k - (double)D.krf);
            D.crf_lo = (float)(c - (double)D.crf);
        } else {
            D.krf = D.crf = D.krf_lo = D.crf_lo = 0.f;
        }
        cell_off += (int)ncells;
        atom_off += d.n_atoms;
    }
    h->n_cells = cell_off;
    // shared-memory tile of the cell kernels: the densest system's expected stencil size
    // with ~3 sigma of Poisson headroom; cells above it take several tiles
    if (o.stencil_tile) {
        h->tile = o.stencil_tile;
    } else {
        double cand = 0.0;
        for (int s = 0; s < n_systems; ++s) {
            const nb_system_desc& d = sys[s];
            const SysDev& D = h->sys_h[s];
            double v = d.n_atoms / (d.box[0] * d.box[1] * d.box[2]);
            for (int k = 0; k < 3; ++k) v *= std::min(D.nc[k], 2 * D.stencil + 1) * d.box[k] / D.nc[k];
            cand = std::max(cand, v);
        }
        long long t = round_up((long long)(cand + 3.0 * std::sqrt(cand) + 96.0), 64);
        h->tile = (int)std::max(256LL, std::min(t, 4096LL));
    }
    h->n_scan_blocks = cdiv(h->n_cells, kScanTile);
    h->blocks_per_cell = o.blocks_per_cell;

    cudaError_t e = cudaSuccess;
#define NB_TRY(x)                        \
    do {                                 \
        e = (x);                         \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    {
        NB_TRY(dalloc(h, &h->sys, n_systems));
        NB_TRY(dalloc(h, &h->sid, N));
        NB_TRY(dalloc(h, &h->params, N));
        NB_TRY(dalloc(h, &h->ex_off, N + 1));
        NB_TRY(dalloc(h, &h->ex_idx, ex_idx_h.size()));
        NB_TRY(dalloc(h, &h->cell_count, h->n_cells));
        NB_TRY(dalloc(h, &h->cell_start, (size_t)h->n_cells + 1));
        NB_TRY(dalloc(h, &h->cell_cursor, h->n_cells));
        NB_TRY(dalloc(h, &h->scan_bsum, h->n_scan_blocks));
        NB_TRY(dalloc(h, &h->cell_sys, h->n_cells));
        {
            std::vector<int> cs((size_t)h->n_cells);
            for (int s = 0; s < n_systems; ++s) {
                const SysDev& D = h->sys_h[s];
                int nc = D.nc[0] * D.nc[1] * D.nc[2];
                for (int k = 0; k < nc; ++k) cs[(size_t)D.cell_off + k] = s;
            }
            NB_TRY(cudaMemcpy(h->cell_sys, cs.data(), sizeof(int) * cs.size(), cudaMemcpyHostToDevice));
        }
        NB_TRY(dalloc(h, &h->cellid, N));
        NB_TRY(dalloc(h, &h->perm_tmp, N));
        NB_TRY(dalloc(h, &h->perm, N));
        NB_TRY(dalloc(h, &h->iperm, N));
        NB_TRY(dalloc(h, &h->xs, N));
        NB_TRY(dalloc(h, &h->xsb, N));
        NB_TRY(dalloc(h, &h->ps, N));
        NB_TRY(dalloc(h, &h->xref, N));
        NB_TRY(dalloc(h, &h->nbr, (size_t)N * h->cap));
        NB_TRY(dalloc(h, &h->nbr_cnt, N));
        NB_TRY(dalloc(h, &h->nbr_out, N));
        NB_TRY(dalloc(h, &h->exp_cnt, N));
        h->excl_w = h->max_excl == 0 ? 0 : (h->max_excl <= 2 ? 2 : 4);
        if (h->excl_w) {
            NB_TRY(dalloc(h, &h->ex_slot, (size_t)N * h->excl_w));
            NB_TRY(dalloc(h, &h->ex_cnt, N));
        }
        NB_TRY(dalloc(h, &h->ffix, 3 * (size_t)N));
        NB_TRY(dalloc(h, &h->e_atom, N));
        NB_TRY(dalloc(h, &h->e_lo, N));
        NB_TRY(dalloc(h, &h->flags, kFlagWords));
        NB_TRY(dalloc(h, &h->build_ticket, 1));
        NB_TRY(cudaMemset(h->build_ticket, 0, sizeof(unsigned)));
        NB_TRY(dalloc(h, &h->bin_ticket, 1));
        NB_TRY(cudaMemset(h->bin_ticket, 0, sizeof(unsigned)));
        if (h->any_prune) {
            NB_TRY(dalloc(h, &h->x_prune, N));
            NB_TRY(dalloc(h, &h->prune_sys, n_systems));
            NB_TRY(cudaMemset(h->prune_sys, 0, sizeof(unsigned) * n_systems));
            NB_TRY(dalloc(h, &h->prune_ticket, 1));
            NB_TRY(cudaMemset(h->prune_ticket, 0, sizeof(unsigned)));
            NB_TRY(dalloc(h, &h->prune_cnt, n_systems));
            NB_TRY(cudaMemset(h->prune_cnt, 0, sizeof(unsigned) * n_systems));
        }
        NB_TRY(dalloc(h, &h->energy, (size_t)n_systems * NB_NE));
        NB_TRY(dalloc(h, &h->ke_atom, N));
        NB_TRY(dalloc(h, &h->vwork, N));
        NB_TRY(dalloc(h, &h->lam, N));
        NB_TRY(dalloc(h, &h->gx_s, N));
        NB_TRY(dalloc(h, &h->gp_s, N));
        NB_TRY(dalloc(h, &h->hbar_atom, N));
        NB_TRY(dalloc(h, &h->jump_atom, N));
        NB_TRY(dalloc(h, &h->e0, (size_t)n_systems * NB_NE));
        NB_TRY(dalloc(h, &h->e1, (size_t)n_systems * NB_NE));
        NB_TRY(dalloc(h, &h->xbar, N));
        NB_TRY(dalloc(h, &h->vbar, N));
        NB_TRY(dalloc(h, &h->xwork, N));
        NB_TRY(dalloc(h, &h->groups, N));
        {
            // no constraints until nb_set_water_constraints: every atom is its own group
            std::vector<int4> g((size_t)N);
            for (long long i = 0; i < N; ++i) g[(size_t)i] = make_int4((int)i, -1, -1, 1);
            NB_TRY(cudaMemcpy(h->groups, g.data(), sizeof(int4) * N, cudaMemcpyHostToDevice));
            h->n_groups = (int)N;
            h->sid_host = sid_h;
        }
        NB_TRY(dalloc(h, &h->counter, 1));
        {
            std::vector<int> rb_sys, rb_off(n_systems + 1, 0);
            for (int s = 0; s < n_systems; ++s) {
                rb_off[s] = (int)rb_sys.size();
                for (int b = 0; b < cdiv(sys[s].n_atoms, red_tile(sys[s].n_atoms)); ++b) rb_sys.push_back(s);
            }
            rb_off[n_systems] = (int)rb_sys.size();
            h->n_red_blocks = (int)rb_sys.size();
            NB_TRY(dalloc(h, &h->red_blk_sys, rb_sys.size()));
            NB_TRY(dalloc(h, &h->red_blk_off, rb_off.size()));
            NB_TRY(dalloc(h, &h->red_part, rb_sys.size() * 6 + (size_t)n_systems * 7));
            NB_TRY(dalloc(h, &h->red_ticket, 1));
            NB_TRY(cudaMemset(h->red_ticket, 0, sizeof(unsigned)));
            NB_TRY(cudaMemcpy(h->red_blk_sys, rb_sys.data(), sizeof(int) * rb_sys.size(), cudaMemcpyHostToDevice));
            NB_TRY(cudaMemcpy(h->red_blk_off, rb_off.data(), sizeof(int) * rb_off.size(), cudaMemcpyHostToDevice));
        }

        std::vector<float2> prm((size_t)N);
        for (long long i = 0; i < N; ++i) prm[(size_t)i] = make_float2(sigma[i], sqrt_eps[i]);
        std::vector<int> ident((size_t)N);
        for (long long i = 0; i < N; ++i) ident[(size_t)i] = (int)i;
        NB_TRY(cudaMemcpy(h->sid, sid_h.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
        NB_TRY(cudaMemcpy(h->params, prm.data(), sizeof(float2) * N, cudaMemcpyHostToDevice));
        NB_TRY(cudaMemcpy(h->ex_off, ex_off_h.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
        if (!ex_idx_h.empty())
            NB_TRY(cudaMemcpy(h->ex_idx, ex_idx_h.data(), sizeof(int) * ex_idx_h.size(), cudaMemcpyHostToDevice));
        NB_TRY(cudaMemcpy(h->perm, ident.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
        NB_TRY(cudaMemcpy(h->iperm, ident.data(), sizeof(int) * N, cudaMemcpyHostToDevice));
        NB_TRY(cudaMemset(h->xref, 0xff, sizeof(float4) * N));  // NaN: the first call rebuilds
        NB_TRY(cudaMemset(h->cell_count, 0, sizeof(int) * h->n_cells));
        NB_TRY(cudaMemset(h->cell_cursor, 0, sizeof(int) * h->n_cells));
        NB_TRY(cudaMemset(h->nbr_cnt, 0, sizeof(int) * N));
        NB_TRY(cudaMemset(h->nbr_out, 0, sizeof(int) * N));
        NB_TRY(cudaMemset(h->ffix, 0, sizeof(long long) * 3 * N));
        NB_TRY(cudaMemset(h->e_atom, 0, sizeof(float4) * N));
        NB_TRY(cudaMemset(h->e_lo, 0, sizeof(float4) * N));
        NB_TRY(cudaMemset(h->ke_atom, 0, sizeof(float) * N));
        NB_TRY(cudaMemset(h->flags, 0, sizeof(unsigned) * kFlagWords));
        NB_TRY(cudaMemset(h->xs, 0, sizeof(float4) * N));
        NB_TRY(cudaMemset(h->xsb, 0, sizeof(float4) * N));
        NB_TRY(build_setup(h));
        NB_TRY(pair_setup(h));
        NB_TRY(pme_setup(h));
        NB_TRY(cudaStreamCreateWithFlags(&h->aux, cudaStreamNonBlocking));
        NB_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
        NB_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        NB_TRY(cudaEventCreateWithFlags(&h->ev_built, cudaEventDisableTiming));
        NB_TRY(cudaMemcpy(h->sys, h->sys_h.data(), sizeof(SysDev) * n_systems, cudaMemcpyHostToDevice));
        NB_TRY(cudaDeviceSynchronize());
    }
#undef NB_TRY
    *out = h;
    return NB_OK;
fail:
    free_all(h);
    delete h;
    cudaGetLastError();
    return e == cudaErrorUnknown ? NB_ERR_CUDA : from_cuda(e);
}

void nb_destroy(nb_handle* h) {
    if (!h) return;
    DeviceGuard g(h->device);
    free_all(h);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    if (h->ev_built) cudaEventDestroy(h->ev_built);
    if (h->aux) cudaStreamDestroy(h->aux);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_used) cudaEventDestroy(e);
    delete h;
}

int64_t nb_num_atoms(const nb_handle* h) { return h ? h->n_atoms : 0; }
int32_t nb_num_systems(const nb_handle* h) { return h ? h->n_sys : 0; }

nb_status nb_check(nb_handle* h, void* stream) {
    if (!h) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaError_t e = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return NB_ERR_CUDA;
    unsigned bits = 0;
    if (cudaMemcpy(&bits, h->flags + 1, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess) return NB_ERR_CUDA;
    if (bits) cudaMemset(h->flags + 1, 0, sizeof(unsigned));
    if (bits & NB_DEVERR_NONFINITE) return NB_ERR_NONFINITE;
    if (bits & NB_DEVERR_LIST_OVERFLOW) return NB_ERR_LIST_OVERFLOW;
    if (bits & NB_DEVERR_FIXEDPOINT) return NB_ERR_FIXEDPOINT_OVERFLOW;
    if (bits & NB_DEVERR_ARG) return NB_ERR_ARG;
    return NB_OK;
}

nb_status nb_blocks_per_cell(const nb_handle* h, int32_t* build, int32_t* pair) {
    if (!h) return NB_ERR_ARG;
    if (build) *build = h->split_build;
    if (pair) *pair = h->split_pair;
    return NB_OK;
}

int64_t nb_rebuild_count(nb_handle* h, void* stream) {
    if (!h) return -1;
    DeviceGuard g(h->device);
    cudaStreamSynchronize(S(stream));
    unsigned long long c = 0;
    cudaMemcpy(&c, h->flags + 2, sizeof(c), cudaMemcpyDeviceToHost);
    return (int64_t)c;
}

nb_status nb_timing_enable(nb_handle* h, int32_t enable) {
    if (!h) return NB_ERR_ARG;
    h->timing = enable ? 1 : 0;
    return NB_OK;
}

nb_status nb_timing_read(nb_handle* h, void* stream, double* ms, int64_t* intervals) {
    if (!h || !ms) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    for (int k = 0; k < NB_NSTAGES; ++k) {
        ms[k] = 0.0;
        if (intervals) intervals[k] = 0;
    }
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return NB_ERR_CUDA;
    for (size_t r = 0; r < h->ev_stage.size(); ++r) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, h->ev_used[2 * r], h->ev_used[2 * r + 1]) == cudaSuccess) {
            ms[h->ev_stage[r]] += t;
            if (intervals) intervals[h->ev_stage[r]] += 1;
        }
    }
    for (cudaEvent_t e : h->ev_used) h->ev_pool.push_back(e);
    h->ev_used.clear();
    h->ev_stage.clear();
    cudaGetLastError();
    return NB_OK;
}

nb_status nl_build(nb_handle* h, const float* xq, int32_t* pairs_out, int64_t max_pairs, int64_t* n_pairs_out,
                   int32_t force_rebuild, void* stream) {
    if (!h || !xq || (pairs_out && max_pairs < 0)) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    prepare(h, F4(xq), force_rebuild != 0, st);
    cudaMemsetAsync(h->counter, 0, sizeof(unsigned long long), st);
    launch_export_pairs(h, reinterpret_cast<int2*>(pairs_out), pairs_out ? max_pairs : 0, h->counter, st);
    nb_status s = launched();
    if (s != NB_OK) return s;
    unsigned long long c = 0;
    if (cudaMemcpyAsync(&c, h->counter, sizeof(c), cudaMemcpyDeviceToHost, st) != cudaSuccess) return NB_ERR_CUDA;
    s = nb_check(h, stream);
    if (n_pairs_out) *n_pairs_out = (int64_t)c;
    return s;
}

nb_status nonbonded_forces(nb_handle* h, const float* xq, float* f_out, double* energies, int32_t terms,
                           void* stream) {
    if (!h || !xq) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    int t = terms & NB_TERM_ALL;
    // with an output to write, the exclusion correction, the force output and the energy
    // reduction run as one epilogue kernel after the pair kernel and the PME gather
    const bool epi = f_out || energies;
    const bool precise = energies && (terms & NB_ENERGY_PRECISE);
    nb_status s = eval(h, F4(xq), t | (epi ? kTermDeferExcl : 0) | (precise ? kTermPrecise : 0),
                       (terms & NB_FORCE_REBUILD) != 0, st, false, energies != nullptr);
    if (s != NB_OK) return s;
    Stage sc(h, NB_STAGE_UPDATE, st);
    if (epi) launch_epilogue(h, t, f_out, energies, st, precise);
    return launched();
}

nb_status nonbonded_forces_allpairs(nb_handle* h, const float* xq, float* f_out, double* energies, void* stream) {
    if (!h || !xq) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    launch_allpairs_lj(h, F4(xq), st);
    if (energies) launch_reduce_energy(h, NB_TERM_LJ, 0, energies, st);
    if (f_out) launch_finalize_forces(h, f_out, st);
    return launched();
}

nb_status pme_spread(nb_handle* h, const float* xq, float* grid, void* stream) {
    if (!h || !xq || !grid) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    launch_load(h, F4(xq), st);
    launch_pme_spread_only(h, grid, st);
    return launched();
}

nb_status pme_gather(nb_handle* h, const float* xq, const float* phi, float* f_out, void* stream) {
    if (!h || !xq || !phi || !f_out) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    launch_load(h, F4(xq), st);
    launch_pme_gather_only(h, phi, f_out, st);
    return launched();
}

nb_status nb_set_water_constraints(nb_handle* h, const int32_t* mols, int32_t n_mol, double d_oh, double d_hh) {
    if (!h || n_mol < 0 || (n_mol > 0 && !mols)) return NB_ERR_ARG;
    if (n_mol > 0 && !(d_oh > 0.0 && d_hh > 0.0 && d_hh < 2.0 * d_oh && std::isfinite(d_oh))) return NB_ERR_ARG;
    const int N = h->n_atoms;
    std::vector<char> used((size_t)N, 0);
    std::vector<int4> g;
    g.reserve((size_t)N);
    for (int m = 0; m < n_mol; ++m) {
        const int a = mols[3 * m], b = mols[3 * m + 1], c = mols[3 * m + 2];
        for (int i : {a, b, c})
            if (i < 0 || i >= N || used[(size_t)i]++) return NB_ERR_ARG;  // out of range or in two molecules
        if (h->sid_host[(size_t)a] != h->sid_host[(size_t)b] || h->sid_host[(size_t)a] != h->sid_host[(size_t)c])
            return NB_ERR_ARG;
        g.push_back(make_int4(a, b, c, 3));
    }
    for (int i = 0; i < N; ++i)
        if (!used[(size_t)i]) g.push_back(make_int4(i, -1, -1, 1));
    DeviceGuard dg(h->device);
    if (cudaMemcpy(h->groups, g.data(), sizeof(int4) * g.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return NB_ERR_CUDA;
    h->n_groups = (int)g.size();
    h->n_water = n_mol;
    h->d_oh = d_oh;
    h->d_hh = d_hh;
    return NB_OK;
}

nb_status langevin_step(nb_handle* h, float* xq, float* v, const float* dt, const float* gamma, double kT,
                        int32_t n_steps, const float* xi, double* energies, int32_t terms, void* stream) {
    if (!h || !xq || !v || !dt || !gamma || !xi || n_steps < 1 || !(kT >= 0.0)) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    const int t = terms & NB_TERM_ALL;
    float4* x4 = F4(xq);
    float4* v4 = F4(v);
    const size_t stride = (size_t)h->n_sys * NB_NE;
    for (int step = 0; step <= n_steps; ++step) {
        if (step == n_steps && !energies) break;  // the final state's forces serve only its energies
        nb_status s = eval(h, x4, t, step == 0 && (terms & NB_FORCE_REBUILD), st, step > 0, energies != nullptr);
        if (s != NB_OK) return s;
        Stage sc(h, NB_STAGE_UPDATE, st);
        if (step < n_steps) launch_langevin(h, x4, v4, dt, gamma, kT, xi + (size_t)step * 3 * h->n_atoms, st, true);
        else launch_kinetic(h, v4, st);
        if (energies) launch_reduce_energy(h, t, 1, energies + (size_t)step * stride, st);
    }
    return launched();
}

nb_status constrain_positions(nb_handle* h, const float* x_ref, float* x, float* v, const float* inv_mass, float dt,
                              void* stream) {
    if (!h || !x_ref || !x || !inv_mass || (v && !(dt > 0.f))) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    launch_settle(h, F4(x_ref), F4(x), v ? F4(v) : nullptr, inv_mass, dt, S(stream));
    return launched();
}

nb_status constrain_velocities(nb_handle* h, const float* x, float* v, void* stream) {
    if (!h || !x || !v) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    launch_rattle(h, F4(x), F4(v), S(stream));
    return launched();
}

nb_status md_step(nb_handle* h, float* xq, float* v, const float* dt, int32_t n_steps, double* energies,
                  int32_t terms, void* stream) {
    if (!h || !xq || !v || !dt || n_steps < 1) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    int t = terms & NB_TERM_ALL;
    float4* x4 = F4(xq);
    float4* v4 = F4(v);
    const size_t stride = (size_t)h->n_sys * NB_NE;
    nb_status s;
    for (int step = 0; step <= n_steps; ++step) {
        // after the first step the integrator has done the check of the new positions
        s = eval(h, x4, t, step == 0 && (terms & NB_FORCE_REBUILD), st, step > 0, energies != nullptr);
        if (s != NB_OK) return s;
        float c_pre = step == 0 ? 0.f : 0.5f;
        float c_post = step == n_steps ? 0.f : 0.5f;
        Stage sc(h, NB_STAGE_UPDATE, st);
        launch_integrate(h, x4, v4, nullptr, dt, c_pre, c_post, step < n_steps, nullptr, nullptr, nullptr, st,
                         StepObs(), step < n_steps);
        if (energies) launch_reduce_energy(h, t, 1, energies + (size_t)step * stride, st);
    }
    return launched();
}

nb_status hmc_trajectory(nb_handle* h, const float* x0, float* x_out, const float* inv_mass, const float* dt,
                         int32_t n_leap, double kT, const float* xi, const double* u, double* stats, float* ckpt,
                         int32_t ckpt_every, int32_t terms, void* stream) {
    if (!h || !x0 || !x_out || x0 == x_out || !inv_mass || !dt || !xi || !u || !stats || n_leap < 1 || !(kT > 0.0))
        return NB_ERR_ARG;
    if (ckpt && ckpt_every < 1) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    int t = terms & NB_TERM_ALL;
    int N = h->n_atoms;
    float4* x = F4(x_out);
    float4* ck = ckpt ? F4(ckpt) : nullptr;
    // precise energies at the two end states (dH)
    const bool precise = (terms & NB_ENERGY_PRECISE) != 0;
    const int tp = t | (precise ? kTermPrecise : 0);
    cudaMemcpyAsync(x_out, x0, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st);
    launch_hmc_init(h, inv_mass, xi, kT, st);
    nb_status s = eval(h, x, tp, ck != nullptr, st);
    if (s != NB_OK) return s;
    launch_reduce_energy(h, t, 1, h->e0, st, StepStat(), precise);
    for (int l = 0; l < n_leap; ++l) {
        float4* cx = nullptr;
        float4* cv = nullptr;
        if (ck && l % ckpt_every == 0) {
            cx = ck + (size_t)(l / ckpt_every) * 2 * N;
            cv = cx + N;
        }
        {
            Stage sc(h, NB_STAGE_UPDATE, st);
            launch_integrate(h, x, h->vwork, inv_mass, dt, l == 0 ? 0.f : 0.5f, 0.5f, 1, cx, cv, nullptr, st,
                             StepObs(), true);
        }
        // the energies of the end state only (dH); the inner steps need forces alone
        const bool last = l == n_leap - 1;
        s = eval(h, x, last ? tp : t, ck != nullptr && (l + 1) % ckpt_every == 0, st, true, last);
        if (s != NB_OK) return s;
    }
    Stage sc(h, NB_STAGE_UPDATE, st);
    launch_integrate(h, x, h->vwork, inv_mass, dt, 0.5f, 0.f, 0, nullptr, nullptr, nullptr, st);
    launch_reduce_energy(h, t, 1, h->e1, st, StepStat(), precise);
    launch_hmc_finish(h, x, F4(x0), kT, u, stats, st);
    return launched();
}

nb_status hmc_trajectory_steps(nb_handle* h, const float* x0, float* x_out, const float* inv_mass, const float* dt,
                               int32_t n_leap, const int32_t* l_prop, double kT, const float* xi, const double* u,
                               double* stats, double* step_stats, float* ckpt, int32_t ckpt_every, int32_t terms,
                               void* stream) {
    if (!h || !x0 || !x_out || x0 == x_out || !inv_mass || !dt || !l_prop || !xi || !u || !stats || !step_stats ||
        n_leap < 1 || !(kT > 0.0))
        return NB_ERR_ARG;
    if (ckpt && ckpt_every < 1) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    int t = terms & NB_TERM_ALL;
    int N = h->n_atoms;
    // the trajectory runs in xwork; x_out receives each system's state at step l_prop[s]
    float4* x = h->xwork;
    float4* ck = ckpt ? F4(ckpt) : nullptr;
    cudaMemcpyAsync(x, x0, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st);
    launch_hmc_init(h, inv_mass, xi, kT, st);
    nb_status s = eval(h, x, t, ck != nullptr, st);
    if (s != NB_OK) return s;
    launch_reduce_energy(h, t, 1, h->e0, st);
    const size_t sstride = (size_t)h->n_sys * 3;
    StepObs ob;
    ob.x0 = F4(x0);
    ob.jump = h->jump_atom;
    ob.l_prop = l_prop;
    ob.x_prop = F4(x_out);
    StepStat ss;
    ss.jump = h->jump_atom;
    ss.e_ref = h->e0;
    ss.kT = kT;
    for (int l = 0; l <= n_leap; ++l) {
        float4* cx = nullptr;
        float4* cv = nullptr;
        if (ck && l < n_leap && l % ckpt_every == 0) {
            cx = ck + (size_t)(l / ckpt_every) * 2 * N;
            cv = cx + N;
        }
        {
            Stage sc(h, NB_STAGE_UPDATE, st);
            ob.step = l;
            launch_integrate(h, x, h->vwork, inv_mass, dt, l == 0 ? 0.f : 0.5f, l == n_leap ? 0.f : 0.5f,
                             l < n_leap, cx, cv, nullptr, st, l > 0 ? ob : StepObs(), l < n_leap);
            if (l > 0) {
                ss.sstat = step_stats + (size_t)(l - 1) * sstride;
                launch_reduce_energy(h, t, 1, h->e1, st, ss);
            }
        }
        if (l == n_leap) break;
        s = eval(h, x, t, ck != nullptr && (l + 1) % ckpt_every == 0, st, true);
        if (s != NB_OK) return s;
    }
    Stage sc(h, NB_STAGE_UPDATE, st);
    launch_hmc_pick(h, F4(x_out), F4(x0), l_prop, n_leap, step_stats, u, stats, st);
    return launched();
}

}  // extern "C"

// Reverse sweep shared by both HMC backward entry points; inj(l) gives the loss
// cotangents entering at state l (1..n_leap).  The recomputation evaluates with the
// energy kernel at the states where the forward pass asked for energies (the ends, or
// every state), since the energy-free kernel rounds the forces differently: so each
// segment repeats the forward trajectory bit for bit.
template <class InjectAt>
static nb_status hmc_backward(nb_handle* h, const float* x0, const float* inv_mass, const float* dt, int n_leap,
                              double kT, const float* xi, const float* ckpt, int k, InjectAt inj, double* g_dt,
                              float* g_inv_mass, int t, bool energy_every_state, cudaStream_t st) {
    auto en_at = [&](int l) { return energy_every_state || l == 0 || l == n_leap; };
    int N = h->n_atoms;
    if (h->seg_k < k) {
        // (k+1) states of positions, velocities and half-step velocities
        float4* p = nullptr;
        if (cudaMalloc(&p, sizeof(float4) * 3 * (size_t)(k + 1) * N) != cudaSuccess) return NB_ERR_NOMEM;
        if (h->seg) {
            cudaFree(h->seg);
            h->allocs.erase(std::remove(h->allocs.begin(), h->allocs.end(), (void*)h->seg), h->allocs.end());
        }
        h->seg = p;
        h->allocs.push_back(p);
        h->seg_k = k;
    }
    const float4* ck = F4(ckpt);
    auto seg_x = [&](int i) { return h->seg + (size_t)i * N; };
    auto seg_v = [&](int i) { return h->seg + (size_t)(h->seg_k + 1 + i) * N; };
    auto seg_p = [&](int i) { return h->seg + (size_t)(2 * (h->seg_k + 1) + i) * N; };
    cudaMemsetAsync(h->hbar_atom, 0, sizeof(double) * N, st);
    cudaMemsetAsync(h->xbar, 0, sizeof(float4) * N, st);
    cudaMemsetAsync(h->vbar, 0, sizeof(float4) * N, st);
    int n_seg = (n_leap + k - 1) / k;
    nb_status s;
    for (int j = n_seg - 1; j >= 0; --j) {
        int s0 = j * k, e = std::min(s0 + k, n_leap), m = e - s0;
        cudaMemcpyAsync(h->xwork, ck + (size_t)j * 2 * N, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st);
        cudaMemcpyAsync(h->vwork, ck + (size_t)j * 2 * N + N, sizeof(float4) * N, cudaMemcpyDeviceToDevice, st);
        s = eval(h, h->xwork, t, true, st, false, en_at(s0));
        if (s != NB_OK) return s;
        for (int q = 0; q < m; ++q) {
            launch_integrate(h, h->xwork, h->vwork, inv_mass, dt, q == 0 ? 0.f : 0.5f, 0.5f, 1, seg_x(q), seg_v(q),
                             seg_p(q + 1), st, StepObs(), true);
            s = eval(h, h->xwork, t, false, st, true, en_at(s0 + q + 1));
            if (s != NB_OK) return s;
        }
        launch_integrate(h, h->xwork, h->vwork, inv_mass, dt, 0.5f, 0.f, 0, seg_x(m), seg_v(m), nullptr, st);
        for (int q = m; q >= 1; --q) {
            const Inject in = inj(s0 + q);
            prepare(h, seg_x(q), false, st);
            launch_bwd_lambda(h, inv_mass, dt, seg_v(q), in, kT, st);
            {
                Stage sc(h, NB_STAGE_PAIR, st);
                launch_vjp(h, t, st);
            }
            if ((t & NB_TERM_PME) && h->has_pme && launch_pme_vjp(h, st)) return NB_ERR_CUDA;
            launch_bwd_adjoint(h, inv_mass, dt, seg_x(q), seg_v(q), F4(x0), in, kT, seg_p(q), g_inv_mass, st);
        }
    }
    s = eval(h, F4(x0), t, false, st, false, true);
    if (s != NB_OK) return s;
    launch_bwd_final(h, inv_mass, dt, xi, kT, g_inv_mass, g_dt, st);
    return launched();
}

extern "C" {

nb_status hmc_trajectory_backward(nb_handle* h, const float* x0, const float* inv_mass, const float* dt,
                                  int32_t n_leap, double kT, const float* xi, const float* ckpt, int32_t ckpt_every,
                                  const double* stats, const double* g_alpha, const double* g_jump, double* g_dt,
                                  float* g_inv_mass, int32_t terms, void* stream) {
    if (!h || !x0 || !inv_mass || !dt || !xi || !ckpt || !stats || !g_alpha || !g_jump || !g_dt || !g_inv_mass ||
        n_leap < 1 || ckpt_every < 1 || !(kT > 0.0))
        return NB_ERR_ARG;
    DeviceGuard g(h->device);
    const int L = n_leap;
    auto inj = [&](int l) {
        Inject in;
        if (l == L) {
            in.ga = g_alpha;
            in.gj = g_jump;
            in.alpha = stats + 1;
            in.a_stride = 4;
        }
        return in;
    };
    // a forward pass with precise energies ran the energy-free pair kernel at the end states:
    // the recomputation does the same (kTermPrecise applies only where energies are asked for)
    return hmc_backward(h, x0, inv_mass, dt, L, kT, xi, ckpt, ckpt_every, inj, g_dt, g_inv_mass,
                        (terms & NB_TERM_ALL) | ((terms & NB_ENERGY_PRECISE) ? kTermPrecise : 0), false,
                        S(stream));
}

nb_status hmc_trajectory_steps_backward(nb_handle* h, const float* x0, const float* inv_mass, const float* dt,
                                        int32_t n_leap, double kT, const float* xi, const float* ckpt,
                                        int32_t ckpt_every, const double* step_stats, const double* g_alpha,
                                        const double* g_jump, double* g_dt, float* g_inv_mass, int32_t terms,
                                        void* stream) {
    if (!h || !x0 || !inv_mass || !dt || !xi || !ckpt || !step_stats || !g_alpha || !g_jump || !g_dt ||
        !g_inv_mass || n_leap < 1 || ckpt_every < 1 || !(kT > 0.0))
        return NB_ERR_ARG;
    DeviceGuard g(h->device);
    const size_t ns = (size_t)h->n_sys;
    auto inj = [&](int l) {
        Inject in;
        in.ga = g_alpha + (size_t)(l - 1) * ns;
        in.gj = g_jump + (size_t)(l - 1) * ns;
        in.alpha = step_stats + (size_t)(l - 1) * ns * 3 + 1;
        in.a_stride = 3;
        return in;
    };
    return hmc_backward(h, x0, inv_mass, dt, n_leap, kT, xi, ckpt, ckpt_every, inj, g_dt, g_inv_mass,
                        terms & NB_TERM_ALL, true, S(stream));
}

nb_status nonbonded_force_vjp(nb_handle* h, const float* xq, const float* lam, float* gx, float* gq, float* gsigma,
                              float* gsqrt_eps, float* f_out, int32_t terms, void* stream) {
    if (!h || !xq || !lam || !gx) return NB_ERR_ARG;
    DeviceGuard g(h->device);
    cudaStream_t st = S(stream);
    int N = h->n_atoms;
    const int t = terms & NB_TERM_ALL;
    prepare(h, F4(xq), false, st);
    launch_pdl(k_lam_scatter, cdiv(N, 256), 256, 0, st, N, lam, h->iperm, h->lam);
    {
        Stage sc(h, NB_STAGE_PAIR, st);
        launch_vjp(h, t & (NB_TERM_LJ | NB_TERM_COUL), st);
    }
    if ((t & NB_TERM_PME) && h->has_pme) {
        Stage sc(h, NB_STAGE_GATHER, st);
        if (launch_pme_vjp(h, st)) return NB_ERR_CUDA;
    }
    Stage sc(h, NB_STAGE_UPDATE, st);
    launch_pdl(k_vjp_out, cdiv(N, 256), 256, 0, st, N, h->gx_s, h->gp_s, h->iperm, gx, gq, gsigma, gsqrt_eps);
    if (f_out) launch_finalize_forces(h, f_out, st);
    return launched();
}

}  // extern "C"
