"""ctypes binding of libnbcore (include/nbcore.h): argument marshalling only.

Every function here checks tensor dtypes, shapes and devices, turns them into
raw device pointers and calls the C entry point of the same name on the
current PyTorch CUDA stream.  All computation happens in the library's CUDA
kernels; if libnbcore.so is missing or no GPU is present the calls raise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnbcore.so")

NB_TERM_LJ = 1
NB_TERM_COUL = 2
NB_TERM_PME = 4
NB_TERM_ALL = 7
NB_FORCE_REBUILD = 256
NB_ENERGY_PRECISE = 512
NB_NE = 6
E_LJ, E_DIR, E_EXCL, E_SELF, E_REC, E_KIN = range(6)

STATUS = {
    0: "ok", 1: "invalid argument", 2: "periodic box edge smaller than 2 r_nl",
    3: "neighbour list capacity exceeded", 4: "fixed-point force accumulator overflow",
    5: "non-finite coordinate", 6: "device wait timed out", 7: "CUDA or cuFFT error",
    8: "device allocation failed",
}

# Every symbol include/nbcore.h declares.
EXPORTS = [
    "nb_status_str", "nb_create", "nb_destroy", "nb_num_atoms", "nb_num_systems", "nb_check",
    "nl_build", "nonbonded_forces", "nonbonded_forces_allpairs", "pme_spread", "pme_gather", "md_step", "hmc_trajectory",
    "hmc_trajectory_backward", "hmc_trajectory_steps", "hmc_trajectory_steps_backward", "autocorrelation",
    "nonbonded_force_vjp", "nb_rebuild_count", "nb_blocks_per_cell", "nb_timing_enable", "nb_timing_read",
    "pme_spread_static", "nb_set_water_constraints", "langevin_step", "constrain_positions", "constrain_velocities",
    "nb_erfc_eval", "nb_erfc_df_eval",
]
STATIC_MESH_MAX = 1 << 20
STAGES = ["check", "rebuild", "pair", "spread", "fft", "convolve", "gather", "update", "build"]


class NbError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = int(status)
        super().__init__("%s: %s (status %d)" % (where, STATUS.get(self.status, "unknown"), self.status))


class SystemDesc(ctypes.Structure):
    _fields_ = [
        ("n_atoms", ctypes.c_int32),
        ("periodic", ctypes.c_int32),
        ("box", ctypes.c_double * 3),
        ("r_cut", ctypes.c_double),
        ("r_skin", ctypes.c_double),
        ("r_switch", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("ke", ctypes.c_double),
        ("pme_grid", ctypes.c_int32 * 3),
        ("pme_order", ctypes.c_int32),
        ("eps_rf", ctypes.c_double),
    ]


class Options(ctypes.Structure):
    _fields_ = [
        ("max_neighbors", ctypes.c_int32),
        ("stencil_tile", ctypes.c_int32),
        ("cell_div", ctypes.c_int32),
        ("force_bits", ctypes.c_int32),
        ("blocks_per_cell", ctypes.c_int32),
        ("prune_skin", ctypes.c_double),
    ]


_lib = None
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_dbl = ctypes.c_double


def load():
    """Load libnbcore.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libnbcore.so not found at %s: build it with "
                           "`python -m paper_2503_20541_b300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    lib.nb_status_str.restype = ctypes.c_char_p
    lib.nb_status_str.argtypes = [ctypes.c_int]
    lib.nb_create.restype = ctypes.c_int
    lib.nb_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(SystemDesc), _i32, _vp, _vp, _vp, _vp,
                              ctypes.POINTER(Options)]
    lib.nb_destroy.restype = None
    lib.nb_destroy.argtypes = [_vp]
    lib.nb_num_atoms.restype = _i64
    lib.nb_num_atoms.argtypes = [_vp]
    lib.nb_num_systems.restype = _i32
    lib.nb_num_systems.argtypes = [_vp]
    lib.nb_check.restype = ctypes.c_int
    lib.nb_check.argtypes = [_vp, _vp]
    lib.nb_rebuild_count.restype = _i64
    lib.nb_rebuild_count.argtypes = [_vp, _vp]
    lib.nl_build.restype = ctypes.c_int
    lib.nl_build.argtypes = [_vp, _vp, _vp, _i64, ctypes.POINTER(_i64), _i32, _vp]
    lib.nonbonded_forces.restype = ctypes.c_int
    lib.nonbonded_forces.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp]
    lib.nonbonded_forces_allpairs.restype = ctypes.c_int
    lib.nonbonded_forces_allpairs.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.pme_spread.restype = ctypes.c_int
    lib.pme_spread.argtypes = [_vp, _vp, _vp, _vp]
    lib.pme_gather.restype = ctypes.c_int
    lib.pme_gather.argtypes = [_vp, _vp, _vp, _vp, _vp]
    lib.md_step.restype = ctypes.c_int
    lib.md_step.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp, _i32, _vp]
    lib.hmc_trajectory.restype = ctypes.c_int
    lib.hmc_trajectory.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _dbl, _vp, _vp, _vp, _vp, _i32, _i32, _vp]
    lib.hmc_trajectory_backward.restype = ctypes.c_int
    lib.hmc_trajectory_backward.argtypes = [_vp, _vp, _vp, _vp, _i32, _dbl, _vp, _vp, _i32, _vp, _vp, _vp, _vp,
                                            _vp, _i32, _vp]
    lib.hmc_trajectory_steps.restype = ctypes.c_int
    lib.hmc_trajectory_steps.argtypes = [_vp, _vp, _vp, _vp, _vp, _i32, _vp, _dbl, _vp, _vp, _vp, _vp, _vp, _i32,
                                         _i32, _vp]
    lib.hmc_trajectory_steps_backward.restype = ctypes.c_int
    lib.hmc_trajectory_steps_backward.argtypes = [_vp, _vp, _vp, _vp, _i32, _dbl, _vp, _vp, _i32, _vp, _vp, _vp,
                                                  _vp, _vp, _i32, _vp]
    lib.autocorrelation.restype = ctypes.c_int
    lib.autocorrelation.argtypes = [_vp, _i32, _i32, _i32, _dbl, _dbl, _vp, _vp, _vp]
    lib.nonbonded_force_vjp.restype = ctypes.c_int
    lib.nonbonded_force_vjp.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i32, _vp]
    lib.nb_set_water_constraints.restype = ctypes.c_int
    lib.nb_set_water_constraints.argtypes = [_vp, _vp, _i32, _dbl, _dbl]
    lib.langevin_step.restype = ctypes.c_int
    lib.langevin_step.argtypes = [_vp, _vp, _vp, _vp, _vp, _dbl, _i32, _vp, _vp, _i32, _vp]
    lib.constrain_positions.restype = ctypes.c_int
    lib.constrain_positions.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_float, _vp]
    lib.constrain_velocities.restype = ctypes.c_int
    lib.constrain_velocities.argtypes = [_vp, _vp, _vp, _vp]
    lib.nb_blocks_per_cell.restype = ctypes.c_int
    lib.nb_blocks_per_cell.argtypes = [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]
    lib.nb_timing_enable.restype = ctypes.c_int
    lib.nb_timing_enable.argtypes = [_vp, _i32]
    lib.nb_timing_read.restype = ctypes.c_int
    lib.nb_timing_read.argtypes = [_vp, _vp, _vp, _vp]
    lib.pme_spread_static.restype = ctypes.c_int
    lib.pme_spread_static.argtypes = [_vp, _i32, _vp, _vp, _vp, _vp]
    lib.nb_erfc_eval.restype = ctypes.c_int
    lib.nb_erfc_eval.argtypes = [_vp, _vp, _i32, _vp]
    lib.nb_erfc_df_eval.restype = ctypes.c_int
    lib.nb_erfc_df_eval.argtypes = [_vp, _vp, _vp, _vp, _i32, _vp]
    _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _stream():
    torch = _torch()
    return _vp(torch.cuda.current_stream().cuda_stream)


def _ptr(t, dtype, shape=None, name="tensor", allow_none=False):
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))
    return _vp(t.data_ptr())


def _ok(status, where):
    if status != 0:
        raise NbError(status, where)


def pme_spread_static(xq, box, mesh, grid):
    """PME charge spreading that allocates no device memory (pme_spread_static in
    include/nbcore.h), for callers that cannot call cudaMalloc.  No handle is involved;
    the library's static mesh is shared by all calls, so calls must not overlap on the GPU."""
    torch = _torch()
    lib = load()
    n = int(xq.shape[0])
    b = np.ascontiguousarray(np.broadcast_to(np.asarray(box, np.float64), (3,)))
    m = np.ascontiguousarray(np.broadcast_to(np.asarray(mesh, np.int32), (3,)))
    _ok(lib.pme_spread_static(_ptr(xq, torch.float32, (n, 4), "xq"), n, b.ctypes.data, m.ctypes.data,
                              _ptr(grid, torch.float32, (int(np.prod(m.astype(np.int64))),), "grid"), _stream()),
        "pme_spread_static")
    return grid


def erfc_eval(x, out=None):
    """erfc(x) of a float32 device tensor x >= 0 with the pair kernels' own evaluation
    (nb_erfc_eval in include/nbcore.h)."""
    torch = _torch()
    lib = load()
    n = int(x.numel())
    if out is None:
        out = torch.empty_like(x)
    _ok(lib.nb_erfc_eval(_ptr(x, torch.float32, (n,), "x"), _ptr(out, torch.float32, (n,), "out"), n, _stream()),
        "nb_erfc_eval")
    return out


def erfc_df_eval(x_hi, x_lo):
    """erfc(x_hi + x_lo) in two-float (float32 device tensors, x >= 0) with the precise-energy
    evaluation's own routine (nb_erfc_df_eval in include/nbcore.h); returns (hi, lo)."""
    torch = _torch()
    lib = load()
    n = int(x_hi.numel())
    hi, lo = torch.empty_like(x_hi), torch.empty_like(x_hi)
    _ok(lib.nb_erfc_df_eval(_ptr(x_hi, torch.float32, (n,), "x_hi"), _ptr(x_lo, torch.float32, (n,), "x_lo"),
                            _ptr(hi, torch.float32, (n,), "out_hi"), _ptr(lo, torch.float32, (n,), "out_lo"), n,
                            _stream()), "nb_erfc_df_eval")
    return hi, lo


def autocorrelation(series, max_lag, a_hi=0.5, a_lo=0.05, acf=None, tau=None):
    """A(k), k = 0..max_lag, and tau_exp of each row of ``series`` ((n_series, n) float64
    on the device) -- autocorrelation in include/nbcore.h.  Returns (acf, tau)."""
    torch = _torch()
    lib = load()
    ns, n = int(series.shape[0]), int(series.shape[1])
    if acf is None:
        acf = torch.empty((ns, max_lag + 1), dtype=torch.float64, device=series.device)
    if tau is None:
        tau = torch.empty(ns, dtype=torch.float64, device=series.device)
    _ok(lib.autocorrelation(_ptr(series, torch.float64, (ns, n), "series"), ns, n, int(max_lag), float(a_hi),
                            float(a_lo), _ptr(acf, torch.float64, (ns, max_lag + 1), "acf"),
                            _ptr(tau, torch.float64, (ns,), "tau"), _stream()), "autocorrelation")
    return acf, tau


def ckpt_size(n_atoms, n_leap, ckpt_every):
    """Number of floats of the checkpoint buffer of hmc_trajectory."""
    return ((n_leap + ckpt_every - 1) // ckpt_every) * 2 * n_atoms * 4


def pack_xq(x, q):
    """(n,3) positions + (n,) charges -> (n,4) float32 numpy array."""
    out = np.zeros((len(q), 4), np.float32)
    out[:, :3] = x
    out[:, 3] = q
    return out


class Handle:
    """Owns an nb_handle: a set of systems with their per-atom parameters.

    ``systems`` is a list of objects with the attributes of
    ``workloads.System`` (n, box, r_cut, r_skin, r_switch, alpha, ke,
    pme_grid, sigma, sqrt_eps, excl_off/excl_idx)."""

    def __init__(self, systems, max_neighbors=0, stencil_tile=0, cell_div=0, force_bits=0, periodic=True,
                 blocks_per_cell=0, prune_skin=0.0):
        lib = load()
        self._h = None
        n_sys = len(systems)
        descs = (SystemDesc * n_sys)()
        sig, sqe, offs, idxs = [], [], [0], []
        base = 0
        for k, s in enumerate(systems):
            d = descs[k]
            d.n_atoms = s.n
            d.periodic = 1 if getattr(s, "periodic", periodic) else 0
            for a in range(3):
                d.box[a] = float(np.broadcast_to(s.box, (3,))[a])
            d.r_cut = s.r_cut
            d.r_skin = s.r_skin
            d.r_switch = s.r_switch
            d.alpha = s.alpha
            d.ke = s.ke
            g = tuple(s.pme_grid) if s.pme_grid else (0, 0, 0)
            for a in range(3):
                d.pme_grid[a] = int(g[a])
            d.pme_order = int(getattr(s, "pme_order", 4))
            d.eps_rf = float(getattr(s, "eps_rf", 0.0) or 0.0)
            sig.append(np.asarray(s.sigma, np.float32))
            sqe.append(np.asarray(s.sqrt_eps, np.float32))
            if s.excl_off is not None:
                o = np.asarray(s.excl_off, np.int64)
                idxs.append(np.asarray(s.excl_idx, np.int64) + base)
                offs.extend((o[1:] + offs[-1]).tolist())
            else:
                offs.extend([offs[-1]] * s.n)
            base += s.n
        self.n_atoms = base
        self.n_sys = n_sys
        self.sigma = np.ascontiguousarray(np.concatenate(sig), np.float32)
        self.sqrt_eps = np.ascontiguousarray(np.concatenate(sqe), np.float32)
        ex_off = np.ascontiguousarray(offs, np.int32)
        ex_idx = np.ascontiguousarray(np.concatenate(idxs) if idxs else np.zeros(0), np.int32)
        opt = Options(int(max_neighbors), int(stencil_tile), int(cell_div), int(force_bits), int(blocks_per_cell),
                      float(prune_skin))
        h = _vp()
        st = lib.nb_create(ctypes.byref(h), descs, n_sys, self.sigma.ctypes.data, self.sqrt_eps.ctypes.data,
                           ex_off.ctypes.data, ex_idx.ctypes.data if ex_idx.size else None, ctypes.byref(opt))
        _ok(st, "nb_create")
        self._h = h
        self._lib = lib
        self.descs = descs
        self.mesh_size = sum(int(np.prod(tuple(s.pme_grid))) for s in systems
                             if s.pme_grid and s.pme_grid[0] > 0)

    def close(self):
        # graphs captured over this handle's buffers (hmc._TrajectoryGraphs) die with it
        self.__dict__.pop("_hmc_graphs", None)
        if getattr(self, "_h", None):
            self._lib.nb_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- calls
    def check(self):
        _ok(self._lib.nb_check(self._h, _stream()), "nb_check")

    def rebuild_count(self):
        return int(self._lib.nb_rebuild_count(self._h, _stream()))

    def timing_enable(self, on=True):
        _ok(self._lib.nb_timing_enable(self._h, 1 if on else 0), "nb_timing_enable")

    def timing_read(self):
        """{stage: (milliseconds, intervals)} since the previous read."""
        ms = np.zeros(len(STAGES), np.float64)
        cnt = np.zeros(len(STAGES), np.int64)
        _ok(self._lib.nb_timing_read(self._h, _stream(), ms.ctypes.data, cnt.ctypes.data), "nb_timing_read")
        return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(STAGES)}

    def set_water_constraints(self, mols, d_oh, d_hh):
        """Rigid water: mols (n_mol, 3) caller indices (O, H1, H2); d_oh, d_hh distances."""
        m = np.ascontiguousarray(np.asarray(mols, dtype=np.int32).reshape(-1, 3))
        _ok(self._lib.nb_set_water_constraints(self._h, m.ctypes.data if m.size else None, int(m.shape[0]),
                                               float(d_oh), float(d_hh)), "nb_set_water_constraints")

    def langevin_step(self, xq, v, dt, gamma, kT, n_steps, xi, energies=None, terms=NB_TERM_ALL):
        torch = _torch()
        N, R = self.n_atoms, self.n_sys
        _ok(self._lib.langevin_step(
            self._h, _ptr(xq, torch.float32, (N, 4), "xq"), _ptr(v, torch.float32, (N, 4), "v"),
            _ptr(dt, torch.float32, (R,), "dt"), _ptr(gamma, torch.float32, (R,), "gamma"), float(kT), int(n_steps),
            _ptr(xi, torch.float32, (n_steps, N, 3), "xi"),
            _ptr(energies, torch.float64, (n_steps + 1, R, NB_NE), "energies", True), int(terms), _stream()),
            "langevin_step")

    def constrain_positions(self, x_ref, x, inv_mass, v=None, dt=0.0):
        torch = _torch()
        N = self.n_atoms
        _ok(self._lib.constrain_positions(
            self._h, _ptr(x_ref, torch.float32, (N, 4), "x_ref"), _ptr(x, torch.float32, (N, 4), "x"),
            _ptr(v, torch.float32, (N, 4), "v", True), _ptr(inv_mass, torch.float32, (N,), "inv_mass"), float(dt),
            _stream()), "constrain_positions")

    def constrain_velocities(self, x, v):
        torch = _torch()
        N = self.n_atoms
        _ok(self._lib.constrain_velocities(self._h, _ptr(x, torch.float32, (N, 4), "x"),
                                           _ptr(v, torch.float32, (N, 4), "v"), _stream()), "constrain_velocities")

    def blocks_per_cell(self):
        """(list build, pair/VJP kernels) thread blocks per cell."""
        b, p = _i32(0), _i32(0)
        _ok(self._lib.nb_blocks_per_cell(self._h, ctypes.byref(b), ctypes.byref(p)), "nb_blocks_per_cell")
        return int(b.value), int(p.value)

    def nl_build(self, xq, max_pairs=0, force_rebuild=False):
        """Return (pairs int32 [n, 2] on the device, n_pairs)."""
        torch = _torch()
        N = self.n_atoms
        n = _i64(0)
        _ok(self._lib.nl_build(self._h, _ptr(xq, torch.float32, (N, 4), "xq"), None, 0, ctypes.byref(n),
                               1 if force_rebuild else 0, _stream()), "nl_build")
        count = int(n.value)
        if max_pairs is None or max_pairs == 0:
            max_pairs = count
        out = torch.empty((max(max_pairs, 1), 2), dtype=torch.int32, device=xq.device)
        _ok(self._lib.nl_build(self._h, _ptr(xq, torch.float32, (N, 4), "xq"), _vp(out.data_ptr()), max_pairs,
                               ctypes.byref(n), 0, _stream()), "nl_build")
        return out[:min(count, max_pairs)], int(n.value)

    def nonbonded_forces(self, xq, f_out=None, energies=None, terms=NB_TERM_ALL, force_rebuild=False,
                         precise=False):
        """precise: energies in two-float arithmetic (NB_ENERGY_PRECISE)."""
        torch = _torch()
        N = self.n_atoms
        t = int(terms) | (NB_FORCE_REBUILD if force_rebuild else 0) | (NB_ENERGY_PRECISE if precise else 0)
        _ok(self._lib.nonbonded_forces(
            self._h, _ptr(xq, torch.float32, (N, 4), "xq"),
            _ptr(f_out, torch.float32, (N, 3), "f_out", True),
            _ptr(energies, torch.float64, (self.n_sys, NB_NE), "energies", True), t, _stream()),
            "nonbonded_forces")
        return f_out, energies

    def nonbonded_forces_allpairs(self, xq, f_out=None, energies=None):
        """All-pairs LJ forces (no list): the O(N^2) comparison baseline."""
        torch = _torch()
        N = self.n_atoms
        _ok(self._lib.nonbonded_forces_allpairs(
            self._h, _ptr(xq, torch.float32, (N, 4), "xq"), _ptr(f_out, torch.float32, (N, 3), "f_out", True),
            _ptr(energies, torch.float64, (self.n_sys, NB_NE), "energies", True), _stream()),
            "nonbonded_forces_allpairs")
        return f_out, energies

    def pme_spread(self, xq, grid):
        torch = _torch()
        _ok(self._lib.pme_spread(self._h, _ptr(xq, torch.float32, (self.n_atoms, 4), "xq"),
                                 _ptr(grid, torch.float32, (self.mesh_size,), "grid"), _stream()), "pme_spread")
        return grid

    def pme_gather(self, xq, phi, f_out):
        torch = _torch()
        _ok(self._lib.pme_gather(self._h, _ptr(xq, torch.float32, (self.n_atoms, 4), "xq"),
                                 _ptr(phi, torch.float32, (self.mesh_size,), "phi"),
                                 _ptr(f_out, torch.float32, (self.n_atoms, 3), "f_out"), _stream()), "pme_gather")
        return f_out

    def md_step(self, xq, v, dt, n_steps, energies=None, terms=NB_TERM_ALL):
        torch = _torch()
        N = self.n_atoms
        _ok(self._lib.md_step(self._h, _ptr(xq, torch.float32, (N, 4), "xq"), _ptr(v, torch.float32, (N, 4), "v"),
                              _ptr(dt, torch.float32, (self.n_sys,), "dt"), int(n_steps),
                              _ptr(energies, torch.float64, (n_steps + 1, self.n_sys, NB_NE), "energies", True),
                              int(terms), _stream()), "md_step")

    def hmc_trajectory(self, x0, x_out, inv_mass, dt, n_leap, kT, xi, u, stats, ckpt=None, ckpt_every=0,
                       terms=NB_TERM_ALL):
        torch = _torch()
        N = self.n_atoms
        ck_shape = (ckpt_size(N, n_leap, ckpt_every),) if ckpt is not None else None
        _ok(self._lib.hmc_trajectory(
            self._h, _ptr(x0, torch.float32, (N, 4), "x0"), _ptr(x_out, torch.float32, (N, 4), "x_out"),
            _ptr(inv_mass, torch.float32, (N,), "inv_mass"), _ptr(dt, torch.float32, (self.n_sys,), "dt"),
            int(n_leap), float(kT), _ptr(xi, torch.float32, (N, 3), "xi"),
            _ptr(u, torch.float64, (self.n_sys,), "u"), _ptr(stats, torch.float64, (self.n_sys, 4), "stats"),
            _ptr(ckpt, torch.float32, ck_shape, "ckpt", True), int(ckpt_every), int(terms), _stream()),
            "hmc_trajectory")

    def _segment_buffer(self, ckpt_every):
        """The backward's first call with a larger checkpoint interval than before
        replaces the library's segment buffer: CUDA graphs captured over the old one
        (hmc._TrajectoryGraphs with a captured backward) are dropped."""
        if int(ckpt_every) > self.__dict__.get("_seg_k", 0):
            self._seg_k = int(ckpt_every)
            cache = self.__dict__.get("_hmc_graphs", {})
            for key in [k for k, g in cache.items() if getattr(g, "bwd", None) is not None]:
                del cache[key]

    def hmc_trajectory_backward(self, x0, inv_mass, dt, n_leap, kT, xi, ckpt, ckpt_every, stats, g_alpha, g_jump,
                                g_dt, g_inv_mass, terms=NB_TERM_LJ | NB_TERM_COUL):
        torch = _torch()
        N = self.n_atoms
        self._segment_buffer(ckpt_every)
        _ok(self._lib.hmc_trajectory_backward(
            self._h, _ptr(x0, torch.float32, (N, 4), "x0"), _ptr(inv_mass, torch.float32, (N,), "inv_mass"),
            _ptr(dt, torch.float32, (self.n_sys,), "dt"), int(n_leap), float(kT),
            _ptr(xi, torch.float32, (N, 3), "xi"),
            _ptr(ckpt, torch.float32, (ckpt_size(N, n_leap, ckpt_every),), "ckpt"), int(ckpt_every),
            _ptr(stats, torch.float64, (self.n_sys, 4), "stats"),
            _ptr(g_alpha, torch.float64, (self.n_sys,), "g_alpha"),
            _ptr(g_jump, torch.float64, (self.n_sys,), "g_jump"),
            _ptr(g_dt, torch.float64, (self.n_sys,), "g_dt"),
            _ptr(g_inv_mass, torch.float32, (N,), "g_inv_mass"), int(terms), _stream()),
            "hmc_trajectory_backward")

    def hmc_trajectory_steps(self, x0, x_out, inv_mass, dt, n_leap, l_prop, kT, xi, u, stats, step_stats, ckpt=None,
                             ckpt_every=0, terms=NB_TERM_ALL):
        torch = _torch()
        N, R = self.n_atoms, self.n_sys
        ck_shape = (ckpt_size(N, n_leap, ckpt_every),) if ckpt is not None else None
        _ok(self._lib.hmc_trajectory_steps(
            self._h, _ptr(x0, torch.float32, (N, 4), "x0"), _ptr(x_out, torch.float32, (N, 4), "x_out"),
            _ptr(inv_mass, torch.float32, (N,), "inv_mass"), _ptr(dt, torch.float32, (R,), "dt"), int(n_leap),
            _ptr(l_prop, torch.int32, (R,), "l_prop"), float(kT), _ptr(xi, torch.float32, (N, 3), "xi"),
            _ptr(u, torch.float64, (R,), "u"), _ptr(stats, torch.float64, (R, 4), "stats"),
            _ptr(step_stats, torch.float64, (n_leap, R, 3), "step_stats"),
            _ptr(ckpt, torch.float32, ck_shape, "ckpt", True), int(ckpt_every), int(terms), _stream()),
            "hmc_trajectory_steps")

    def hmc_trajectory_steps_backward(self, x0, inv_mass, dt, n_leap, kT, xi, ckpt, ckpt_every, step_stats, g_alpha,
                                      g_jump, g_dt, g_inv_mass, terms=NB_TERM_LJ | NB_TERM_COUL):
        torch = _torch()
        N, R = self.n_atoms, self.n_sys
        self._segment_buffer(ckpt_every)
        _ok(self._lib.hmc_trajectory_steps_backward(
            self._h, _ptr(x0, torch.float32, (N, 4), "x0"), _ptr(inv_mass, torch.float32, (N,), "inv_mass"),
            _ptr(dt, torch.float32, (R,), "dt"), int(n_leap), float(kT), _ptr(xi, torch.float32, (N, 3), "xi"),
            _ptr(ckpt, torch.float32, (ckpt_size(N, n_leap, ckpt_every),), "ckpt"), int(ckpt_every),
            _ptr(step_stats, torch.float64, (n_leap, R, 3), "step_stats"),
            _ptr(g_alpha, torch.float64, (n_leap, R), "g_alpha"), _ptr(g_jump, torch.float64, (n_leap, R), "g_jump"),
            _ptr(g_dt, torch.float64, (R,), "g_dt"), _ptr(g_inv_mass, torch.float32, (N,), "g_inv_mass"),
            int(terms), _stream()), "hmc_trajectory_steps_backward")

    def nonbonded_force_vjp(self, xq, lam, gx, gq=None, gsigma=None, gsqrt_eps=None, f_out=None,
                            terms=NB_TERM_LJ | NB_TERM_COUL):
        torch = _torch()
        N = self.n_atoms
        _ok(self._lib.nonbonded_force_vjp(
            self._h, _ptr(xq, torch.float32, (N, 4), "xq"), _ptr(lam, torch.float32, (N, 3), "lam"),
            _ptr(gx, torch.float32, (N, 3), "gx"), _ptr(gq, torch.float32, (N,), "gq", True),
            _ptr(gsigma, torch.float32, (N,), "gsigma", True), _ptr(gsqrt_eps, torch.float32, (N,), "gsqrt_eps", True),
            _ptr(f_out, torch.float32, (N, 3), "f_out", True), int(terms), _stream()), "nonbonded_force_vjp")
