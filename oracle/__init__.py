"""FP64 CPU oracle for the nonbonded force / MD / HMC path of arXiv 2503.20541.

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the CPU
baseline arm of ``bench.py`` are the only code allowed to import this package.
It shares no code with the CUDA library ``paper_2503_20541_b300`` and never
imports it.

Contents (each cites the passage of the paper it follows):
  * ``nonbonded`` / ``nonbonded_rows`` -- all-pairs LJ (Eq. lj, Lorentz-Berthelot
    mixing, optional switch S(x)) + Ewald direct erfc sum + exclusion correction +
    self energy, or the reaction field (Eq. RFA) instead of the Ewald terms
    (Sec. 2.1.2), in C (oracle.c).
  * ``nonbonded_cells`` -- the same sums over the candidates of a cell list (Sec. 2.1.2,
    "Neighborlists"), pinned equal to ``nonbonded``; for CPU timings at large N.
  * ``ewald_recip`` -- exact reciprocal-space structure-factor sum (Sec. 2.1.2).
  * ``neighbor_pairs`` -- brute-force Verlet pair set at r_nl = r_c + r_g.
  * ``force_vjp`` -- analytic pair-Jacobian vector product of the real-space forces.
  * ``pme`` -- smooth PME with recursive B-splines (module ``oracle.pme``).
  * ``dynamics`` -- velocity Verlet (Sec. 2.2.1) and the HMC proposal / ESJD loss
    (Sec. 4, Eqs. loss and acceptance).
  * ``constraints`` -- rigid-water constraints as their defining equations (SHAKE by
    Newton's method, RATTLE by a linear solve) and the Langevin middle scheme
    (Sec. 2.2.1).
  * ``tuning`` -- the folded-normal trajectory length, the step-length-weighted loss
    L_HMC truncated at L_q (Sec. 4, Eq. loss_steps), per-step HMC statistics, and the
    autocorrelation A(k) / tau_exp (Sec. 4).

Parity status: every function is pinned by tests/test_oracle_pins.py,
tests/test_oracle_tuning.py and tests/test_oracle_constraints.py (closed forms, lattice sums, finite differences,
brute-force invariants, scipy's folded normal).
"""
import ctypes
import numpy as np

from . import build as _build

_lib = None


class OrcParams(ctypes.Structure):
    _fields_ = [
        ("box", ctypes.c_double * 3),
        ("periodic", ctypes.c_int32),
        ("pad_", ctypes.c_int32),
        ("r_cut", ctypes.c_double),
        ("r_switch", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("ke", ctypes.c_double),
        ("eps_rf", ctypes.c_double),
    ]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = ctypes.CDLL(path)
        _lib.orc_neighbor_pairs.restype = ctypes.c_int64
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def make_params(box, r_cut, r_switch=-1.0, alpha=0.0, ke=0.0, periodic=True, eps_rf=0.0):
    """Oracle parameters; eps_rf > 0 selects the reaction field (Eq. RFA) with solvent
    dielectric eps_rf in place of the Ewald direct term (alpha must then be 0)."""
    assert not (eps_rf > 0.0 and alpha > 0.0)
    p = OrcParams()
    b = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    for k in range(3):
        p.box[k] = float(b[k])
    p.periodic = 1 if periodic else 0
    p.r_cut = float(r_cut)
    p.r_switch = float(r_switch)
    p.alpha = float(alpha)
    p.ke = float(ke)
    p.eps_rf = float(eps_rf)
    return p


def _excl(excl, n):
    if excl is None:
        return None, None
    off, idx = excl
    off = np.ascontiguousarray(off, dtype=np.int32)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    assert off.shape == (n + 1,)
    return off, idx


def nonbonded(x, q, sigma, sqrt_eps, params, excl=None):
    """All-pairs energies (E_lj, E_dir, E_excl, E_self) and forces (n,3), FP64."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    q, sigma, sqrt_eps = _d(q), _d(sigma), _d(sqrt_eps)
    off, idx = _excl(excl, n)
    e = np.zeros(4)
    f = np.zeros((n, 3))
    lib().orc_nonbonded(ctypes.c_int(n), _p(x), _p(q), _p(sigma), _p(sqrt_eps), ctypes.byref(params),
                        _p(off), _p(idx), _p(e), _p(f))
    return e, f


def nonbonded_rows(x, q, sigma, sqrt_eps, params, rows, excl=None):
    """Force on each atom in ``rows`` (summed over all j) and its half pair energies."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    q, sigma, sqrt_eps = _d(q), _d(sigma), _d(sqrt_eps)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    off, idx = _excl(excl, n)
    er = np.zeros((rows.size, 3))
    fr = np.zeros((rows.size, 3))
    lib().orc_nonbonded_rows(ctypes.c_int(n), _p(x), _p(q), _p(sigma), _p(sqrt_eps), ctypes.byref(params),
                             _p(off), _p(idx), ctypes.c_int(rows.size), _p(rows), _p(er), _p(fr))
    return er, fr


def nonbonded_cells(x, q, sigma, sqrt_eps, params, excl=None):
    """The quantities of ``nonbonded`` summed per atom over the candidates of a cell list
    of edge >= r_c (Sec. 2.1.2, "Neighborlists"); all pairs for open or small boxes."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    q, sigma, sqrt_eps = _d(q), _d(sigma), _d(sqrt_eps)
    off, idx = _excl(excl, n)
    e = np.zeros(4)
    f = np.zeros((n, 3))
    rc = lib().orc_nonbonded_cells(ctypes.c_int(n), _p(x), _p(q), _p(sigma), _p(sqrt_eps),
                                   ctypes.byref(params), _p(off), _p(idx), _p(e), _p(f))
    if rc != 0:
        raise MemoryError("orc_nonbonded_cells: allocation failed")
    return e, f


def num_threads():
    return int(lib().orc_num_threads())


def set_num_threads(n):
    """Threads of the oracle's parallel loops from here on (single-thread timings)."""
    lib().orc_set_num_threads(ctypes.c_int(int(n)))


def ewald_recip(x, q, box, alpha, ke, mmax):
    """Exact Ewald reciprocal energy and forces, |n_d| <= mmax[d]."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    q = _d(q)
    box = _d(np.broadcast_to(np.asarray(box, dtype=np.float64), (3,)))
    mm = np.ascontiguousarray(np.broadcast_to(np.asarray(mmax), (3,)), dtype=np.int32)
    e = np.zeros(1)
    f = np.zeros((n, 3))
    lib().orc_ewald_recip(ctypes.c_int(n), _p(x), _p(q), _p(box), ctypes.c_double(alpha),
                          ctypes.c_double(ke), _p(mm), _p(e), _p(f))
    return float(e[0]), f


def neighbor_pairs(x, params, r_nl, excl=None, band=0.0):
    """Brute-force pair set {(i<j): r^2 < r_nl^2, not excluded}; returns (pairs, n_band)."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    off, idx = _excl(excl, n)
    nb = np.zeros(1, dtype=np.int64)
    cnt = lib().orc_neighbor_pairs(ctypes.c_int(n), _p(x), ctypes.byref(params), ctypes.c_double(r_nl),
                                   _p(off), _p(idx), ctypes.c_int64(0), None, ctypes.c_double(band), _p(nb))
    pairs = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    lib().orc_neighbor_pairs(ctypes.c_int(n), _p(x), ctypes.byref(params), ctypes.c_double(r_nl),
                             _p(off), _p(idx), ctypes.c_int64(cnt), _p(pairs), ctypes.c_double(band), _p(nb))
    return pairs[:cnt], int(nb[0])


def force_vjp(x, q, sigma, sqrt_eps, params, lam, excl=None):
    """(dF/dx)^T lam and gradients of lam.F wrt q, sigma, sqrt(eps) (real-space terms)."""
    x = _d(x).reshape(-1, 3)
    n = x.shape[0]
    q, sigma, sqrt_eps = _d(q), _d(sigma), _d(sqrt_eps)
    lam = _d(lam).reshape(-1, 3)
    off, idx = _excl(excl, n)
    gx = np.zeros((n, 3))
    gq = np.zeros(n)
    gs = np.zeros(n)
    ge = np.zeros(n)
    lib().orc_force_vjp(ctypes.c_int(n), _p(x), _p(q), _p(sigma), _p(sqrt_eps), ctypes.byref(params),
                        _p(off), _p(idx), _p(lam), _p(gx), _p(gq), _p(gs), _p(ge))
    return gx, gq, gs, ge


COULOMB_KJ_MOL_ANGSTROM = 1389.35457644  # ke in kJ/mol * Angstrom / e^2


def ewald_alpha(delta, r_cut):
    """alpha = sqrt(-log(2 delta)) / r_c (Sec. 2.1.2, Eq. alpha)."""
    return float(np.sqrt(-np.log(2.0 * delta)) / r_cut)
