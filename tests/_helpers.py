"""Shared helpers for the GPU parity tests (inputs, oracle calls, comparisons)."""
import numpy as np

import oracle
from oracle import pme as opme
from paper_2503_20541_b300 import nbcore


def dev_xq(s):
    import torch
    return torch.from_numpy(nbcore.pack_xq(s.x, s.q)).cuda()


def oracle_params(s):
    return oracle.make_params(s.box, r_cut=s.r_cut, r_switch=s.r_switch, alpha=s.alpha, ke=s.ke,
                              periodic=getattr(s, "periodic", True), eps_rf=getattr(s, "eps_rf", 0.0) or 0.0)


def oracle_real_space(s, x=None):
    """(energies[4], forces) of LJ + Ewald direct + exclusion + self, FP64 all pairs."""
    x = s.x.astype(np.float64) if x is None else x
    return oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, oracle_params(s), excl=s.excl)


def oracle_pme(s, x=None):
    x = s.x.astype(np.float64) if x is None else x
    return opme.pme(x, s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)


def rel_rms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def band(r_nl):
    """FP32 ambiguity band of the r^2 < r_nl^2 test (8 ulp of r_nl^2)."""
    return 8.0 * float(np.spacing(np.float32(r_nl * r_nl)))


def pair_set(pairs):
    p = np.asarray(pairs)
    return set(map(tuple, p.tolist()))


def pairs_near_boundary(x, box, r_nl, width):
    """Unordered pairs whose FP64 r^2 lies within `width` of r_nl^2 (brute force)."""
    x = np.asarray(x, np.float64)
    L = np.asarray(box, np.float64)
    out = set()
    for i in range(len(x) - 1):
        d = x[i + 1:] - x[i]
        d -= L * np.round(d / L)
        r2 = np.einsum("ij,ij->i", d, d)
        for j in np.nonzero(np.abs(r2 - r_nl * r_nl) <= width)[0]:
            out.add((i, i + 1 + int(j)))
    return out


EPS32 = 2.0 ** -24  # unit roundoff of FP32


def rf_rounding_scale(s, chunk=600, rows=None):
    """sqrt(sum over unordered non-excluded pairs r < r_c of m_ij^2), m_ij = ke |q_i q_j|
    (1/r + c + k r^2): the sum of the magnitudes of the parts of each reaction-field pair
    energy (Eq. RFA).  Every FP32 pair energy is rounded at ~EPS32 m_ij and the errors of
    independent pairs add like a random walk, so EPS32 times this is the expected error
    of E_RF; it matters because water's pair energies cancel ~10^4-fold in the sum.
    With ``rows``, the sum of squares is estimated from those rows, scaled by n/len(rows)."""
    x = s.x.astype(np.float64)
    q = s.q.astype(np.float64)
    L = np.broadcast_to(np.asarray(s.box, dtype=np.float64), (3,))
    rc, eps, ke = float(s.r_cut), float(s.eps_rf), float(s.ke)
    k = (eps - 1.0) / ((2.0 * eps + 1.0) * rc ** 3)
    c = 3.0 * eps / ((2.0 * eps + 1.0) * rc)
    n = s.n
    rows = np.arange(n) if rows is None else np.asarray(rows)
    tot = 0.0
    for c0 in range(0, rows.size, chunk):
        rr = rows[c0:c0 + chunk]
        d = x[rr, None, :] - x[None, :, :]
        d -= L * np.round(d / L)
        r2 = np.einsum("ijk,ijk->ij", d, d)
        ii = rr[:, None]
        jj = np.arange(n)[None, :]
        m = (r2 < rc * rc) & (jj != ii)
        if s.excl_off is not None:
            for a, i in enumerate(rr):
                m[a, s.excl_idx[s.excl_off[i]:s.excl_off[i + 1]]] = False
        r = np.sqrt(np.where(m, r2, 1.0))
        mag = np.where(m, np.abs(ke * q[ii] * q[jj]) * (1.0 / r + c + k * r * r), 0.0)
        tot += float(np.sum(mag * mag))
    return float(np.sqrt(0.5 * tot * n / rows.size))
