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
                              periodic=getattr(s, "periodic", True))


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
