"""Edge cases and full-size sampled parity through the C ABI.

Degenerate inputs: a single atom, a dimer across the periodic boundary (LJ minimum,
just inside and just outside r_c), a sparse gas with mostly empty cells, a dense
cluster in a large box (list overflow reported cleanly, then correct with a larger
capacity; its stencils exceed the shared-memory tile), an empty system (refused).
Full sizes: the 8.19M-atom LJ fluid (forces and neighbour sets of sampled atoms against
brute force) and the 256-system batch (sampled atoms of LJ and water systems,
including PME, against the oracle).
"""
import numpy as np
import pytest

import oracle
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import band, dev_xq, oracle_params, oracle_pme, oracle_real_space, pair_set, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-6


def _lj(x, L, r_cut=2.5, r_skin=0.3):
    n = len(x)
    box = np.array([L, L, L], dtype=np.float64)
    s = wl.System(name="custom", x=np.zeros((n, 3), np.float32), q=np.zeros(n, np.float32),
                  sigma=np.ones(n, np.float32), sqrt_eps=np.ones(n, np.float32), mass=np.ones(n, np.float32),
                  box=box, r_cut=r_cut, r_skin=r_skin, types=np.zeros(n, np.int32))
    s.x = np.mod(np.asarray(x, np.float64), s.box).astype(np.float32)
    return s


def _forces(h, s, terms=nbcore.NB_TERM_LJ):
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    h.nonbonded_forces(dev_xq(s), f, e, terms=terms)
    h.check()
    return f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0]


def test_single_atom_has_no_pairs():
    s = _lj([[3.0, 4.0, 5.0]], 10.0)
    with nbcore.Handle([s]) as h:
        _, n = h.nl_build(dev_xq(s), force_rebuild=True)
        f, e = _forces(h, s)
    assert n == 0
    assert np.all(f == 0.0) and np.all(e == 0.0)


@pytest.mark.parametrize("r", [2.0 ** (1.0 / 6.0), 2.4999, 2.5001])
def test_dimer_across_the_periodic_boundary(r):
    L = 10.0
    s = _lj([[0.3, 5.0, 5.0], [0.3 - r, 5.0, 5.0]], L)
    with nbcore.Handle([s]) as h:
        _, n = h.nl_build(dev_xq(s), force_rebuild=True)
        f, e = _forces(h, s)
    eo, fo = oracle_real_space(s)
    assert n == 1  # within r_nl = 2.8 in every case
    if r > 2.5:
        assert e[0] == 0.0 and np.all(f == 0.0) and eo[0] == 0.0
    else:
        assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])
        # at the minimum the force is a cancellation of 48 s^12/r and 24 s^6/r: the FP32
        # error is bounded against the magnitude of those terms, not against F ~ 0
        s6 = r ** -6.0
        scale = 24.0 * (2.0 * s6 * s6 + s6) / r
        assert np.abs(f - fo).max() <= 1e-5 * scale
    if r < 1.2:
        assert e[0] == pytest.approx(-1.0, rel=1e-6)


def test_sparse_gas_with_mostly_empty_cells():
    rng = np.random.default_rng(11)
    L = 60.0
    pts = []
    while len(pts) < 300:
        p = rng.uniform(0, L, 3)
        if all(np.linalg.norm((p - q) - L * np.round((p - q) / L)) > 0.95 for q in pts):
            pts.append(p)
    s = _lj(np.array(pts), L)
    with nbcore.Handle([s]) as h:
        pairs, n = h.nl_build(dev_xq(s), force_rebuild=True)
        gpu = pair_set(pairs.cpu().numpy())
        f, e = _forces(h, s)
    ref, _ = oracle.neighbor_pairs(s.x.astype(np.float64), oracle_params(s), 2.8, band=band(2.8))
    assert gpu == pair_set(ref)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])


def test_dense_cluster_overflows_default_list_then_fits():
    # 1000 atoms at rho* 0.8442 in a corner of a box of volume 60x theirs, r_c = 5:
    # ~520 neighbours each against a capacity sized from the average density, and
    # stencils far above the automatic shared-memory tile
    c = wl.lj_random(1000, seed=12, r_cut=5.0)
    L = 4.0 * float(c.box[0])
    s = _lj(c.x.astype(np.float64), L, r_cut=5.0)
    xq = dev_xq(s)
    with nbcore.Handle([s]) as h:
        with pytest.raises(nbcore.NbError) as ei:
            h.nl_build(xq, force_rebuild=True)
        assert ei.value.status == 3  # NB_ERR_LIST_OVERFLOW
    with nbcore.Handle([s], max_neighbors=1024) as h:
        f, e = _forces(h, s)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])


def test_empty_system_is_refused():
    s = _lj(np.zeros((0, 3)), 10.0)
    with pytest.raises(nbcore.NbError) as ei:
        nbcore.Handle([s])
    assert ei.value.status == 1  # NB_ERR_ARG


def _min_image_d2(x, xi, L):
    d = x - xi
    d -= L * np.round(d / L)
    return np.einsum("ij,ij->i", d, d)


def test_lj_8m_full_size_sampled():
    """The largest LJ sweep point in the bench's configuration: forces of 32 sampled
    atoms against FP64 rows over all 8.19M atoms, and their neighbour sets against a
    brute-force scan (outside the FP32 band around r_nl)."""
    s = wl.lj_random(8192000, seed=500 + 8192000 % 997, kT=1.0)
    xq = dev_xq(s)
    rng = np.random.default_rng(3)
    rows = np.sort(rng.choice(s.n, 32, replace=False))
    r_nl = s.r_cut + s.r_skin
    with nbcore.Handle([s]) as h:
        f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        h.nonbonded_forces(xq, f, None, terms=nbcore.NB_TERM_LJ, force_rebuild=True)
        pairs, n = h.nl_build(xq)
        h.check()
        p = pairs[:n]
        sel = torch.from_numpy(rows.astype(np.int32)).cuda()
        m = torch.isin(p[:, 0], sel) | torch.isin(p[:, 1], sel)
        sub = p[m].cpu().numpy()
        fs = f[torch.from_numpy(rows).cuda()].cpu().numpy().astype(np.float64)
        del pairs, p, f
    er, fr = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), rows)
    assert rel_rms(fs, fr) <= F_TOL
    x64 = s.x.astype(np.float64)
    L = float(s.box[0])
    b = band(r_nl)
    for i in rows:
        d2 = _min_image_d2(x64, x64[i], L)
        d2[i] = np.inf
        want = set(np.nonzero(d2 < r_nl * r_nl)[0].tolist())
        amb = set(np.nonzero(np.abs(d2 - r_nl * r_nl) <= b)[0].tolist())
        got = set(sub[sub[:, 0] == i, 1].tolist()) | set(sub[sub[:, 1] == i, 0].tolist())
        assert got - amb == want - amb, i


def test_batched_256_full_size_sampled():
    """The 256-system batch of the bench: sampled atoms of three LJ and three water
    systems (real space + PME) against the oracle, and those systems bitwise equal to
    their single-system handles."""
    systems = wl.batched_mix(256)
    offs = np.cumsum([0] + [s.n for s in systems])
    xq = torch.cat([dev_xq(s) for s in systems])
    n = int(offs[-1])
    f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((256, 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems, cell_div=1) as h:
        h.nonbonded_forces(xq, f, e)
        h.check()
    fb = f.cpu().numpy().astype(np.float64)
    eb = e.cpu().numpy()
    rng = np.random.default_rng(8)
    for k in (0, 2, 100, 1, 3, 101):
        s = systems[k]
        fk = fb[offs[k]:offs[k + 1]]
        rows = np.sort(rng.choice(s.n, min(40, s.n), replace=False))
        er, fr = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), rows,
                                       excl=s.excl)
        if s.pme_grid and s.pme_grid[0] > 0:
            Ep, Fp = oracle_pme(s)
            fr = fr + Fp[rows]
            assert abs(eb[k, 4] - Ep) <= E_TOL * abs(Ep)
        assert rel_rms(fk[rows], fr) <= F_TOL, k
        with nbcore.Handle([s], cell_div=1) as h1:
            f1 = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
            e1 = torch.empty((1, 6), dtype=torch.float64, device="cuda")
            h1.nonbonded_forces(dev_xq(s), f1, e1)
            h1.check()
        assert np.array_equal(f1.cpu().numpy().astype(np.float64), fk), k
        assert np.array_equal(e1.cpu().numpy()[0], eb[k]), k


def test_orthorhombic_water_box_against_the_oracle():
    """A non-cubic box: the molecules of the lowest 8 of the 10 lattice layers of a 31.05 A
    water box, in a 31.05 x 31.05 x 24.84 A cell (the lattice period along z, so the
    spacing across the boundary is regular; a different cell count, image shift and PME
    mesh size along z): forces, LJ, exclusion, self and reciprocal energies against the FP64 oracle, and the
    direct-space energy within its FP32 rounding bound (a sum that cancels by ~10^3)."""
    s = wl.water_slab(seed=7)
    with nbcore.Handle([s]) as h:
        f, e = _forces(h, s, terms=nbcore.NB_TERM_ALL)
    eo, fo = oracle_real_space(s)
    Ep, Fp = oracle_pme(s)
    assert rel_rms(f, fo + Fp) <= F_TOL
    for c in (0, 2, 3):
        assert abs(e[c] - eo[c]) <= E_TOL * abs(eo[c]), (c, e[c], eo[c])
    assert abs(e[4] - Ep) <= E_TOL * abs(Ep)
    # direct space: the random walk of FP32 roundings of the pair terms
    x = s.x.astype(np.float64)
    pairs, _ = oracle.neighbor_pairs(x, oracle_params(s), s.r_cut, excl=s.excl)
    d = x[pairs[:, 0]] - x[pairs[:, 1]]
    d -= s.box * np.round(d / s.box)
    r = np.sqrt(np.sum(d * d, axis=1))
    from scipy.special import erfc
    t = s.ke * s.q[pairs[:, 0]].astype(np.float64) * s.q[pairs[:, 1]] * erfc(s.alpha * r) / r
    bound = E_TOL * abs(eo[1]) + 6.0 * np.finfo(np.float32).eps * np.sqrt(np.sum(t * t))
    assert abs(e[1] - eo[1]) <= bound, (e[1], eo[1], bound)
    # precise (two-float) energies: every component at the flat bar
    with nbcore.Handle([s]) as h:
        ep = torch.empty((1, 6), dtype=torch.float64, device="cuda")
        h.nonbonded_forces(torch.from_numpy(nbcore.pack_xq(s.x, s.q)).cuda(), None, ep, precise=True)
        h.check()
        ep = ep.cpu().numpy()[0]
    for c in range(4):
        assert abs(ep[c] - eo[c]) <= E_TOL * abs(eo[c]), (c, ep[c], eo[c])
    assert abs(ep[4] - Ep) <= E_TOL * abs(Ep)
