"""Pins of the FP64 oracle against values fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: closed forms
(LJ dimer, lattice Madelung sums, B-spline pieces, the discrete harmonic
solution of velocity Verlet), invariances (Ewald alpha-independence, translation,
Newton III, Hessian symmetry), finite differences, and library routines for
special cases (scipy's KD-tree for the pair set).  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import pme as opme
from paper_2503_20541_b300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()[:2]
            vals[k] = float(v)
    return vals


# ---------------------------------------------------------------- LJ (Eq. lj)

def _dimer(r, g, r_cut=10.0, r_switch=-1.0):
    x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    sig = np.array([g["sigma1"], g["sigma2"]])
    sqe = np.sqrt([g["eps1"], g["eps2"]])
    p = oracle.make_params(40.0, r_cut=r_cut, r_switch=r_switch)
    return oracle.nonbonded(x, np.zeros(2), sig, sqe, p)


def test_lj_dimer_minimum_depth_and_zero_crossing():
    g = golden("lj_dimer.txt")
    e, f = _dimer(g["r_min"], g)
    assert e[0] == pytest.approx(g["U_min"], rel=1e-12)
    assert np.abs(f).max() < 1e-12
    for h in (1e-3, -1e-3):
        assert _dimer(g["r_min"] + h, g)[0][0] > g["U_min"]
    e0, _ = _dimer(0.5 * (g["sigma1"] + g["sigma2"]), g)
    assert abs(e0[0]) < 1e-13
    # repulsive inside sigma: force pushes atom 1 (at +x) further along +x
    _, fr = _dimer(1.2, g)
    assert fr[1, 0] > 0 and fr[0, 0] < 0


def test_lj_switch_continuity_and_symmetry():
    g = golden("lj_dimer.txt")
    rc, rs = 2.5, 2.0
    # energy and force vanish as r -> r_c with the switch, not without it
    e_sw, f_sw = _dimer(rc - 1e-7, g, r_cut=rc, r_switch=rs)
    e_ns, _ = _dimer(rc - 1e-7, g, r_cut=rc)
    assert abs(e_sw[0]) < 1e-15 and abs(e_ns[0]) > 1e-3
    assert np.abs(f_sw).max() < 1e-10
    # S(x) + S(1-x) = 1 and S(1/2) = 1/2 for the smoothstep S = 1 - 6x^5 + 15x^4 - 10x^3
    def S(x):
        r = rs + x * (rc - rs)
        return _dimer(r, g, r_cut=rc, r_switch=rs)[0][0] / _dimer(r, g, r_cut=rc)[0][0]
    for x in (0.1, 0.3, 0.45):
        assert S(x) + S(1 - x) == pytest.approx(1.0, abs=1e-12)
    assert S(0.5) == pytest.approx(0.5, abs=1e-12)
    # unchanged inside r_s
    assert _dimer(1.9, g, r_cut=rc, r_switch=rs)[0][0] == _dimer(1.9, g, r_cut=rc)[0][0]


# ------------------------------------------------------------ Ewald (Sec. 2.1.2)

def _rocksalt(n_cells, r0=1.0):
    a = 2.0 * r0
    na = wl.fcc_sites(n_cells, a)
    cl = na + np.array([r0, 0.0, 0.0])
    x = np.concatenate([na, cl])
    q = np.concatenate([np.ones(len(na)), -np.ones(len(cl))])
    L = n_cells * a
    return x - L * np.floor(x / L), q, L


def _ewald_total(x, q, L, alpha, r_cut, mmax, excl=None, ke=1.0):
    p = oracle.make_params(L, r_cut=r_cut, alpha=alpha, ke=ke)
    n = len(q)
    e, f = oracle.nonbonded(x, q, np.ones(n), np.zeros(n), p, excl=excl)
    er, fr = oracle.ewald_recip(x, q, L, alpha, ke, mmax)
    return e[1] + e[2] + e[3] + er, f + fr


def test_ewald_nacl_madelung():
    g = golden("madelung_nacl.txt")
    x, q, L = _rocksalt(4)
    E, F = _ewald_total(x, q, L, alpha=1.4, r_cut=L / 2, mmax=22)
    expected = -0.5 * len(q) * g["M"] / 1.0
    assert E == pytest.approx(expected, rel=g["tolerance_rel"])
    assert np.abs(F).max() < 1e-8  # perfect lattice: every ion at a symmetry centre


def _charges_on_lattice(seed, L=10.0, side=4, jitter=0.5):
    rng = np.random.default_rng(seed)
    g = (np.arange(side) + 0.5) * L / side
    x = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    x = x + rng.uniform(-jitter, jitter, x.shape)
    q = np.where(np.arange(len(x)) % 2 == 0, 1.0, -1.0) * rng.uniform(0.5, 1.5, len(x))
    q -= q.mean()
    return x - L * np.floor(x / L), q, L


def test_ewald_total_is_alpha_independent():
    x, q, L = _charges_on_lattice(7)
    E1, F1 = _ewald_total(x, q, L, alpha=1.15, r_cut=L / 2, mmax=24)
    E2, F2 = _ewald_total(x, q, L, alpha=1.4, r_cut=L / 2, mmax=28)
    assert E1 == pytest.approx(E2, rel=1e-10)
    assert np.abs(F1 - F2).max() < 1e-8 * np.abs(F1).max()


def test_exclusion_correction_removes_bare_pair():
    x, q, L = _charges_on_lattice(11)
    x[1] = x[0] + np.array([0.9, 0.3, -0.2])  # a bonded-like pair
    x[3] = x[2] + np.array([-0.5, 0.8, 0.1])
    n = len(q)
    excl_pairs = [(0, 1), (2, 3)]
    lists = [[] for _ in range(n)]
    for i, j in excl_pairs:
        lists[i].append(j)
        lists[j].append(i)
    off = np.cumsum([0] + [len(l) for l in lists]).astype(np.int32)
    idx = np.array([j for l in lists for j in l], dtype=np.int32)
    for alpha, mm in ((1.15, 24), (1.4, 28)):
        Ee, Fe = _ewald_total(x, q, L, alpha, L / 2, mm, excl=(off, idx))
        Ea, Fa = _ewald_total(x, q, L, alpha, L / 2, mm)
        bare = 0.0
        Fb = np.zeros_like(Fa)
        for i, j in excl_pairs:
            d = x[i] - x[j]
            r = np.linalg.norm(d)
            bare += q[i] * q[j] / r
            Fb[i] += q[i] * q[j] * d / r ** 3
            Fb[j] -= q[i] * q[j] * d / r ** 3
        assert Ee == pytest.approx(Ea - bare, rel=1e-10)
        assert np.abs(Fe - (Fa - Fb)).max() < 1e-8 * np.abs(Fa).max()


# -------------------------------------------------------------- PME / B-splines

def test_bspline_recursion_matches_cubic_pieces():
    t = np.linspace(0.0, 1.0, 11)
    M = lambda u: opme.bspline(4, u)
    np.testing.assert_allclose(M(t), t ** 3 / 6, atol=1e-15)
    np.testing.assert_allclose(M(t + 1), (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6, atol=1e-15)
    np.testing.assert_allclose(M(t + 2), (3 * t ** 3 - 6 * t ** 2 + 4) / 6, atol=1e-15)
    np.testing.assert_allclose(M(t + 3), (1 - t) ** 3 / 6, atol=1e-15)
    for n in (3, 4, 5, 6):
        s = sum(opme.bspline(n, t + j) for j in range(n))
        np.testing.assert_allclose(s, 1.0, atol=1e-14)  # partition of unity
        u = np.linspace(0.3, n - 0.3, 7)
        h = 1e-6
        fd = (opme.bspline(n, u + h) - opme.bspline(n, u - h)) / (2 * h)
        np.testing.assert_allclose(opme.dbspline(n, u), fd, atol=1e-8)


def test_bspline_moduli_closed_form_order4():
    K = 64
    m = np.arange(K)
    expect = 9.0 / (2.0 + np.cos(2 * np.pi * m / K)) ** 2
    np.testing.assert_allclose(opme.bspline_moduli(4, K), expect, rtol=1e-13)


def test_pme_converges_to_exact_reciprocal_sum():
    x, q, L = _charges_on_lattice(3)
    alpha = 0.7
    Ee, Fe = oracle.ewald_recip(x, q, L, alpha, 1.0, mmax=14)
    errs = []
    for K in (16, 32, 64, 128):
        Ep, Fp = opme.pme(x, q, L, alpha, 1.0, K)
        errs.append((abs(Ep - Ee) / abs(Ee), np.linalg.norm(Fp - Fe) / np.linalg.norm(Fe)))
    # order-4 cardinal B-splines: energy error O(h^4), force error O(h^3)
    for a, b in zip(errs[:-1], errs[1:]):
        assert b[0] < a[0] / 12 and b[1] < a[1] / 6
    assert errs[-1][0] < 1e-6 and errs[-1][1] < 5e-5


def test_pme_forces_are_gradient_of_pme_energy():
    x, q, L = _charges_on_lattice(5, side=3)
    rng = np.random.default_rng(0)
    E, F = opme.pme(x, q, L, 0.8, 1.0, 20)
    h = 1e-6
    for _ in range(6):
        i, d = rng.integers(len(q)), rng.integers(3)
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        fd = -(opme.pme(xp, q, L, 0.8, 1.0, 20)[0] - opme.pme(xm, q, L, 0.8, 1.0, 20)[0]) / (2 * h)
        assert fd == pytest.approx(F[i, d], rel=1e-6, abs=1e-8)


# ------------------------------------------------------------ neighbour set

@pytest.mark.parametrize("factor,shells", [(1.1, 12 + 6), (1.3, 12 + 6 + 24)])
def test_neighbor_pairs_fcc_shell_counts(factor, shells):
    a = 1.5
    x = wl.fcc_sites(5, a)
    L = 5 * a
    p = oracle.make_params(L, r_cut=1.0)
    pairs, _ = oracle.neighbor_pairs(x, p, factor * a)
    assert len(pairs) == len(x) * shells // 2
    assert np.all(pairs[:, 0] < pairs[:, 1])


def test_neighbor_pairs_match_kdtree():
    from scipy.spatial import cKDTree
    s = wl.lj_random(1500, seed=5)
    L = s.box[0]
    x = s.x.astype(np.float64)
    r_nl = 2.8
    p = oracle.make_params(L, r_cut=2.5)
    pairs, _ = oracle.neighbor_pairs(x, p, r_nl)
    ref = cKDTree(x, boxsize=L).query_pairs(r_nl, output_type="ndarray")
    ref = {tuple(sorted(t)) for t in ref.tolist()}
    assert {tuple(t) for t in pairs.tolist()} == ref
    # open system: the same set without periodic images
    po = oracle.make_params(L, r_cut=2.5, periodic=False)
    pairs_o, _ = oracle.neighbor_pairs(x, po, r_nl)
    ref_o = {tuple(sorted(t)) for t in cKDTree(x).query_pairs(r_nl, output_type="ndarray").tolist()}
    assert {tuple(t) for t in pairs_o.tolist()} == ref_o


def test_neighbor_pairs_drop_exclusions():
    s = wl.water_box(n_side=4, L=12.4, seed=2, r_cut=6.0)
    x = s.x.astype(np.float64)
    p = oracle.make_params(s.box, r_cut=6.0)
    with_ex, _ = oracle.neighbor_pairs(x, p, 6.0, excl=s.excl)
    without, _ = oracle.neighbor_pairs(x, p, 6.0)
    assert len(without) - len(with_ex) == 3 * (s.n // 3)  # three intramolecular pairs each


# ------------------------------------------------ forces, invariances, VJP

def _small_water(seed=4, elec="ewald"):
    s = wl.water_box(n_side=3, L=9.6, seed=seed, r_cut=4.6, alpha=0.8)
    if elec == "rf":
        p = oracle.make_params(s.box, r_cut=4.6, r_switch=4.0, ke=wl.KE_KJ_MOL_A, eps_rf=78.5)
    else:
        p = oracle.make_params(s.box, r_cut=4.6, r_switch=4.0, alpha=0.8, ke=wl.KE_KJ_MOL_A)
    return s, p


def _near_cutoff(x, i, p, rc, tol=2e-3):
    d = x - x[i]
    d -= p.box[0] * np.round(d / p.box[0])
    r = np.linalg.norm(d, axis=1)
    return np.any(np.abs(r - rc) < tol)


@pytest.mark.parametrize("elec", ["ewald", "rf"])
def test_forces_are_minus_gradient_real_space(elec):
    s, p = _small_water(elec=elec)
    x = s.x.astype(np.float64)
    e, F = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
    rng = np.random.default_rng(1)
    h = 1e-6
    checked = 0
    while checked < 12:
        i, d = int(rng.integers(s.n)), int(rng.integers(3))
        if _near_cutoff(x, i, p, 4.6):
            continue
        xp, xm = x.copy(), x.copy()
        xp[i, d] += h
        xm[i, d] -= h
        Ep = oracle.nonbonded(xp, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)[0][:3].sum()
        Em = oracle.nonbonded(xm, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)[0][:3].sum()
        assert -(Ep - Em) / (2 * h) == pytest.approx(F[i, d], rel=1e-6, abs=1e-6)
        checked += 1


def test_forces_are_minus_gradient_reciprocal():
    x, q, L = _charges_on_lattice(9, side=3)
    E, F = oracle.ewald_recip(x, q, L, 0.9, 1.0, 10)
    h = 1e-3  # fourth-order stencil: truncation O(h^4), round-off ~1e-13/h

    def E_at(i, d, dx):
        xs = x.copy()
        xs[i, d] += dx
        return oracle.ewald_recip(xs, q, L, 0.9, 1.0, 10)[0]
    for i, d in ((0, 0), (5, 1), (13, 2)):
        fd = -(E_at(i, d, -2 * h) - 8 * E_at(i, d, -h) + 8 * E_at(i, d, h) - E_at(i, d, 2 * h)) / (12 * h)
        assert fd == pytest.approx(F[i, d], rel=1e-8, abs=1e-10)


def test_newton_third_law_and_translation_invariance():
    s, p = _small_water()
    x = s.x.astype(np.float64)
    e, F = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
    assert np.abs(F.sum(axis=0)).max() < 1e-9 * np.abs(F).max()
    e2, F2 = oracle.nonbonded(x + np.array([0.37, -1.3, 2.1]), s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
    np.testing.assert_allclose(e2, e, rtol=1e-10)
    np.testing.assert_allclose(F2, F, atol=1e-8 * np.abs(F).max())


@pytest.mark.parametrize("elec", ["ewald", "rf"])
def test_force_vjp_matches_finite_differences(elec):
    s, p = _small_water(6, elec=elec)
    x = s.x.astype(np.float64)
    n = s.n
    rng = np.random.default_rng(2)
    lam = rng.standard_normal((n, 3))
    gx, gq, gs, ge = oracle.force_vjp(x, s.q, s.sigma, s.sqrt_eps, p, lam, excl=s.excl)
    h = 1e-6
    checked = 0
    while checked < 10:
        k, d = int(rng.integers(n)), int(rng.integers(3))
        if _near_cutoff(x, k, p, 4.6):
            continue
        xp, xm = x.copy(), x.copy()
        xp[k, d] += h
        xm[k, d] -= h
        Fp = oracle.nonbonded(xp, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)[1]
        Fm = oracle.nonbonded(xm, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)[1]
        fd = float(np.sum(lam * (Fp - Fm)) / (2 * h))
        assert gx[k, d] == pytest.approx(fd, rel=1e-5, abs=1e-4)
        checked += 1
    # parameter gradients of lam . F
    def lamF(q=s.q, sig=s.sigma, sqe=s.sqrt_eps):
        return float(np.sum(lam * oracle.nonbonded(x, q, sig, sqe, p, excl=s.excl)[1]))
    for k in (0, 1, 4):
        for arr, g in ((s.q, gq), (s.sigma, gs), (s.sqrt_eps, ge)):
            ap, am = arr.astype(np.float64).copy(), arr.astype(np.float64).copy()
            ap[k] += h
            am[k] -= h
            kw = {0: "q", 1: "sig", 2: "sqe"}[[id(s.q), id(s.sigma), id(s.sqrt_eps)].index(id(arr))]
            fd = (lamF(**{kw: ap}) - lamF(**{kw: am})) / (2 * h)
            assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-4)


@pytest.mark.parametrize("elec", ["ewald", "rf"])
def test_force_jacobian_is_symmetric(elec):
    s, p = _small_water(8, elec=elec)
    x = s.x.astype(np.float64)
    rng = np.random.default_rng(3)
    g1, g2 = rng.standard_normal((2, s.n, 3))
    v1 = oracle.force_vjp(x, s.q, s.sigma, s.sqrt_eps, p, g1, excl=s.excl)[0]
    v2 = oracle.force_vjp(x, s.q, s.sigma, s.sqrt_eps, p, g2, excl=s.excl)[0]
    assert np.sum(g2 * v1) == pytest.approx(np.sum(g1 * v2), rel=1e-11)


# ------------------------------------------------------------ reaction field (Eq. RFA)

def _rf_dimer(r, eps_rf, rc=9.0, excl=False):
    x = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    q = np.array([0.7, -0.4])
    p = oracle.make_params(40.0, r_cut=rc, ke=wl.KE_KJ_MOL_A, eps_rf=eps_rf)
    ex = (np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32)) if excl else None
    return oracle.nonbonded(x, q, np.ones(2), np.zeros(2), p, excl=ex)


def test_reaction_field_special_cases():
    rc = 9.0
    qq = wl.KE_KJ_MOL_A * 0.7 * -0.4
    # eps_s = 1 (no dielectric beyond r_c): Coulomb shifted to vanish at r_c, force unchanged
    for r in (1.0, 3.7, 8.5):
        e, f = _rf_dimer(r, 1.0)
        assert e[1] == pytest.approx(qq * (1.0 / r - 1.0 / rc), rel=1e-13)
        assert f[0, 0] == pytest.approx(-qq / (r * r), rel=1e-13)
        assert f[1, 0] == pytest.approx(qq / (r * r), rel=1e-13)
        assert e[2] == 0.0 and e[3] == 0.0
    # conducting boundary (eps_s -> infinity): k r_c^3 -> 1/2, c r_c -> 3/2
    r = 4.5
    e, f = _rf_dimer(r, 1e15)
    assert e[1] == pytest.approx(qq * (1.0 / r + r * r / (2 * rc ** 3) - 1.5 / rc), rel=1e-12)
    assert f[0, 0] == pytest.approx(-qq * (1.0 / (r * r) - r / rc ** 3), rel=1e-12)
    # the energy goes to zero at the cut-off and is cut beyond it
    e_in, _ = _rf_dimer(rc * (1 - 1e-12), 78.5)
    e_out, f_out = _rf_dimer(rc * (1 + 1e-12), 78.5)
    assert abs(e_in[1]) < 1e-9 * abs(qq) / rc
    assert e_out[1] == 0.0 and np.all(f_out == 0.0)
    # excluded pairs do not interact under the reaction field
    e, f = _rf_dimer(1.0, 78.5, excl=True)
    assert np.all(e == 0.0) and np.all(f == 0.0)


# ------------------------------------------------------------ dynamics / HMC

def test_velocity_verlet_harmonic_closed_form():
    # x'' = -w^2 x under velocity Verlet: x_n = cos(n theta), cos(theta) = 1 - (w dt)^2/2
    w2, dt = 2.0, 0.1
    fe = lambda x: (-w2 * x, 0.5 * w2 * float(np.sum(x ** 2)))
    x0 = np.array([[1.0, 0.0, 0.0]])
    v0 = np.zeros((1, 3))
    th = math.acos(1 - w2 * dt * dt / 2)
    for n in (1, 7, 50):
        x, v, _, _ = odyn.velocity_verlet(x0, v0, np.ones(1), dt, n, fe)
        assert x[0, 0] == pytest.approx(math.cos(n * th), abs=1e-12)


def _lj_fe(s, p):
    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    return fe


def test_velocity_verlet_reversible_and_second_order():
    s = wl.lj_fcc(n_cells=3, kT=0.72)
    p = oracle.make_params(s.box, r_cut=2.5, r_switch=2.2)
    fe = _lj_fe(s, p)
    x0 = s.x.astype(np.float64)
    v0 = s.v.astype(np.float64)
    w = np.ones(s.n)
    x1, v1, _, _ = odyn.velocity_verlet(x0, v0, w, 0.005, 40, fe)
    x2, v2, _, _ = odyn.velocity_verlet(x1, -v1, w, 0.005, 40, fe)
    assert np.abs(x2 - x0).max() < 1e-9 and np.abs(v2 + v0).max() < 1e-9
    # energy error of the leapfrog is O(dt^2)
    errs = []
    for dt in (0.004, 0.002):
        _, _, U, K = odyn.velocity_verlet(x0, v0, w, dt, int(round(0.2 / dt)), fe)
        H = U + K
        errs.append(np.abs(H - H[0]).max())
    assert 3.0 < errs[0] / errs[1] < 5.0


def test_hmc_acceptance_and_mass_repartition():
    s = wl.lj_random(108, seed=3, n_types=2)
    # smooth switch: with plain truncation, cutoff crossings add O(1) energy jumps to dH
    p = oracle.make_params(s.box, r_cut=2.5, r_switch=2.2)
    fe = _lj_fe(s, p)
    rng = np.random.default_rng(4)
    xi = rng.standard_normal((s.n, 3))
    dHs = []
    for dt in (0.004, 0.002, 0.001):
        out = odyn.hmc_proposal(s.x.astype(np.float64), xi, np.ones(s.n), dt, int(round(0.032 / dt)), 1.0, fe, s.box)
        assert 0.0 <= out["alpha"] <= 1.0
        assert out["alpha"] == pytest.approx(min(1.0, math.exp(-out["dH"])), rel=1e-12)
        # the kinetic energy of the Maxwell-Boltzmann draw is kT/2 sum xi^2, independent of masses
        assert out["K0"] == pytest.approx(0.5 * np.sum(xi ** 2), rel=1e-12)
        dHs.append(abs(out["dH"]))
    assert dHs[0] / dHs[1] > 2.5 and dHs[1] / dHs[2] > 2.5
    m = odyn.masses_from_logits([0.3, -0.2], s.types, float(s.n))
    assert m.sum() == pytest.approx(s.n, rel=1e-14)
    assert m[0] / m[1] == pytest.approx(math.exp(0.5), rel=1e-14)
    np.testing.assert_allclose(odyn.masses_from_logits([0.0, 0.0], s.types, 7.0 * s.n), 7.0)


def test_ewald_alpha_heuristic():
    # alpha = sqrt(-log(2 delta))/r_c; with r_c = 9 and alpha = 0.32 the tolerance is ~1.3e-4
    a = oracle.ewald_alpha(1.3e-4, 9.0)
    assert a == pytest.approx(0.32, rel=0.01)
    assert math.exp(-(a * 9.0) ** 2) == pytest.approx(2 * 1.3e-4, rel=1e-12)


def test_oracle_and_library_share_no_code():
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    pat_o = re.compile(r"^\s*(import|from)\s+paper_2503_20541_b300|#\s*include\s*[<\"].*(nbcore|csrc)", re.M)
    for dirpath, _, files in os.walk(os.path.join(root, "oracle")):
        for fn in files:
            if fn.endswith((".py", ".c", ".h")):
                assert not pat_o.search(open(os.path.join(dirpath, fn)).read()), fn
    pat_p = re.compile(r"^\s*(import|from)\s+oracle\b|#\s*include\s*[<\"].*oracle", re.M)
    for dirpath, _, files in os.walk(os.path.join(root, "paper_2503_20541_b300")):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                assert not pat_p.search(open(os.path.join(dirpath, fn)).read()), fn


def test_pme_force_vjp_matches_central_differences_and_is_symmetric():
    """The reciprocal-space force VJP: d(lam . F_rec)/dx and /dq by FP64 central
    differences of the forward PME forces, and <h, VJP(g)> = <g, VJP(h)> (the position
    Hessian of E_rec is symmetric)."""
    from oracle import pme as opme
    rng = np.random.default_rng(7)
    n, L, K = 24, np.array([9.0, 9.0, 9.0]), (12, 12, 12)
    x = rng.uniform(0, 9.0, (n, 3))
    q = rng.uniform(-1, 1, n)
    q -= q.mean()
    alpha, ke = 0.45, 1.0
    lam = rng.standard_normal((n, 3))
    gx, gq = opme.pme_force_vjp(x, q, L, alpha, ke, K, lam)

    def lf(xx, qq):
        return float(np.sum(lam * opme.pme(xx, qq, L, alpha, ke, K)[1]))
    h = 1e-5
    for i in (0, 5, 17):
        for d in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, d] += h
            xm[i, d] -= h
            fd = (lf(xp, q) - lf(xm, q)) / (2 * h)
            assert abs(gx[i, d] - fd) <= 1e-6 * (1.0 + abs(fd)), (i, d, gx[i, d], fd)
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd = (lf(x, qp) - lf(x, qm)) / (2 * h)
        assert abs(gq[i] - fd) <= 1e-6 * (1.0 + abs(fd)), (i, gq[i], fd)
    g2 = rng.standard_normal((n, 3))
    gx2, _ = opme.pme_force_vjp(x, q, L, alpha, ke, K, g2)
    a, b = float(np.sum(g2 * gx)), float(np.sum(lam * gx2))
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))
