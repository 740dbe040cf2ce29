"""GPU parity of rigid water and Langevin dynamics (Sec. 2.2.1) through the C ABI.

SETTLE and the velocity constraint against the oracle's SHAKE and RATTLE solutions of
the defining equations; Langevin trajectories of rigid reaction-field water against the
FP64 oracle integrator with the same normals; gamma = 0 without constraints against the
FP64 velocity Verlet; the thermostat's kinetic energy against equipartition over the six
degrees of freedom of each rigid molecule; a captured graph equal to eager launches.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import constraints as con
from oracle import dynamics as odyn
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import EPS32, dev_xq, oracle_params, rf_rounding_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

D_OH = wl.WATER_ROH
D_HH = 2.0 * wl.WATER_ROH * math.sin(math.radians(wl.WATER_HOH_DEG) / 2.0)
KT = 2.494  # kJ/mol at 300 K
TERMS = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL


def _water(n_mol=200, seed=11):
    s = wl.water_rf_density(n_mol, seed=seed, r_cut=8.0, r_skin=1.0)
    mols = np.arange(s.n).reshape(-1, 3)
    m = s.mass.astype(np.float64)
    x = con.constrain_positions(s.x.astype(np.float64), s.x.astype(np.float64), m, mols, D_OH, D_HH)
    s.x = x.astype(np.float32)
    return s, mols, m


def _bonds(x, mols):
    a, b, c = x[mols[:, 0]], x[mols[:, 1]], x[mols[:, 2]]
    return np.stack([np.linalg.norm(a - b, axis=1), np.linalg.norm(a - c, axis=1), np.linalg.norm(b - c, axis=1)], 1)


def _v4(v, m):
    out = np.zeros((len(m), 4), np.float32)
    out[:, :3] = v
    out[:, 3] = 1.0 / m
    return torch.from_numpy(out).cuda()


def test_settle_and_velocity_constraint_match_oracle():
    s, mols, m = _water()
    rng = np.random.default_rng(1)
    x0 = s.x.astype(np.float64)
    x1 = (x0 + 0.02 * rng.standard_normal(x0.shape)).astype(np.float32).astype(np.float64)
    ref = con.constrain_positions(x0, x1, m, mols, D_OH, D_HH)
    dt = 0.01
    v = rng.standard_normal((s.n, 3)).astype(np.float32)
    with nbcore.Handle([s]) as h:
        h.set_water_constraints(mols, D_OH, D_HH)
        xr = dev_xq(s)
        xn = torch.from_numpy(nbcore.pack_xq(x1, s.q)).cuda()
        vd = _v4(v, m)
        h.constrain_positions(xr, xn, torch.from_numpy((1.0 / m).astype(np.float32)).cuda(), vd, dt)
        h.check()
        xg = xn.cpu().numpy()[:, :3].astype(np.float64)
        vg = vd.cpu().numpy()[:, :3].astype(np.float64)
        np.testing.assert_allclose(xg, ref, rtol=0, atol=2e-5)
        np.testing.assert_allclose(_bonds(xg, mols), np.tile([D_OH, D_OH, D_HH], (len(mols), 1)), rtol=0, atol=1e-5)
        np.testing.assert_allclose(vg, v + (ref - x1) / dt, rtol=0, atol=5e-3)
        # velocity constraint at the constrained positions
        vr = rng.standard_normal((s.n, 3)).astype(np.float32)
        vd = _v4(vr, m)
        h.constrain_velocities(xn, vd)
        h.check()
    vo = con.constrain_velocities(xg, vr.astype(np.float64), m, mols, D_OH, D_HH)
    np.testing.assert_allclose(vd.cpu().numpy()[:, :3], vo, rtol=0, atol=2e-5)


def _oracle_fe(s):
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
        return f, float(e[:4].sum())
    return fe


@pytest.mark.parametrize("gamma", [0.0, 10.0])
def test_rigid_water_langevin_matches_oracle(gamma):
    s, mols, m = _water()
    rng = np.random.default_rng(2)
    v0 = con.constrain_velocities(s.x.astype(np.float64), np.sqrt(KT / m)[:, None] * rng.standard_normal((s.n, 3)),
                                  m, mols, D_OH, D_HH).astype(np.float32)
    n_steps, dt = 10, 0.01
    xi = rng.standard_normal((n_steps, s.n, 3)).astype(np.float32)
    xo, vo, Uo, Ko = con.langevin_middle(s.x.astype(np.float64), v0.astype(np.float64), m, dt, gamma, KT,
                                         xi.astype(np.float64), n_steps, _oracle_fe(s), mols, D_OH, D_HH)
    with nbcore.Handle([s]) as h:
        h.set_water_constraints(mols, D_OH, D_HH)
        x = dev_xq(s)
        v = _v4(v0, m)
        e = torch.empty((n_steps + 1, 1, 6), dtype=torch.float64, device="cuda")
        h.langevin_step(x, v, torch.tensor([dt], device="cuda"), torch.tensor([gamma], device="cuda"), KT, n_steps,
                        torch.from_numpy(xi).cuda(), e, terms=TERMS)
        h.check()
    xg = x.cpu().numpy()[:, :3].astype(np.float64)
    vg = v.cpu().numpy()[:, :3].astype(np.float64)
    # measured: 5e-6 A, 1.6e-5, 1.8e-6 A, |dU| at the reaction-field rounding scale, K 4e-7
    np.testing.assert_allclose(xg, xo, rtol=0, atol=2e-5)
    assert np.sqrt(np.mean((vg - vo) ** 2) / np.mean(vo ** 2)) < 5e-5
    np.testing.assert_allclose(_bonds(xg, mols), np.tile([D_OH, D_OH, D_HH], (len(mols), 1)), rtol=0, atol=6e-6)
    eg = e.cpu().numpy()[:, 0]
    U = eg[:, :5].sum(axis=1)
    tol_u = 1e-6 * np.abs(Uo).max() + 6 * EPS32 * rf_rounding_scale(s)
    assert np.abs(U - Uo).max() <= tol_u, (np.abs(U - Uo).max(), tol_u)
    np.testing.assert_allclose(eg[:, 5], Ko, rtol=2e-6)


def test_frictionless_unconstrained_langevin_is_velocity_verlet():
    s = wl.lj_fcc(n_cells=6, kT=0.72)
    p = oracle.make_params(s.box, r_cut=2.5)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    dt, n_steps = 0.005, 20
    x0, v0 = s.x.astype(np.float64), s.v.astype(np.float64)
    F0, _ = fe(x0)
    vh = (v0 - 0.5 * dt * F0).astype(np.float32)  # v_{-1/2} for the leapfrog form
    xv, _, Uv, _ = odyn.velocity_verlet(x0, v0, np.ones(s.n), dt, n_steps, fe)
    with nbcore.Handle([s]) as h:
        x = dev_xq(s)
        v = _v4(vh, np.ones(s.n))
        e = torch.empty((n_steps + 1, 1, 6), dtype=torch.float64, device="cuda")
        h.langevin_step(x, v, torch.tensor([dt], device="cuda"), torch.tensor([0.0], device="cuda"), 1.0, n_steps,
                        torch.zeros((n_steps, s.n, 3), device="cuda"), e, terms=nbcore.NB_TERM_LJ)
        h.check()
    d = x.cpu().numpy()[:, :3].astype(np.float64) - xv
    d -= s.box * np.round(d / s.box)
    assert np.abs(d).max() < 2e-5
    np.testing.assert_allclose(e.cpu().numpy()[:, 0, 0], Uv, rtol=2e-6)


def test_thermostat_equipartition_of_rigid_water():
    s, mols, m = _water(n_mol=300, seed=12)
    rng = np.random.default_rng(3)
    v0 = con.constrain_velocities(s.x.astype(np.float64), np.sqrt(KT / m)[:, None] * rng.standard_normal((s.n, 3)),
                                  m, mols, D_OH, D_HH).astype(np.float32)
    n_steps, dt, gamma = 1500, 0.005, 10.0
    with nbcore.Handle([s]) as h:
        h.set_water_constraints(mols, D_OH, D_HH)
        x = dev_xq(s)
        v = _v4(v0, m)
        e = torch.empty((n_steps + 1, 1, 6), dtype=torch.float64, device="cuda")
        xi = torch.randn((n_steps, s.n, 3), device="cuda", generator=torch.Generator(device="cuda").manual_seed(4))
        h.langevin_step(x, v, torch.tensor([dt], device="cuda"), torch.tensor([gamma], device="cuda"), KT, n_steps,
                        xi, e, terms=TERMS)
        h.check()
        xg = x.cpu().numpy()[:, :3].astype(np.float64)
    K = e.cpu().numpy()[n_steps // 3:n_steps, 0, 5]
    # six degrees of freedom per rigid molecule; the mean of the half-step kinetic energies
    # carries an O((gamma dt)^2, (omega dt)^2) bias well below the 3% bound
    assert K.mean() == pytest.approx(0.5 * 6 * len(mols) * KT, rel=0.03)
    np.testing.assert_allclose(_bonds(xg, mols), np.tile([D_OH, D_OH, D_HH], (len(mols), 1)), rtol=0, atol=6e-6)


def test_captured_langevin_equals_eager():
    from paper_2503_20541_b300.graphs import CapturedStep
    s, mols, m = _water()
    rng = np.random.default_rng(5)
    v0 = (np.sqrt(KT / m)[:, None] * rng.standard_normal((s.n, 3))).astype(np.float32)
    xi = torch.from_numpy(rng.standard_normal((5, s.n, 3)).astype(np.float32)).cuda()
    dt = torch.tensor([0.005], device="cuda")
    g = torch.tensor([10.0], device="cuda")
    out = []
    for captured in (False, True):
        with nbcore.Handle([s]) as h:
            h.set_water_constraints(mols, D_OH, D_HH)
            x = dev_xq(s)
            v = _v4(v0, m)
            x_init, v_init = x.clone(), v.clone()
            fn = lambda: h.langevin_step(x, v, dt, g, KT, 5, xi, terms=TERMS)  # noqa: E731
            if captured:
                step = CapturedStep(fn, warmup=1)
                x.copy_(x_init)
                v.copy_(v_init)
                h.nl_build(x, max_pairs=1, force_rebuild=True)
                step.replay()
            else:
                fn()
                x.copy_(x_init)
                v.copy_(v_init)
                h.nl_build(x, max_pairs=1, force_rebuild=True)
                fn()
            torch.cuda.synchronize()
            h.check()
            out.append((x.cpu().numpy(), v.cpu().numpy()))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_water_constraint_descriptor_checks():
    s, mols, m = _water()
    with nbcore.Handle([s]) as h:
        for bad in (np.array([[0, 1, 1]]), np.array([[0, 1, 2], [2, 4, 5]]), np.array([[0, 1, s.n]])):
            with pytest.raises(nbcore.NbError):
                h.set_water_constraints(bad, D_OH, D_HH)
        with pytest.raises(nbcore.NbError):
            h.set_water_constraints(mols, D_OH, 2.5 * D_OH)
        h.set_water_constraints(mols, D_OH, D_HH)
        h.set_water_constraints(np.zeros((0, 3), np.int32), D_OH, D_HH)  # removes them
    s2, _, _ = _water(seed=13)
    with nbcore.Handle([s, s2]) as h:  # a molecule across two systems
        with pytest.raises(nbcore.NbError):
            h.set_water_constraints(np.array([[s.n - 1, s.n, s.n + 1]]), D_OH, D_HH)
