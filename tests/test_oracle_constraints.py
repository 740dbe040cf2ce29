"""Pins of the constraint and Langevin oracle (oracle.constraints).

SHAKE: the solution satisfies the constraints, keeps the momentum, moves each atom only
within the old molecular plane with zero net torque about the old positions (the
properties that make it unique and that SETTLE's closed form is built on), and leaves a
rigidly moved molecule unchanged.  RATTLE: a projection (idempotent) that zeroes the
bond-length rates and leaves rigid-body velocities unchanged.  Langevin: with gamma = 0
and no constraints the positions are those of the pinned velocity Verlet; the O step
preserves the Maxwell-Boltzmann variance; constrained NVE water conserves energy to
second order in dt with the constraints held at every step.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import constraints as con
from oracle import dynamics as odyn
from paper_2503_20541_b300 import workloads as wl

D_OH = wl.WATER_ROH
D_HH = 2.0 * wl.WATER_ROH * math.sin(math.radians(wl.WATER_HOH_DEG) / 2.0)
M = np.array([wl.MASS_O, wl.MASS_H, wl.MASS_H])


def _molecule(rng):
    th = math.radians(wl.WATER_HOH_DEG) / 2.0
    ref = np.array([[0.0, 0.0, 0.0], [D_OH * math.sin(th), D_OH * math.cos(th), 0.0],
                    [-D_OH * math.sin(th), D_OH * math.cos(th), 0.0]])
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    return ref @ q.T + rng.uniform(-5, 5, 3)


def _bonds(x):
    return np.array([np.linalg.norm(x[0] - x[1]), np.linalg.norm(x[0] - x[2]), np.linalg.norm(x[1] - x[2])])


def test_shake_solution_properties():
    rng = np.random.default_rng(1)
    for _ in range(20):
        x0 = _molecule(rng)
        x1 = x0 + 0.05 * rng.standard_normal((3, 3))
        x3 = con.shake_molecule(x0, x1, M, D_OH, D_HH)
        np.testing.assert_allclose(_bonds(x3), [D_OH, D_OH, D_HH], rtol=0, atol=1e-12)
        d = x3 - x1
        np.testing.assert_allclose(M @ d, 0.0, atol=1e-13)  # momentum
        n0 = np.cross(x0[1] - x0[0], x0[2] - x0[0])
        np.testing.assert_allclose(d @ n0, 0.0, atol=1e-13)  # in the old plane
        torque = np.sum(M[:, None] * np.cross(x0, d), axis=0)
        np.testing.assert_allclose(torque, 0.0, atol=1e-12)


def test_shake_leaves_rigid_motion_unchanged():
    rng = np.random.default_rng(2)
    x0 = _molecule(rng)
    q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    c = x0.mean(axis=0)
    x1 = (x0 - c) @ q.T + c + np.array([0.3, -0.2, 0.1])
    np.testing.assert_allclose(con.shake_molecule(x0, x1, M, D_OH, D_HH), x1, atol=1e-12)


def test_rattle_is_a_projection_keeping_rigid_body_velocities():
    rng = np.random.default_rng(3)
    x = _molecule(rng)
    v = rng.standard_normal((3, 3))
    p = con.rattle_molecule(x, v, M, D_OH, D_HH)
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        assert abs(np.dot(x[i] - x[j], p[i] - p[j])) < 1e-12
    np.testing.assert_allclose(M @ p, M @ v, atol=1e-12)
    np.testing.assert_allclose(con.rattle_molecule(x, p, M, D_OH, D_HH), p, atol=1e-12)
    assert np.sum(M[:, None] * p * p) <= np.sum(M[:, None] * v * v)
    w, V = rng.standard_normal(3), rng.standard_normal(3)
    rigid = np.cross(w, x - x.mean(axis=0)) + V
    np.testing.assert_allclose(con.rattle_molecule(x, rigid, M, D_OH, D_HH), rigid, atol=1e-12)


def _lj_fe(s, p):
    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    return fe


def test_langevin_without_friction_is_velocity_verlet():
    s = wl.lj_fcc(n_cells=3, kT=0.72)
    p = oracle.make_params(s.box, r_cut=2.5, r_switch=2.2)
    fe = _lj_fe(s, p)
    x0, v0 = s.x.astype(np.float64), s.v.astype(np.float64)
    m = np.ones(s.n)
    dt = 0.005
    F0, _ = fe(x0)
    xi = np.zeros((12, s.n, 3))
    x_lf, _, U_lf, _ = con.langevin_middle(x0, v0 - 0.5 * dt * F0, m, dt, 0.0, 1.0, xi, 12, fe)
    x_vv, _, U_vv, _ = odyn.velocity_verlet(x0, v0, m, dt, 12, fe)
    np.testing.assert_allclose(x_lf, x_vv, rtol=0, atol=1e-11)
    np.testing.assert_allclose(U_lf, U_vv, rtol=1e-11)


def test_ornstein_uhlenbeck_step_keeps_maxwell_boltzmann():
    rng = np.random.default_rng(4)
    n, kT = 200000, 2.5
    m = rng.choice([1.0, 16.0], n)
    v0 = np.sqrt(kT / m)[:, None] * rng.standard_normal((n, 3))
    fe = lambda x: (np.zeros_like(x), 0.0)  # noqa: E731
    for gamma in (0.0, 3.0, 1e6):
        _, v, _, _ = con.langevin_middle(np.zeros((n, 3)), v0, m, 0.01, gamma, kT, rng.standard_normal((1, n, 3)), 1,
                                         fe)
        z = v * np.sqrt(m / kT)[:, None]
        assert np.mean(z * z) == pytest.approx(1.0, abs=0.01)
    # gamma -> infinity: the old velocities are forgotten
    _, v, _, _ = con.langevin_middle(np.zeros((n, 3)), v0, m, 0.01, 1e6, kT, np.zeros((1, n, 3)), 1, fe)
    assert np.abs(v).max() < 1e-12


def _rigid_water():
    s = wl.water_rf_density(200, seed=11, r_cut=8.0, r_skin=1.0)
    p = oracle.make_params(s.box, r_cut=s.r_cut, ke=s.ke, eps_rf=s.eps_rf, r_switch=-1.0)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
        return f, float(e[:4].sum())
    mols = np.arange(s.n).reshape(-1, 3)
    return s, fe, mols


def test_constrained_nve_water_is_second_order_and_rigid():
    s, fe, mols = _rigid_water()
    m = s.mass.astype(np.float64)
    x0 = s.x.astype(np.float64)
    x0 = con.constrain_positions(x0, x0, m, mols, D_OH, D_HH)  # exact geometry
    rng = np.random.default_rng(5)
    kT = 2.494
    v0 = con.constrain_velocities(x0, np.sqrt(kT / m)[:, None] * rng.standard_normal((s.n, 3)), m, mols, D_OH,
                                  D_HH)
    errs = []
    for dt in (0.008, 0.004):
        n = int(round(0.08 / dt))
        x, v, U, K = con.langevin_middle(x0, v0, m, dt, 0.0, kT, np.zeros((n, s.n, 3)), n, fe, mols, D_OH, D_HH)
        for mol in mols:
            np.testing.assert_allclose(_bonds(x[mol]), [D_OH, D_OH, D_HH], rtol=0, atol=1e-10)
        H = U[:-1] + K[:-1]
        errs.append(np.abs(H - H[0]).max())
    assert 3.0 < errs[0] / errs[1] < 5.0
