"""Batched MD and HMC (Sec. 2.2.1 velocity Verlet; Sec. 4 HMC proposal with the FP64 dH
acceptance) over uneven LJ systems of the 256-system mix (its LJ half, sizes log-uniform
in [500, 20000]): one handle for all systems, every system's trajectory checked against
the FP64 oracle integrator, and every system bitwise equal to the same system run alone
in its own handle while the list rebuild schedules agree (a batched handle rebuilds every
system's list when one system needs it; the step sizes keep the displacements below the
rebuild threshold, and the check is made only when no rebuild followed the first build)."""
import copy

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KT = 1.0


def _mix_lj(k=5):
    """The smallest LJ systems of the mix (500-534 atoms: boxes with folded axes) and one
    of ~2,000 atoms (a full cell stencil)."""
    mix = wl.batched_mix(256)
    lj = sorted([s for s in mix if s.ke == 0.0], key=lambda s: s.n)
    mid = min(lj, key=lambda s: abs(s.n - 2000))
    return lj[:k - 1] + [mid]


def _oracle_fe(s):
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded_cells(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    return fe


def _velocities(systems, seed):
    rng = np.random.default_rng(seed)
    return [(np.sqrt(KT) * rng.standard_normal((s.n, 3))).astype(np.float32) for s in systems]


def _md(systems, vs, dt, n_steps):
    n = sum(s.n for s in systems)
    xq = torch.cat([dev_xq(s) for s in systems])
    v = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    v[:, :3] = torch.from_numpy(np.concatenate(vs)).cuda()
    v[:, 3] = 1.0
    E = torch.zeros((n_steps + 1, len(systems), 6), dtype=torch.float64, device="cuda")
    with nbcore.Handle(systems) as h:
        h.md_step(xq, v, torch.full((len(systems),), dt, dtype=torch.float32, device="cuda"), n_steps, E,
                  terms=nbcore.NB_TERM_LJ)
        h.check()
        rebuilds = h.rebuild_count()
    return xq.cpu().numpy(), v.cpu().numpy(), E.cpu().numpy(), rebuilds


def test_batched_md_matches_oracle_and_single_systems():
    systems = _mix_lj()
    vs = _velocities(systems, 21)
    n_steps, dt = 10, 0.002
    xb, vb, Eb, rb = _md(systems, vs, dt, n_steps)
    off = 0
    for k, s in enumerate(systems):
        sl = slice(off, off + s.n)
        off += s.n
        # bitwise: the system alone in its own handle
        xs1, vs1, Es1, r1 = _md([s], [vs[k]], dt, n_steps)
        if rb == 1 and r1 == 1:
            assert np.array_equal(xs1, xb[sl]) and np.array_equal(vs1, vb[sl])
            assert np.array_equal(Es1[:, 0, :], Eb[:, k, :])
        # the FP64 velocity-Verlet trajectory
        xo, vo, Uo, Ko = odyn.velocity_verlet(s.x.astype(np.float64), vs[k].astype(np.float64), np.ones(s.n),
                                              dt, n_steps, _oracle_fe(s))
        # the potential energy of a relaxing jittered lattice crosses zero: its FP32 error is
        # bounded against the energy scale |U| + K of the trajectory, as the dH of HMC is
        scale = np.abs(Uo).max() + Ko.max()
        assert np.abs(Eb[:, k, 0] - Uo).max() <= 2e-6 * scale, (k, Eb[:, k, 0], Uo)
        np.testing.assert_allclose(Eb[:, k, 5], Ko, rtol=1e-5)
        d = odyn.min_image(xb[sl, :3].astype(np.float64) - xo, s.box)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4


def test_batched_hmc_matches_oracle_and_single_systems():
    systems = [copy.copy(s) for s in _mix_lj()]
    for s in systems:
        s.r_switch = 2.2  # a smooth potential: dH is compared per system
    R, L = len(systems), 10
    n = sum(s.n for s in systems)
    rng = np.random.default_rng(5)
    xi = [rng.standard_normal((s.n, 3)).astype(np.float32) for s in systems]
    u = rng.uniform(size=R)
    dts = np.array([0.002, 0.0025, 0.003, 0.0022, 0.0028][:R], np.float32)

    def run(sys_list, xis, us, dt):
        N = sum(s.n for s in sys_list)
        x0 = torch.cat([dev_xq(s) for s in sys_list])
        x1 = torch.empty_like(x0)
        st = torch.empty((len(sys_list), 4), dtype=torch.float64, device="cuda")
        with nbcore.Handle(sys_list) as h:
            h.hmc_trajectory(x0, x1, torch.ones(N, dtype=torch.float32, device="cuda"), torch.from_numpy(dt).cuda(),
                             L, KT, torch.from_numpy(np.concatenate(xis)).cuda(), torch.from_numpy(us).cuda(), st,
                             terms=nbcore.NB_TERM_LJ)
            h.check()
            rebuilds = h.rebuild_count()
        return x1.cpu().numpy(), st.cpu().numpy(), rebuilds
    xb, sb, rb = run(systems, xi, u, dts)
    off = 0
    for k, s in enumerate(systems):
        sl = slice(off, off + s.n)
        off += s.n
        x1, s1, r1 = run([s], [xi[k]], u[k:k + 1], dts[k:k + 1])
        if rb == 1 and r1 == 1:
            assert np.array_equal(x1, xb[sl]) and np.array_equal(s1[0], sb[k])
        o = odyn.hmc_proposal(s.x.astype(np.float64), xi[k].astype(np.float64), np.ones(s.n), float(dts[k]), L,
                              KT, _oracle_fe(s), s.box)
        scale = abs(o["U0"]) + o["K0"]
        assert abs(sb[k, 0] - o["dH"]) <= 2e-6 * scale, (k, sb[k, 0], o["dH"])
        assert sb[k, 2] == pytest.approx(o["jump"], rel=1e-4)
        assert sb[k, 3] == (1.0 if u[k] < sb[k, 1] else 0.0)
