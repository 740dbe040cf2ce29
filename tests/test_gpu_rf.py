"""GPU parity of the reaction-field electrostatics (Eq. RFA) through the C ABI.

Forces and energies of water boxes with the reaction field against the FP64 all-pairs
oracle (the small box element by element, the 24,000-atom box on sampled rows with all
rows for the energies), the force VJP under the reaction field, and the descriptor
checks (invalid dielectric, RF with Ewald splitting or a PME mesh, charged systems of
both kinds in one handle).
"""
import numpy as np
import pytest

import oracle
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import EPS32, dev_xq, oracle_params, oracle_real_space, rel_rms, rf_rounding_scale

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F_TOL = 1e-5
E_TOL = 1e-6
TERMS = nbcore.NB_TERM_LJ | nbcore.NB_TERM_COUL


def _forces(h, s, terms=TERMS, precise=False):
    f = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
    e = torch.empty((1, 6), dtype=torch.float64, device="cuda")
    h.nonbonded_forces(dev_xq(s), f, e, terms=terms, precise=precise)
    h.check()
    return f.cpu().numpy().astype(np.float64), e.cpu().numpy()[0]


def _rf_tol(s, e_ref, rows=None):
    """E_RF of water is a ~10^4-fold cancelling sum of FP32 pair energies: its error is
    bounded by 1e-6 relative plus six times the random-walk sum of the pairs' rounding
    (EPS32 times the root sum of squares of their parts' magnitudes)."""
    return E_TOL * abs(e_ref) + 6.0 * EPS32 * rf_rounding_scale(s, rows=rows)


@pytest.mark.parametrize("tile", [0, 256])
def test_reaction_field_water_matches_oracle(tile):
    s = wl.water_rf_density(600, seed=3)  # 1800 atoms, r_c 10 A, the paper's scaling setting
    with nbcore.Handle([s], stencil_tile=tile) as h:
        f, e = _forces(h, s)
        _, ep = _forces(h, s, precise=True)
    eo, fo = oracle_real_space(s)
    assert rel_rms(f, fo) <= F_TOL
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0])
    assert abs(e[1] - eo[1]) <= _rf_tol(s, eo[1]), (e[1], eo[1], _rf_tol(s, eo[1]))
    # precise (two-float) energies: the flat bar
    for c in (0, 1):
        assert abs(ep[c] - eo[c]) <= E_TOL * abs(eo[c]), (c, ep[c], eo[c])
    assert e[2] == 0.0 and e[3] == 0.0 and e[4] == 0.0  # no exclusion correction, self or mesh
    assert eo[2] == 0.0 and eo[3] == 0.0


def test_reaction_field_water_24k_sampled():
    """The benchmark's 8000-molecule box with the reaction field in place of Ewald + PME."""
    s = wl.as_reaction_field(wl.water_box())
    with nbcore.Handle([s]) as h:
        f, e = _forces(h, s)
        _, ep = _forces(h, s, precise=True)
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(s.n, 400, replace=False))
    er, fr = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), rows,
                                   excl=s.excl)
    assert rel_rms(f[rows], fr) <= F_TOL
    er_all, _ = oracle.nonbonded_rows(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                      np.arange(s.n), excl=s.excl)
    eo = er_all.sum(axis=0)
    assert abs(e[0] - eo[0]) <= E_TOL * abs(eo[0]), (e[0], eo[0])
    tol = _rf_tol(s, eo[1], rows=np.arange(0, s.n, 11))  # every 11th row: O and H alike
    assert abs(e[1] - eo[1]) <= tol, (e[1], eo[1], tol)
    for c in (0, 1):
        assert abs(ep[c] - eo[c]) <= E_TOL * abs(eo[c]), (c, ep[c], eo[c])


def test_reaction_field_vjp_matches_oracle():
    s = wl.water_rf_density(600, seed=4)
    rng = np.random.default_rng(5)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    gxo, gqo, gso, geo = oracle.force_vjp(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s),
                                          lam, excl=s.excl)
    with nbcore.Handle([s]) as h:
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gq = torch.empty(s.n, dtype=torch.float32, device="cuda")
        gs = torch.empty(s.n, dtype=torch.float32, device="cuda")
        ge = torch.empty(s.n, dtype=torch.float32, device="cuda")
        fo = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(dev_xq(s), torch.from_numpy(lam).cuda(), gx, gq, gs, ge, f_out=fo)
        h.check()
    assert rel_rms(gx.cpu().numpy(), gxo) <= 1e-5
    assert rel_rms(gq.cpu().numpy(), gqo) <= 1e-5
    o = s.sqrt_eps > 0
    assert rel_rms(gs.cpu().numpy()[o], gso[o]) <= 1e-5
    assert rel_rms(ge.cpu().numpy(), geo) <= 1e-5
    assert rel_rms(fo.cpu().numpy(), oracle_real_space(s)[1]) <= F_TOL


def test_reaction_field_descriptor_checks():
    def refused(s_list):
        with pytest.raises(nbcore.NbError) as ei:
            nbcore.Handle(s_list)
        assert ei.value.status == 1

    s = wl.water_rf_density(600, seed=6)
    s.eps_rf = 0.5  # below 1
    refused([s])
    s = wl.water_rf_density(600, seed=6)
    s.alpha = 0.32  # RF and Ewald splitting together
    refused([s])
    s = wl.water_rf_density(600, seed=6)
    s.pme_grid = (32, 32, 32)  # RF with a mesh
    refused([s])
    refused([wl.water_rf_density(600, seed=6), wl.water_box_density(600, seed=7)])  # two kinds
    # an uncharged LJ system may share a handle with reaction-field water
    lj = wl.lj_random(500, seed=8)
    sw = wl.water_rf_density(600, seed=9)
    with nbcore.Handle([lj, sw]) as h:
        n = lj.n + sw.n
        f = torch.empty((n, 3), dtype=torch.float32, device="cuda")
        e = torch.empty((2, 6), dtype=torch.float64, device="cuda")
        h.nonbonded_forces(torch.cat([dev_xq(lj), dev_xq(sw)]), f, e, terms=TERMS)
        h.check()
    eo, fo = oracle_real_space(sw)
    assert rel_rms(f.cpu().numpy()[lj.n:].astype(np.float64), fo) <= F_TOL
    assert abs(e.cpu().numpy()[1, 1] - eo[1]) <= _rf_tol(sw, eo[1])


R_HMC, N_LEAP, K_CKPT, KT = 3, 8, 4, 2.494


def _rf_water(r):
    return wl.as_reaction_field(wl.water_box(n_side=4, L=12.42, seed=80 + r, r_cut=5.0, r_skin=0.5, alpha=0.0,
                                             pme_grid=16))


def _oracle_hmc_loss(s, xi, w, dt):
    from oracle import dynamics as odyn
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
        return f, float(e.sum())
    o = odyn.hmc_proposal(s.x.astype(np.float64), xi.astype(np.float64), w, float(dt), N_LEAP, KT, fe, s.box)
    return o["alpha"] * o["jump"] / (R_HMC * N_LEAP), o


def test_hmc_backward_with_reaction_field_matches_finite_differences():
    systems = [_rf_water(r) for r in range(R_HMC)]
    n = systems[0].n
    mass = np.where(systems[0].q < 0, 15.999, 1.008)
    w = np.tile(1.0 / mass, R_HMC).astype(np.float32)
    dts = np.array([0.01, 0.014, 0.012], np.float32)
    xi, u = wl.hmc_randoms(R_HMC, n, seed=6)
    with nbcore.Handle(systems) as h:
        x0 = torch.cat([dev_xq(s) for s in systems])
        x_out = torch.empty_like(x0)
        stats = torch.empty((R_HMC, 4), dtype=torch.float64, device="cuda")
        ck = torch.empty(nbcore.ckpt_size(R_HMC * n, N_LEAP, K_CKPT), dtype=torch.float32, device="cuda")
        wt, dtt = torch.from_numpy(w).cuda(), torch.from_numpy(dts).cuda()
        xit, ut = torch.from_numpy(xi.reshape(-1, 3)).cuda(), torch.from_numpy(u).cuda()
        h.hmc_trajectory(x0, x_out, wt, dtt, N_LEAP, KT, xit, ut, stats, ck, K_CKPT, terms=TERMS)
        st = stats.cpu().numpy()
        g_alpha = torch.from_numpy(st[:, 2] / (R_HMC * N_LEAP)).cuda()
        g_jump = torch.from_numpy(st[:, 1] / (R_HMC * N_LEAP)).cuda()
        g_dt = torch.zeros(R_HMC, dtype=torch.float64, device="cuda")
        g_w = torch.zeros(R_HMC * n, dtype=torch.float32, device="cuda")
        h.hmc_trajectory_backward(x0, wt, dtt, N_LEAP, KT, xit, ck, K_CKPT, stats, g_alpha, g_jump, g_dt, g_w,
                                  terms=TERMS)
        h.check()
    gdt = g_dt.cpu().numpy()
    gw = g_w.cpu().numpy().astype(np.float64)
    w64, d64 = w.astype(np.float64), dts.astype(np.float64)
    checked = 0
    for r in range(R_HMC):
        s = systems[r]
        wr = w64[r * n:(r + 1) * n]
        _, o = _oracle_hmc_loss(s, xi[r], wr, d64[r])
        # dH = H1 - H0: two reaction-field energies, each within its rounding bound
        tol_dh = 2.0 * _rf_tol(s, o["U0"]) + 1e-6 * (abs(o["U0"]) + o["K0"])
        assert abs(st[r, 0] - o["dH"]) <= tol_dh, (r, st[r, 0], o["dH"], tol_dh)
        if abs(o["dH"]) < 10.0 * abs(st[r, 0] - o["dH"]) or (o["dH"] > 0) != (st[r, 0] > 0):
            continue  # within the measured dH error of the alpha = 1 kink
        checked += 1
        hs = 1e-5 * d64[r]
        fd = (_oracle_hmc_loss(s, xi[r], wr, d64[r] + hs)[0] - _oracle_hmc_loss(s, xi[r], wr, d64[r] - hs)[0]) / (
            2 * hs)
        assert gdt[r] == pytest.approx(fd, rel=2e-3, abs=1e-9), (r, gdt[r], fd)
        dirv = np.where(s.q < 0, 1.0, -0.5) * wr
        eps = 1e-5
        fdw = (_oracle_hmc_loss(s, xi[r], wr + eps * dirv, d64[r])[0] -
               _oracle_hmc_loss(s, xi[r], wr - eps * dirv, d64[r])[0]) / (2 * eps)
        g = gw[r * n:(r + 1) * n]
        tol = 2e-3 * abs(fdw) + 1e-4 * float(np.abs(g * dirv).sum())
        assert abs(float(np.dot(g, dirv)) - fdw) <= tol, (r, float(np.dot(g, dirv)), fdw, tol)
    assert checked >= 1
