"""The reciprocal-space force VJP (PME backward) through the C ABI: the full VJP (real
space + PME) of a water box against the FP64 oracle (oracle.force_vjp + the PME VJP), and
the HMC backward of a small water system with PME against FP64 central differences of
the oracle loss (real-space + smooth-PME energies, all random numbers frozen)."""
import math

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import pme as opme
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_params, rel_rms

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_force_vjp_with_pme_matches_oracle():
    s = wl.water_box(n_side=8, L=24.84, seed=14, pme_grid=24)
    rng = np.random.default_rng(9)
    lam = rng.standard_normal((s.n, 3)).astype(np.float32)
    gxr, gqr, _, _ = oracle.force_vjp(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), lam,
                                      excl=s.excl)
    gxk, gqk = opme.pme_force_vjp(s.x.astype(np.float64), s.q.astype(np.float64), s.box, s.alpha, s.ke,
                                  s.pme_grid, lam.astype(np.float64))
    with nbcore.Handle([s]) as h:
        gx = torch.empty((s.n, 3), dtype=torch.float32, device="cuda")
        gq = torch.empty(s.n, dtype=torch.float32, device="cuda")
        h.nonbonded_force_vjp(dev_xq(s), torch.from_numpy(lam).cuda(), gx, gq, terms=nbcore.NB_TERM_ALL)
        h.check()
    assert rel_rms(gx.cpu().numpy(), gxr + gxk) <= 1e-5
    assert rel_rms(gq.cpu().numpy(), gqr + gqk) <= 1e-5
    # the reciprocal part alone is checked too (it is small next to real space)
    with nbcore.Handle([s]) as h:
        gx2 = torch.empty_like(gx)
        gq2 = torch.empty_like(gq)
        h.nonbonded_force_vjp(dev_xq(s), torch.from_numpy(lam).cuda(), gx2, gq2, terms=nbcore.NB_TERM_PME)
        h.check()
    assert rel_rms(gx2.cpu().numpy(), gxk) <= 1e-4
    assert rel_rms(gq2.cpu().numpy(), gqk) <= 1e-4


R, N_LEAP, K_CKPT, KT = 3, 8, 4, 2.494


def _water(r):
    return wl.water_box(n_side=4, L=12.42, seed=70 + r, r_cut=5.0, r_skin=0.5, alpha=0.6, pme_grid=16)


def _oracle_loss(s, xi, w, dt):
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p, excl=s.excl)
        ep, fp = opme.pme(x, s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)
        return f + fp, float(e.sum() + ep)
    o = odyn.hmc_proposal(s.x.astype(np.float64), xi.astype(np.float64), w, float(dt), N_LEAP, KT, fe, s.box)
    return o["alpha"] * o["jump"] / (R * N_LEAP), o


def test_hmc_backward_with_pme_matches_finite_differences():
    systems = [_water(r) for r in range(R)]
    n = systems[0].n
    mass = np.where(systems[0].q < 0, 15.999, 1.008)
    w = np.tile(1.0 / mass, R).astype(np.float32)
    dts = np.array([0.01, 0.014, 0.012], np.float32)
    xi, u = wl.hmc_randoms(R, n, seed=5)
    with nbcore.Handle(systems) as h:
        x0 = torch.cat([dev_xq(s) for s in systems])
        x_out = torch.empty_like(x0)
        stats = torch.empty((R, 4), dtype=torch.float64, device="cuda")
        ck = torch.empty(nbcore.ckpt_size(R * n, N_LEAP, K_CKPT), dtype=torch.float32, device="cuda")
        wt, dtt = torch.from_numpy(w).cuda(), torch.from_numpy(dts).cuda()
        xit, ut = torch.from_numpy(xi.reshape(-1, 3)).cuda(), torch.from_numpy(u).cuda()
        h.hmc_trajectory(x0, x_out, wt, dtt, N_LEAP, KT, xit, ut, stats, ck, K_CKPT, terms=nbcore.NB_TERM_ALL)
        st = stats.cpu().numpy()
        g_alpha = torch.from_numpy(st[:, 2] / (R * N_LEAP)).cuda()
        g_jump = torch.from_numpy(st[:, 1] / (R * N_LEAP)).cuda()
        g_dt = torch.zeros(R, dtype=torch.float64, device="cuda")
        g_w = torch.zeros(R * n, dtype=torch.float32, device="cuda")
        h.hmc_trajectory_backward(x0, wt, dtt, N_LEAP, KT, xit, ck, K_CKPT, stats, g_alpha, g_jump, g_dt, g_w,
                                  terms=nbcore.NB_TERM_ALL)
        h.check()
    gdt = g_dt.cpu().numpy()
    gw = g_w.cpu().numpy().astype(np.float64)
    w64, d64 = w.astype(np.float64), dts.astype(np.float64)
    checked = 0
    for r in range(R):
        s = systems[r]
        wr = w64[r * n:(r + 1) * n]
        _, o = _oracle_loss(s, xi[r], wr, d64[r])
        # U is a small residual of large exclusion and self terms here: dH's FP32 error is
        # bounded against the summed component magnitudes
        e0, _ = oracle.nonbonded(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, oracle_params(s), excl=s.excl)
        ep0, _ = opme.pme(s.x.astype(np.float64), s.q.astype(np.float64), s.box, s.alpha, s.ke, s.pme_grid)
        scale = float(np.abs(e0).sum() + abs(ep0)) + o["K0"]
        assert abs(st[r, 0] - o["dH"]) <= 2e-6 * scale, (r, st[r, 0], o["dH"], scale)
        if abs(o["dH"]) < 10.0 * abs(st[r, 0] - o["dH"]) or (o["dH"] > 0) != (st[r, 0] > 0):
            continue  # within the measured dH error of the alpha = 1 kink
        checked += 1
        hs = 1e-5 * d64[r]
        fd = (_oracle_loss(s, xi[r], wr, d64[r] + hs)[0] - _oracle_loss(s, xi[r], wr, d64[r] - hs)[0]) / (2 * hs)
        assert gdt[r] == pytest.approx(fd, rel=2e-3, abs=1e-9), (r, gdt[r], fd)
        dirv = np.where(s.q < 0, 1.0, -0.5) * wr
        eps = 1e-5
        fdw = (_oracle_loss(s, xi[r], wr + eps * dirv, d64[r])[0] -
               _oracle_loss(s, xi[r], wr - eps * dirv, d64[r])[0]) / (2 * eps)
        g = gw[r * n:(r + 1) * n]
        tol = 2e-3 * abs(fdw) + 1e-4 * float(np.abs(g * dirv).sum())
        assert abs(float(np.dot(g, dirv)) - fdw) <= tol, (r, float(np.dot(g, dirv)), fdw, tol)
    assert checked >= 1
