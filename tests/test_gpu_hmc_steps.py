"""GPU parity of the folded-normal-length HMC (Sec. 4, Eq. loss_steps) and of A(k).

Forward: dH, acceptance probability and squared jump of every intermediate state of
every replica against the FP64 oracle trajectory; the proposal after the drawn length;
with every length at L_q, the fixed-length proposal's chain state (to FP32 rounding).  Backward:
the gradient of the step-weighted loss with respect to dt and the inverse masses against
FP64 central differences of the oracle loss.  A(k) and tau_exp against the oracle.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import tuning as tun
from paper_2503_20541_b300 import nbcore, workloads as wl

from _helpers import dev_xq, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R = 3
MU_L = 10.0
L_Q = tun.length_cutoff(MU_L)  # 14
K_CKPT = 4
KT = 1.0


def _setup(n=216):
    systems = []
    for r in range(R):
        s = wl.lj_random(n, seed=60 + r, n_types=2)
        s.r_switch = 2.2
        systems.append(s)
    masses = odyn.masses_from_logits([0.25, -0.1], systems[0].types, float(n))
    w = np.tile(1.0 / masses, R).astype(np.float32)
    dts = np.array([0.004, 0.0055, 0.0045], np.float32)
    xi, u = wl.hmc_randoms(R, n, seed=77)
    return systems, w, dts, xi, u


def _oracle_steps(s, xi, w, dt, n_steps=L_Q):
    p = oracle_params(s)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])
    return tun.hmc_proposal_steps(s.x.astype(np.float64), xi.astype(np.float64), w.astype(np.float64), float(dt),
                                  n_steps, KT, fe, s.box)


def _energy_scale(s, xi, w):
    p = oracle_params(s)
    e, _ = oracle.nonbonded(s.x.astype(np.float64), s.q, s.sigma, s.sqrt_eps, p)
    return abs(float(e[0])) + 0.5 * KT * float(np.sum(xi.astype(np.float64) ** 2))


def _gpu_steps(h, systems, w, dts, xi, u, l_prop):
    n_tot = sum(s.n for s in systems)
    x0 = torch.cat([dev_xq(s) for s in systems])
    x_out = torch.empty_like(x0)
    stats = torch.empty((R, 4), dtype=torch.float64, device="cuda")
    sst = torch.empty((L_Q, R, 3), dtype=torch.float64, device="cuda")
    ck = torch.empty(nbcore.ckpt_size(n_tot, L_Q, K_CKPT), dtype=torch.float32, device="cuda")
    a = dict(inv_mass=torch.from_numpy(w).cuda(), dt=torch.from_numpy(dts).cuda(),
             xi=torch.from_numpy(xi.reshape(-1, 3)).cuda(), u=torch.from_numpy(u).cuda(),
             l_prop=torch.tensor(l_prop, dtype=torch.int32, device="cuda"))
    h.hmc_trajectory_steps(x0, x_out, a["inv_mass"], a["dt"], L_Q, a["l_prop"], KT, a["xi"], a["u"], stats, sst, ck,
                           K_CKPT, terms=nbcore.NB_TERM_LJ)
    return x0, x_out, stats, sst, ck, a


def test_steps_forward_matches_oracle():
    systems, w, dts, xi, u = _setup()
    n = systems[0].n
    l_prop = [L_Q, 3, 9]
    with nbcore.Handle(systems) as h:
        _, x_out, stats, sst, _, _ = _gpu_steps(h, systems, w, dts, xi, u, l_prop)
        h.check()
    st = stats.cpu().numpy()
    ss = sst.cpu().numpy()
    xo = x_out.cpu().numpy()
    for r, s in enumerate(systems):
        wr = w[r * n:(r + 1) * n]
        o = _oracle_steps(s, xi[r], wr, dts[r])
        scale = _energy_scale(s, xi[r], wr)
        for l in range(L_Q):
            # FP32 energies: |error| ~ 1e-7 of the energy scale
            assert abs(ss[l, r, 0] - o["dH"][l]) <= 2e-6 * scale, (r, l, ss[l, r, 0], o["dH"][l])
            assert ss[l, r, 1] == pytest.approx(min(1.0, math.exp(-ss[l, r, 0] / KT)), rel=1e-12)
            assert ss[l, r, 1] == pytest.approx(o["alpha"][l], abs=2e-6 * scale)
            assert ss[l, r, 2] == pytest.approx(o["jump"][l], rel=1e-4)
        lp = l_prop[r]
        np.testing.assert_array_equal(st[r, :3], ss[lp - 1, r])
        acc = u[r] < st[r, 1]
        assert st[r, 3] == (1.0 if acc else 0.0)
        ref = o["x"][lp - 1] if acc else s.x.astype(np.float64)
        d = xo[r * n:(r + 1) * n, :3].astype(np.float64) - ref
        d -= s.box * np.round(d / s.box)
        assert np.sqrt(np.mean(d ** 2)) < 1e-4
        np.testing.assert_array_equal(xo[r * n:(r + 1) * n, 3], s.q)


def test_steps_at_full_length_equal_the_fixed_length_proposal():
    systems, w, dts, xi, u = _setup()
    u = np.array([0.0, 0.999999, 0.5])  # one sure accept, one near-sure reject, one either way
    with nbcore.Handle(systems) as h:
        x0, x_a, st_a, sst, ck_a, a = _gpu_steps(h, systems, w, dts, xi, u, [L_Q] * R)
        x_b = torch.empty_like(x0)
        st_b = torch.empty((R, 4), dtype=torch.float64, device="cuda")
        ck_b = torch.empty_like(ck_a)
        h.hmc_trajectory(x0, x_b, a["inv_mass"], a["dt"], L_Q, KT, a["xi"], a["u"], st_b, ck_b, K_CKPT,
                         terms=nbcore.NB_TERM_LJ)
        h.check()
    # same integrator and list rebuild schedule (the checkpoints force the same
    # rebuilds).  The fixed-length proposal asks for energies only at its last step, so
    # its other force evaluations take the energy-free kernel (another erfc and 1/r^2,
    # another reduction tree): states agree to FP32 rounding, not bit for bit.
    ca, cb = ck_a.cpu().numpy().astype(np.float64), ck_b.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(ca - cb)) <= 1e-4 * max(1.0, float(np.max(np.abs(ca))))
    xa, xb = x_a.cpu().numpy().astype(np.float64), x_b.cpu().numpy().astype(np.float64)
    d = xa[:, :3] - xb[:, :3]
    d -= systems[0].box * np.round(d / systems[0].box)
    assert np.max(np.abs(d)) <= 1e-4
    np.testing.assert_array_equal(xa[:, 3], xb[:, 3])
    sa, sb = st_a.cpu().numpy(), st_b.cpu().numpy()
    n = systems[0].n
    for r, s in enumerate(systems):
        scale = _energy_scale(s, xi[r], w[r * n:(r + 1) * n])
        assert abs(sa[r, 0] - sb[r, 0]) <= 2e-6 * scale, (r, sa[r, 0], sb[r, 0])
        assert abs(sa[r, 1] - sb[r, 1]) <= 2e-6 * scale
        assert sa[r, 3] == sb[r, 3]  # u keeps off the FP32 band of alpha
    np.testing.assert_allclose(sa[:, 2], sb[:, 2], rtol=1e-4)


def _oracle_loss(s, xi, w, dt, coef):
    """sum_l coef_l alpha_l jump_l of one replica (the Eq. loss_steps terms with the
    weights w_l / (R l) folded into coef)."""
    o = _oracle_steps(s, xi, w, dt)
    return float(np.sum(coef * o["alpha"] * o["jump"]))


def test_steps_backward_matches_finite_differences():
    systems, w, dts, xi, u = _setup()
    n = systems[0].n
    wl_ = tun.step_weights(MU_L, 1.0, L_Q) / (R * np.arange(1, L_Q + 1))
    w64, d64 = w.astype(np.float64), dts.astype(np.float64)
    orc = [_oracle_steps(s, xi[r], w64[r * n:(r + 1) * n], d64[r]) for r, s in enumerate(systems)]
    with nbcore.Handle(systems) as h:
        x0, _, _, sst, ck, a = _gpu_steps(h, systems, w, dts, xi, u, [5, 7, L_Q])
        ss = sst.cpu().numpy()
        # states whose dH sits within the FP32 error band of alpha's kink at dH = 0 (or on
        # the other side of it in the oracle) carry no loss term: central differences
        # across the kink are meaningless
        scales = [_energy_scale(s, xi[r], w[r * n:(r + 1) * n]) for r, s in enumerate(systems)]
        mask = np.array([[abs(ss[l, r, 0]) > 5e-6 * scales[r] and (ss[l, r, 0] > 0) == (orc[r]["dH"][l] > 0)
                          for r in range(R)] for l in range(L_Q)])
        coef = wl_[:, None] * mask
        g_alpha = torch.from_numpy(np.ascontiguousarray(coef * ss[:, :, 2])).cuda()
        g_jump = torch.from_numpy(np.ascontiguousarray(coef * ss[:, :, 1])).cuda()
        g_dt = torch.zeros(R, dtype=torch.float64, device="cuda")
        g_w = torch.zeros(R * n, dtype=torch.float32, device="cuda")
        h.hmc_trajectory_steps_backward(x0, a["inv_mass"], a["dt"], L_Q, KT, a["xi"], ck, K_CKPT, sst, g_alpha,
                                        g_jump, g_dt, g_w, terms=nbcore.NB_TERM_LJ)
        h.check()
    assert mask.sum() >= 3 * R
    gdt = g_dt.cpu().numpy()
    gw = g_w.cpu().numpy().astype(np.float64)
    for r in range(R):
        s = systems[r]
        wr = w64[r * n:(r + 1) * n]
        c = coef[:, r]
        hstep = 1e-5 * d64[r]
        fd = (_oracle_loss(s, xi[r], wr, d64[r] + hstep, c) - _oracle_loss(s, xi[r], wr, d64[r] - hstep, c)) / (
            2 * hstep)
        assert gdt[r] == pytest.approx(fd, rel=2e-3, abs=1e-9), (r, gdt[r], fd)
        dirv = np.where(s.types == 0, 1.0, -0.7) * wr
        eps = 1e-5
        fdw = (_oracle_loss(s, xi[r], wr + eps * dirv, d64[r], c) -
               _oracle_loss(s, xi[r], wr - eps * dirv, d64[r], c)) / (2 * eps)
        g = gw[r * n:(r + 1) * n]
        # mixed-sign direction: bound the FP32 error against sum |g_i v_i|
        tol = 2e-3 * abs(fdw) + 1e-4 * float(np.abs(g * dirv).sum())
        assert abs(float(np.dot(g, dirv)) - fdw) <= tol, (r, float(np.dot(g, dirv)), fdw, tol)


def test_autograd_function_and_loss_match_the_direct_calls():
    from paper_2503_20541_b300 import hmc
    systems, w, dts, xi, u = _setup()
    n = systems[0].n
    l_prop = [5, 7, L_Q]
    mu_L = torch.tensor(MU_L, dtype=torch.float64, device="cuda", requires_grad=True)
    with nbcore.Handle(systems) as h:
        x0, _, _, sst, ck, a = _gpu_steps(h, systems, w, dts, xi, u, l_prop)
        wt = a["inv_mass"].clone().requires_grad_(True)
        dtt = a["dt"].clone().requires_grad_(True)
        alpha, jump, x_out, stats = hmc.HMCStepsProposal.apply(wt, dtt, h, x0, a["xi"], a["u"], a["l_prop"], L_Q, KT,
                                                               K_CKPT, nbcore.NB_TERM_LJ)
        loss = hmc.lhmc_loss(alpha, jump, mu_L)
        loss.backward()
        ss = sst.cpu().numpy()
        assert np.array_equal(alpha.detach().cpu().numpy(), ss[:, :, 1])
        assert float(loss.detach()) == pytest.approx(tun.lhmc_loss(ss[:, :, 1].T, ss[:, :, 2].T, MU_L), rel=1e-13)
        # the same cotangents through the direct entry point
        coef = tun.step_weights(MU_L, 1.0, L_Q) / (R * np.arange(1, L_Q + 1))
        g_dt = torch.zeros(R, dtype=torch.float64, device="cuda")
        g_w = torch.zeros(R * n, dtype=torch.float32, device="cuda")
        h.hmc_trajectory_steps_backward(x0, a["inv_mass"], a["dt"], L_Q, KT, a["xi"], ck, K_CKPT, sst,
                                        torch.from_numpy(np.ascontiguousarray(coef[:, None] * ss[:, :, 2])).cuda(),
                                        torch.from_numpy(np.ascontiguousarray(coef[:, None] * ss[:, :, 1])).cuda(),
                                        g_dt, g_w, terms=nbcore.NB_TERM_LJ)
        h.check()
    np.testing.assert_allclose(dtt.grad.cpu().numpy(), g_dt.cpu().numpy().astype(np.float32), rtol=1e-6)
    np.testing.assert_allclose(wt.grad.cpu().numpy(), g_w.cpu().numpy(), rtol=1e-5, atol=1e-6 * float(
        g_w.abs().max()))
    # d L_HMC / d mu_L = (1/R) sum alpha jump / l  d w_l / d mu_L, against central differences
    fd = (tun.lhmc_loss(ss[:, :, 1].T, ss[:, :, 2].T, MU_L + 1e-5) -
          tun.lhmc_loss(ss[:, :, 1].T, ss[:, :, 2].T, MU_L - 1e-5)) / 2e-5
    assert float(mu_L.grad) == pytest.approx(fd, rel=1e-6)


def test_out_of_range_length_is_reported_and_keeps_x0():
    systems, w, dts, xi, u = _setup()
    n = systems[0].n
    with nbcore.Handle(systems) as h:
        x0, x_out, stats, sst, _, _ = _gpu_steps(h, systems, w, dts, xi, np.zeros(R), [0, 3, L_Q + 1])
        with pytest.raises(nbcore.NbError) as ei:
            h.check()
        assert ei.value.status == 1
        st = stats.cpu().numpy()
        ss = sst.cpu().numpy()
    assert np.all(st[0] == 0.0) and np.all(st[2] == 0.0)
    np.testing.assert_array_equal(st[1, :3], ss[2, 1])
    assert torch.equal(x_out[:n], x0[:n]) and torch.equal(x_out[2 * n:], x0[2 * n:])


def test_autocorrelation_matches_oracle():
    from scipy import signal
    rng = np.random.default_rng(21)
    n, max_lag = 30000, 120
    rows = []
    for phi in (0.5, 0.8, 0.95):
        rows.append(signal.lfilter([1.0], [1.0, -phi], rng.standard_normal(n + 500))[500:])
    rows.append(3.0 * rows[1] - 600.0)  # an offset a hundred times the spread, as in an energy trace
    rows.append(np.array([(-1.0) ** t for t in range(n)]))
    series = np.ascontiguousarray(np.stack(rows))
    acf, tau = nbcore.autocorrelation(torch.from_numpy(series).cuda(), max_lag)
    acf = acf.cpu().numpy()
    tau = tau.cpu().numpy()
    for i, o in enumerate(rows):
        ref = tun.autocorrelation(o, max_lag)
        np.testing.assert_allclose(acf[i], ref, rtol=0, atol=1e-11)
        t_ref = tun.tau_exp(ref)
        if math.isnan(t_ref):
            assert math.isnan(tau[i])
        else:
            assert tau[i] == pytest.approx(t_ref, rel=1e-9)
    # A(k) is unchanged by O -> a O + b
    np.testing.assert_allclose(acf[3], acf[1], rtol=0, atol=1e-11)
    assert tau[1] == pytest.approx(-1.0 / math.log(0.8), rel=0.1)


def test_autocorrelation_rejects_bad_arguments():
    s = torch.zeros((1, 10), dtype=torch.float64, device="cuda")
    for lag, hi, lo in ((10, 0.5, 0.05), (0, 0.5, 0.05), (3, 0.05, 0.5), (3, 1.5, 0.05)):
        with pytest.raises(nbcore.NbError):
            nbcore.autocorrelation(s, lag, a_hi=hi, a_lo=lo)
