"""The torch.autograd.Function over the HMC proposal (Sec. 4): gradients of the ESJD
loss with respect to log mu and the mass logits, taken through torch autograd (the
folded-normal step and the fixed-total-mass parameterisation on the torch side, the
hand-written adjoint in the library), against FP64 central differences of the oracle
loss with all random numbers frozen; and a short Adam run of the training loop."""
import math

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from paper_2503_20541_b300 import nbcore, workloads as wl
from paper_2503_20541_b300 import hmc

from _helpers import dev_xq, oracle_params

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

R, N_LEAP, K_CKPT, KT = 3, 16, 4, 1.0


def _systems(n=216):
    out = []
    for r in range(R):
        s = wl.lj_random(n, seed=60 + r, n_types=2)
        s.r_switch = 2.2
        out.append(s)
    return out


def _oracle_loss(systems, xi, log_mu, eps, logits):
    total = 0.0
    for r, s in enumerate(systems):
        p = oracle_params(s)

        def fe(x, s=s, p=p):
            e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
            return f, float(e[0])
        m = odyn.masses_from_logits(logits, s.types, float(s.n))
        dt = odyn.step_from_folded_normal(math.exp(log_mu), eps[r])
        o = odyn.hmc_proposal(s.x.astype(np.float64), xi[r].astype(np.float64), 1.0 / m, dt, N_LEAP, KT, fe, s.box)
        total += o["alpha"] * o["jump"]
    return total / (R * N_LEAP)


def test_autograd_gradients_match_oracle_finite_differences():
    systems = _systems()
    n = systems[0].n
    rng = np.random.default_rng(5)
    xi = rng.standard_normal((R, n, 3)).astype(np.float32)
    eps = rng.standard_normal(R)
    u = np.full(R, 0.5)
    log_mu0, logits0 = math.log(0.005), np.array([0.1, -0.2])
    types = torch.from_numpy(systems[0].types.astype(np.int64)).cuda()
    with nbcore.Handle(systems) as h:
        log_mu = torch.tensor(log_mu0, dtype=torch.float64, device="cuda", requires_grad=True)
        logits = torch.tensor(logits0, dtype=torch.float64, device="cuda", requires_grad=True)
        dt = hmc.folded_normal_step(log_mu, torch.from_numpy(eps).cuda())
        w = (1.0 / hmc.masses_from_logits(logits, types, float(n))).repeat(R)
        dt.retain_grad()
        w.retain_grad()
        x0 = torch.cat([dev_xq(s) for s in systems])
        alpha, jump, _, _ = hmc.HMCProposal.apply(w, dt, h, x0, torch.from_numpy(xi.reshape(-1, 3)).cuda(),
                                                  torch.from_numpy(u).cuda(), N_LEAP, KT, K_CKPT, nbcore.NB_TERM_LJ)
        loss = (alpha * jump).mean() / N_LEAP
        loss.backward()
        g_mu, g_lg = log_mu.grad, logits.grad
        h.check()
        # magnitudes of the summed terms (the FP32 adjoint's error is bounded against them)
        d = torch.tensor([1.0, -1.0], dtype=torch.float64, device="cuda")
        with torch.no_grad():
            hh = 1e-6
            wv = ((1.0 / hmc.masses_from_logits(logits + hh * d, types, float(n))).repeat(R) -
                  (1.0 / hmc.masses_from_logits(logits - hh * d, types, float(n))).repeat(R)) / (2 * hh)
            mag_lg = float(torch.sum(torch.abs(w.grad.double() * wv)))
            mag_mu = float(torch.sum(torch.abs(dt.grad.double() * dt.double())))
    o0 = _oracle_loss(systems, xi, log_mu0, eps, logits0)
    assert float(loss.detach()) == pytest.approx(o0, rel=2e-3)
    hs = 1e-4
    fd_mu = (_oracle_loss(systems, xi, log_mu0 + hs, eps, logits0) -
             _oracle_loss(systems, xi, log_mu0 - hs, eps, logits0)) / (2 * hs)
    assert abs(float(g_mu) - fd_mu) <= 5e-3 * abs(fd_mu) + 1e-4 * mag_mu, (float(g_mu), fd_mu, mag_mu)
    # (1, -1) is the only non-degenerate logit direction: a common shift leaves the masses
    dn = np.array([1.0, -1.0])
    fd_lg = (_oracle_loss(systems, xi, log_mu0, eps, logits0 + hs * dn) -
             _oracle_loss(systems, xi, log_mu0, eps, logits0 - hs * dn)) / (2 * hs)
    got = float(torch.dot(g_lg, d))
    assert abs(got - fd_lg) <= 2e-2 * abs(fd_lg) + 1e-4 * mag_lg, (got, fd_lg, mag_lg)
    assert abs(float(g_lg.sum())) <= 1e-9 * float(g_lg.abs().sum()) + 1e-15  # shift invariance


def test_training_loop_runs_and_moves_parameters():
    systems = _systems()
    types = torch.from_numpy(systems[0].types.astype(np.int64)).cuda()
    x0 = torch.cat([dev_xq(s) for s in systems])
    with nbcore.Handle(systems) as h:
        hist = hmc.train_esjd(h, x0, types, float(systems[0].n), iters=6, n_leap=N_LEAP, ckpt_every=K_CKPT, lr=0.05,
                              seed=3)
        h.check()
    assert len(hist) == 6
    assert all(np.isfinite(r["loss"]) and r["loss"] >= 0 for r in hist)
    assert hist[-1]["mu"] != hist[0]["mu"]
    assert abs(sum(m * c for m, c in zip(hist[-1]["mass_per_type"], np.bincount(systems[0].types))) -
               systems[0].n) < 1e-9 * systems[0].n


def _grads(h, systems, types, xi, eps, u, k):
    n = systems[0].n
    log_mu = torch.tensor(math.log(0.005), dtype=torch.float64, device="cuda", requires_grad=True)
    logits = torch.tensor([0.1, -0.2], dtype=torch.float64, device="cuda", requires_grad=True)
    dt = hmc.folded_normal_step(log_mu, eps)
    w = (1.0 / hmc.masses_from_logits(logits, types, float(n))).repeat(R)
    x0 = torch.cat([dev_xq(s) for s in systems])
    alpha, jump, x_out, _ = hmc.HMCProposal.apply(w, dt, h, x0, xi, u, N_LEAP, KT, k, nbcore.NB_TERM_LJ)
    loss = (alpha * jump).mean() / N_LEAP
    loss.backward()
    return torch.cat([log_mu.grad.reshape(1), logits.grad, loss.detach().reshape(1)]), x_out


def test_graph_replays_equal_direct_calls_across_checkpoint_intervals():
    """The autograd function replays its forward and adjoint as CUDA graphs: gradients,
    loss and proposals equal those of the direct library calls bitwise, also after a call
    with a larger checkpoint interval has replaced the library's segment buffer (the
    graphs captured over the old buffer are dropped, and captured again)."""
    systems = _systems()
    n = systems[0].n
    rng = np.random.default_rng(9)
    xi = torch.from_numpy(rng.standard_normal((R * n, 3)).astype(np.float32)).cuda()
    eps = torch.from_numpy(rng.standard_normal(R)).cuda()
    u = torch.full((R,), 0.5, dtype=torch.float64, device="cuda")
    types = torch.from_numpy(systems[0].types.astype(np.int64)).cuda()
    saved = hmc.USE_GRAPHS
    try:
        hmc.USE_GRAPHS = False
        with nbcore.Handle(systems) as h:
            ref = {k: _grads(h, systems, types, xi, eps, u, k) for k in (4, 8)}
            h.check()
        hmc.USE_GRAPHS = True
        with nbcore.Handle(systems) as h:
            # 4 captures over the first segment buffer; 8 replaces it (dropping those graphs)
            for k in (4, 4, 8, 4, 8):
                g, x_out = _grads(h, systems, types, xi, eps, u, k)
                assert torch.equal(g, ref[k][0]), k
                assert torch.equal(x_out, ref[k][1]), k
            h.check()
    finally:
        hmc.USE_GRAPHS = saved
