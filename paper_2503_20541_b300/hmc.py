"""Differentiable HMC (Sec. 4) through libnbcore.

``HMCProposal`` is a torch.autograd.Function over one batched HMC proposal per replica:
the forward is ``hmc_trajectory`` (Maxwell-Boltzmann draw, L velocity-Verlet steps,
FP64 dH, Metropolis test; checkpoints every k steps) and the backward is
``hmc_trajectory_backward`` (the hand-written adjoint: reverse leapfrog with the force
VJP, recomputing each segment from its checkpoint).  It is differentiable in the
per-atom inverse masses and the per-replica step sizes, which is what the paper's
tuning of step size and mass scale needs.

The parameterisations of Sec. 4 sit on the torch side: the step size is a folded normal
dt = |mu + 0.01 mu eps| (reparameterised, eps frozen per iteration), and the per-type
masses keep the total mass fixed, m_t = M s_t / sum_t n_t s_t with s_t = exp(logit_t).
``train_esjd`` maximises the expected squared jump distance per force evaluation,
(1/R) sum_r alpha_r |x'_r - x_r|^2 / L, with Adam over (log mu, mass logits).
"""
import math

import torch

from . import nbcore


class HMCProposal(torch.autograd.Function):
    """(alpha, jump, x_out, accepted) = HMCProposal.apply(w, dt, h, x0, xi, u, n_leap, kT, ckpt_every, terms)

    w: per-atom inverse masses (N,), dt: per-replica step sizes (R,) -- both float32 on
    the device; h: an ``nbcore.Handle`` over the R replicas; x0: positions and charges
    (N, 4); xi: standard normals (N, 3); u: Metropolis uniforms (R,) float64.
    Gradients flow to w and dt through alpha and jump (float64, per replica).
    """

    @staticmethod
    def forward(ctx, w, dt, h, x0, xi, u, n_leap, kT, ckpt_every, terms):
        R, N = h.n_sys, h.n_atoms
        wd = w.detach().to(torch.float32).contiguous()
        dtd = dt.detach().to(torch.float32).contiguous()
        x_out = torch.empty_like(x0)
        stats = torch.empty((R, 4), dtype=torch.float64, device=x0.device)
        ck = torch.empty(nbcore.ckpt_size(N, n_leap, ckpt_every), dtype=torch.float32, device=x0.device)
        h.hmc_trajectory(x0, x_out, wd, dtd, n_leap, kT, xi, u, stats, ck, ckpt_every, terms=terms)
        ctx.h = h
        ctx.cfg = (n_leap, kT, ckpt_every, terms, w.dtype, dt.dtype)
        ctx.save_for_backward(wd, dtd, x0, xi, ck, stats)
        accepted = stats[:, 3].clone()
        ctx.mark_non_differentiable(x_out, accepted)
        return stats[:, 1].clone(), stats[:, 2].clone(), x_out, accepted

    @staticmethod
    def backward(ctx, g_alpha, g_jump, g_x, g_acc):
        wd, dtd, x0, xi, ck, stats = ctx.saved_tensors
        n_leap, kT, ckpt_every, terms, w_dtype, dt_dtype = ctx.cfg
        h = ctx.h
        R, N = h.n_sys, h.n_atoms
        z = torch.zeros(R, dtype=torch.float64, device=x0.device)
        ga = z if g_alpha is None else g_alpha.to(torch.float64).contiguous()
        gj = z if g_jump is None else g_jump.to(torch.float64).contiguous()
        g_dt = torch.zeros(R, dtype=torch.float64, device=x0.device)
        g_w = torch.zeros(N, dtype=torch.float32, device=x0.device)
        h.hmc_trajectory_backward(x0, wd, dtd, n_leap, kT, xi, ck, ckpt_every, stats, ga, gj, g_dt, g_w, terms=terms)
        return (g_w.to(w_dtype), g_dt.to(dt_dtype), None, None, None, None, None, None, None, None)


def folded_normal_step(log_mu, eps, rel_sigma=0.01):
    """dt = |mu + rel_sigma mu eps| per replica, mu = exp(log_mu) (reparameterised)."""
    mu = torch.exp(log_mu)
    return torch.abs(mu + rel_sigma * mu * eps)


def masses_from_logits(logits, types, m_total):
    """Per-atom masses m = m_t[type], m_t = m_total s_t / sum_t n_t s_t, s_t = exp(logit_t)."""
    s = torch.exp(logits)
    counts = torch.bincount(types, minlength=s.numel()).to(s.dtype)
    mt = m_total * s / torch.sum(counts * s)
    return mt[types]


def train_esjd(h, x0, types, m_total, iters=200, n_leap=32, kT=1.0, ckpt_every=8, lr=0.05, log_mu0=math.log(0.005),
               logits0=None, seed=0, terms=nbcore.NB_TERM_LJ, callback=None):
    """Adam on (log mu, mass logits) maximising the ESJD per force evaluation.

    h: handle over R replicas of one system (N atoms each, ``types`` (N,) int64 on the
    device, ``m_total`` its total mass); x0: (R N, 4) start positions.  Each iteration
    draws eps (R,), xi (R N, 3), u (R,) from a seeded generator, runs one proposal per
    replica, steps the optimiser and continues every chain from its accepted/rejected
    state.  Returns the per-iteration history (loss, mu, masses per type, mean alpha).
    """
    dev = x0.device
    R = h.n_sys
    n = types.numel()
    n_types = int(types.max().item()) + 1
    log_mu = torch.tensor(log_mu0, dtype=torch.float64, device=dev, requires_grad=True)
    logits = torch.zeros(n_types, dtype=torch.float64, device=dev) if logits0 is None else \
        torch.as_tensor(logits0, dtype=torch.float64, device=dev).clone()
    logits.requires_grad_(True)
    opt = torch.optim.Adam([log_mu, logits], lr=lr)
    gen = torch.Generator(device=dev).manual_seed(seed)
    x = x0.clone()
    hist = []
    for it in range(iters):
        eps = torch.randn(R, dtype=torch.float64, device=dev, generator=gen)
        xi = torch.randn((R * n, 3), dtype=torch.float32, device=dev, generator=gen)
        u = torch.rand(R, dtype=torch.float64, device=dev, generator=gen)
        dt = folded_normal_step(log_mu, eps)
        w = (1.0 / masses_from_logits(logits, types, m_total)).repeat(R)
        alpha, jump, x_new, acc = HMCProposal.apply(w, dt, h, x, xi, u, n_leap, kT, ckpt_every, terms)
        loss = -(alpha * jump).mean() / n_leap
        opt.zero_grad()
        loss.backward()
        opt.step()
        x = x_new
        rec = {"it": it, "loss": -float(loss.detach()), "mu": float(torch.exp(log_mu.detach())),
               "alpha": float(alpha.detach().mean()), "accepted": float(acc.mean())}
        with torch.no_grad():
            s = torch.exp(logits)
            counts = torch.bincount(types, minlength=n_types).to(s.dtype)
            rec["mass_per_type"] = (m_total * s / torch.sum(counts * s)).tolist()
        hist.append(rec)
        if callback is not None:
            callback(rec)
    return hist
