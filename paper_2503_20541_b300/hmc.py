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

The trajectory length of Sec. 4 is a folded normal N_F(mu_L, sigma_L = 1) as well:
``HMCStepsProposal`` runs L_q steps (L_q = ceil of the 0.999 quantile) and returns the
acceptance probability and squared jump of every intermediate state, the proposal being
the state after a length drawn from the discretised N_F.  ``lhmc_loss`` is Eq. loss_steps,
(1/R) sum_i sum_{l<=L_q} N_F(l; mu_L, sigma_L) alpha_{i,l} |x_{i,l} - x_i|^2 / l, which is
differentiable in mu_L through the weights; ``train_lhmc`` maximises it over (log dt mean,
log mu_L, mass logits).  Only the parameterisations (weights, quantile, length draw) are
torch or host arithmetic; the trajectories and their adjoint run in libnbcore.
"""
import math

import torch

from . import nbcore

# The forward and the adjoint of a proposal are each some hundreds of kernel launches;
# issued from Python through the autograd engine they make a training iteration
# host-bound.  With USE_GRAPHS each is captured once per handle and configuration as a
# CUDA graph over static buffers (inputs copied in, outputs and saved tensors copied out),
# and replayed: the same kernels on the same data, so the results are bitwise those of
# the direct calls.
USE_GRAPHS = True


class _TrajectoryGraphs:
    """Static buffers and CUDA graphs of one handle's HMC forward and adjoint for one
    configuration (n_leap, kT, ckpt_every, terms, and for the step-statistics variant the
    per-state outputs).  Graphs are captured on first use, after the inputs are in place
    (the capture's warm-up runs compute with them)."""

    def __init__(self, h, dev, n_leap, kT, ckpt_every, terms, steps):
        R, N = h.n_sys, h.n_atoms
        f32, f64 = torch.float32, torch.float64
        self.h, self.cfg, self.steps = h, (n_leap, kT, ckpt_every, terms), steps
        self.w = torch.zeros(N, dtype=f32, device=dev)
        self.dt = torch.zeros(R, dtype=f32, device=dev)
        self.x0 = torch.zeros((N, 4), dtype=f32, device=dev)
        self.xi = torch.zeros((N, 3), dtype=f32, device=dev)
        self.u = torch.zeros(R, dtype=f64, device=dev)
        self.l_prop = torch.ones(R, dtype=torch.int32, device=dev)
        self.x_out = torch.zeros((N, 4), dtype=f32, device=dev)
        self.stats = torch.zeros((R, 4), dtype=f64, device=dev)
        self.sst = torch.zeros((n_leap, R, 3), dtype=f64, device=dev) if steps else None
        self.ck = torch.zeros(nbcore.ckpt_size(N, n_leap, ckpt_every), dtype=f32, device=dev)
        gshape = (n_leap, R) if steps else (R,)
        self.ga = torch.zeros(gshape, dtype=f64, device=dev)
        self.gj = torch.zeros(gshape, dtype=f64, device=dev)
        self.g_dt = torch.zeros(R, dtype=f64, device=dev)
        self.g_w = torch.zeros(N, dtype=f32, device=dev)
        self.fwd = None
        self.bwd = None

    def run_fwd(self):
        n_leap, kT, k, terms = self.cfg
        if self.steps:
            self.h.hmc_trajectory_steps(self.x0, self.x_out, self.w, self.dt, n_leap, self.l_prop, kT, self.xi,
                                        self.u, self.stats, self.sst, self.ck, k, terms=terms)
        else:
            self.h.hmc_trajectory(self.x0, self.x_out, self.w, self.dt, n_leap, kT, self.xi, self.u, self.stats,
                                  self.ck, k, terms=terms)

    def run_bwd(self):
        n_leap, kT, k, terms = self.cfg
        self.g_dt.zero_()
        self.g_w.zero_()
        if self.steps:
            self.h.hmc_trajectory_steps_backward(self.x0, self.w, self.dt, n_leap, kT, self.xi, self.ck, k,
                                                 self.sst, self.ga, self.gj, self.g_dt, self.g_w, terms=terms)
        else:
            self.h.hmc_trajectory_backward(self.x0, self.w, self.dt, n_leap, kT, self.xi, self.ck, k, self.stats,
                                           self.ga, self.gj, self.g_dt, self.g_w, terms=terms)

    def forward(self):
        if self.fwd is None:
            from .graphs import CapturedStep
            self.fwd = CapturedStep(self.run_fwd)
        self.fwd.replay()

    def backward(self):
        if self.bwd is None:
            from .graphs import CapturedStep
            self.bwd = CapturedStep(self.run_bwd)
        self.bwd.replay()


def _use_graphs():
    """Graphs unless disabled, or unless the caller is capturing a graph of their own (the
    direct calls are then recorded into it)."""
    return USE_GRAPHS and not torch.cuda.is_current_stream_capturing()


def _graphs(h, dev, n_leap, kT, ckpt_every, terms, steps):
    cache = h.__dict__.setdefault("_hmc_graphs", {})
    key = (steps, int(n_leap), float(kT), int(ckpt_every), int(terms), h.n_sys, h.n_atoms)
    g = cache.get(key)
    if g is None:
        g = cache[key] = _TrajectoryGraphs(h, dev, n_leap, kT, ckpt_every, terms, steps)
    return g


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
        if _use_graphs():
            g = _graphs(h, x0.device, n_leap, kT, ckpt_every, terms, False)
            for dst, src in ((g.w, wd), (g.dt, dtd), (g.x0, x0), (g.xi, xi), (g.u, u)):
                dst.copy_(src)
            g.forward()
            x_out, stats, ck = g.x_out.clone(), g.stats.clone(), g.ck.clone()
        else:
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
        if _use_graphs():
            g = _graphs(h, x0.device, n_leap, kT, ckpt_every, terms, False)
            for dst, src in ((g.w, wd), (g.dt, dtd), (g.x0, x0), (g.xi, xi), (g.ck, ck), (g.stats, stats),
                             (g.ga, ga), (g.gj, gj)):
                dst.copy_(src)
            g.backward()
            g_w, g_dt = g.g_w.clone(), g.g_dt.clone()
        else:
            g_dt = torch.zeros(R, dtype=torch.float64, device=x0.device)
            g_w = torch.zeros(N, dtype=torch.float32, device=x0.device)
            h.hmc_trajectory_backward(x0, wd, dtd, n_leap, kT, xi, ck, ckpt_every, stats, ga, gj, g_dt, g_w,
                                      terms=terms)
        return (g_w.to(w_dtype), g_dt.to(dt_dtype), None, None, None, None, None, None, None, None)


class HMCStepsProposal(torch.autograd.Function):
    """(alpha, jump, x_out, stats) = HMCStepsProposal.apply(w, dt, h, x0, xi, u, l_prop, n_leap, kT, ckpt_every, terms)

    As ``HMCProposal``, with n_leap = L_q steps per replica and the proposal taken after
    l_prop[r] steps (int32, (R,), in [1, n_leap]).  alpha and jump are (n_leap, R) float64:
    the acceptance probability and squared jump of every state l = 1..n_leap.  stats is
    (R, 4) float64 (dH, alpha, jump, accepted) of the proposal.  Gradients flow to w and dt
    through alpha and jump.
    """

    @staticmethod
    def forward(ctx, w, dt, h, x0, xi, u, l_prop, n_leap, kT, ckpt_every, terms):
        R, N = h.n_sys, h.n_atoms
        wd = w.detach().to(torch.float32).contiguous()
        dtd = dt.detach().to(torch.float32).contiguous()
        if _use_graphs():
            g = _graphs(h, x0.device, n_leap, kT, ckpt_every, terms, True)
            for dst, src in ((g.w, wd), (g.dt, dtd), (g.x0, x0), (g.xi, xi), (g.u, u), (g.l_prop, l_prop)):
                dst.copy_(src)
            g.forward()
            x_out, stats, sst, ck = g.x_out.clone(), g.stats.clone(), g.sst.clone(), g.ck.clone()
        else:
            x_out = torch.empty_like(x0)
            stats = torch.empty((R, 4), dtype=torch.float64, device=x0.device)
            sst = torch.empty((n_leap, R, 3), dtype=torch.float64, device=x0.device)
            ck = torch.empty(nbcore.ckpt_size(N, n_leap, ckpt_every), dtype=torch.float32, device=x0.device)
            h.hmc_trajectory_steps(x0, x_out, wd, dtd, n_leap, l_prop, kT, xi, u, stats, sst, ck, ckpt_every,
                                   terms=terms)
        ctx.h = h
        ctx.cfg = (n_leap, kT, ckpt_every, terms, w.dtype, dt.dtype)
        ctx.save_for_backward(wd, dtd, x0, xi, ck, sst)
        ctx.mark_non_differentiable(x_out, stats)
        return sst[:, :, 1].clone(), sst[:, :, 2].clone(), x_out, stats

    @staticmethod
    def backward(ctx, g_alpha, g_jump, g_x, g_stats):
        wd, dtd, x0, xi, ck, sst = ctx.saved_tensors
        n_leap, kT, ckpt_every, terms, w_dtype, dt_dtype = ctx.cfg
        h = ctx.h
        R, N = h.n_sys, h.n_atoms
        z = torch.zeros((n_leap, R), dtype=torch.float64, device=x0.device)
        ga = z if g_alpha is None else g_alpha.to(torch.float64).contiguous()
        gj = z if g_jump is None else g_jump.to(torch.float64).contiguous()
        if _use_graphs():
            g = _graphs(h, x0.device, n_leap, kT, ckpt_every, terms, True)
            for dst, src in ((g.w, wd), (g.dt, dtd), (g.x0, x0), (g.xi, xi), (g.ck, ck), (g.sst, sst),
                             (g.ga, ga), (g.gj, gj)):
                dst.copy_(src)
            g.backward()
            g_w, g_dt = g.g_w.clone(), g.g_dt.clone()
        else:
            g_dt = torch.zeros(R, dtype=torch.float64, device=x0.device)
            g_w = torch.zeros(N, dtype=torch.float32, device=x0.device)
            h.hmc_trajectory_steps_backward(x0, wd, dtd, n_leap, kT, xi, ck, ckpt_every, sst, ga, gj, g_dt, g_w,
                                            terms=terms)
        return (g_w.to(w_dtype), g_dt.to(dt_dtype), None, None, None, None, None, None, None, None, None)


def folded_normal_pdf(x, mu, sigma):
    """N_F(x; mu, sigma) = N(x; mu, sigma) + N(-x; mu, sigma) (Sec. 4), differentiable in mu."""
    c = 1.0 / math.sqrt(2.0 * math.pi * sigma * sigma)
    return c * (torch.exp(-(x - mu) ** 2 / (2.0 * sigma * sigma)) + torch.exp(-(x + mu) ** 2 / (2.0 * sigma * sigma)))


def folded_normal_quantile(p, mu, sigma):
    """Q(p) of N_F(mu, sigma) by bisection on its CDF 1/2 [erf((x+mu)/(s sqrt2)) + erf((x-mu)/(s sqrt2))]."""
    s = sigma * math.sqrt(2.0)
    cdf = lambda x: 0.5 * (math.erf((x + mu) / s) + math.erf((x - mu) / s))  # noqa: E731
    lo, hi = 0.0, abs(mu) + sigma
    while cdf(hi) < p:
        hi *= 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cdf(mid) < p:
            lo = mid
        else:
            hi = mid
        if hi - lo <= 1e-13 * max(1.0, hi):
            break
    return 0.5 * (lo + hi)


def length_cutoff(mu_L, sigma_L=1.0, p=0.999):
    """L_q = ceil(Q(0.999)) of N_F(mu_L, sigma_L): the trajectory length every replica runs."""
    return max(1, int(math.ceil(folded_normal_quantile(p, float(mu_L), sigma_L))))


def draw_lengths(mu_L, sigma_L, L_q, u):
    """Proposal lengths l in 1..L_q with probabilities proportional to N_F(l; mu_L, sigma_L),
    by inverse transform of the uniforms u (R,) -> int32 (R,) on u's device."""
    ell = torch.arange(1, L_q + 1, dtype=torch.float64, device=u.device)
    w = folded_normal_pdf(ell, torch.as_tensor(float(mu_L), dtype=torch.float64, device=u.device), sigma_L)
    c = torch.cumsum(w, 0) / torch.sum(w)
    return (torch.searchsorted(c, u.to(torch.float64).contiguous(), right=True) + 1).clamp_(max=L_q).to(torch.int32)


def lhmc_loss(alpha, jump, mu_L, sigma_L=1.0):
    """Eq. loss_steps: (1/R) sum_i sum_{l=1}^{L_q} w_l alpha_{i,l} jump_{i,l} / l, with
    alpha, jump (L_q, R) and w_l = N_F(l; mu_L, sigma_L) (mu_L a tensor: differentiable)."""
    L_q, R = alpha.shape
    ell = torch.arange(1, L_q + 1, dtype=alpha.dtype, device=alpha.device)
    w = folded_normal_pdf(ell, mu_L.to(alpha.dtype), sigma_L)
    return torch.sum((w / ell)[:, None] * alpha * jump) / R


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
    counts = torch.bincount(types, minlength=n_types).to(torch.float64)
    keys = ("loss", "mu", "alpha", "accepted")
    x = x0.clone()
    hist, rows = [], []
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
        with torch.no_grad():
            row = torch.stack([-loss, torch.exp(log_mu), alpha.mean(), acc.to(torch.float64).mean()])
            row = torch.cat([row, _type_masses(logits, counts, m_total)])
        _record(it, row, keys, {}, hist, rows, callback)
    return _finish(hist, rows, keys, [{} for _ in rows])


def _type_masses(logits, counts, m_total):
    s = torch.exp(logits)
    return m_total * s / torch.sum(counts * s)


def _record(it, row, keys, extra, hist, rows, callback):
    """One iteration's history: kept on the device (read once by ``_finish``) unless a
    callback wants it now, so that the host does not wait for every iteration."""
    if callback is None:
        rows.append(row)
        return
    rec = _as_record(it, row.cpu().tolist(), keys, extra)
    hist.append(rec)
    callback(rec)


def _as_record(it, vals, keys, extra):
    rec = {"it": it}
    rec.update(zip(keys, vals[:len(keys)]))
    rec.update(extra)
    rec["mass_per_type"] = vals[len(keys):]
    return rec


def _finish(hist, rows, keys, extras):
    if rows:
        vals = torch.stack(rows).cpu().tolist()
        hist = [_as_record(it, v, keys, e) for it, (v, e) in enumerate(zip(vals, extras))]
    return hist


def train_lhmc(h, x0, types, m_total, iters=200, kT=1.0, ckpt_every=8, lr=0.05, log_mu0=math.log(0.005),
               mu_L0=32.0, sigma_L=1.0, logits0=None, seed=0, terms=nbcore.NB_TERM_LJ, callback=None):
    """Adam on (log dt mean, log mu_L, mass logits) maximising L_HMC (Eq. loss_steps).

    Each iteration: L_q from the current mu_L, dt per replica from its folded normal,
    proposal lengths drawn from the discretised N_F(mu_L, sigma_L), one L_q-step
    trajectory per replica, the gradient of L_HMC through the weights (mu_L) and the
    trajectories (dt, masses), and every chain continues from its accepted/rejected state.
    Returns the per-iteration history (loss, dt mean, mu_L, L_q, masses per type, mean
    alpha of the proposals, acceptance).
    """
    dev = x0.device
    R = h.n_sys
    n = types.numel()
    n_types = int(types.max().item()) + 1
    log_mu = torch.tensor(log_mu0, dtype=torch.float64, device=dev, requires_grad=True)
    log_mu_L = torch.tensor(math.log(mu_L0), dtype=torch.float64, device=dev, requires_grad=True)
    logits = torch.zeros(n_types, dtype=torch.float64, device=dev) if logits0 is None else \
        torch.as_tensor(logits0, dtype=torch.float64, device=dev).clone()
    logits.requires_grad_(True)
    opt = torch.optim.Adam([log_mu, log_mu_L, logits], lr=lr)
    gen = torch.Generator(device=dev).manual_seed(seed)
    counts = torch.bincount(types, minlength=n_types).to(torch.float64)
    keys = ("loss", "mu", "mu_L", "alpha", "accepted")
    x = x0.clone()
    hist, rows, extras = [], [], []
    for it in range(iters):
        mu_L = torch.exp(log_mu_L)
        L_q = length_cutoff(float(mu_L.detach()), sigma_L)
        eps = torch.randn(R, dtype=torch.float64, device=dev, generator=gen)
        xi = torch.randn((R * n, 3), dtype=torch.float32, device=dev, generator=gen)
        u = torch.rand(R, dtype=torch.float64, device=dev, generator=gen)
        ul = torch.rand(R, dtype=torch.float64, device=dev, generator=gen)
        l_prop = draw_lengths(float(mu_L.detach()), sigma_L, L_q, ul)
        dt = folded_normal_step(log_mu, eps)
        w = (1.0 / masses_from_logits(logits, types, m_total)).repeat(R)
        alpha, jump, x_new, stats = HMCStepsProposal.apply(w, dt, h, x, xi, u, l_prop, L_q, kT, ckpt_every, terms)
        loss = -lhmc_loss(alpha, jump, mu_L, sigma_L)
        opt.zero_grad()
        loss.backward()
        opt.step()
        x = x_new
        with torch.no_grad():
            row = torch.stack([-loss, torch.exp(log_mu), mu_L, stats[:, 1].mean(), stats[:, 3].mean()])
            row = torch.cat([row, _type_masses(logits, counts, m_total)])
        extras.append({"L_q": L_q})
        _record(it, row, keys, {"L_q": L_q}, hist, rows, callback)
    return _finish(hist, rows, keys, extras)
