"""FP64 reference of the HMC tuning objective of Sec. 4: the folded-normal trajectory
length, the step-length-weighted loss L_HMC (Eq. loss_steps) truncated at the 0.999
quantile L_q, the per-step HMC statistics it needs, and the autocorrelation function
A(k) with the exponential autocorrelation time tau_exp used to evaluate the tuning.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Readings where the paper leaves a choice open:
  * L_q = ceil(Q(0.999)), Q the quantile function of N_F(mu_L, sigma_L): the sum runs
    over integer step counts, so the quantile is rounded up.
  * w_l is the folded-normal density itself, evaluated at the integer l (no
    renormalisation over 1..L_q); the same discretised weights, normalised, are the
    distribution the proposal's length is drawn from.
  * A(k) replaces the thermodynamic averages by averages over one stationary series, in
    the centred form: for expectations <O_t O_{t+k}> - <O>^2 = <(O_t - <O>)(O_{t+k} - <O>)>,
    and A is unchanged by O -> a O + b; with finite series only the centred estimator
    keeps that invariance (the plain one carries an O(k/n) edge term times <O>^2, which
    swamps the covariance of an energy trace whose mean is far larger than its spread).
    So A(k) = [1/(n-k) sum_{t<n-k} d_t d_{t+k}] / [1/n sum_t d_t^2], d_t = O_t - mean(O).
  * tau_exp is the least-squares slope of ln A(k) against k over the lags k >= 1 from
    the first with A(k) <= a_hi up to the last before A(k) first falls below a_lo
    (the decay region above the noise floor); fewer than two such lags give NaN.
"""
import math

import numpy as np


def folded_normal_pdf(x, mu, sigma):
    """N_F(x; mu, sigma): the normal density at x plus its mirror image at -x (Sec. 4)."""
    x = np.asarray(x, dtype=np.float64)
    c = 1.0 / math.sqrt(2.0 * math.pi * sigma * sigma)
    return c * np.exp(-(x - mu) ** 2 / (2.0 * sigma * sigma)) + c * np.exp(-(x + mu) ** 2 / (2.0 * sigma * sigma))


def folded_normal_cdf(x, mu, sigma):
    """P(X <= x) for X ~ N_F(mu, sigma), x >= 0: the integral of the density from 0,
    1/2 [erf((x + mu)/(sigma sqrt 2)) + erf((x - mu)/(sigma sqrt 2))]."""
    s = sigma * math.sqrt(2.0)
    return 0.5 * (math.erf((x + mu) / s) + math.erf((x - mu) / s))


def folded_normal_quantile(p, mu, sigma, tol=1e-13):
    """Q(p): the x >= 0 with folded_normal_cdf(x) = p, by bisection."""
    lo, hi = 0.0, abs(mu) + sigma
    while folded_normal_cdf(hi, mu, sigma) < p:
        hi *= 2.0
    while hi - lo > tol * max(1.0, hi):
        mid = 0.5 * (lo + hi)
        if folded_normal_cdf(mid, mu, sigma) < p:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def length_cutoff(mu_L, sigma_L=1.0, p=0.999):
    """L_q: the truncation of the sum over step lengths in Eq. loss_steps."""
    return int(math.ceil(folded_normal_quantile(p, mu_L, sigma_L)))


def step_weights(mu_L, sigma_L, L_q):
    """w_l = N_F(l; mu_L, sigma_L) for l = 1..L_q."""
    return folded_normal_pdf(np.arange(1, L_q + 1, dtype=np.float64), mu_L, sigma_L)


def draw_length(mu_L, sigma_L, L_q, u):
    """The proposal's length l ~ the discretised folded normal on 1..L_q (probabilities
    proportional to w_l), by inverse transform of a uniform u in [0, 1)."""
    w = step_weights(mu_L, sigma_L, L_q)
    c = np.cumsum(w) / np.sum(w)
    return int(np.searchsorted(c, u, side="right")) + 1


def hmc_proposal_steps(x0, xi, inv_mass, dt, n_steps, kT, force_energy, box):
    """One HMC trajectory of n_steps velocity-Verlet steps (Sec. 4) with the statistics of
    every intermediate state l = 1..n_steps: dH_l = E(x_l, v_l) - E(x_0, v_0), the
    acceptance probability alpha_l = min(1, exp(-dH_l/kT)) of proposing (x_l, v_l), and the
    squared jump |mi(x_l - x_0)|^2.  Velocities v0 = sqrt(kT/m) xi as in hmc_proposal."""
    w = np.asarray(inv_mass, dtype=np.float64)
    x0 = np.asarray(x0, dtype=np.float64)
    wv = w[:, None]
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    x = x0.copy()
    v = np.sqrt(kT * w)[:, None] * np.asarray(xi, dtype=np.float64)
    F, U = force_energy(x)
    H0 = U + 0.5 * float(np.sum(np.sum(v * v, axis=1) / w))
    dH, alpha, jump, xs = [], [], [], []
    for _ in range(n_steps):
        v = v + 0.5 * dt * wv * F
        x = x + dt * v
        F, U = force_energy(x)
        v = v + 0.5 * dt * wv * F
        d = x - x0
        d = d - L * np.round(d / L)
        h = U + 0.5 * float(np.sum(np.sum(v * v, axis=1) / w)) - H0
        dH.append(h)
        alpha.append(min(1.0, math.exp(-h / kT)) if h == h else 0.0)
        jump.append(float(np.sum(d * d)))
        xs.append(x.copy())
    return {"dH": np.array(dH), "alpha": np.array(alpha), "jump": np.array(jump), "x": xs}


def lhmc_loss(alpha, jump, mu_L, sigma_L=1.0):
    """Eq. loss_steps: (1/R) sum_i sum_{l=1}^{L_q} w_l alpha_{i,l} |O'_{i,l} - O_{i,l}|^2 / l
    with alpha, jump of shape (R, L_q) and w_l = N_F(l; mu_L, sigma_L)."""
    a = np.asarray(alpha, dtype=np.float64)
    j = np.asarray(jump, dtype=np.float64)
    L_q = a.shape[1]
    w = step_weights(mu_L, sigma_L, L_q)
    ell = np.arange(1, L_q + 1, dtype=np.float64)
    return float(np.sum(w[None, :] * a * j / ell[None, :]) / a.shape[0])


def autocorrelation(o, max_lag):
    """A(k) for k = 0..max_lag of one series (Sec. 4): the lagged covariance over the
    variance, both about the series mean (see the module header)."""
    o = np.asarray(o, dtype=np.float64)
    n = o.size
    d = o - float(np.mean(o))
    var = float(np.mean(d * d))
    out = np.empty(max_lag + 1)
    for k in range(max_lag + 1):
        out[k] = float(np.mean(d[:n - k] * d[k:])) / var
    return out


def tau_exp(acf, a_hi=0.5, a_lo=0.05):
    """Exponential autocorrelation time: A(k) -> exp(-k / tau_exp), fitted over the decay
    region (see the module header)."""
    a = np.asarray(acf, dtype=np.float64)
    k0 = None
    ks = []
    for k in range(1, a.size):
        if a[k] < a_lo:
            break
        if k0 is None and a[k] <= a_hi:
            k0 = k
        if k0 is not None:
            ks.append(k)
    if len(ks) < 2:
        return float("nan")
    kk = np.array(ks, dtype=np.float64)
    slope = np.polyfit(kk, np.log(a[ks]), 1)[0]
    return float(-1.0 / slope)
