"""Pins of the HMC tuning oracle (oracle.tuning): the folded normal against scipy's
foldnorm and the half-normal special case, the discretised weights against Poisson
summation, the step-weighted loss against its ballistic closed form, the per-step HMC
statistics against the pinned single-length proposal, and A(k) / tau_exp against
closed forms (an alternating series, an exact exponential) and an AR(1) process."""
import math

import numpy as np
import pytest

import oracle
from oracle import dynamics as odyn
from oracle import tuning as tun
from paper_2503_20541_b300 import workloads as wl

scipy_stats = pytest.importorskip("scipy.stats")
from scipy import integrate, signal  # noqa: E402


@pytest.mark.parametrize("mu,sigma", [(0.0, 1.0), (0.8, 1.0), (3.0, 1.0), (60.0, 1.0), (0.01, 1e-4)])
def test_folded_normal_density_and_cdf_match_foldnorm(mu, sigma):
    ref = scipy_stats.foldnorm(mu / sigma, scale=sigma)
    x = np.linspace(0.0, mu + 6 * sigma, 57)
    np.testing.assert_allclose(tun.folded_normal_pdf(x, mu, sigma), ref.pdf(x), rtol=1e-12, atol=1e-300)
    for xv in x[1::7]:
        assert tun.folded_normal_cdf(xv, mu, sigma) == pytest.approx(ref.cdf(xv), rel=1e-12, abs=1e-15)
    total, _ = integrate.quad(lambda t: float(tun.folded_normal_pdf(t, mu, sigma)), 0.0, mu + 40 * sigma,
                              points=[mu], limit=200)
    assert total == pytest.approx(1.0, abs=1e-9)


@pytest.mark.parametrize("mu,sigma", [(0.0, 1.0), (0.7, 1.0), (10.0, 1.0), (60.0, 1.0), (0.5, 0.005)])
def test_quantile_matches_foldnorm_ppf(mu, sigma):
    for p in (0.5, 0.9, 0.999):
        q = tun.folded_normal_quantile(p, mu, sigma)
        assert q == pytest.approx(scipy_stats.foldnorm.ppf(p, mu / sigma, scale=sigma), rel=1e-9)
    if mu == 0.0:
        # half-normal: Q(p) = sigma Phi^-1((1 + p)/2)
        assert tun.folded_normal_quantile(0.999, 0.0, sigma) == pytest.approx(
            sigma * scipy_stats.norm.ppf(0.9995), rel=1e-10)


def test_length_cutoff():
    assert tun.length_cutoff(60.0) == math.ceil(scipy_stats.foldnorm.ppf(0.999, 60.0)) == 64
    assert tun.length_cutoff(10.0) == 14
    assert tun.length_cutoff(0.2) == math.ceil(scipy_stats.foldnorm.ppf(0.999, 0.2))


def test_integer_weights_sum_to_one_by_poisson_summation():
    # sum_l phi(l - mu) over the integers is 1 + 2 sum_k exp(-2 pi^2 k^2 sigma^2) cos(2 pi k mu):
    # within 5.4e-9 of 1 for sigma = 1, whatever mu
    for mu in (20.0, 30.37, 45.5):
        w = tun.step_weights(mu, 1.0, 200)
        assert abs(w.sum() - 1.0) < 6e-9
        assert abs(w.sum() - (1.0 + 2.0 * math.exp(-2.0 * math.pi ** 2) * math.cos(2 * math.pi * mu))) < 1e-15 + 1e-12


def test_lhmc_loss_ballistic_closed_form():
    # alpha = 1 and |O'_l - O_l|^2 = c l: every term is w_l c, so the loss is c times the
    # truncated weight sum, between 0.999 c and c for mu far from 0
    mu = 30.37
    L_q = tun.length_cutoff(mu)
    c = 2.5
    R = 4
    ell = np.arange(1, L_q + 1, dtype=np.float64)
    loss = tun.lhmc_loss(np.ones((R, L_q)), np.tile(c * ell, (R, 1)), mu)
    assert 0.999 * c <= loss <= c * (1.0 + 1e-8)
    # the replica average: one replica with zero jumps halves the loss of two
    two = tun.lhmc_loss(np.ones((2, L_q)), np.stack([c * ell, 0 * ell]), mu)
    assert two == pytest.approx(0.5 * loss, rel=1e-14)
    # a jump that grows like l^2 weights the mean length: sum_l w_l l ~ mu
    quad = tun.lhmc_loss(np.ones((1, L_q)), (ell * ell)[None, :], mu)
    assert quad == pytest.approx(mu, rel=2e-3)


def test_draw_length_follows_the_discretised_weights():
    mu, L_q = 12.3, tun.length_cutoff(12.3)
    w = tun.step_weights(mu, 1.0, L_q)
    p = w / w.sum()
    M = 20000
    draws = np.array([tun.draw_length(mu, 1.0, L_q, (k + 0.5) / M) for k in range(M)])
    assert draws.min() >= 1 and draws.max() <= L_q
    counts = np.bincount(draws, minlength=L_q + 1)[1:] / M
    assert np.abs(counts - p).max() <= 1.0 / M + 1e-12
    assert np.all(np.diff(draws) >= 0)  # inverse transform: monotone in u


def test_per_step_statistics_match_single_length_proposals():
    s = wl.lj_random(108, seed=3, n_types=2)
    p = oracle.make_params(s.box, r_cut=2.5, r_switch=2.2)

    def fe(x):
        e, f = oracle.nonbonded(x, s.q, s.sigma, s.sqrt_eps, p)
        return f, float(e[0])

    rng = np.random.default_rng(5)
    xi = rng.standard_normal((s.n, 3))
    w = 1.0 / odyn.masses_from_logits([0.2, -0.1], s.types, float(s.n))
    x0 = s.x.astype(np.float64)
    out = tun.hmc_proposal_steps(x0, xi, w, 0.004, 9, 1.0, fe, s.box)
    for ell in (1, 4, 9):
        ref = odyn.hmc_proposal(x0, xi, w, 0.004, ell, 1.0, fe, s.box)
        assert out["dH"][ell - 1] == pytest.approx(ref["dH"], rel=1e-12, abs=1e-13)
        assert out["alpha"][ell - 1] == pytest.approx(ref["alpha"], rel=1e-12)
        assert out["jump"][ell - 1] == pytest.approx(ref["jump"], rel=1e-12)
        np.testing.assert_allclose(out["x"][ell - 1], ref["x"], rtol=0, atol=1e-12)


def test_autocorrelation_closed_forms():
    o = np.array([(-1.0) ** t for t in range(1000)])
    a = tun.autocorrelation(o, 4)
    np.testing.assert_allclose(a, [1.0, -1.0, 1.0, -1.0, 1.0], rtol=0, atol=1e-14)
    # an exact exponential: the fit returns its decay time
    k = np.arange(60)
    assert tun.tau_exp(np.exp(-k / 7.3)) == pytest.approx(7.3, rel=1e-10)
    # white noise has no decay region above the noise floor
    rng = np.random.default_rng(0)
    assert math.isnan(tun.tau_exp(tun.autocorrelation(rng.standard_normal(20000), 10)))


def test_autocorrelation_is_invariant_under_affine_maps():
    # A(k) is a correlation: O -> a O + b (a > 0) leaves it unchanged, also with an offset
    # two hundred times the spread, as for a potential-energy trace
    rng = np.random.default_rng(4)
    o = signal.lfilter([1.0], [1.0, -0.7], rng.standard_normal(5000))
    a = tun.autocorrelation(o, 30)
    np.testing.assert_allclose(tun.autocorrelation(3.0 * o - 600.0, 30), a, rtol=0, atol=1e-11)
    np.testing.assert_allclose(tun.autocorrelation(-2.0 * o, 30), a, rtol=0, atol=1e-13)


def test_autocorrelation_of_ar1_process():
    # o_t = phi o_{t-1} + e_t has A(k) = phi^k and tau_exp = -1/ln(phi)
    phi = 0.8
    rng = np.random.default_rng(1)
    o = signal.lfilter([1.0], [1.0, -phi], rng.standard_normal(1_000_000))[1000:]
    a = tun.autocorrelation(o, 20)
    np.testing.assert_allclose(a[:11], phi ** np.arange(11), rtol=0, atol=0.01)
    assert tun.tau_exp(a) == pytest.approx(-1.0 / math.log(phi), rel=0.06)
