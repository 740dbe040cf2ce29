"""The host/torch side of the HMC tuning (paper_2503_20541_b300.hmc) against the oracle:
L_q, the discretised length draw, the folded-normal weights and Eq. loss_steps with its
derivative in mu_L.  CPU tensors only."""
import math

import numpy as np
import pytest

from oracle import tuning as tun

torch = pytest.importorskip("torch")
from paper_2503_20541_b300 import hmc  # noqa: E402


@pytest.mark.parametrize("mu", [0.3, 1.0, 10.0, 32.0, 60.0, 61.7])
def test_length_cutoff_matches_oracle(mu):
    assert hmc.length_cutoff(mu) == tun.length_cutoff(mu)
    assert hmc.folded_normal_quantile(0.999, mu, 1.0) == pytest.approx(tun.folded_normal_quantile(0.999, mu, 1.0),
                                                                        rel=1e-12)


def test_draw_lengths_match_oracle():
    mu = 23.4
    L_q = tun.length_cutoff(mu)
    u = torch.linspace(0.0, 0.999999, 5001, dtype=torch.float64)
    got = hmc.draw_lengths(mu, 1.0, L_q, u).numpy()
    ref = np.array([tun.draw_length(mu, 1.0, L_q, float(x)) for x in u])
    # the cumulative sums are formed in different orders: a uniform within rounding of a
    # bin edge may land on either side
    assert np.mean(got == ref) > 0.999 and np.abs(got - ref).max() <= 1
    assert got.dtype == np.int32 and got.min() >= 1 and got.max() <= L_q


def test_lhmc_loss_and_mu_gradient_match_oracle():
    rng = np.random.default_rng(2)
    mu = 12.6
    L_q = tun.length_cutoff(mu)
    R = 5
    alpha = rng.uniform(0.0, 1.0, (L_q, R))
    jump = rng.uniform(0.0, 3.0, (L_q, R)) * np.arange(1, L_q + 1)[:, None]
    m = torch.tensor(mu, dtype=torch.float64, requires_grad=True)
    loss = hmc.lhmc_loss(torch.from_numpy(alpha), torch.from_numpy(jump), m)
    loss.backward()
    assert float(loss) == pytest.approx(tun.lhmc_loss(alpha.T, jump.T, mu), rel=1e-13)
    fd = (tun.lhmc_loss(alpha.T, jump.T, mu + 1e-6) - tun.lhmc_loss(alpha.T, jump.T, mu - 1e-6)) / 2e-6
    assert float(m.grad) == pytest.approx(fd, rel=1e-7)
    xs = torch.linspace(0.0, 40.0, 81, dtype=torch.float64)
    np.testing.assert_allclose(hmc.folded_normal_pdf(xs, torch.tensor(mu, dtype=torch.float64), 1.0).numpy(),
                               tun.folded_normal_pdf(xs.numpy(), mu, 1.0), rtol=1e-14, atol=1e-300)
    assert math.isclose(float(hmc.folded_normal_step(torch.tensor(math.log(0.004), dtype=torch.float64),
                                                            torch.tensor(-1.5, dtype=torch.float64))),
                        abs(0.004 - 0.01 * 0.004 * 1.5), rel_tol=1e-12)
