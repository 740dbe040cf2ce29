"""Coefficients of the complementary error function used by the pair kernels (erfc.cuh).

    python paper_2503_20541_b300/csrc/erfc_fit.py

erfc(x) = exp(-x^2) erfcx(x) for x >= 0, and with t = 1 / (1 + x/2) (0 < t <= 1 maps
the whole half-line x >= 0) erfcx(x) / t is a smooth function of t that a polynomial
in u = 2t - 1 represents to ~1e-9 relative at degree 12.  The fit is a Chebyshev least
squares fit (numpy) of erfcx(x)/t, with relative weights iteratively raised where the
error is largest (a Lawson-style approach toward the minimax fit), to the values of
scipy.special.erfcx; the Chebyshev series is converted to monomials in u for Horner's
rule.  Prints the coefficients (lowest order first) and the fit's max relative error.
"""
import numpy as np
from numpy.polynomial import chebyshev as C
from scipy.special import erfcx

DEG = 12


def fit(deg=DEG, n=6000, iters=30):
    """Monomial coefficients in u = 2t - 1, lowest order first, each exactly an FP32 value.

    After the FP64 fit, the coefficients are rounded to FP32 one at a time from the lowest
    order up, and the ones not yet rounded are refitted (same weights, least squares in the
    monomial basis) to absorb the rounding: rounding all of them at once left a systematic
    relative bias of ~2e-8, mostly from the constant term."""
    t = np.cos(np.pi * (np.arange(n) + 0.5) / n) * 0.5 + 0.5   # Chebyshev nodes on (0, 1)
    x = 2.0 * (1.0 / t - 1.0)
    y = erfcx(x) / t
    u = 2.0 * t - 1.0
    w = 1.0 / y
    for _ in range(iters):
        c = C.chebfit(u, y, deg, w=w)
        r = np.abs(C.chebval(u, c) / y - 1.0)
        w = w * (1.0 + 50.0 * r / r.max()) ** 0.5
    m = C.cheb2poly(c)
    V = np.vander(u, deg + 1, increasing=True)
    for k in range(deg + 1):
        m[k] = float(np.float32(m[k]))
        if k < deg:
            rest = y - V[:, :k + 1] @ m[:k + 1]
            m[k + 1:] = np.linalg.lstsq(V[:, k + 1:] * w[:, None], rest * w, rcond=None)[0]
    return m


def max_rel_error(mono, x):
    t = 1.0 / (1.0 + 0.5 * x)
    return float(np.max(np.abs(t * np.polynomial.polynomial.polyval(2.0 * t - 1.0, mono) / erfcx(x) - 1.0)))


if __name__ == "__main__":
    m = fit()
    for k, v in enumerate(m):
        print("c%-2d = %.9e" % (k, np.float32(v)))
    print("max relative error of the fit on [0, 10]: %.2e" % max_rel_error(m, np.linspace(0.0, 10.0, 200001)))
