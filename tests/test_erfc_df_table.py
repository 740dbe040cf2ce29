"""The two-float erfc table of the precise energies (csrc/erfc_df.cuh) against scipy's FP64
erfc, on the host: the stored coefficients (hi + lo, exact in FP64) of every interval,
evaluated by Horner's rule in FP64 on a dense grid, within 1e-13 relative of erfc, and
the pieces meeting at the interval ends.  The table is written by csrc/erfc_df_fit.py from
mpmath's erfc; scipy's erfc is an independent implementation."""
import os
import re

import numpy as np
from scipy.special import erfc

HDR = os.path.join(os.path.dirname(__file__), "..", "paper_2503_20541_b300", "csrc", "erfc_df.cuh")


def _table():
    src = open(HDR).read()
    H = float(re.search(r"kErfcDfH = ([0-9.eE+-]+)f;", src).group(1))
    n_int = int(re.search(r"kErfcDfIntervals = (\d+);", src).group(1))
    deg = int(re.search(r"kErfcDfDeg = (\d+);", src).group(1))
    body = src[src.index("g_erfc_df"):]
    pairs = re.findall(r"\{([-+0-9.eE]+)f, ([-+0-9.eE]+)f\}", body)
    c = np.array([[float(a), float(b)] for a, b in pairs], dtype=np.float64)
    assert c.shape == (n_int * (deg + 1), 2)
    # the literals carry 10 significant digits: each names one FP32 number, the value the
    # compiler stores (within 1e-9 relative of it, far from a rounding midpoint)
    c32 = c.astype(np.float32).astype(np.float64)
    nz = c != 0.0
    assert np.all(np.abs(c32[nz] - c[nz]) <= 1e-9 * np.abs(c[nz]))
    c = c32
    return H, n_int, deg, (c[:, 0] + c[:, 1]).reshape(n_int, deg + 1), c.reshape(n_int, deg + 1, 2)


def _eval(coef, t):
    p = np.full_like(t, coef[-1])
    for m in range(coef.size - 2, -1, -1):
        p = p * t + coef[m]
    return p


def test_table_matches_fp64_erfc():
    H, n_int, deg, coef, _ = _table()
    assert H == 0.25 and n_int * H == 6.0
    worst = 0.0
    for k in range(n_int):
        t = np.linspace(0.0, H, 2001)
        got = _eval(coef[k], t)
        ref = erfc(k * H + t)
        worst = max(worst, float(np.max(np.abs(got - ref) / ref)))
    assert worst <= 1e-13, worst


def test_pieces_meet_at_the_interval_ends():
    H, n_int, deg, coef, _ = _table()
    for k in range(n_int - 1):
        end = _eval(coef[k], np.array([H]))[0]
        start = coef[k + 1][0]
        assert abs(end - start) <= 1e-13 * start, k


def test_lo_parts_are_roundings_of_hi():
    # |lo| <= ulp(hi)/2: each pair is a normalised two-float number
    *_, pairs = _table()
    hi, lo = pairs[..., 0], pairs[..., 1]
    nz = hi != 0.0
    assert np.all(np.abs(lo[nz]) <= 0.5 * np.spacing(np.abs(hi[nz]).astype(np.float32)).astype(np.float64))
