"""CPU pins of the pair kernels' erfc (csrc/erfc.cuh): its coefficients are the output of
csrc/erfc_fit.py, the fit meets its stated accuracy against scipy's erfcx, and an FP32
emulation of the kernel's evaluation order (numpy, every FMA rounded once) stays within a
few ulp of the FP64 erfc over the Ewald range."""
import os
import re
import sys

import numpy as np
from scipy.special import erfc as erfc64, erfcx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_20541_b300", "csrc")
sys.path.insert(0, CSRC)
import erfc_fit  # noqa: E402

f32 = np.float32


def header_coefficients():
    src = open(os.path.join(CSRC, "erfc.cuh")).read()
    body = src[src.index("float p = "):src.index("return E * (t * p);")]
    vals = [float(v) for v in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    return np.array(vals[::-1], np.float32)  # Horner runs from the top coefficient down


def test_header_coefficients_are_the_fit():
    assert np.array_equal(header_coefficients(), erfc_fit.fit().astype(np.float32))


def test_fit_accuracy_on_the_half_line():
    m = erfc_fit.fit()
    x = np.linspace(0.0, 10.0, 100001)
    assert erfc_fit.max_rel_error(m, x) < 2.5e-8        # below half an FP32 ulp
    t = 1.0 / (1.0 + 0.5 * x[x <= 4.0])
    rel = t * np.polynomial.polynomial.polyval(2.0 * t - 1.0, m) / erfcx(x[x <= 4.0]) - 1.0
    assert abs(rel.mean()) < 1e-8                        # no systematic bias
    # the variable t = 1/(1 + x/2) covers x -> infinity: erfcx(x) ~ 1/(sqrt(pi) x)
    x = np.array([50.0, 1e3, 1e5])
    t = 1.0 / (1.0 + 0.5 * x)
    approx = t * np.polynomial.polynomial.polyval(2.0 * t - 1.0, m)
    assert np.all(np.abs(approx / erfcx(x) - 1.0) < 2.5e-8)


def _fma(a, b, c):
    return (np.float64(a) * np.float64(b) + np.float64(c)).astype(np.float32)


def emulate(x):
    """The kernel's operation order in FP32 (2^y taken correctly rounded)."""
    c = header_coefficients()
    L, L_lo, ln2 = f32(1.4426950408889634), f32(1.92596299e-08), f32(0.693147182)
    s = (x * x).astype(np.float32)
    s_lo = _fma(x, x, -s)
    y = (-s * L).astype(np.float32)
    y_lo = (_fma(-s, L, -y) - _fma(s, L_lo, (s_lo * L).astype(np.float32))).astype(np.float32)
    e = np.exp2(np.float64(y)).astype(np.float32)
    E = _fma(e, (y_lo * ln2).astype(np.float32), e)
    d = _fma(f32(0.5), x, f32(1.0))
    d_lo = _fma(f32(0.5), x, (f32(1.0) - d).astype(np.float32))
    t = (1.0 / np.float64(d)).astype(np.float32)
    t = _fma(t, (_fma(-d, t, f32(1.0)) - (d_lo * t).astype(np.float32)).astype(np.float32), t)
    u = _fma(f32(2.0), t, f32(-1.0))
    p = np.full_like(x, c[-1])
    for k in range(len(c) - 2, -1, -1):
        p = _fma(p, u, c[k])
    return (E * (t * p).astype(np.float32)).astype(np.float32)


def test_fp32_emulation_stays_within_a_few_ulp():
    x = np.linspace(0.0, 4.5, 200001, dtype=np.float32)
    ref = erfc64(x.astype(np.float64))
    ulp = np.spacing(ref.astype(np.float32)).astype(np.float64)
    err = np.abs(emulate(x).astype(np.float64) - ref) / ulp
    assert err.max() <= 5.0 and err.mean() <= 1.0
