"""Writes erfc_df.cuh: erfc(x) on [0, X_MAX) as piecewise polynomials with two-float
coefficients, for the double-float energies of the pair terms (ke q_i q_j erfc(alpha r)/r,
Sec. 2.1.2) in the precise-energy evaluation.

Interval k covers [k H, (k + 1) H); on it erfc(k H + t) = sum_m c_{k,m} t^m, t in [0, H].
The coefficients interpolate erfc at the DEG + 1 Chebyshev points of the interval,
computed with mpmath at 60 significant digits (solving the Vandermonde system in t at that
precision), and each is stored as hi = fl32(c), lo = fl32(c - hi).  The script checks the
interpolant against mpmath's erfc on a dense grid of every interval and refuses to write
the table if the largest relative error exceeds TOL (the interpolation error itself is
below 1e-15; the two-float rounding of the coefficients dominates what is left).

Run from this directory:  python erfc_df_fit.py  (rewrites erfc_df.cuh)."""
import os
import struct

import mpmath as mp

H = 0.25       # interval width: t = x - k H is exact in FP32 for x in [k H, (k + 1) H)
X_MAX = 6.0    # erfc(6) = 2.2e-17: beyond it the terms are far below any energy's rounding
DEG = 15
TOL = 1e-13    # relative, of the stored interpolant: rounding the power-basis coefficients
               # to two floats (~4e-15 each) dominates, up to 5e-14 where the series alternates (x ~ 6)
mp.mp.dps = 60


def f32(v):
    return struct.unpack("f", struct.pack("f", float(v)))[0]


def fit_interval(a):
    n = DEG + 1
    ts = [mp.mpf(H) / 2 * (1 - mp.cos(mp.pi * (k + mp.mpf(1) / 2) / n)) for k in range(n)]
    A = mp.matrix(n, n)
    b = mp.matrix(n, 1)
    for i, t in enumerate(ts):
        for m in range(n):
            A[i, m] = t ** m
        b[i] = mp.erfc(a + t)
    return list(mp.lu_solve(A, b))


def main():
    n_int = int(round(X_MAX / H))
    rows, worst = [], 0.0
    for k in range(n_int):
        a = mp.mpf(k) * mp.mpf(H)
        c = fit_interval(a)
        pairs = []
        for v in c:
            hi = f32(v)
            lo = f32(v - mp.mpf(hi))
            pairs.append((hi, lo))
        # the stored (hi + lo) coefficients against erfc on a dense grid of the interval
        for s in range(401):
            t = mp.mpf(H) * s / 400
            p = mp.mpf(0)
            for hi, lo in reversed(pairs):
                p = p * t + (mp.mpf(hi) + mp.mpf(lo))
            ref = mp.erfc(a + t)
            worst = max(worst, float(abs(p - ref) / ref))
        rows.append(pairs)
    if worst > TOL:
        raise SystemExit("fit error %.3e above %.1e: raise DEG or narrow H" % (worst, TOL))
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "erfc_df.cuh")
    with open(out, "w") as fh:
        fh.write("// erfc_df.cuh -- written by erfc_df_fit.py; do not edit.\n")
        fh.write("// erfc(k H + t) = sum_m c[k][m] t^m for t in [0, H), two-float coefficients (hi, lo);\n")
        fh.write("// Chebyshev-point interpolants of degree %d, largest relative error of the\n" % DEG)
        fh.write("// interpolant %.2e over [0, %.1f).\n" % (worst, X_MAX))
        fh.write("#pragma once\n\nnamespace nb {\n\n")
        fh.write("constexpr float kErfcDfH = %sf;\n" % repr(float(H)))
        fh.write("constexpr float kErfcDfInvH = %sf;\n" % repr(1.0 / H))
        fh.write("constexpr int kErfcDfIntervals = %d;\n" % n_int)
        fh.write("constexpr int kErfcDfDeg = %d;\n\n" % DEG)
        fh.write("static __device__ const float2 g_erfc_df[kErfcDfIntervals][kErfcDfDeg + 1] = {\n")
        for k, pairs in enumerate(rows):
            fh.write("    {  // [%.2f, %.2f)\n" % (k * H, (k + 1) * H))
            for hi, lo in pairs:
                fh.write("        {%s, %s},\n" % (repr_f(hi), repr_f(lo)))
            fh.write("    },\n")
        fh.write("};\n\n}  // namespace nb\n")
    print("wrote", out, "worst relative error %.3e" % worst)


def repr_f(v):
    s = "%.9e" % v
    return s + "f"


if __name__ == "__main__":
    main()
