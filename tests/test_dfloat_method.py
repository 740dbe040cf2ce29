"""The two-float arithmetic of the precise energies (csrc/dfloat.cuh), restated on the host
with numpy float32 operations (IEEE round-to-nearest, as the _rn intrinsics; an FMA as the
exact float64 product plus the addend, rounded once to float32 -- exact for the product
error that two_prod forms), and checked against float64 / exact rational arithmetic:
TwoSum and the FMA product error are exact, the accurate two-float sum and product keep
~2^-47 relative error, Dekker's addition ~2^-46 of the operands' size, and the division-free
1/sqrt (hardware estimate plus one Newton step) 1.5 e0^2 for an estimate off by e0: below
2.5e-13 with the hardware reciprocal square root modelled as the correctly rounded one
perturbed by up to 2 ulp, below 1e-13 when it is within 1 ulp."""
from fractions import Fraction

import numpy as np

F = np.float32
RNG = np.random.default_rng(17)


def fma(a, b, c):
    return F(float(a) * float(b) + float(c))


def two_sum(a, b):
    s = F(a + b)
    bb = F(s - a)
    return s, F(F(a - F(s - bb)) + F(b - bb))


def fast_two_sum(a, b):
    s = F(a + b)
    return s, F(b - F(s - a))


def two_prod(a, b):
    p = F(a * b)
    return p, fma(a, b, -p)


def df_add(a, b):
    s = two_sum(a[0], b[0])
    t = two_sum(a[1], b[1])
    s = fast_two_sum(s[0], F(s[1] + t[0]))
    return fast_two_sum(s[0], F(s[1] + t[1]))


def df_add_fast(a, b):
    s = two_sum(a[0], b[0])
    return fast_two_sum(s[0], F(s[1] + F(a[1] + b[1])))


def df_mul(a, b):
    p = two_prod(a[0], b[0])
    return fast_two_sum(p[0], fma(a[0], b[1], fma(a[1], b[0], p[1])))


def df_rsqrt(a, ulp_off=0):
    y = F(1.0 / np.sqrt(float(a[0])))
    for _ in range(abs(ulp_off)):
        y = np.nextafter(y, F(np.inf) if ulp_off > 0 else F(0))
    m = df_mul(a, two_prod(y, y))
    e = two_sum(F(-m[0]), F(1.0))
    e = fast_two_sum(e[0], F(e[1] - m[1]))
    return fast_two_sum(y, F(F(y * e[0]) * F(0.5)))


def exact(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def rand_df(n, lo=-3, hi=3):
    out = []
    for _ in range(n):
        h = F(RNG.uniform(1, 2) * 10.0 ** RNG.uniform(lo, hi) * RNG.choice([-1, 1]))
        l = F(float(h) * RNG.uniform(-1, 1) * 2.0 ** -25)
        out.append(fast_two_sum(h, l))
    return out


def test_two_sum_and_two_prod_are_exact():
    for _ in range(2000):
        a, b = F(RNG.normal() * 10 ** RNG.uniform(-4, 4)), F(RNG.normal() * 10 ** RNG.uniform(-4, 4))
        s, e = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e)) == Fraction(float(a)) + Fraction(float(b))
        p, q = two_prod(a, b)
        assert Fraction(float(p)) + Fraction(float(q)) == Fraction(float(a)) * Fraction(float(b))


def test_two_float_sum_and_product_errors():
    xs, ys = rand_df(1500), rand_df(1500)
    for x, y in zip(xs, ys):
        ref = exact(x) + exact(y)
        got = exact(df_add(x, y))
        assert abs(got - ref) <= 2.0 ** -46 * abs(ref) + 2.0 ** -70
        got = exact(df_add_fast(x, y))
        assert abs(got - ref) <= 2.0 ** -45 * (abs(exact(x)) + abs(exact(y)))
        ref = exact(x) * exact(y)
        got = exact(df_mul(x, y))
        assert abs(got - ref) <= 2.0 ** -45 * abs(ref)


def test_division_free_rsqrt():
    worst = {0: 0.0, 1: 0.0, 2: 0.0}
    for a in rand_df(1500, lo=-1, hi=3):
        a = (F(abs(a[0])), F(abs(a[1])) if a[1] * a[0] > 0 else F(-abs(a[1])))
        val = float(exact(a))
        for off in (-2, -1, 0, 1, 2):  # the hardware estimate within a couple of ulp
            r = exact(df_rsqrt(a, off))
            rel = abs(float(r) * np.sqrt(val) - 1.0)
            worst[abs(off)] = max(worst[abs(off)], rel)
    assert worst[0] <= 2e-14 and worst[1] <= 1e-13 and worst[2] <= 2.5e-13, worst
