"""The rounding of the float-float FP64 step, checked on the host.

The step forms each result f*_i = w_i + x ulp(w_i) as a float-float value
x = x.h + x.l (two FP32 numbers) and rounds it to an integer count of ulps
with FP32 operations only: t = x.h + 1.5 2^47 (the floats in [2^47, 2^48)
are the multiples of 2^24, so bits(t) - bits(1.5 2^47) counts them), the
remainder rem = x.h - (t - 1.5 2^47) (exact), then one conversion of
rem + x.l.  With |x.h| < 2^46 and |x.l| < 1.5 2^24 the result is within one
unit of x.  This test replays those FP32 operations bit for bit with numpy
(round to nearest even, as the device intrinsics) and checks the bound
against the exact value of x.h + x.l, including the extremes of both ranges,
and that the bound needs the limit on x.l.
"""
from fractions import Fraction

import numpy as np

M = np.float32(1.5 * 2.0 ** 47)


def _round_units(xh, xl):
    xh, xl = np.float32(xh), np.float32(xl)
    t = np.float32(xh + M)
    rem = np.float32(xh - np.float32(t - M))
    lo = np.float32(rem + xl)
    k = int(np.int64(t.view(np.int32)) - np.int64(M.view(np.int32)))  # multiples of 2^24
    return k * (1 << 24) + int(np.rint(lo))


def _exact(xh, xl):
    return Fraction(float(np.float32(xh))) + Fraction(float(np.float32(xl)))


def _random_pairs(rng, n, xl_bound):
    # magnitudes spread over every binade up to the limits
    eh = rng.uniform(-30, 46, n)
    el = rng.uniform(-30, np.log2(xl_bound), n)
    xh = np.float32(rng.choice([-1, 1], n) * 2.0 ** eh)
    xl = np.float32(rng.choice([-1, 1], n) * 2.0 ** el)
    keep = (np.abs(xh) < 2.0 ** 46) & (np.abs(xl) < xl_bound)
    return xh[keep], xl[keep]


def test_within_one_unit_over_the_ranges():
    rng = np.random.default_rng(7)
    xh, xl = _random_pairs(rng, 4000, 1.5 * 2.0 ** 24)
    worst = Fraction(0)
    for h, l in zip(xh, xl):
        err = abs(_round_units(h, l) - _exact(h, l))
        worst = max(worst, err)
        assert err <= 1, (float(h), float(l), float(err))
    assert worst > Fraction(1, 2)  # the bound is reached in places, not beaten by accident


def test_extremes():
    big = np.nextafter(np.float32(2.0 ** 46), np.float32(0))
    low = np.nextafter(np.float32(1.5 * 2.0 ** 24), np.float32(0))
    for h in (big, -big, np.float32(2.0 ** 23 * 3), np.float32(0.0), np.float32(-0.75)):
        for l in (low, -low, np.float32(0.5), np.float32(-2.0 ** -20), np.float32(0.0)):
            assert abs(_round_units(h, l) - _exact(h, l)) <= 1, (float(h), float(l))


def test_integers_are_kept():
    rng = np.random.default_rng(8)
    for n in rng.integers(-(1 << 45), 1 << 45, 500):
        h = np.float32(n)          # the nearest float
        rest = int(n) - int(h)     # exact remainder, |rest| < 2^22
        l = np.float32(rest)
        assert _round_units(h, l) == int(n)


def test_needs_the_low_part_limit():
    # far beyond 1.5 2^24 the FP32 sum rem + x.l rounds away more than a unit
    h, l = np.float32(5.0), np.float32(2.0 ** 30 + 2.0 ** 7 * 3)  # rem = 5 lost in the spacing of 128
    assert abs(_round_units(h, l) - _exact(h, l)) > 1


# ---- lazy float-float sums that feed a product -------------------------------
f32 = np.float32


def _fma(a, b, c):
    # a*b is exact in FP64 (two 24-bit significands); the sum is rounded once
    # to FP64 and then to FP32 (a second rounding only on exact FP64 ties)
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _add_lazy(x, y):
    s, e = _two_sum(x[0], y[0])
    return s, f32(e + f32(x[1] + y[1]))


def _mul(x, y):
    p = f32(x[0] * y[0])
    e = _fma(x[0], y[0], -p)
    e = _fma(x[0], y[1], e)
    e = _fma(x[1], y[0], e)
    return p, e


def _ff(rng, mag):
    h = f32(rng.choice([-1, 1]) * rng.uniform(0.5, 1.0) * mag)
    return h, f32(rng.uniform(-0.5, 0.5) * np.spacing(h))


def _val(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def test_lazy_sum_feeding_a_product_keeps_the_error_of_the_operands():
    """(a + b) c with the sum left unnormalised errs by at most a few 2^-47
    of max(|a|, |b|) |c|, also when a + b cancels to a tiny value: the same
    order as with the sum renormalised first (worst cases over these draws
    1.5 and 1.8 2^-47)."""
    rng = np.random.default_rng(9)
    worst = 0.0
    for k in range(3000):
        a = _ff(rng, 2.0 ** rng.uniform(-20, 20))
        if k % 3 == 0:  # near-total cancellation
            b = (f32(-a[0] * f32(1 + rng.uniform(-1e-6, 1e-6))), f32(-a[1]))
        else:
            b = _ff(rng, abs(float(a[0])) * 2.0 ** rng.uniform(-10, 10))
        c = _ff(rng, 2.0 ** rng.uniform(-20, 20))
        got = _val(_mul(_add_lazy(a, b), c))
        exact = (_val(a) + _val(b)) * _val(c)
        scale = max(abs(float(a[0])), abs(float(b[0]))) * abs(float(c[0]))
        worst = max(worst, abs(float(got - exact)) / scale)
    assert worst < 3 * 2.0 ** -47, worst
