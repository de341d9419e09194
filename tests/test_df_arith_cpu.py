"""The double-float arithmetic of the refinement residual (CPU emulation of the same steps:
split of an FP64 value into hi + lo floats, Knuth's two-sum, Dekker's product through FMA):
a 3R-pair stencil sum keeps its rounding error near 2^-48 of the summed magnitudes, which is
what allows it at Sternheimer tolerances >= 1e-8."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def _fma(a, b, c):
    return f32(float(a) * float(b) + float(c))  # product exact in float64


def _two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def _fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def _split(x):
    h = f32(x)
    return h, f32(x - float(h))


def _add(a, b):
    s, e = _two_sum(a[0], b[0])
    return _fast_two_sum(s, f32(e + f32(a[1] + b[1])))


def _fma_df(acc, c, x):
    p = f32(c[0] * x[0])
    e = _fma(c[0], x[0], -p)
    e = _fma(c[0], x[1], _fma(c[1], x[0], e))
    s, e2 = _two_sum(acc[0], p)
    return _fast_two_sum(s, f32(e2 + f32(acc[1] + e)))


def test_double_float_stencil_sum_error():
    rng = np.random.default_rng(0)
    worst = 0.0
    for _ in range(300):
        R = 6
        coef = rng.standard_normal(3 * R) * 10
        xs = rng.standard_normal((3 * R, 2)) * 100
        acc = (f32(0), f32(0))
        exact, mag = Fraction(0), 0.0
        for k in range(3 * R):
            acc = _fma_df(acc, _split(coef[k]), _add(_split(xs[k, 0]), _split(xs[k, 1])))
            exact += Fraction(coef[k]) * (Fraction(xs[k, 0]) + Fraction(xs[k, 1]))
            mag += abs(coef[k]) * (abs(xs[k, 0]) + abs(xs[k, 1]))
        got = Fraction(float(acc[0])) + Fraction(float(acc[1]))
        worst = max(worst, abs(float(got - exact)) / mag)
    assert worst < 4 * 2.0 ** -48
    assert worst > 2.0 ** -60  # it is not secretly FP64
