"""The float-float arithmetic of the merger (hi + lo pairs of float32 built from
Knuth's TwoSum, Dekker's Fast2Sum and the FMA TwoProduct; division by one
long-division step, square root by one Newton step from the float32 root),
modelled step by step in numpy float32 and checked against exact rational
arithmetic: every operation is accurate to a few 2^-46 relative, which is what
the merger's refit and compatibility tests rely on."""
from fractions import Fraction

import numpy as np

f32 = np.float32


def fma(a, b, c):
    """float32 fused multiply-add: the exact a*b + c rounded once (a*b is exact in float64)."""
    return f32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    return s, f32(f32(a - f32(s - bb)) + f32(b - bb))


def fast_two_sum(a, b):
    s = f32(a + b)
    return s, f32(b - f32(s - a))


def add(x, y):
    s, e = two_sum(x[0], y[0])
    return fast_two_sum(s, f32(e + f32(x[1] + y[1])))


def mul(x, y):
    p = f32(x[0] * y[0])
    e = fma(x[0], y[0], -p)
    e = fma(x[0], y[1], e)
    e = fma(x[1], y[0], e)
    return fast_two_sum(p, e)


def mul_f(x, b):
    p = f32(x[0] * b)
    return fast_two_sum(p, fma(x[1], b, fma(x[0], b, -p)))


def div(x, y):
    q1 = f32(x[0] / y[0])
    r = add(x, (-mul_f(y, q1)[0], -mul_f(y, q1)[1]))
    return fast_two_sum(q1, f32(r[0] / y[0]))


def sqrt(x):
    if not x[0] > 0:
        return f32(0), f32(0)
    r = f32(np.sqrt(x[0]))
    p = f32(r * r)
    res = f32(f32(f32(x[0] - p) - fma(r, r, -p)) + x[1])
    return fast_two_sum(r, f32(res * f32(f32(0.5) / r)))


def from_double(v):
    hi = f32(v)
    return hi, f32(v - float(hi))


def value(x):
    return Fraction(float(x[0])) + Fraction(float(x[1]))


def rel(got, want):
    return abs(got - want) / abs(want) if want != 0 else abs(got - want)


def test_float_float_operations_are_accurate_to_a_few_2_pow_minus_46():
    rng = np.random.default_rng(7)
    bound = Fraction(8, 2 ** 46)
    worst = {k: Fraction(0) for k in ("add", "mul", "div", "sqrt", "from")}
    for _ in range(3000):
        a = rng.uniform(-300, 300) * 10 ** rng.uniform(-3, 3)
        b = rng.uniform(-300, 300) * 10 ** rng.uniform(-3, 3)
        x, y = from_double(a), from_double(b)
        worst["from"] = max(worst["from"], rel(value(x), Fraction(a)))
        vx, vy = value(x), value(y)
        # additions are bounded relative to the terms (like an FP64 sum), the rest relative to the result
        s = add(x, y)
        worst["add"] = max(worst["add"], abs(value(s) - (vx + vy)) / (abs(vx) + abs(vy)))
        worst["mul"] = max(worst["mul"], rel(value(mul(x, y)), vx * vy))
        worst["div"] = max(worst["div"], rel(value(div(x, y)), vx / vy))
        sq = sqrt((abs(x[0]), x[1] if x[0] > 0 else -x[1]))
        want = abs(vx)
        got = value(sq) ** 2
        worst["sqrt"] = max(worst["sqrt"], rel(got, want) / 2)  # relative error of the root
    for k, v in worst.items():
        assert v < bound, (k, float(v) * 2 ** 46)
