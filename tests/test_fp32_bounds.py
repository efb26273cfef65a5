"""CPU checks of the FP32 candidate pass's bounds on an exact emulation of
its float32 arithmetic (Fractions as the reference): the score is the
sequential fused multiply-add chain over k = 0..f-1, the norms are the
float32 sums of squares lifted by (1 + (f + 2) 2^-23), and
  H = fma(gamma nhat_u, nhat_i, s~) >= u^T i >= fma(-gamma nhat_u, nhat_i, s~) = L,
  gamma = (f + 4) 2^-23,
on random, cancelling, opposite and wide-dynamic-range rows."""
from fractions import Fraction
import math

import numpy as np
import pytest

f32 = np.float32


def rn32(q):
    """A Fraction rounded to the nearest float32 (ties to even)."""
    x = f32(float(q))
    best = None
    for c in (np.nextafter(x, f32(-np.inf)), x, np.nextafter(x, f32(np.inf))):
        d = abs(Fraction(float(c)) - q)
        even = (int(np.array([c], dtype=np.float32).view(np.uint32)[0]) & 1) == 0
        key = (d, not even)
        if best is None or key < best[0]:
            best = (key, c)
    return best[1]


def fma(a, b, c):
    return rn32(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def norm_ub(x):
    ss = f32(0)
    for v in x:
        ss = fma(v, v, ss)
    return f32(f32(math.sqrt(float(ss))) * f32(1.0 + (len(x) + 2) * 1.1920929e-07))


def pairs(rng, f, n):
    for t in range(n):
        kind = t % 4
        u = rng.standard_normal(f) * math.exp(rng.uniform(-4, 4))
        if kind == 0:
            i = rng.standard_normal(f)
        elif kind == 1:
            i = rng.standard_normal(f)
            i = i - (i @ u) / (u @ u) * u
        elif kind == 2:
            i = -u
        else:
            u = u * np.exp(rng.uniform(-10, 10, f))
            i = rng.standard_normal(f) * np.exp(rng.uniform(-10, 10, f))
        yield u.astype(np.float32), (i * math.exp(rng.uniform(-4, 4))).astype(np.float32)


def test_rn32_rounds_to_nearest_even():
    assert rn32(Fraction(1) + Fraction(1, 2 ** 24)) == 1.0            # tie to even
    assert rn32(Fraction(1) + Fraction(3, 2 ** 24)) == 1.0 + 2 ** -22  # tie to even upward
    assert rn32(Fraction(1, 3)) == f32(1 / 3)


@pytest.mark.parametrize("f", [1, 7, 50, 128])
def test_fp32_filter_bounds(f):
    rng = np.random.default_rng(200 + f)
    gamma = f32(f32(f + 4) * f32(5.9604645e-08) * f32(2.0))
    for u, i in pairs(rng, f, 80):
        s = f32(0)
        for a, b in zip(u, i):
            s = fma(a, b, s)
        gu = f32(gamma * norm_ub(u))
        ni = norm_ub(i)
        H = fma(gu, ni, s)
        L = fma(f32(-gu), ni, s)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, i))
        assert Fraction(float(H)) >= exact >= Fraction(float(L))
