"""CPU checks of the constants in the exactness argument of the fast path
(the rescore's compensated dot product and its tie-check margin), on a
bit-faithful float32 emulation of the rescore's arithmetic:

  * TwoProduct (p = fl(a b), e = fma(a, b, -p)) and TwoSum split exactly;
  * the compensated dot product (Ogita, Rump, Oishi 2005, Algorithm Dot2:
    TwoProduct + TwoSum per term, errors summed in float32, hi + lo in
    double) stays within (2 gamma_2f gamma_f + (f + 2) 2^-53) ||u|| ||i|| of
    the exact u^T i -- the per-score bound whose double is the rescore's
    relative error and whose quadruple is its tie-check gap -- on random,
    cancelling and wide-dynamic-range inputs;
  * the FP64 definition's sequential sum is within the same bound, so two
    compensated scores further apart than the gap are ordered as the
    definition orders them.
Exact values are Python Fractions."""
from fractions import Fraction

import numpy as np
import pytest

f32 = np.float32


def two_product(a, b):
    p = f32(a * b)
    e = f32(Fraction(float(a)) * Fraction(float(b)) - Fraction(float(p)))  # fma(a, b, -p), exact
    return p, e


def two_sum(a, b):
    s = f32(a + b)
    bb = f32(s - a)
    e = f32(f32(a - f32(s - bb)) + f32(b - bb))
    return s, e


def dot2(u, v):
    hi, lo = f32(0), f32(0)
    for a, b in zip(u, v):
        p, pe = two_product(a, b)
        s, se = two_sum(hi, p)
        hi = s
        lo = f32(lo + f32(pe + se))
    return float(hi) + float(lo)


def exact_dot(u, v):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, v))


def seq_f64(u, v):
    s = 0.0
    for a, b in zip(u, v):
        s = s + float(a) * float(b)
    return s


def bound(f):
    uf = 2.0 ** -24
    gf = f * uf / (1 - f * uf)
    g2f = 2 * f * uf / (1 - 2 * f * uf)
    return 2 * g2f * gf + (f + 2) * 2.0 ** -53


def cases(rng, f, n):
    for t in range(n):
        kind = t % 3
        u = rng.standard_normal(f)
        if kind == 0:       # random
            v = rng.standard_normal(f)
        elif kind == 1:     # heavy cancellation: v nearly orthogonal to u
            v = rng.standard_normal(f)
            v = v - (v @ u) / (u @ u) * u + 1e-7 * rng.standard_normal(f)
        else:               # wide dynamic range
            u = u * np.exp(rng.uniform(-20, 20, f))
            v = rng.standard_normal(f) * np.exp(rng.uniform(-20, 20, f))
        yield u.astype(np.float32), v.astype(np.float32)


def test_error_free_transformations():
    rng = np.random.default_rng(0)
    for _ in range(2000):
        a, b = (rng.standard_normal(2) * np.exp(rng.uniform(-30, 30, 2))).astype(np.float32)
        p, e = two_product(a, b)
        assert Fraction(float(p)) + Fraction(float(e)) == Fraction(float(a)) * Fraction(float(b))
        s, e2 = two_sum(a, b)
        assert Fraction(float(s)) + Fraction(float(e2)) == Fraction(float(a)) + Fraction(float(b))


@pytest.mark.parametrize("f", [2, 17, 50, 128])
def test_dot2_and_fp64_within_the_rescore_bound(f):
    rng = np.random.default_rng(f)
    worst = 0.0
    for u, v in cases(rng, f, 240):
        ex = exact_dot(u, v)
        scale = float(np.linalg.norm(u.astype(np.float64)) * np.linalg.norm(v.astype(np.float64)))
        e_dot2 = abs(Fraction(dot2(u, v)) - ex)
        e_f64 = abs(Fraction(seq_f64(u, v)) - ex)
        b = Fraction(bound(f)) * Fraction(scale)
        assert e_dot2 <= b and e_f64 <= b
        worst = max(worst, float(e_dot2) / (bound(f) * scale))
    assert worst < 1.0


def test_gap_above_margin_keeps_the_definitions_order():
    # two items whose compensated scores differ by more than twice the bound
    # (the rescore's tie-check gap is twice its doubled bound) rank as the
    # FP64 definition ranks them
    rng = np.random.default_rng(7)
    f = 50
    for _ in range(300):
        u = rng.standard_normal(f).astype(np.float32)
        a = rng.standard_normal(f).astype(np.float32)
        b = (a + 1e-5 * rng.standard_normal(f)).astype(np.float32)
        sa, sb = dot2(u, a), dot2(u, b)
        nu = float(np.linalg.norm(u.astype(np.float64)))
        nmax = max(float(np.linalg.norm(a.astype(np.float64))), float(np.linalg.norm(b.astype(np.float64))))
        gap = 2 * (2 * bound(f)) * nu * nmax
        if abs(sa - sb) > gap:
            assert (sa > sb) == (seq_f64(u, a) > seq_f64(u, b))
