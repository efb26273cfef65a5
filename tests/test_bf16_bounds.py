"""CPU checks of the BF16 candidate pass's bound arithmetic (the operand
rows' bound columns and the select's lower bound), on an emulation of the
same float32 / BF16 roundings with exact Fractions as the reference:

  * the operand row of u holds RN_bf16(u) and two bound columns (beta_u,
    nhat_u), the item row RN_bf16(i) and (nhat_i, alpha_i), each rounded up
    to BF16 after the float32 arithmetic that builds it;
  * whatever the tensor core's FP32 accumulation of the row product does
    within g (the sum of the magnitudes of the terms), the accumulated H is
    at least u^T i: no item of the exact top-K falls under the filter;
  * the select's lower bound L = (H - slack) - |H| 2^-22,
    slack = (2 A + g (nhat_u nhat_i + A)) (1 + 2^-18), never exceeds u^T i,
    so the threshold (the K-th largest L) never passes the K-th exact score.
Inputs: random rows of several norms and dimensions, near-parallel and
opposite pairs, rows with wide dynamic range, rows exactly representable
in BF16."""
from fractions import Fraction
import math

import numpy as np
import pytest

f32 = np.float32
U24 = 2.0 ** -24


def row_len(f):
    n = f + 2
    if n <= 16:
        return 16
    if n <= 32:
        return 32
    if n <= 64:
        return 64
    full, rem = n // 64 * 64, n % 64
    return full if rem == 0 else full + (16 if rem <= 16 else 32 if rem <= 32 else 64)


def bf16_rn(x):
    b = np.array([x], dtype=np.float32).view(np.uint32)[0]
    b = (int(b) + 0x7FFF + ((int(b) >> 16) & 1)) & 0xFFFF0000
    return np.array([b], dtype=np.uint32).view(np.float32)[0]


def bf16_ru_pos(x):  # x > 0
    b = int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    if b & 0xFFFF:
        b = (b & 0xFFFF0000) + 0x10000
    return np.array([b], dtype=np.uint32).view(np.float32)[0]


def f32_ru(q):  # Fraction -> float32 rounded up
    x = f32(float(q))
    if Fraction(float(x)) < q:
        x = np.nextafter(x, f32(np.inf))
    return x


def f32_rn(q):  # Fraction -> float32 round to nearest (via double: q is exact in double here)
    return f32(float(q))


def fma_rn(a, b, c):
    return f32_rn(Fraction(float(a)) * Fraction(float(b)) + Fraction(float(c)))


def norm_ub(ss, f):
    return f32(f32(math.sqrt(float(ss))) * f32(1.0 + (f + 2) * 1.1920929e-07))


def operand(x, role):
    """(RN_bf16 row, first bound column, second bound column) as prep.cu builds them."""
    f = len(x)
    fp = row_len(f)
    t = np.array([bf16_rn(v) for v in x], dtype=np.float32)
    d = (x - t).astype(np.float32)  # exact: t has 8 significant bits of x
    ss_x = ss_t = ss_d = f32(0)
    for k in range(f):
        ss_x = fma_rn(x[k], x[k], ss_x)
        ss_t = fma_rn(t[k], t[k], ss_t)
        ss_d = fma_rn(d[k], d[k], ss_d)
    g = f32(f32(fp + 4) * f32(9.5367432e-07) + f32(f) * f32(8.8817842e-16))
    nhat = max(norm_ub(ss_x, f), norm_ub(ss_t, f))
    errn = norm_ub(ss_d, f)
    nhat_b = bf16_ru_pos(nhat)
    inner = f32_ru(Fraction(float(g)) * Fraction(float(nhat)) + Fraction(float(errn)))
    eb_b = bf16_ru_pos(f32_ru(Fraction(float(inner)) * Fraction(float(f32(1.0) + g))))
    return (t, eb_b, nhat_b, g) if role == 0 else (t, nhat_b, eb_b, g)


def lower(H, beta_u, nhat_u, nhat_i, alpha_i, g):
    A = fma_rn(beta_u, nhat_i, f32(nhat_u * alpha_i))
    nn = f32(nhat_u * nhat_i)
    slack = f32(fma_rn(f32(2.0), A, f32(g * f32(nn + A))) * f32(1.0 + 3.814697265625e-06))
    return f32(f32(H - slack) - f32(abs(H) * f32(2.384185791015625e-07)))


def pairs(rng, f, n):
    for t in range(n):
        kind = t % 5
        u = rng.standard_normal(f) * math.exp(rng.uniform(-3, 3))
        if kind == 0:
            i = rng.standard_normal(f)
        elif kind == 1:
            i = u + 1e-3 * rng.standard_normal(f)
        elif kind == 2:
            i = -u
        elif kind == 3:
            u = u * np.exp(rng.uniform(-8, 8, f))
            i = rng.standard_normal(f) * np.exp(rng.uniform(-8, 8, f))
        else:
            u = np.round(u * 4) / 4
            i = np.round(rng.standard_normal(f) * 4) / 4
        yield u.astype(np.float32), (i * math.exp(rng.uniform(-3, 3))).astype(np.float32)


@pytest.mark.parametrize("f", [3, 16, 50, 100, 128])
def test_filter_upper_and_lower_bounds(f):
    rng = np.random.default_rng(100 + f)
    for u, i in pairs(rng, f, 60):
        ut, beta_u, nhat_u, g = operand(u, 0)
        it, nhat_i, alpha_i, _ = operand(i, 1)
        exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, i))
        terms = [Fraction(float(a)) * Fraction(float(b)) for a, b in zip(ut, it)]
        A = Fraction(float(beta_u)) * Fraction(float(nhat_i)) + Fraction(float(nhat_u)) * Fraction(float(alpha_i))
        H_exact = sum(terms) + A
        err = Fraction(float(g)) * (sum(abs(x) for x in terms) + A)
        # any FP32 accumulation within the error bound stays above u^T i
        assert H_exact - err >= exact
        # the lower bound from any accumulated value in that range stays below u^T i
        for H in (f32_ru(H_exact + err), f32(float(H_exact)), f32_ru(H_exact - err)):
            L = lower(H, beta_u, nhat_u, nhat_i, alpha_i, g)
            assert Fraction(float(L)) <= exact


def test_bf16_helpers():
    assert bf16_rn(f32(1.0)) == 1.0
    assert bf16_rn(f32(1.0 + 2 ** -8)) == 1.0             # tie to even
    assert bf16_rn(f32(1.0 + 3 * 2 ** -8)) == 1.0 + 2 ** -6
    assert bf16_ru_pos(f32(1.0 + 2 ** -20)) == 1.0 + 2 ** -7
    assert bf16_ru_pos(f32(1.5)) == 1.5
    assert row_len(50) == 64 and row_len(128) == 144 and row_len(100) == 128 and row_len(14) == 16
