"""CPU checks of the rounding margins of the GPU's Maximus bounds, on an
exact emulation of their float32 arithmetic (Fractions as the reference).

theta_b: the cluster's smallest member cosine, each computed as
d / (sqrt(su) sqrt(sc)) - (2f + 8) 2^-23 with FMA-summed d, su, sc (a lower
bound of the true smallest cosine).  CBound(i) = ||i|| g with
g = cos(theta_ic - theta_b) from the angle-difference identity, computed
from x = cos(theta_ic) + (2f + 8) 2^-23 and y = cos(theta_b) plus 2^-20 and
a final outward factor (Eq. appx_bound; the upper-bound lemma of Sec. III-B).
The lemma must hold as computed: u^T i <= ||u|| CBound(i) for every member
u and every item i -- checked on members spread over a cone and items at,
inside and outside its edge, aligned and opposite to the centroid."""
from fractions import Fraction
import math

import numpy as np
import pytest

f32 = np.float32


def rn32(q):
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


def dot_fma(a, b):
    s = f32(0)
    for x, y in zip(a, b):
        s = fma(x, y, s)
    return s


def sqrt32(x):
    return f32(np.sqrt(f32(x)))  # correctly rounded float32 square root


def cos_lower(u, c):
    f = len(u)
    d, su, sc = dot_fma(u, c), dot_fma(u, u), dot_fma(c, c)
    q = f32(d / f32(sqrt32(su) * sqrt32(sc)))
    return max(f32(q - f32(f32(2 * f + 8) * f32(5.9604645e-08) * f32(2.0))), f32(-1.0))


def norm_ub(x):
    ss = dot_fma(x, x)
    return f32(sqrt32(ss) * f32(1.0 + (len(x) + 2) * 1.1920929e-07))


def cbound(c, i, y):
    f = len(i)
    d, sc, si, ni = dot_fma(c, i), dot_fma(c, c), dot_fma(i, i), norm_ub(i)
    if si == 0:
        g = f32(0)
    elif sc == 0 or y <= -1:
        g = f32(1)
    else:
        x = f32(f32(d / f32(sqrt32(sc) * sqrt32(si))) + f32(f32(2 * f + 8) * f32(5.9604645e-08) * f32(2.0)))
        x = min(x, f32(1.0))
        if x >= y:
            g = f32(1)
        else:
            sx = sqrt32(f32(f32(1 - x) * f32(1 + x)))
            sy = sqrt32(f32(f32(1 - y) * f32(1 + y)))
            g = min(f32(1), f32(fma(x, y, f32(sx * sy)) + f32(9.5367432e-07)))
    if g >= 0:
        return f32(f32(ni * g) * f32(1.0 + 2.3841858e-07))
    return f32(f32(f32(ni * f32(1.0 - (2 * f + 4) * 1.1920929e-07)) * g) * f32(1.0 - 2.3841858e-07))


def lemma_holds(u, i, b):
    s = sum(Fraction(float(a)) * Fraction(float(v)) for a, v in zip(u, i))
    nu2 = sum(Fraction(float(a)) ** 2 for a in u)
    B = Fraction(float(b))
    if s <= 0 <= B:
        return True
    if s > 0:
        return B > 0 and s * s <= nu2 * B * B
    return B < 0 and s * s >= nu2 * B * B  # both negative: |s| >= ||u|| |B|


def unit(v):
    return v / np.linalg.norm(v)


@pytest.mark.parametrize("f,spread", [(2, 0.3), (8, 0.5), (32, 0.2), (51, 1.5)])
def test_cbound_lemma_as_computed(f, spread):
    rng = np.random.default_rng(f)
    c = unit(rng.standard_normal(f))
    members = [(unit(c + spread * rng.standard_normal(f)) * math.exp(rng.uniform(-2, 2))).astype(np.float32)
               for _ in range(40)]
    c32 = (c * 1.7).astype(np.float32)
    perp = rng.standard_normal(f)
    perp = unit(perp - (perp @ c) * c)
    # a member on the cone's edge in the (c, perp) plane: the items in that
    # plane just outside the edge are where the lemma is tight
    alpha = max(math.acos(max(-1.0, min(1.0, float(unit(u.astype(np.float64)) @ c)))) for u in members)
    members.append(((math.cos(alpha) * c + math.sin(alpha) * perp) * 2.3).astype(np.float32))
    y = min(cos_lower(u, c32) for u in members)
    theta_b = math.acos(max(-1.0, min(1.0, float(y))))
    items = []
    for _ in range(40):
        items.append(rng.standard_normal(f))
    for ang in (0.0, alpha * 0.5, alpha, alpha + 1e-6, alpha + 1e-3, alpha + 0.1, theta_b, theta_b * 1.5,
                math.pi / 2, alpha + math.pi / 2, math.pi - 1e-3, math.pi):
        items.append(math.cos(ang) * c + math.sin(ang) * perp)
    items = [(v * math.exp(rng.uniform(-2, 2))).astype(np.float32) for v in items]
    items.append(np.zeros(f, dtype=np.float32))
    for i in items:
        b = cbound(c32, i, y)
        for u in members:
            assert lemma_holds(u, i, b)


def test_zero_centroid_gives_norm_bound():
    i = np.array([3.0, -4.0], dtype=np.float32)
    b = cbound(np.zeros(2, dtype=np.float32), i, f32(0.5))
    assert float(b) >= 5.0
