"""CPU checks of the per-cluster list keys (the 16-bit radix sort of the
CBound keys and the bound each list rank carries), on a bit-exact model of
the key transform: a float's descending key keeps its order; a rank's bound
is the upper edge of its 16-bit bucket, which is never below the bound of
any item at that rank or later, never increases along the list, and for
positive bounds lies at most 2^-7 above the item's own bound."""
import numpy as np

M = 0xFFFFFFFF
KEY_BITS = 16


def float_desc_key(x):
    b = int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    asc = (~b & M) if (b & 0x80000000) else (b | 0x80000000)
    return ~asc & M


def ord2f(o):
    b = (o & 0x7FFFFFFF) if (o & 0x80000000) else (~o & M)
    return float(np.array([b], dtype=np.uint32).view(np.float32)[0])


def bucket_edge(key):
    mask = ~((1 << (32 - KEY_BITS)) - 1) & M
    return ord2f(~(key & mask) & M)


def sample(rng, n):
    x = np.concatenate([
        rng.standard_normal(n) * np.exp(rng.uniform(-30, 30, n)),
        np.array([0.0, -0.0, 1.0, -1.0, 1e-40, -1e-40, 3.4e38, -3.4e38]),
        np.nextafter(np.float32(1.0), np.float32(2.0)) * np.ones(3),
    ]).astype(np.float32)
    return x


def test_keys_order_and_bucket_edges():
    rng = np.random.default_rng(0)
    x = sample(rng, 20000)
    keys = np.array([float_desc_key(v) for v in x], dtype=np.uint64)
    # descending keys: a larger float has a smaller key (ties only for equal values, +0 == -0 aside)
    order = np.argsort(keys, kind="stable")
    xs = x[order].astype(np.float64)
    assert (np.diff(xs) <= 0).all()
    # the 16-bit sort: stable by the top bits only; edges along the list
    top = keys >> np.uint64(32 - KEY_BITS)
    order16 = np.argsort(top, kind="stable")
    edges = np.array([bucket_edge(int(k)) for k in keys[order16]])
    vals = x[order16].astype(np.float64)
    assert (np.diff(edges) <= 0).all()                       # non-increasing along the list
    suffix_max = np.maximum.accumulate(vals[::-1])[::-1]
    assert (edges >= suffix_max).all()                       # covers every later item
    pos = vals > 1e-37
    assert (edges[pos] <= vals[pos] * (1 + 2.0 ** -7)).all()  # at most 2^-7 looser for positive bounds
