"""Seeded synthetic factor matrices shaped like the paper's workloads.

This module holds only input generation: counter-based random numbers,
normal variates and row rescaling.  It contains none of the search
method's arithmetic, so both the CPU oracle and the CUDA path can take
their inputs from it without sharing any part of the computation.

Random stream: SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to a counter
(stream key + element index), giving 53-bit uniforms in (0, 1);
normals come from the Box-Muller transform.  Every array is a pure
function of (seed, stream id, shape), so any subset can be regenerated.

Workload recipes (the paper's datasets are not available, so these
stand in for them; shapes follow the paper's Table I):
  * ``gaussian_rows``: x[r, d] ~ N(0, 1) / sqrt(d + 1), d = 0..f-1,
    then each row rescaled to a norm drawn from LogNormal(mu, sigma).
  * ``clustered_users``: 256 random unit directions, mixture weights
    proportional to LogNormal(0, 1) draws; a user is its direction plus
    N(0, noise^2 I) noise, renormalised, times a LogNormal norm.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)
_STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# stream ids, one per independent random array of a workload
S_USERS, S_ITEMS, S_USER_NORMS, S_ITEM_NORMS = 1, 2, 3, 4
S_DIRS, S_DIR_WEIGHTS, S_USER_DIR, S_INIT, S_SAMPLE = 5, 6, 7, 8, 9
S_SERVE = 10


def _splitmix64(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = x + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _splitmix64(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
        return _splitmix64(np.array([s ^ (np.uint64(stream) * _STREAM_MUL)],
                                    dtype=np.uint64))[0]


def uniform(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniforms in (0, 1), float64, elements [offset, offset + n) of a stream."""
    key = _stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(offset, offset + n, dtype=np.uint64) * _GOLDEN + key
    bits = _splitmix64(ctr) >> np.uint64(11)
    return (bits.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, n: int, offset: int = 0) -> np.ndarray:
    """n standard normals (Box-Muller over consecutive uniform pairs)."""
    start = offset - (offset % 2)
    m = n + (offset - start)
    pairs = (m + 1) // 2
    u = uniform(seed, stream, 2 * pairs, 2 * (start // 2))
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    z = np.empty(2 * pairs, dtype=np.float64)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[offset - start: offset - start + n]


def _rescale_rows(x: np.ndarray, norms: np.ndarray) -> np.ndarray:
    cur = np.sqrt(np.einsum("ij,ij->i", x, x))
    cur[cur == 0.0] = 1.0
    return x * (norms / cur)[:, None]


def gaussian_rows(n: int, f: int, seed: int, stream: int,
                  norm_stream: int | None = None,
                  lognormal: tuple[float, float] | None = None,
                  chunk: int = 1 << 20, offset: int = 0) -> np.ndarray:
    """float32 [n][f]: N(0,1)/sqrt(d+1) entries, rows optionally rescaled
    to LogNormal(mu, sigma) norms drawn from ``norm_stream``.  The rows are
    rows [offset, offset + n) of the same recipe's larger matrix."""
    out = np.empty((n, f), dtype=np.float32)
    dim_scale = 1.0 / np.sqrt(np.arange(1, f + 1, dtype=np.float64))
    rows_per = max(1, chunk // max(f, 1))
    for r0 in range(0, n, rows_per):
        r1 = min(n, r0 + rows_per)
        z = normal(seed, stream, (r1 - r0) * f, (offset + r0) * f).reshape(r1 - r0, f)
        x = z * dim_scale[None, :]
        if lognormal is not None:
            mu, sigma = lognormal
            rho = np.exp(mu + sigma * normal(seed, norm_stream, r1 - r0, offset + r0))
            x = _rescale_rows(x, rho)
        out[r0:r1] = x.astype(np.float32)
    return out


def clustered_users(n: int, f: int, seed: int, n_dirs: int = 256,
                    noise: float = 0.2, lognormal=(0.0, 0.3),
                    chunk: int = 1 << 20, offset: int = 0) -> np.ndarray:
    """float32 [n][f] users drawn from a mixture of ``n_dirs`` angular
    clusters with uneven (LogNormal(0,1)-weighted) sizes: rows
    [offset, offset + n) of the recipe's larger matrix."""
    dirs = normal(seed, S_DIRS, n_dirs * f).reshape(n_dirs, f)
    dirs /= np.sqrt(np.einsum("ij,ij->i", dirs, dirs))[:, None]
    w = np.exp(normal(seed, S_DIR_WEIGHTS, n_dirs))
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    pick = np.searchsorted(cdf, uniform(seed, S_USER_DIR, n, offset), side="right")
    pick = np.minimum(pick, n_dirs - 1)
    out = np.empty((n, f), dtype=np.float32)
    rows_per = max(1, chunk // max(f, 1))
    mu, sigma = lognormal
    for r0 in range(0, n, rows_per):
        r1 = min(n, r0 + rows_per)
        z = normal(seed, S_USERS, (r1 - r0) * f, (offset + r0) * f).reshape(r1 - r0, f)
        x = dirs[pick[r0:r1]] + noise * z
        rho = np.exp(mu + sigma * normal(seed, S_USER_NORMS, r1 - r0, offset + r0))
        out[r0:r1] = _rescale_rows(x, rho).astype(np.float32)
    return out


def distinct_ids(n: int, count: int, seed: int, stream: int) -> np.ndarray:
    """``count`` distinct ids from range(n), int64, in draw order
    (the first ``count`` of a random permutation keyed by uniforms)."""
    if count > n:
        raise ValueError("count > n")
    keys = uniform(seed, stream, n)
    return np.argsort(keys, kind="stable")[:count].astype(np.int64)


# --------------------------------------------------------------------------
# Workloads.  Sizes follow the paper's Table I; recipes are stated above.
# --------------------------------------------------------------------------
WORKLOADS = {
    # small FP32 case: 2,048 users x 1,024 items, f=32
    "small-2048x1024-f32": dict(n_users=2048, n_items=1024, f=32, ks=(1, 10),
                                users="plain", item_norm=(0.0, 0.5)),
    # Netflix-shaped: 480,189 users x 17,770 items
    "netflix-480189x17770": dict(n_users=480189, n_items=17770, f=50,
                                 fs=(10, 50, 100), ks=(1, 5, 10, 50),
                                 users="lognormal", user_norm=(0.0, 0.3),
                                 item_norm=(0.0, 0.5)),
    # KDD-shaped clustered users: 1,000,000 x 624,961, f=51
    "kdd-1000000x624961": dict(n_users=1000000, n_items=624961, f=51, ks=(10,),
                               users="clustered", user_norm=(0.0, 0.3),
                               item_norm=(0.0, 0.7)),
    # serving: resident 1,000,000-item f=128 catalogue; requests of 1..4096
    # N(0,1)/sqrt(f) users with K in {1, 10, 100} (see serving_users)
    "serve-1000000x128": dict(n_users=4096, n_items=1000000, f=128, ks=(1, 10, 100),
                              users="serve", item_norm=(0.0, 0.5)),
    # R2-shaped large catalogue: 1,823,179 x 136,736, f=50
    "r2-1823179x136736": dict(n_users=1823179, n_items=136736, f=50,
                              ks=(1, 10, 50), users="lognormal",
                              user_norm=(0.0, 0.3), item_norm=(0.0, 1.0)),
}


def make_users(spec: dict, seed: int, n: int | None = None, f: int | None = None,
               offset: int = 0) -> np.ndarray:
    """The workload's users: rows [offset, offset + n) of its user recipe."""
    n = spec["n_users"] if n is None else n
    f = spec["f"] if f is None else f
    kind = spec["users"]
    if kind == "plain":
        return gaussian_rows(n, f, seed, S_USERS, offset=offset)
    if kind == "lognormal":
        return gaussian_rows(n, f, seed, S_USERS, S_USER_NORMS, spec["user_norm"], offset=offset)
    if kind == "clustered":
        return clustered_users(n, f, seed, lognormal=spec["user_norm"], offset=offset)
    if kind == "serve":
        return serving_users(n, f, seed, offset)
    raise ValueError(kind)


def make_items(spec: dict, seed: int, n: int | None = None, f: int | None = None) -> np.ndarray:
    n = spec["n_items"] if n is None else n
    f = spec["f"] if f is None else f
    return gaussian_rows(n, f, seed, S_ITEMS, S_ITEM_NORMS, spec["item_norm"])


def serving_users(n: int, f: int, seed: int, offset: int = 0) -> np.ndarray:
    """Serving-query users: N(0,1)/sqrt(f) entries (no per-dimension decay)."""
    z = normal(seed, S_SERVE, n * f, offset * f).reshape(n, f)
    return (z / np.sqrt(f)).astype(np.float32)
