"""CPU oracle for exact batch top-K MIPS -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never loads it.  The
arithmetic lives in ``mips_oracle.c`` (plain C, FP64, OpenMP over users);
this module builds it with gcc on first use and wraps it with ctypes.

Functions and the passages they follow:
  * ``topk``       -- the problem (Sec. II-B) by brute force (Sec. II-C):
                      sequential FP64 dots, full sort per user, ties to the
                      smaller item index.
  * ``dot``        -- one FP64 inner product u^T i.
  * ``kmeans``     -- Lloyd k-means used by ConstructIndex (Algorithm 1).
  * ``theta_b``    -- max user/centroid angle per cluster (Algorithm 1).
  * ``cbound``     -- Eq. (appx_bound), per (cluster, item).
  * ``maximus``    -- Algorithm 1 end to end (ConstructIndex + QueryIndex).
Pins for every function are in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mips_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libmips_oracle.so")
_lib = None


def compile_source(src: str, out: str) -> str:
    """gcc-compile one oracle C source into a shared library at ``out``."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp",
                           "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile mips_oracle.c into oracle/_build/libmips_oracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_source(_SRC, _LIB_PATH)
    return _LIB_PATH


def _bind(path: str):
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_dot.restype = dbl
    lib.oracle_dot.argtypes = [P, P, i32]
    lib.oracle_topk.restype = i32
    lib.oracle_topk.argtypes = [P, i64, P, i64, i32, i32, i32, P, P]
    lib.oracle_kmeans.restype = None
    lib.oracle_kmeans.argtypes = [P, i64, i32, i32, i32, P, i32, P, P, P]
    lib.oracle_kmeans_objective.restype = dbl
    lib.oracle_kmeans_objective.argtypes = [P, i64, i32, P, P]
    lib.oracle_theta_b.restype = None
    lib.oracle_theta_b.argtypes = [P, i64, i32, i32, P, P, P]
    lib.oracle_cbound.restype = dbl
    lib.oracle_cbound.argtypes = [P, P, i32, dbl]
    lib.oracle_cbound_all.restype = None
    lib.oracle_cbound_all.argtypes = [P, i32, P, i64, i32, P, i32, P]
    lib.oracle_maximus.restype = i32
    lib.oracle_maximus.argtypes = [P, i64, P, i64, i32, i32, i32, i32, P, i32, P, P, P, P, P, P]
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(build())
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def dot(u, i, lib=None) -> float:
    u, i = _f32(u), _f32(i)
    return (lib or _load()).oracle_dot(_ptr(u), _ptr(i), u.shape[-1])


def topk(U, I, K: int, nthreads: int = 0, return_threads: bool = False, lib=None):
    """Brute-force exact top-K: (idx int32 [nU][K], score float64 [nU][K])."""
    U, I = _f32(U), _f32(I)
    nU, f = U.shape
    nI = I.shape[0]
    if not (1 <= K <= nI) or I.shape[1] != f:
        raise ValueError("bad shapes or K")
    idx = np.empty((nU, K), dtype=np.int32)
    sc = np.empty((nU, K), dtype=np.float64)
    nt = (lib or _load()).oracle_topk(_ptr(U), nU, _ptr(I), nI, f, K, nthreads, _ptr(idx), _ptr(sc))
    return (idx, sc, nt) if return_threads else (idx, sc)


def kmeans(U, C: int, iters: int, init_ids, nthreads: int = 0, lib=None):
    """(centroids float64 [C][f], assign int32 [nU], objective per iteration)."""
    U = _f32(U)
    nU, f = U.shape
    init = np.ascontiguousarray(init_ids, dtype=np.int64)
    cent = np.empty((C, f), dtype=np.float64)
    assign = np.empty(nU, dtype=np.int32)
    trace = np.empty(max(iters, 1), dtype=np.float64)
    (lib or _load()).oracle_kmeans(_ptr(U), nU, f, C, iters, _ptr(init), nthreads, _ptr(cent), _ptr(assign), _ptr(trace))
    return cent, assign, trace[:iters]


def kmeans_objective(U, cent, assign, lib=None) -> float:
    U = _f32(U)
    cent = np.ascontiguousarray(cent, dtype=np.float64)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    return (lib or _load()).oracle_kmeans_objective(_ptr(U), U.shape[0], U.shape[1], _ptr(cent), _ptr(assign))


def theta_b(U, cent, assign, lib=None):
    U = _f32(U)
    cent = np.ascontiguousarray(cent, dtype=np.float64)
    assign = np.ascontiguousarray(assign, dtype=np.int32)
    out = np.empty(cent.shape[0], dtype=np.float64)
    (lib or _load()).oracle_theta_b(_ptr(U), U.shape[0], U.shape[1], cent.shape[0], _ptr(cent), _ptr(assign), _ptr(out))
    return out


def cbound(c, i, theta: float, lib=None) -> float:
    c = np.ascontiguousarray(c, dtype=np.float64)
    i = _f32(i)
    return (lib or _load()).oracle_cbound(_ptr(c), _ptr(i), i.shape[-1], float(theta))


def cbound_all(cent, I, theta, nthreads: int = 0, lib=None):
    cent = np.ascontiguousarray(cent, dtype=np.float64)
    I = _f32(I)
    th = np.ascontiguousarray(theta, dtype=np.float64)
    out = np.empty((cent.shape[0], I.shape[0]), dtype=np.float64)
    (lib or _load()).oracle_cbound_all(_ptr(cent), cent.shape[0], _ptr(I), I.shape[0], I.shape[1], _ptr(th), nthreads, _ptr(out))
    return out


def maximus(U, I, K: int, C: int, iters: int, init_ids, nthreads: int = 0, lib=None):
    """Algorithm 1 end to end.  Returns a dict with idx, score, visited,
    centroids, assign, theta_b, threads."""
    U, I = _f32(U), _f32(I)
    nU, f = U.shape
    nI = I.shape[0]
    if not (1 <= K <= nI) or I.shape[1] != f or not (1 <= C <= nU):
        raise ValueError("bad shapes, K or C")
    init = np.ascontiguousarray(init_ids, dtype=np.int64)
    idx = np.empty((nU, K), dtype=np.int32)
    sc = np.empty((nU, K), dtype=np.float64)
    vis = np.empty(nU, dtype=np.int64)
    cent = np.empty((C, f), dtype=np.float64)
    assign = np.empty(nU, dtype=np.int32)
    th = np.empty(C, dtype=np.float64)
    nt = (lib or _load()).oracle_maximus(_ptr(U), nU, _ptr(I), nI, f, K, C, iters, _ptr(init), nthreads,
                                _ptr(idx), _ptr(sc), _ptr(vis), _ptr(cent), _ptr(assign), _ptr(th))
    return dict(idx=idx, score=sc, visited=vis, centroids=cent, assign=assign, theta_b=th, threads=nt)


class Oracle:
    """The oracle bound to one compiled library (the default build, or a
    variant the tests compile with a deliberately planted mistake)."""

    def __init__(self, lib_path: str | None = None):
        self.lib = _bind(lib_path) if lib_path else _load()

    def __getattr__(self, name):
        fn = globals()[name]
        return lambda *a, **k: fn(*a, lib=self.lib, **k)
