"""Pins for the CPU oracle: checks against what the paper and mathematics
fix, independent of the oracle's own code.

* Brute force (Sec. II-B/C): exact rational arithmetic on tiny inputs,
  integer closed forms, hand-worked fixture (tests/golden), one-hot and
  Cauchy-Schwarz cases, tie rule, zero user, power-of-two and positive
  scaling (ranking invariance noted under Eq. max), item permutation.
* CBound (Eq. appx_bound): worked values (tests/golden), a dense scan of
  the angle interval of Eq. (max), the Lemma "upper bound in index lists"
  on every pair, the tight single-user case and the theta_b >= theta_ic
  branch.
* theta_b: a planar construction with a known maximum angle.
* k-means: exact means of integer blobs, objective non-increasing, every
  user at an argmin centroid.
* Maximus (Algorithm 1, Theorem "exact"): equal to brute force on every
  seed, and it must actually prune on clustered users.

Every pin is a function of an oracle handle, so the last test can plant a
mistake in a copy of the oracle source and check that some pin fails.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_dot(u, i):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(u, i))


def exact_topk(U, I, K):
    out = []
    for u in U:
        s = [(exact_dot(u, it), j) for j, it in enumerate(I)]
        s.sort(key=lambda t: (-t[0], t[1]))
        out.append([j for _, j in s[:K]])
    return np.array(out, dtype=np.int32)


# ---------------------------------------------------------------- brute force
def pin_exact_rational(o):
    rng = np.random.default_rng(7)
    for f in (1, 3, 7, 16):
        U = rng.standard_normal((5, f)).astype(np.float32)
        I = rng.standard_normal((37, f)).astype(np.float32)
        K = 6
        idx, sc = o.topk(U, I, K)
        assert (idx == exact_topk(U, I, K)).all()
        for u in range(U.shape[0]):
            for k in range(K):
                ex = exact_dot(U[u], I[idx[u, k]])
                sabs = sum(abs(float(a) * float(b)) for a, b in zip(U[u], I[idx[u, k]]))
                # sequential FP64 summation: |err| <= f * 2^-53 * sum |p|
                assert abs(float(Fraction(sc[u, k]) - ex)) <= f * 2.0**-53 * sabs * 1.0001


def pin_integer_closed_form(o):
    rng = np.random.default_rng(11)
    U = rng.integers(-20, 21, size=(9, 5)).astype(np.float32)
    I = rng.integers(-20, 21, size=(50, 5)).astype(np.float32)
    K = 7
    idx, sc = o.topk(U, I, K)
    for u in range(9):
        s = [(int(sum(int(a) * int(b) for a, b in zip(U[u], I[j]))), j) for j in range(50)]
        s.sort(key=lambda t: (-t[0], t[1]))
        assert [j for _, j in s[:K]] == idx[u].tolist()
        assert [float(v) for v, _ in s[:K]] == sc[u].tolist()


def pin_golden_hand_example(o):
    items, users, exp_idx, exp_sc = [], [], [], []
    for line in open(os.path.join(GOLDEN, "hand_example_f2.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        if line.startswith("item"):
            items.append([float(x) for x in line.split()[1:]])
        else:
            lhs, rhs = line.split("->")
            ids, scs = rhs.split("|")
            users.append([float(x) for x in lhs.split()[1:]])
            exp_idx.append([int(x) for x in ids.split()])
            exp_sc.append([float(x) for x in scs.split()])
    idx, sc = o.topk(np.array(users), np.array(items), 3)
    assert idx.tolist() == exp_idx
    assert sc.tolist() == exp_sc


def pin_one_hot(o):
    f = 6
    w = np.array([5.0, 3.0, 8.0, 1.0, 7.0, 2.0, 4.0, 6.0, 9.0, 0.5, 2.5, 3.5])
    I = np.zeros((12, f), dtype=np.float32)
    for j in range(12):
        I[j, j % f] = w[j]
    for k in range(f):
        U = np.zeros((1, f), dtype=np.float32)
        U[0, k] = 1.0
        idx, sc = o.topk(U, I, 1)
        cand = [j for j in range(12) if j % f == k]
        best = max(cand, key=lambda j: w[j])
        assert idx[0, 0] == best and sc[0, 0] == w[best]


def pin_cauchy_schwarz(o):
    rng = np.random.default_rng(3)
    I = rng.standard_normal((40, 8))
    I /= np.linalg.norm(I, axis=1, keepdims=True)
    I = I.astype(np.float32)
    for j in (0, 17, 39):
        idx, _ = o.topk(I[j:j + 1], I, 1)
        assert idx[0, 0] == j


def pin_ties_and_zero_user(o):
    rng = np.random.default_rng(5)
    base = rng.standard_normal((10, 4)).astype(np.float32)
    I = np.concatenate([base, base[[3, 7]]])  # items 10, 11 duplicate 3, 7
    U = rng.standard_normal((6, 4)).astype(np.float32)
    idx, sc = o.topk(U, I, 12)
    for u in range(6):
        row = idx[u].tolist()
        assert row.index(3) < row.index(10) and row.index(7) < row.index(11)
        assert row.index(10) == row.index(3) + 1 or sc[u, row.index(3) + 1] == sc[u, row.index(3)]
    idx, sc = o.topk(np.zeros((2, 4), dtype=np.float32), I, 5)
    assert idx.tolist() == [[0, 1, 2, 3, 4]] * 2 and (sc == 0).all()


def pin_scaling(o):
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U = synth.make_users(W, 1, n=64)
    I = synth.make_items(W, 1, n=300)
    idx, sc = o.topk(U, I, 10)
    idx2, sc2 = o.topk(U * np.float32(8.0), I * np.float32(2.0**-5), 10)
    assert (idx == idx2).all() and (sc2 == sc * 2.0**-2).all()
    idx3, _ = o.topk(U * np.float32(1.37), I, 10)
    assert (idx3 == idx).all()


def pin_permutation(o):
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U = synth.make_users(W, 2, n=32)
    I = synth.make_items(W, 2, n=200)
    perm = np.random.default_rng(1).permutation(200)
    idx, sc = o.topk(U, I, 8)
    idxp, scp = o.topk(U, I[perm], 8)
    assert (perm[idxp] == idx).all() and (scp == sc).all()


# ---------------------------------------------------------------- CBound
def _planar(r, phi_deg):
    p = math.radians(phi_deg)
    return np.array([r * math.cos(p), r * math.sin(p)], dtype=np.float32)


def pin_cbound_worked(o):
    c = np.array([1.0, 0.0])
    for line in open(os.path.join(GOLDEN, "cbound_worked.txt")):
        line = line.split("#")[0].strip()
        if not line:
            continue
        r, phi, tb, exp = (float(x) for x in line.split())
        got = o.cbound(c, _planar(r, phi), math.radians(tb))
        assert abs(got - exp) <= 1e-6 * max(1.0, abs(exp)), (line, got)


def pin_cbound_dense_angle_scan(o):
    """Eq. (max): the bound is max ||i|| cos(theta) over the interval
    [theta_ic - theta_b, theta_ic + theta_b]; scan it densely."""
    rng = np.random.default_rng(9)
    for _ in range(40):
        f = int(rng.integers(2, 9))
        c = rng.standard_normal(f)
        i = rng.standard_normal(f).astype(np.float32)
        tb = float(rng.uniform(0, math.pi))
        ni = float(np.linalg.norm(i.astype(np.float64)))
        cosic = float(np.dot(c, i.astype(np.float64)) / (np.linalg.norm(c) * ni))
        tic = math.acos(max(-1.0, min(1.0, cosic)))
        grid = np.linspace(tic - tb, tic + tb, 200001)
        scan = ni * np.cos(grid).max()
        got = o.cbound(c, i, tb)
        assert abs(got - scan) <= 1e-8 * ni, (got, scan)


def _clustered_small(seed, n_users=300, n_items=400, f=6, C=5):
    W = dict(synth.WORKLOADS["kdd-1000000x624961"])
    U = synth.clustered_users(n_users, f, seed, n_dirs=C, noise=0.15)
    I = synth.gaussian_rows(n_items, f, seed, synth.S_ITEMS, synth.S_ITEM_NORMS, W["item_norm"])
    return U, I


def pin_cbound_lemma(o):
    """Lemma (upper bound in index lists): ||u|| CBound(c, i, theta_b) >= u^T i
    for every user u of the cluster and every item i."""
    for seed in (0, 1):
        U, I = _clustered_small(seed)
        C = 5
        init = synth.distinct_ids(U.shape[0], C, seed, synth.S_INIT)
        cent, assign, _ = o.kmeans(U, C, 3, init)
        th = o.theta_b(U, cent, assign)
        B = o.cbound_all(cent, I, th)
        S = U.astype(np.float64) @ I.astype(np.float64).T
        nu = np.linalg.norm(U.astype(np.float64), axis=1)
        slack = 1e-12 * nu[:, None] * np.linalg.norm(I.astype(np.float64), axis=1)[None, :]
        assert (nu[:, None] * B[assign] + slack >= S).all()


def pin_cbound_tight_and_branch(o):
    rng = np.random.default_rng(4)
    u = rng.standard_normal(5).astype(np.float32)
    I = rng.standard_normal((30, 5)).astype(np.float32)
    c = u.astype(np.float64)  # single-user cluster at its own centroid: theta_b = 0
    th = o.theta_b(u[None, :], c[None, :], np.zeros(1, np.int32))
    assert th[0] <= 1e-7
    nu = float(np.linalg.norm(u.astype(np.float64)))
    for i in I:
        b = o.cbound(c, i, float(th[0]))
        assert abs(nu * b - float(exact_dot(u, i))) <= 1e-6 * nu * float(np.linalg.norm(i))
    # theta_ic <= theta_b: bound is ||i||
    i = _planar(3.0, 20.0)
    assert o.cbound(np.array([1.0, 0.0]), i, math.radians(25.0)) == pytest.approx(3.0, rel=1e-7)


def pin_theta_b_planar(o):
    angles = [30.0, -30.0, 10.0, -10.0, 0.0]
    U = np.array([_planar(1.0 + 0.1 * k, a) for k, a in enumerate(angles)], dtype=np.float32)
    cent = np.array([[2.0, 0.0]])
    th = o.theta_b(U, cent, np.zeros(len(angles), np.int32))
    assert abs(th[0] - math.radians(30.0)) < 1e-6


# ---------------------------------------------------------------- k-means
def pin_kmeans_blobs(o):
    a = np.array([[0, 0], [2, 0], [0, 2], [2, 2]], dtype=np.float32)
    b = a + np.float32(100.0)
    U = np.concatenate([a, b, a[:2] + np.float32(1.0)])
    cent, assign, _ = o.kmeans(U, 2, 1, np.array([0, 5]))
    assert (assign == np.array([0, 0, 0, 0, 1, 1, 1, 1, 0, 0])).all()
    m0 = np.concatenate([a, a[:2] + 1.0]).astype(np.float64).mean(axis=0)
    assert np.array_equal(cent[0], m0) and np.array_equal(cent[1], b.astype(np.float64).mean(axis=0))


def pin_kmeans_monotone_argmin(o):
    U, _ = _clustered_small(3, n_users=500, C=7)
    init = synth.distinct_ids(500, 7, 3, synth.S_INIT)
    cent, assign, trace = o.kmeans(U, 7, 6, init)
    assert all(trace[t + 1] <= trace[t] * (1 + 1e-12) for t in range(len(trace) - 1))
    # the objective after the final update is no larger than the last assignment's
    assert o.kmeans_objective(U, cent, assign) <= trace[-1] * (1 + 1e-12)
    # every user sits at a nearest centroid of the centroids it was assigned to:
    cent5, assign5, _ = o.kmeans(U, 7, 5, init)
    cent6, assign6, _ = o.kmeans(U, 7, 6, init)
    d = ((U[:, None, :].astype(np.float64) - cent5[None, :, :]) ** 2).sum(-1)
    assert (d[np.arange(500), assign6] <= d.min(axis=1) * (1 + 1e-12)).all()


# ---------------------------------------------------------------- Maximus
def pin_maximus_exact(o):
    for seed in (0, 1, 2):
        U, I = _clustered_small(seed, n_users=400, n_items=600, f=8, C=6)
        for C, K in ((1, 1), (6, 5), (12, 10)):
            init = synth.distinct_ids(U.shape[0], C, seed, synth.S_INIT)
            r = o.maximus(U, I, K, C, 3, init)
            idx, sc = o.topk(U, I, K)
            assert (r["idx"] == idx).all() and (r["score"] == sc).all()


def pin_maximus_prunes(o):
    U, I = _clustered_small(5, n_users=400, n_items=2000, f=8, C=4)
    init = synth.distinct_ids(400, 8, 5, synth.S_INIT)
    r = o.maximus(U, I, 5, 8, 3, init)
    assert r["visited"].mean() < 0.5 * I.shape[0]
    assert (r["visited"] >= 5).all()


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]


@pytest.mark.parametrize("pin", PINS, ids=[p.__name__ for p in PINS])
def test_pin(pin):
    pin(oracle.Oracle())


# Mistakes planted in a copy of the oracle source; each must trip a pin.
MUTANTS = {
    "dropped_last_term": ("for (int k = 0; k < f; ++k) s += (double)u[k] * (double)i[k];",
                          "for (int k = 0; k + 1 < f; ++k) s += (double)u[k] * (double)i[k];"),
    "tie_to_larger_index": ("return sa > sb || (sa == sb && ia < ib);",
                            "return sa > sb || (sa == sb && ia > ib);"),
    "bound_without_theta_b": ("return theta_b < theta_ic ? ni * cos(theta_ic - theta_b) : ni;",
                              "return ni * cos(theta_ic);"),
    "bound_sign_flip": ("return theta_b < theta_ic ? ni * cos(theta_ic - theta_b) : ni;",
                        "return theta_b < theta_ic ? ni * cos(theta_ic + theta_b) : ni;"),
    "walk_without_user_norm": ("double bound = nu * L[t].b * (1.0 + margin) + margin * nu * item_norm[it];",
                               "double bound = L[t].b * (1.0 + margin);"),
    "theta_b_min_not_max": ("if (th > theta_b[j]) theta_b[j] = th;",
                            "if (theta_b[j] == 0.0 || th < theta_b[j]) theta_b[j] = th;"),
    "kmeans_update_skipped": ("cent[(size_t)j * f + k] = sums[(size_t)j * f + k] / (double)cnt[j];",
                              "cent[(size_t)j * f + k] += 0.0 * sums[(size_t)j * f + k];"),
    "transposed_scores": ("row[j].s = oracle_dot(uv, I + (size_t)j * f, f);",
                          "row[j].s = oracle_dot(U + (size_t)(j % n_users) * f, I + (size_t)u % n_items * f, f);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name, tmp_path):
    src = open(oracle._SRC).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = oracle.compile_source(str(path), str(tmp_path / "libmutant.so"))
    o = oracle.Oracle(lib)
    failed = []
    for pin in PINS:
        try:
            pin(o)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"no pin caught planted mistake {name}"
