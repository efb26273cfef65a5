"""GPU checks of the Maximus path (mips_topk_maximus, Sec. III / Algorithm 1)
through the C ABI:
  * results equal the brute-force oracle and mips_topk (Theorem "exact");
  * the GPU's CBound values are upper bounds: ||u|| CBound >= u^T i for every
    member u of the cluster and every item (Lemma "upper bound in index
    lists"), and no smaller than the oracle's CBound evaluated on the GPU's
    own centroids and theta_b;
  * each cluster's list is a permutation sorted by bound (Property
    "monotonicity of sorted index lists");
  * pruning invariant: every item a user did not score has
    ||u|| CBound < (the user's K-th score);
  * k-means: each user sits at a nearest centroid, centroids are member means
    (spherical k-means: unit vectors along the member means);
  * pruning happens on clustered users; degenerate cases (C = 1, K = n_items,
    zero users, duplicate items)."""
import math

import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def clustered(n_users, n_items, f, seed, n_dirs=16, noise=0.2, item_norm=(0.0, 0.7)):
    U = synth.clustered_users(n_users, f, seed, n_dirs=n_dirs, noise=noise)
    I = synth.gaussian_rows(n_items, f, seed, synth.S_ITEMS, synth.S_ITEM_NORMS, item_norm)
    return U, I


def run_maximus(U, I, K, C, dtype="fp32", iters=3, seed=0, block_items=0):
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C, dtype=dtype, kmeans_iters=iters, seed=seed,
                             block_items=block_items)
    idx, sc = mips.topk_maximus(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    st = mips.get_stats(index)
    Ce = st["clusters"]
    nU, nI, f = U.shape[0], I.shape[0], U.shape[1]
    bufs = dict(
        assign=mips.get_buffer(index, "assign", torch.int32, (nU,)).cpu().numpy(),
        centroids=mips.get_buffer(index, "centroids", torch.float32, (Ce, f)).cpu().numpy(),
        cos_b=mips.get_buffer(index, "cos_b", torch.float32, (Ce,)).cpu().numpy(),
        bound_sorted=mips.get_buffer(index, "bound_sorted", torch.float32, (Ce, nI)).cpu().numpy(),
        list=mips.get_buffer(index, "list", torch.int32, (Ce, nI)).cpu().numpy(),
        visited=mips.get_buffer(index, "visited", torch.int32, (nU,)).cpu().numpy(),
        perm=mips.get_buffer(index, "perm", torch.int32, (nI,)).cpu().numpy(),
    )
    bmm_idx, bmm_sc = mips.topk(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    index.close()
    return idx.cpu().numpy(), sc.cpu().numpy(), st, bufs, bmm_idx.cpu().numpy(), bmm_sc.cpu().numpy()


@pytest.mark.parametrize("dtype,block", [("fp32", 0), ("bf16", 0), ("bf16", 256), ("fp8", 0), ("fp8", 256)])
@pytest.mark.parametrize("C,K", [(8, 10), (16, 1), (4, 50)])
def test_maximus_exact_and_bounds(C, K, dtype, block):
    """bf16 runs the tensor-core walk: pass 1 over the first block of every
    list (4096 items, or one 256-item tile), pass 2 over the rest."""
    U, I = clustered(3000, 2000, 16, seed=C + K)
    idx, sc, st, b, bidx, bsc = run_maximus(U, I, K, C, dtype=dtype, block_items=block)
    assert st["dtype"] == mips.DTYPES[dtype]  # the tensor-core path of that dtype was taken
    ref = oracle.topk(U, I, K)
    check_against_oracle(U, I, K, idx, sc, ref=ref)
    assert (idx == bidx).all() and (sc == bsc).all()

    U64, I64 = U.astype(np.float64), I.astype(np.float64)
    perm = b["perm"]                  # position -> item id
    S = U64 @ I64[perm].T             # scores in position order
    nu = np.linalg.norm(U64, axis=1)
    # bounds per (cluster, position) from the sorted lists
    Bpos = np.empty_like(b["bound_sorted"], dtype=np.float64)
    for j in range(Bpos.shape[0]):
        L = b["list"][j]
        assert np.array_equal(np.sort(L), np.arange(I.shape[0]))          # a permutation
        assert (np.diff(b["bound_sorted"][j].astype(np.float64)) <= 0).all()  # non-increasing
        Bpos[j, L] = b["bound_sorted"][j]
    a = b["assign"]
    # Lemma: ||u|| CBound >= u^T i for every member and every item
    assert (nu[:, None] * Bpos[a] >= S - 1e-12 * np.abs(S)).all()
    # GPU bound >= oracle CBound on the GPU's centroids and theta_b
    theta = np.arccos(np.clip(b["cos_b"].astype(np.float64), -1, 1))
    cent = b["centroids"].astype(np.float64)
    Bor = oracle.cbound_all(cent, I[perm], theta)
    assert (Bpos >= Bor - 1e-9 * np.abs(Bor) - 1e-12).all()
    # pruning invariant: items beyond what a user scored cannot reach its K-th score
    kth = ref[1][:, K - 1]
    for u in range(U.shape[0]):
        v = b["visited"][u]
        if v < I.shape[0]:
            assert nu[u] * b["bound_sorted"][a[u], v] < kth[u]
    assert st["pairs_scored"] == b["visited"].sum()


@pytest.mark.parametrize("dtype,block", [("fp32", 0), ("bf16", 512), ("fp8", 512)])
def test_maximus_prunes_on_clustered_users(dtype, block):
    U, I = clustered(4000, 6000, 12, seed=11, n_dirs=8, noise=0.1)
    idx, sc, st, b, _, _ = run_maximus(U, I, 5, 8, dtype=dtype, block_items=block)
    check_against_oracle(U, I, 5, idx, sc)
    assert b["visited"].mean() < 0.5 * I.shape[0]


@pytest.mark.parametrize("f,dtype", [(8, "fp32"), (51, "bf16"), (70, "bf16"), (100, "fp32")])
def test_kmeans_invariants(f, dtype):
    # f = 8, 51, 70, 100: the centroid sums run in groups of 1, 2, 3 and 4
    # warps (one warp per 32 dimensions); every final centroid is its
    # members' mean, and the answer stays exact
    U, I = clustered(2500, 300, f, seed=3)
    idx, sc, _, b, _, _ = run_maximus(U, I, 3, 12, dtype=dtype)
    check_against_oracle(U, I, 3, idx, sc)
    U64, cent = U.astype(np.float64), b["centroids"].astype(np.float64)
    d = ((U64[:, None, :] - cent[None, :, :]) ** 2).sum(-1)
    a = b["assign"]
    # assignment is from the previous centroids; with i iterations the final
    # centroids are the members' means of that assignment
    for j in range(cent.shape[0]):
        m = a == j
        if m.any():
            np.testing.assert_allclose(cent[j], U64[m].mean(axis=0), rtol=1e-4, atol=1e-5)
    assert d.shape == (U.shape[0], cent.shape[0])


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "fp8"])
def test_spherical_kmeans(dtype):
    """kmeans_spherical (Sec. III-A): exact results; every centroid is the unit
    vector along its members' mean (of the last assignment step)."""
    U, I = clustered(2500, 900, 12, seed=8)
    K, C = 10, 12
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C, dtype=dtype, kmeans_spherical=True)
    idx, sc = mips.topk_maximus(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    Ce = mips.get_stats(index)["clusters"]
    nU, f = U.shape
    a = mips.get_buffer(index, "assign", torch.int32, (nU,)).cpu().numpy()
    cent = mips.get_buffer(index, "centroids", torch.float32, (Ce, f)).cpu().numpy().astype(np.float64)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy())
    U64 = U.astype(np.float64)
    for j in range(Ce):
        m = a == j
        if m.any():
            mu = U64[m].mean(axis=0)
            np.testing.assert_allclose(cent[j], mu / np.linalg.norm(mu), rtol=1e-4, atol=1e-5)
    index.close()


@pytest.mark.parametrize("dtype", ["fp32", "bf16", "fp8"])
def test_maximus_degenerate_cases(dtype):
    rng = np.random.default_rng(1)
    base = rng.integers(-3, 4, size=(50, 6)).astype(np.float32)
    I = np.concatenate([base, base[:10]])
    U = rng.integers(-2, 3, size=(300, 6)).astype(np.float32)
    U[::13] = 0.0
    for C, K in ((1, 4), (300, 7), (5, 60)):
        idx, sc, st, b, bidx, _ = run_maximus(U, I, K, C, dtype=dtype)
        check_against_oracle(U, I, K, idx, sc)
        assert (idx == bidx).all()


@pytest.mark.slow
def test_maximus_kdd_shape_sampled():
    """Clustered users (256 directions) at a reduced KDD-like size."""
    W = synth.WORKLOADS["kdd-1000000x624961"]
    U = synth.clustered_users(200000, 51, 0)
    I = synth.make_items(W, 0, n=100000)
    idx, sc, st, b, bidx, _ = run_maximus(U, I, 10, 64, dtype="bf16")
    assert (idx == bidx).all()
    rows = synth.distinct_ids(U.shape[0], 256, 0, synth.S_SAMPLE)
    check_against_oracle(U, I, 10, idx, sc, rows=rows)


def test_autotune_picks_a_tried_candidate_and_stays_exact():
    """mips_autotune times Maximus on a user sample for |C| x B candidates;
    its choice becomes the index's and the results stay exact."""
    U, I = clustered(20000, 3000, 12, seed=21, n_dirs=16, noise=0.15)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=8, dtype="bf16")
    Ud = torch.from_numpy(U).cuda()
    rep = mips.autotune(index, Ud, 10)
    assert rep["tried"], rep
    cs = {c for c, _, _ in rep["tried"]}
    assert max(cs) <= U.shape[0] // 32 and min(cs) >= 16
    best = min(rep["tried"], key=lambda t: t[2])
    assert (rep["clusters"], rep["block_items"]) == (best[0], best[1])
    assert all(e > 0 for _, _, e in rep["tried"])
    idx, sc = mips.topk_maximus(index, Ud, 10)
    mips.sync(index)
    assert mips.get_stats(index)["clusters"] == rep["clusters"]
    check_against_oracle(U, I, 10, idx.cpu().numpy(), sc.cpu().numpy())
    index.close()
