"""GPU checks of fitted centroids (mips_fit_clusters; Sec. III-E, practical
usage: cluster an initial set of users once, then only assign later users
to the extant centroids):
  * Maximus results stay equal to the brute-force oracle when k-means ran on
    a 10 % sample and the call's users are only assigned (both walks);
  * each user sits at a nearest fitted centroid, and the kept clusters are
    exactly those that received users (small batches walk few clusters);
  * CBound stays an upper bound for every member of every kept cluster;
  * dropping the fit returns to per-call clustering; graphs captured before
    a fit are not replayed after it; servers and autotune see the fit."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def data(n_users, n_items, f, seed):
    U = synth.clustered_users(n_users, f, seed, n_dirs=16, noise=0.2)
    I = synth.gaussian_rows(n_items, f, seed, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    return U, I


def kmeans_err_bound(U64, cent):
    """Bound on |computed - exact| of u . c_j - ||c_j||^2 / 2 for the tensor-core
    assignment: BF16 operands (unit roundoff 2^-8) give at most
    (2^-7 + 2^-16) ||u|| ||c_j|| for the product and 2^-8 ||c_j||^2 / 2 for the
    bias column, the FP32 sum f 2^-23 ||u|| ||c_j|| more; 2^-6 (||u|| ||c_j|| +
    ||c_j||^2 / 2) covers them twice over."""
    nu = np.linalg.norm(U64, axis=1)[:, None]
    nc = np.linalg.norm(cent, axis=1)[None, :]
    return 2.0 ** -6 * (nu * nc + 0.5 * nc * nc)


def fitted_index(I, U_fit, C, dtype="bf16", block_items=0):
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C, dtype=dtype, block_items=block_items)
    mips.fit_clusters(index, torch.from_numpy(U_fit).cuda())
    return index


@pytest.mark.parametrize("dtype,block", [("bf16", 0), ("bf16", 256), ("fp32", 0)])
def test_fit_on_sample_then_assign_is_exact(dtype, block):
    U, I = data(4000, 2500, 24, seed=11)
    K, C = 10, 16
    index = fitted_index(I, U[:400], C, dtype=dtype, block_items=block)
    Ud = torch.from_numpy(U).cuda()
    idx, sc = mips.topk_maximus(index, Ud, K)
    mips.sync(index)
    st = mips.get_stats(index)
    Ce, nU, nI, f = st["clusters"], U.shape[0], I.shape[0], U.shape[1]
    assert 1 <= Ce <= C
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy())

    assign = mips.get_buffer(index, "assign", torch.int32, (nU,)).cpu().numpy()
    cent = mips.get_buffer(index, "centroids", torch.float32, (Ce, f)).cpu().numpy().astype(np.float64)
    bound = mips.get_buffer(index, "bound_sorted", torch.float32, (Ce, nI)).cpu().numpy().astype(np.float64)
    lists = mips.get_buffer(index, "list", torch.int32, (Ce, nI)).cpu().numpy()
    perm = mips.get_buffer(index, "perm", torch.int32, (nI,)).cpu().numpy()
    # every kept slot holds users; every user at a nearest kept centroid
    assert set(np.unique(assign).tolist()) == set(range(Ce))
    U64 = U.astype(np.float64)
    obj = U64 @ cent.T - 0.5 * (cent * cent).sum(axis=1)[None, :]
    mine = obj[np.arange(nU), assign]
    if dtype == "bf16":  # tcgen05 assignment: each objective within its BF16 bound (kmeans_err_bound)
        e = kmeans_err_bound(U64, cent)
        assert (mine + e[np.arange(nU), assign] >= (obj - e).max(axis=1)).all()
    else:
        assert (mine >= obj.max(axis=1) - 1e-4 * (1 + np.abs(obj).max(axis=1))).all()
    # CBound upper bound for every member and item
    S = U64 @ I.astype(np.float64)[perm].T
    nu = np.linalg.norm(U64, axis=1)
    for j in range(Ce):
        Bpos = np.empty(nI)
        Bpos[lists[j]] = bound[j]
        m = assign == j
        assert (nu[m, None] * Bpos[None, :] * (1 + 1e-5) + 1e-6 >= S[m]).all()
    index.close()


def test_small_batches_walk_only_used_clusters():
    U, I = data(3000, 1500, 16, seed=5)
    C, K = 64, 5
    index = fitted_index(I, U[:2000], C)
    for n in (1, 3, 37):
        Un = U[2000:2000 + n]
        idx, sc = mips.topk_maximus(index, torch.from_numpy(Un).cuda(), K)
        mips.sync(index)
        st = mips.get_stats(index)
        assert 1 <= st["clusters"] <= n
        check_against_oracle(Un, I, K, idx.cpu().numpy(), sc.cpu().numpy())
    index.close()


def test_clear_graphs_servers_autotune():
    U, I = data(6000, 1200, 16, seed=9)
    C, K = 8, 10
    ref = oracle.topk(U, I, K)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=C)
    Ud = torch.from_numpy(U).cuda()
    oi = torch.empty((U.shape[0], K), dtype=torch.int32, device="cuda")
    osc = torch.empty((U.shape[0], K), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):  # plain + capture, then a replay
            mips.topk_graph(index, Ud, K, method="maximus", out_idx=oi, out_score=osc, stream=s)
        mips.sync(index, s)
        launches_per_call = mips.get_stats(index)["launches"]
        check_against_oracle(U, I, K, oi.cpu().numpy(), osc.cpu().numpy(), ref=ref)

        mips.fit_clusters(index, Ud[:600], stream=s)
        oi.zero_()
        for _ in range(2):  # the fit invalidates the captured graph
            mips.topk_graph(index, Ud, K, method="maximus", out_idx=oi, out_score=osc, stream=s)
        mips.sync(index, s)
        st = mips.get_stats(index)
        assert st["launches"] != launches_per_call  # assignment only, no k-means iterations
        check_against_oracle(U, I, K, oi.cpu().numpy(), osc.cpu().numpy(), ref=ref)

        rep = mips.autotune(index, Ud, K, stream=s)
        assert rep["clusters"] == C and all(c == C for c, _, _ in rep["tried"])
        assert index_clusters_after(index, Ud, K, s) <= C

    srv = mips.Server(index, method="maximus", slots=2)
    rid = srv.submit(U[:500], K)
    gi, gs, _ = srv.wait(rid)
    srv.close()
    check_against_oracle(U[:500], I, K, gi, gs, ref=(ref[0][:500], ref[1][:500]))

    mips.fit_clusters(index, None)
    idx, sc = mips.topk_maximus(index, Ud, K)
    mips.sync(index)
    assert mips.get_stats(index)["clusters"] == C
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), ref=ref)
    index.close()


def index_clusters_after(index, Ud, K, s):
    mips.topk_maximus(index, Ud, K, stream=s)
    mips.sync(index, s)
    return mips.get_stats(index)["clusters"]


def test_fit_argument_errors():
    I = synth.gaussian_rows(300, 8, 0, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4)
    lib = mips.load()
    import ctypes
    fake = ctypes.c_void_p(16)
    assert lib.mips_fit_clusters(index.handle, None, 5, None) == mips.MIPS_ERR_ARG
    assert lib.mips_fit_clusters(index.handle, fake, -1, None) == mips.MIPS_ERR_ARG
    assert lib.mips_fit_clusters(index.handle, None, 0, None) == mips.MIPS_OK  # nothing fitted: a no-op
    # fewer users than clusters: as many centroids as users
    U = synth.gaussian_rows(3, 8, 1, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    mips.fit_clusters(index, torch.from_numpy(U).cuda())
    idx, sc = mips.topk_maximus(index, torch.from_numpy(U).cuda(), 2)
    mips.sync(index)
    assert mips.get_stats(index)["clusters"] <= 3
    check_against_oracle(U, I, 2, idx.cpu().numpy(), sc.cpu().numpy())
    index.close()
