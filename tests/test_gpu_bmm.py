"""GPU parity of the blocked multiply + fused top-K path (mips_topk) with
the oracle, through the C ABI, on every candidate-pass dtype the library
builds.  Covers several tiles with ragged tails, edge shapes and the
degenerate cases (ties, duplicates, zero users, K = n_items, overflowing
candidate lists, non-finite input)."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DTYPES = ["fp32", "bf16", "fp8"]


def _dtype_or_skip(dtype, I, **kw):
    try:
        return mips.build_index(torch.from_numpy(I).cuda(), dtype=dtype, **kw)
    except mips.MipsError as e:
        if e.status == mips.MIPS_ERR_UNIMPLEMENTED:
            pytest.skip(f"{dtype} not built")
        raise


def run_topk(U, I, K, dtype, method="topk"):
    index = _dtype_or_skip(dtype, I)
    fn = getattr(mips, method)
    idx, sc = fn(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    stats = mips.get_stats(index)
    index.close()
    return idx.cpu().numpy(), sc.cpu().numpy(), stats


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("K", [1, 10])
def test_small_workload_all_users(dtype, K):
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U, I = synth.make_users(W, 0), synth.make_items(W, 0)
    idx, sc, st = run_topk(U, I, K, dtype)
    check_against_oracle(U, I, K, idx, sc)
    assert st["users_overflow"] == 0


@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("nU,nI,f,K", [(1, 1, 1, 1), (31, 33, 3, 5), (129, 257, 31, 7), (200, 1000, 33, 50),
                                        (300, 700, 64, 128), (130, 999, 100, 16), (77, 500, 128, 3),
                                        (513, 4097, 50, 10), (64, 40, 10, 40)])
def test_ragged_shapes(dtype, nU, nI, f, K):
    U = synth.gaussian_rows(nU, f, 3, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    I = synth.gaussian_rows(nI, f, 3, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    idx, sc, _ = run_topk(U, I, K, dtype)
    check_against_oracle(U, I, K, idx, sc)


@pytest.mark.parametrize("f,K", [(63, 10), (64, 1), (78, 16), (80, 10), (94, 5), (120, 3), (126, 16), (128, 10),
                                 (128, 1), (128, 100), (64, 128)])
def test_tail_chunk_rows(f, K):
    """Operand rows of 64 + 16 or 64 + 32 BF16 elements (f + 2 = 65..96,
    129..130): full 128-byte swizzled chunks plus a 32- or 64-byte tail
    chunk with its own tensor map and swizzle; for f near 128 the item tile
    is loaded as two 128-row halves (N = 128 MMAs) to fit shared memory, and
    a large-K heap that still does not fit lives in global memory.  The
    tensor-core path must be the one used."""
    U = synth.gaussian_rows(700, f, 9, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    I = synth.gaussian_rows(3000, f, 9, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    idx, sc, st = run_topk(U, I, K, "bf16")
    assert st["dtype"] == 1, "BF16 tensor-core path not taken"
    check_against_oracle(U, I, K, idx, sc)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4, dtype="bf16")
    mi, ms = mips.topk_maximus(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    assert mips.get_stats(index)["dtype"] == 1
    index.close()
    check_against_oracle(U, I, K, mi.cpu().numpy(), ms.cpu().numpy())


@pytest.mark.parametrize("dtype", DTYPES)
def test_ties_duplicates_zero_users(dtype):
    rng = np.random.default_rng(0)
    base = rng.integers(-3, 4, size=(60, 8)).astype(np.float32)
    I = np.concatenate([base, base[:20], base[5:9]])      # duplicated items -> exact ties
    U = rng.integers(-2, 3, size=(150, 8)).astype(np.float32)
    U[::17] = 0.0                                           # zero users
    for K in (1, 5, 33):
        idx, sc, st = run_topk(U, I, K, dtype)
        check_against_oracle(U, I, K, idx, sc)
    assert st["users_fp64"] > 0  # integer data: exact ties resolved by the FP64 check


@pytest.mark.parametrize("dtype", DTYPES)
def test_all_items_identical_overflow(dtype):
    """Every item equal: every user's candidate list overflows and the
    exhaustive rescore must return items 0..K-1."""
    I = np.tile(np.array([[0.5, -1.0, 2.0, 0.25]], dtype=np.float32), (3000, 1))
    U = synth.gaussian_rows(40, 4, 1, synth.S_USERS)
    idx, sc, st = run_topk(U, I, 7, dtype)
    check_against_oracle(U, I, 7, idx, sc)
    assert st["users_overflow"] == 40


@pytest.mark.parametrize("dtype", DTYPES)
def test_k_equals_n_items(dtype):
    U = synth.gaussian_rows(70, 12, 5, synth.S_USERS)
    I = synth.gaussian_rows(90, 12, 5, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    idx, sc, _ = run_topk(U, I, 90, dtype)
    check_against_oracle(U, I, 90, idx, sc)


@pytest.mark.parametrize("dtype", DTYPES)
def test_scaling_invariance(dtype):
    """Power-of-two scaling: identical indices and exactly scaled scores."""
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U, I = synth.make_users(W, 1, n=256), synth.make_items(W, 1)
    idx, sc, _ = run_topk(U, I, 10, dtype)
    idx2, sc2, _ = run_topk(U * np.float32(4.0), I * np.float32(0.125), 10, dtype)
    assert (idx == idx2).all()
    np.testing.assert_allclose(sc2, sc * 0.5, rtol=1e-12, atol=0)


@pytest.mark.parametrize("dtype", DTYPES)
def test_nonfinite_input_reported(dtype):
    I = synth.gaussian_rows(100, 8, 0, synth.S_ITEMS)
    U = synth.gaussian_rows(10, 8, 0, synth.S_USERS)
    U[3, 2] = np.nan
    index = _dtype_or_skip(dtype, I)
    mips.topk(index, torch.from_numpy(U).cuda(), 3)
    with pytest.raises(mips.MipsError) as e:
        mips.sync(index)
    assert e.value.status == mips.MIPS_ERR_NONFINITE
    I[7, 1] = np.inf
    with pytest.raises(mips.MipsError) as e:
        mips.build_index(torch.from_numpy(I).cuda(), dtype=dtype)
    assert e.value.status == mips.MIPS_ERR_NONFINITE


def test_argument_errors():
    I = synth.gaussian_rows(50, 8, 0, synth.S_ITEMS)
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="fp32")
    U = torch.from_numpy(synth.gaussian_rows(5, 8, 0, synth.S_USERS)).cuda()
    for K in (0, 51, 129):
        with pytest.raises(mips.MipsError) as e:
            mips.topk(index, U, K)
        assert e.value.status == mips.MIPS_ERR_ARG
    with pytest.raises(ValueError):
        mips.topk(index, torch.zeros((5, 9), device="cuda"), 3)


@pytest.mark.parametrize("dtype", DTYPES)
def test_host_entry_point_matches_device(dtype):
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U, I = synth.make_users(W, 2, n=500), synth.make_items(W, 2)
    index = _dtype_or_skip(dtype, I)
    d_idx, d_sc = mips.topk(index, torch.from_numpy(U).cuda(), 10)
    h_idx, h_sc = mips.topk_host(index, torch.from_numpy(U).pin_memory(), 10)
    assert (d_idx.cpu() == h_idx).all() and (d_sc.cpu() == h_sc).all()
    h2_idx, h2_sc = mips.topk_host(index, U, 10)   # pageable host memory too
    assert (h2_idx == h_idx).all()
    index.close()


def test_host_entry_point_chunked_overlap():
    """140,000 users: the host path runs three user chunks whose copies
    overlap the compute; results equal the device call's bit for bit, with
    pinned and with pageable host buffers, and the oracle's on sampled rows."""
    U = synth.gaussian_rows(140000, 16, 4, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    I = synth.gaussian_rows(300, 16, 4, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    d_idx, d_sc = mips.topk(index, torch.from_numpy(U).cuda(), 7)
    h_idx, h_sc = mips.topk_host(index, torch.from_numpy(U).pin_memory(), 7)
    assert (d_idx.cpu() == h_idx).all() and (d_sc.cpu() == h_sc).all()
    h2_idx, h2_sc = mips.topk_host(index, U, 7)   # pageable
    assert (h2_idx == h_idx).all() and (h2_sc == h_sc).all()
    rows = np.random.default_rng(0).choice(U.shape[0], 400, replace=False)
    check_against_oracle(U, I, 7, h_idx.numpy(), h_sc.numpy(), rows=np.sort(rows))
    index.close()


@pytest.mark.slow
@pytest.mark.parametrize("dtype", DTYPES)
@pytest.mark.parametrize("f,K", [(10, 1), (50, 10), (100, 50)])
def test_netflix_shape_full_size_sampled(dtype, f, K):
    """480,189 x 17,770 at full size (the benchmark's workload); the oracle
    checks a seeded sample of users plus the largest-norm users."""
    W = synth.WORKLOADS["netflix-480189x17770"]
    U, I = synth.make_users(W, 0, f=f), synth.make_items(W, 0, f=f)
    idx, sc, st = run_topk(U, I, K, dtype)
    rows = np.union1d(synth.distinct_ids(U.shape[0], 384, 0, synth.S_SAMPLE),
                      np.argsort(-np.linalg.norm(U, axis=1))[:64])
    check_against_oracle(U, I, K, idx, sc, rows=rows)


@pytest.mark.parametrize("nU,nI,f,K", [(1, 20000, 32, 10), (300, 50000, 50, 5), (1000, 30000, 24, 1),
                                        (2000, 9000, 64, 16), (700, 12000, 40, 50)])
def test_item_chunked_small_batches(nU, nI, f, K):
    """Few user tiles against many item tiles: the blocked multiply splits
    the items into chunks (a work item per user tile and chunk, two
    sub-lists per user and chunk); the rescore takes the union."""
    U = synth.gaussian_rows(nU, f, 13, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    I = synth.gaussian_rows(nI, f, 13, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    idx, sc, st = run_topk(U, I, K, "bf16")
    assert st["dtype"] == 1
    check_against_oracle(U, I, K, idx, sc)
