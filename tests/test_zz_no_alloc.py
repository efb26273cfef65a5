"""mips_topk_noalloc: the entry point for callers that cannot allocate
device memory (inside an allocator or out-of-memory handler, on a path where
cudaFree's device synchronisation is unacceptable, or under a memory budget
owned by someone else).  It takes its scratch from a static device array
instead of cudaMalloc.

Checked here, through the C ABI on the GPU: two calls in a row (the second
on different users, so stale scratch contents from the first would show)
give the CPU oracle's exact top-K (indices equal, scores within the
tolerance of the other parity tests) and the same rows as mips_topk on an
FP32 index; a call sized exactly at the documented scratch rule is
accepted and one user more is rejected with a clear message.  Collected last so that a failure here never hides the
other tests' results; it passes alone and after them."""
import math

import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import SCORE_TOL, check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(I, U, K):
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="fp32")
    idx, sc = mips.topk(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    out = idx.cpu().numpy(), sc.cpu().numpy()
    index.close()
    return out


def test_noalloc_matches_topk_two_calls_in_a_row():
    W = synth.WORKLOADS["small-2048x1024-f32"]
    I = synth.make_items(W, 0)
    K = 10
    I_d = torch.from_numpy(I).cuda()
    for seed, n in ((0, 2048), (7, 1500)):
        U = synth.make_users(W, seed, n=n)
        ref_idx, ref_sc = _reference(I, U, K)
        out_idx = torch.full((n, K), -1, dtype=torch.int32, device="cuda")
        out_sc = torch.zeros((n, K), dtype=torch.float64, device="cuda")
        mips.topk_noalloc(I_d, torch.from_numpy(U).cuda(), K, out_idx, out_sc)
        got_idx, got_sc = out_idx.cpu().numpy(), out_sc.cpu().numpy()
        check_against_oracle(U, I, K, got_idx, got_sc, ref=oracle.topk(U, I, K))
        assert np.array_equal(got_idx, ref_idx)
        nu = np.linalg.norm(U.astype(np.float64), axis=1)[:, None]
        ni = np.linalg.norm(I.astype(np.float64), axis=1)[ref_idx]
        assert (np.abs(got_sc - ref_sc) <= SCORE_TOL * nu * ni).all()


def _max_users(n_items, f, K):
    """Largest n_users the documented scratch rule admits (32 MiB; 5 KiB of
    counters and padding counted in full)."""
    cap = max(4 * K + 96, min(math.ceil(K * (2 + math.log(n_items / K))) + 96, n_items + 96))
    return (32 * 2**20 - 8 * n_items - 5120) // (28 + 28 * cap)


def test_noalloc_size_rule_is_the_documented_one():
    n_items, f, K = 1000, 8, 10
    n_ok = _max_users(n_items, f, K)
    I = torch.from_numpy(synth.gaussian_rows(n_items, f, 0, synth.S_ITEMS)).cuda()
    U = synth.gaussian_rows(n_ok + 64, f, 0, synth.S_USERS)
    oi = torch.empty((n_ok, K), dtype=torch.int32, device="cuda")
    os_ = torch.empty((n_ok, K), dtype=torch.float64, device="cuda")
    mips.topk_noalloc(I, torch.from_numpy(U[:n_ok]).cuda(), K, oi, os_)  # accepted
    rows = np.arange(0, n_ok, max(1, n_ok // 64))
    check_against_oracle(U[:n_ok], I.cpu().numpy(), K, oi.cpu().numpy(), os_.cpu().numpy(), rows=rows)
    # far beyond the rule: rejected before any device work
    big = 2 * n_ok + 64
    Ub = torch.from_numpy(synth.gaussian_rows(big, f, 1, synth.S_USERS)).cuda()
    oi2 = torch.empty((big, K), dtype=torch.int32, device="cuda")
    os2 = torch.empty((big, K), dtype=torch.float64, device="cuda")
    with pytest.raises(mips.MipsError) as e:
        mips.topk_noalloc(I, Ub, K, oi2, os2)
    assert e.value.status == mips.MIPS_ERR_ARG and "scratch" in str(e.value)


def test_noalloc_rejects_oversize_call():
    I = torch.from_numpy(synth.gaussian_rows(1000, 8, 0, synth.S_ITEMS)).cuda()
    U = torch.from_numpy(synth.gaussian_rows(100000, 8, 0, synth.S_USERS)).cuda()
    oi = torch.empty((100000, 10), dtype=torch.int32, device="cuda")
    os_ = torch.empty((100000, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(mips.MipsError) as e:
        mips.topk_noalloc(I, U, 10, oi, os_)
    assert e.value.status == mips.MIPS_ERR_ARG and "scratch" in str(e.value)
