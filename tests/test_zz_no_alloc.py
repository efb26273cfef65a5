"""mips_topk_noalloc: the entry point for callers that cannot allocate
device memory (inside an allocator or out-of-memory handler, on a path where
cudaFree's device synchronisation is unacceptable, or under a memory budget
owned by someone else).  It takes its scratch from a static device array
instead of cudaMalloc.

Checked here, through the C ABI on the GPU: two calls in a row (the second
on different users, so stale scratch contents from the first would show)
give the same indices as mips_topk on an FP32 index and scores within the
tolerance of the other parity tests; the oversize call is rejected with a
clear message.  Collected last so that a failure here never hides the
other tests' results; it passes alone and after them."""
import numpy as np
import pytest

from paper_1706_01449_gb300 import mips, synth
from parity_util import SCORE_TOL

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
        assert np.array_equal(got_idx, ref_idx)
        nu = np.linalg.norm(U.astype(np.float64), axis=1)[:, None]
        ni = np.linalg.norm(I.astype(np.float64), axis=1)[ref_idx]
        assert (np.abs(got_sc - ref_sc) <= SCORE_TOL * nu * ni).all()


def test_noalloc_rejects_oversize_call():
    I = torch.from_numpy(synth.gaussian_rows(1000, 8, 0, synth.S_ITEMS)).cuda()
    U = torch.from_numpy(synth.gaussian_rows(100000, 8, 0, synth.S_USERS)).cuda()
    oi = torch.empty((100000, 10), dtype=torch.int32, device="cuda")
    os_ = torch.empty((100000, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(mips.MipsError) as e:
        mips.topk_noalloc(I, U, 10, oi, os_)
    assert e.value.status == mips.MIPS_ERR_ARG and "scratch" in str(e.value)
