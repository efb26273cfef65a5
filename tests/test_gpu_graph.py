"""GPU checks of mips_topk_graph (whole call captured into a CUDA graph,
replayed for the same arguments): replays give the plain call's results,
read new input values at the same address, keep per-argument graphs apart,
and re-capture after the workspace grows."""
import numpy as np
import pytest

from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _users(n, f, seed):
    return synth.clustered_users(n, f, seed, n_dirs=8, noise=0.2)


@pytest.mark.parametrize("method,dtype", [("bmm", "bf16"), ("maximus", "bf16"), ("maximus", "fp32")])
def test_graph_replay_matches_plain(method, dtype):
    f, K = 24, 10
    I = synth.gaussian_rows(3000, f, 5, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=8, dtype=dtype)
    s = torch.cuda.Stream()
    plain = mips.topk if method == "bmm" else mips.topk_maximus
    U0, U1 = _users(2500, f, 1), _users(2500, f, 2)
    Ud = torch.from_numpy(U0).cuda()
    oi = torch.empty((2500, K), dtype=torch.int32, device="cuda")
    osc = torch.empty((2500, K), dtype=torch.float64, device="cuda")
    with torch.cuda.stream(s):
        for it in range(3):  # first call captures, then replays
            mips.topk_graph(index, Ud, K, method, oi, osc, stream=s)
            mips.sync(index, stream=s)
            check_against_oracle(U0, I, K, oi.cpu().numpy(), osc.cpu().numpy())
        st = mips.get_stats(index)
        assert st["n_users"] == 2500 and st["ms_total"] > 0
        # new values at the same address: the replay reads them
        Ud.copy_(torch.from_numpy(U1))
        mips.topk_graph(index, Ud, K, method, oi, osc, stream=s)
        mips.sync(index, stream=s)
        check_against_oracle(U1, I, K, oi.cpu().numpy(), osc.cpu().numpy())
        ri, rs = plain(index, Ud, K, stream=s)
        mips.sync(index, stream=s)
        assert (ri.cpu().numpy() == oi.cpu().numpy()).all() and (rs.cpu().numpy() == osc.cpu().numpy()).all()
    index.close()


def test_graph_workspace_growth_and_separate_arguments():
    f, K = 16, 5
    I = synth.gaussian_rows(1500, f, 7, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4, dtype="bf16")
    s = torch.cuda.Stream()
    small, large = _users(600, f, 3), _users(9000, f, 4)
    Us, Ul = torch.from_numpy(small).cuda(), torch.from_numpy(large).cuda()
    with torch.cuda.stream(s):
        a = mips.topk_graph(index, Us, K, "maximus", stream=s)  # capture (small workspace)
        mips.sync(index, stream=s)
        b = mips.topk_graph(index, Ul, K, "maximus", stream=s)  # grows the workspace
        mips.sync(index, stream=s)
        check_against_oracle(large, I, K, b[0].cpu().numpy(), b[1].cpu().numpy())
        # the small call's graph is stale now: the call re-captures and stays exact
        for _ in range(2):
            c = mips.topk_graph(index, Us, K, "maximus", a[0], a[1], stream=s)
            mips.sync(index, stream=s)
            check_against_oracle(small, I, K, c[0].cpu().numpy(), c[1].cpu().numpy())
        # other K, other method: their own graphs
        for method, k in (("bmm", K), ("maximus", 1)):
            for _ in range(2):
                d = mips.topk_graph(index, Us, k, method, stream=s)
                mips.sync(index, stream=s)
                check_against_oracle(small, I, k, d[0].cpu().numpy(), d[1].cpu().numpy())
    # a method outside {0, 1} is an argument error
    import ctypes
    lib = mips.load()
    st = lib.mips_topk_graph(index.handle, ctypes.c_void_p(Us.data_ptr()), Us.shape[0], K, 2,
                             ctypes.c_void_p(a[0].data_ptr()), ctypes.c_void_p(a[1].data_ptr()),
                             ctypes.c_void_p(s.cuda_stream))
    assert st == mips.MIPS_ERR_ARG
    index.close()
