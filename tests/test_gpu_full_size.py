"""Full-size workloads in the launch configuration the benchmark times,
checked against the oracle on sampled users (seeded sample plus the users
of largest norm):
  * R2 shape (1,823,179 users x 136,736 items, f = 50, heavy item-norm skew):
    blocked multiply, Maximus (autotuned |C| and B) and Optimus, K = 1 / 10 / 50;
  * KDD shape through the captured-graph path (Maximus, autotuned);
  * serving on the 1,000,000-item f = 128 catalogue: requests of mixed size
    and K through the server, sampled rows of every request."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def _rows(U, n_sample, seed):
    return np.union1d(synth.distinct_ids(U.shape[0], n_sample, seed, synth.S_SAMPLE),
                      np.argsort(-np.linalg.norm(U, axis=1))[:32])


@pytest.fixture(scope="module")
def r2():
    W = synth.WORKLOADS["r2-1823179x136736"]
    U, I = synth.make_users(W, 0), synth.make_items(W, 0)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=64, dtype="bf16")
    Ud = torch.from_numpy(U).cuda()
    yield U, I, index, Ud
    index.close()


@pytest.mark.parametrize("K", [1, 10, 50])
def test_r2_bmm_maximus_optimus(r2, K):
    U, I, index, Ud = r2
    rows = _rows(U, 160, K)
    ref = oracle.topk(U[rows], I, K)
    bi, bs = mips.topk(index, Ud, K)
    mips.sync(index)
    check_against_oracle(U, I, K, bi.cpu().numpy(), bs.cpu().numpy(), rows=rows, ref=ref)
    mips.autotune(index, Ud, K)
    mi, ms = mips.topk_maximus(index, Ud, K)
    mips.sync(index)
    check_against_oracle(U, I, K, mi.cpu().numpy(), ms.cpu().numpy(), rows=rows, ref=ref)
    si, ss, rep = mips.select(index, Ud, K)
    mips.sync(index)
    check_against_oracle(U, I, K, si.cpu().numpy(), ss.cpu().numpy(), rows=rows, ref=ref)
    assert rep["choice"] in (0, 1)


def test_kdd_maximus_graph_replay():
    W = synth.WORKLOADS["kdd-1000000x624961"]
    U, I = synth.make_users(W, 0), synth.make_items(W, 0)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=64, dtype="bf16")
    s = torch.cuda.Stream()
    Ud = torch.from_numpy(U).cuda()
    rows = _rows(U, 128, 7)
    ref = oracle.topk(U[rows], I, 10)
    with torch.cuda.stream(s):
        mips.autotune(index, Ud, 10, stream=s)
        for _ in range(2):  # capture, then replay
            gi, gs = mips.topk_graph(index, Ud, 10, "maximus", stream=s)
            mips.sync(index, stream=s)
            check_against_oracle(U, I, 10, gi.cpu().numpy(), gs.cpu().numpy(), rows=rows, ref=ref)
    index.close()


def test_serving_full_catalogue_sampled():
    W = synth.WORKLOADS["serve-1000000x128"]
    I = synth.make_items(W, 0)
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    rng = np.random.default_rng(5)
    reqs, off = [], 0
    for _ in range(12):
        n = int(round(np.exp(rng.uniform(0, np.log(4096)))))
        reqs.append((synth.serving_users(n, 128, 2, off), int(rng.choice([1, 10, 100]))))
        off += n
    srv = mips.Server(index, slots=2, max_batch_users=8192)
    ids = [srv.submit(U, K) for U, K in reqs]
    got = [srv.wait(i, timeout=300) for i in ids]
    srv.close()
    for (U, K), (gi, gs, _) in zip(reqs, got):
        rows = np.arange(U.shape[0]) if U.shape[0] <= 16 else synth.distinct_ids(U.shape[0], 16, K, synth.S_SAMPLE)
        check_against_oracle(U, I, K, gi, gs, rows=rows)
    index.close()
