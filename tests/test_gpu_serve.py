"""GPU checks of the serving loop (mips_server_*): requests of mixed sizes
and K submitted at once are batched (several requests per batch, mixed K
inside a batch, batches in flight on different stream slots at the same
time), and every request's result is bit-identical to the same request
run alone, and exact against the oracle (every request).  Memory
admission: a batch's admitted bytes are exactly the workspace its call
took plus its buffers, and with a budget the batches in flight never hold
more than the budget."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _requests(n_req, f, seed, max_users=600, ks=(1, 5, 10, 50, 100)):
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        n = int(round(np.exp(rng.uniform(0, np.log(max_users)))))
        U = (rng.standard_normal((n, f)) / np.sqrt(f)).astype(np.float32)
        out.append((U, int(rng.choice(ks))))
    return out


@pytest.mark.parametrize("method", ["bmm", "maximus"])
def test_mixed_requests_alone_equals_in_the_mix(method):
    f = 32
    I = synth.gaussian_rows(20000, f, 11, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=8, dtype="bf16")
    reqs = _requests(40 if method == "bmm" else 16, f, 3)
    srv = mips.Server(index, method=method, slots=2, max_batch_users=1024)
    ids = [srv.submit(U, K) for U, K in reqs]
    got = [srv.wait(i, timeout=120) for i in ids]
    srv.close()
    m = {"bmm": "bmm", "maximus": "maximus"}[method]
    for (U, K), (gi, gs, info) in zip(reqs, got):
        ai, asc = mips.topk_host(index, U, K, m)
        assert (gi == ai).all() and (gs == asc).all()
        assert info["batch_K"] >= K and info["batch_users"] >= U.shape[0]
        assert info["t_submit"] <= info["t_start"] <= info["t_done"]
    for (U, K), (gi, gs, _) in zip(reqs, got):
        check_against_oracle(U, I, K, gi, gs, ref=oracle.topk(U, I, K))
    infos = [g[2] for g in got]
    # several requests per batch, and mixed K inside one batch (5 and 10,
    # 50 and 100 share a K class)
    assert any(i["batch_users"] > U.shape[0] for (U, _), i in zip(reqs, infos))
    assert any(i["batch_K"] > K for (_, K), i in zip(reqs, infos))
    if method == "bmm":
        # two batches on different slots were in flight at the same time
        spans = {}
        for i in infos:
            spans[i["batch"]] = (i["t_start"], i["t_done"], i["slot"])
        b = sorted(spans.values())
        assert any(b[j][2] != b[j + 1][2] and b[j + 1][0] < b[j][1] for j in range(len(b) - 1))
    index.close()


def test_memory_budget_admission_and_errors():
    f = 16
    I = synth.gaussian_rows(3000, f, 12, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    reqs = _requests(12, f, 5, max_users=300, ks=(1, 10))
    # a budget below any batch: one batch in flight at a time, all complete
    srv = mips.Server(index, slots=3, max_batch_users=256, mem_budget=1)
    ids = [srv.submit(U, K) for U, K in reqs]
    got = [srv.wait(i, timeout=120) for i in ids]
    spans = sorted({(g[2]["t_start"], g[2]["t_done"]) for g in got})
    assert all(spans[j + 1][0] >= spans[j][1] for j in range(len(spans) - 1))
    for (U, K), (gi, gs, _) in zip(reqs, got):
        ai, asc = mips.topk_host(index, U, K, "bmm")
        assert (gi == ai).all() and (gs == asc).all()
    # K above n_items and unknown ids are argument errors; nothing hangs
    with pytest.raises(mips.MipsError):
        srv.submit(reqs[0][0], I.shape[0] + 1)
    with pytest.raises(mips.MipsError):
        srv.wait(10 ** 9, timeout=0.01)
    srv.close()
    index.close()


def test_admission_bytes_are_the_calls_workspace_and_budget_holds():
    f = 32
    I = synth.gaussian_rows(20000, f, 13, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    reqs = _requests(24, f, 9, max_users=400, ks=(1, 10, 100))

    def run(**kw):
        srv = mips.Server(index, slots=3, max_batch_users=512, **kw)
        ids = [srv.submit(U, K) for U, K in reqs]
        got = [srv.wait(i, timeout=120) for i in ids]
        srv.close()
        return got

    free = run()
    for (U, K), (gi, gs, info) in zip(reqs, free):
        io = info["batch_users"] * (f * 4 + info["batch_K"] * 12)
        # the admitted workspace is what the call laid out and took
        assert info["batch_ws_bytes"] > 0 and info["batch_bytes"] == info["batch_ws_bytes"] + io
        check_against_oracle(U, I, K, gi, gs, ref=oracle.topk(U, I, K))
    biggest = max(g[2]["batch_bytes"] for g in free)
    budget = int(biggest * 1.5)  # room for one batch, not always two
    capped = run(mem_budget=budget)
    # admission: a batch starts only if everything in flight fits the
    # budget, or it runs alone
    for g in capped:
        assert g[2]["inflight_bytes"] <= max(budget, g[2]["batch_bytes"])
        assert g[2]["batch_bytes"] == g[2]["batch_ws_bytes"] + g[2]["batch_users"] * (f * 4 + g[2]["batch_K"] * 12)
    for (gi, gs, _), (fi, fs, _) in zip(capped, free):
        assert (gi == fi).all() and (gs == fs).all()
    index.close()
