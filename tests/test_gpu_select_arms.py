"""GPU checks of the multi-arm selector (mips_select_arms; Sec. IV's Optimus
with more arms: the FP32, BF16 and FP8 candidate passes times the blocked
multiply and Maximus, chosen from repeated timings of one user sample):
  * the result is the exact top-K (oracle on sampled rows; every arm is
    exact, so the choice cannot change it);
  * the report is consistent: one arm per (index, method), the choice has
    the smallest mean estimate, every arm was timed at least three rounds
    unless it was dropped, intervals are non-negative, and the sampling
    overhead is reported;
  * on the Netflix shape the BF16 blocked multiply is chosen and on the R2
    shape (heavy item-norm skew) BF16 Maximus, the forms the full-size runs
    measure fastest there;
  * argument errors."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DT = {0: "fp32", 1: "bf16", 2: "fp8"}
METH = {0: "bmm", 1: "maximus"}


def _indexes(I, clusters):
    Id = torch.from_numpy(I).cuda()
    return [mips.build_index(Id, clusters=clusters, dtype=d) for d in ("fp32", "bf16", "fp8")]


def _check_report(rep, n_users):
    assert rep["n_arms"] == 6
    arms = rep["arms"]
    assert sorted((a["index"], a["method"]) for a in arms) == [(i, m) for i in range(3) for m in range(2)]
    means = [a["est_mean"] for a in arms]
    assert rep["choice"] == int(np.argmin(means))
    for a in arms:
        assert a["rounds"] >= 3 or a["dropped"]
        assert a["est_ci"] >= 0.0 and a["est_mean"] > 0.0
    assert 3 <= rep["rounds"] <= 6
    assert 0 < rep["sample_users"] <= n_users
    assert 0.0 < rep["t_sample"] <= rep["t_total"]


def _run(workload, n_users, K, clusters, rows=300):
    spec = synth.WORKLOADS[workload]
    U = synth.make_users(spec, 0, n=n_users)
    I = synth.make_items(spec, 0)
    ix = _indexes(I, clusters)
    idx, sc, rep = mips.select_arms(ix, torch.from_numpy(U).cuda(), K)
    torch.cuda.synchronize()
    r = np.random.default_rng(1).choice(n_users, size=min(rows, n_users), replace=False)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), rows=r)
    _check_report(rep, n_users)
    for x in ix:
        x.close()
    ch = rep["arms"][rep["choice"]]
    return DT[ch["dtype"]], METH[ch["method"]], rep


def test_netflix_shape_picks_bf16_blocked_multiply():
    dt, meth, rep = _run("netflix-480189x17770", 480189, 10, 64)
    assert (dt, meth) == ("bf16", "bmm"), rep


def test_r2_shape_picks_bf16_maximus():
    dt, meth, rep = _run("r2-1823179x136736", 1823179, 10, 32)
    assert (dt, meth) == ("bf16", "maximus"), rep


def test_small_input_all_users_in_the_sample():
    # fewer users than the sample floor: every user is timed, none is left
    U = synth.gaussian_rows(3000, 24, 4, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    I = synth.gaussian_rows(2500, 24, 4, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    ix = _indexes(I, 8)
    idx, sc, rep = mips.select_arms(ix, torch.from_numpy(U).cuda(), 7, max_rounds=4)
    check_against_oracle(U, I, 7, idx.cpu().numpy(), sc.cpu().numpy())
    _check_report(rep, U.shape[0])
    assert rep["sample_users"] == U.shape[0] and rep["rounds"] <= 4
    for x in ix:
        x.close()


def test_select_arms_argument_errors():
    I = synth.gaussian_rows(500, 16, 2, synth.S_ITEMS)
    U = torch.from_numpy(synth.gaussian_rows(64, 16, 2, synth.S_USERS)).cuda()
    a = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    b = mips.build_index(torch.from_numpy(I[:400]).cuda(), dtype="fp32")
    for bad, kw in (([a, b], {}), ([a], {"max_rounds": 2}), ([a], {"max_rounds": 17}), ([a] * 9, {})):
        with pytest.raises(mips.MipsError) as e:
            mips.select_arms(bad, U, 5, **kw)
        assert e.value.status == mips.MIPS_ERR_ARG
    a.close()
    b.close()
