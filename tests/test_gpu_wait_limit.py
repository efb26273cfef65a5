"""GPU check of the score kernel's bounded waits (through the C ABI).

Every wait inside the tensor-core kernel gives up after a limit, raises a
timeout, lets the other roles drain their copies and MMAs, frees the tensor
memory and exits.  Here the test hook makes the next launch publish no
work item, with a 5 ms limit: the call's sync must report
MIPS_ERR_TIMEOUT, and the context must stay usable -- the next calls (on
the same index and on a fresh one) return the oracle's exact top-K."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_expired_wait_reports_timeout_and_the_next_calls_are_exact():
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U, I = synth.make_users(W, 0), synth.make_items(W, 0)
    K = 10
    index = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    Ud = torch.from_numpy(U).cuda()
    mips.test_expire_next_wait(5_000_000)
    mips.topk(index, Ud, K)  # asynchronous: the status comes with the sync
    with pytest.raises(mips.MipsError) as e:
        mips.sync(index)
    assert e.value.status == mips.MIPS_ERR_TIMEOUT
    ref = oracle.topk(U, I, K)
    idx, sc = mips.topk(index, Ud, K)  # the hook was used up: an ordinary call
    mips.sync(index)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), ref=ref)
    index.close()
    fresh = mips.build_index(torch.from_numpy(I).cuda(), dtype="bf16")
    idx, sc = mips.topk(fresh, Ud, K)
    mips.sync(fresh)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), ref=ref)
    fresh.close()

