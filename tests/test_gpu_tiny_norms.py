"""GPU checks of users at the bottom of the FP32 range (through the C ABI):
zero users, users whose squared entries all underflow (||u||^2 = 0 in FP32
though u != 0), users with a subnormal ||u||^2 and users with subnormal
entries, mixed with ordinary users in one call.  The blocked multiply (both
candidate passes) and Maximus must return the oracle's exact top-K for all
of them: the rescore sends every non-zero user with ||u||^2 < 2^-100 to the
exhaustive FP64 scoring."""
import numpy as np
import pytest

import oracle
from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def tiny_users(f, seed):
    U = synth.gaussian_rows(64, f, seed, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    U[0:6] *= np.float32(1e-24)    # squares underflow: ||u||^2 = 0 in FP32
    U[6:12] *= np.float32(1e-30)
    U[12:18] *= np.float32(1e-17)  # ||u||^2 ~ 1e-34: subnormal range of the sum
    U[18:21] = 0.0                 # zero users
    U[21] = 0.0
    U[21, 3] = np.float32(1e-40)   # one subnormal entry
    U[22] = 0.0
    U[22, :4] = np.float32([1e-42, -3e-41, 2e-45, 7e-39])
    return U.astype(np.float32)


@pytest.mark.parametrize("method,dtype", [("bmm", "bf16"), ("bmm", "fp32"), ("maximus", "bf16"),
                                          ("maximus", "fp32")])
@pytest.mark.parametrize("K", [1, 10])
def test_tiny_and_zero_users_exact(method, dtype, K):
    f = 24
    U = tiny_users(f, seed=3)
    I = synth.gaussian_rows(700, f, 3, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4, dtype=dtype)
    fn = mips.topk if method == "bmm" else mips.topk_maximus
    idx, sc = fn(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    ref = oracle.topk(U, I, K)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), ref=ref)
    # the tiny users' scores are the FP64 definition's values, not zeros
    assert (np.abs(sc.cpu().numpy()[:18, 0]) > 0).all()
    index.close()
