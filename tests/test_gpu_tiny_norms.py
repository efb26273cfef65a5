"""GPU checks of rows at the bottom of the FP32 range (through the C ABI).

Users: zero users, users whose squared entries all underflow (||u||^2 = 0
in FP32 though u != 0), users with a subnormal ||u||^2 and users with
subnormal entries, mixed with ordinary users in one call; the rescore sends
every non-zero user with ||u||^2 < 2^-100 to the exhaustive FP64 scoring.

Items: a catalogue whose ordinary items all score negative for users along
-e1, so that those users' top-K lies among items scaled by 1e-22 (squared
norms ~1e-44, below the FP32 normal range) and 1e-30 (squares underflow to
0); the norm bounds, the bound columns of the BF16 pass, the FP32 pass's
error term and Maximus's CBound must all stay valid for them.

The blocked multiply (both candidate passes) and Maximus must return the
oracle's exact top-K for all of them."""
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


@pytest.mark.parametrize("method,dtype", [("bmm", "bf16"), ("bmm", "fp32"), ("bmm", "fp8"), ("maximus", "bf16"),
                                          ("maximus", "fp32"), ("maximus", "fp8")])
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


def tiny_item_catalogue(f, seed):
    I = synth.gaussian_rows(600, f, seed, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    I[:, 0] = np.abs(I[:, 0]) + np.float32(0.5)     # every ordinary item: positive first coordinate
    T = synth.gaussian_rows(60, f, seed + 1, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.5))
    T[:40] *= np.float32(1e-22)                       # ||i||^2 ~ 1e-44: subnormal in FP32
    T[40:56] *= np.float32(1e-30)                     # squares underflow to 0 in FP32
    T[56:] = 0.0                                      # zero items
    I = np.concatenate([I[:300], T, I[300:]]).astype(np.float32)  # tiny items in the middle of the ids
    return I


def neg_e1_users(f, seed):
    U = synth.gaussian_rows(48, f, seed, synth.S_USERS, synth.S_USER_NORMS, (0.0, 0.3))
    D = synth.gaussian_rows(16, f, seed + 2, synth.S_USERS)
    D = 0.01 * D
    D[:, 0] = -1.0                                    # along -e1: every ordinary item scores below 0
    return np.concatenate([D, U]).astype(np.float32)


@pytest.mark.parametrize("method,dtype", [("bmm", "bf16"), ("bmm", "fp32"), ("bmm", "fp8"), ("maximus", "bf16"),
                                          ("maximus", "fp32"), ("maximus", "fp8")])
@pytest.mark.parametrize("K", [1, 10])
def test_tiny_items_exact(method, dtype, K):
    f = 24
    I = tiny_item_catalogue(f, seed=5)
    U = neg_e1_users(f, seed=5)
    ref = oracle.topk(U, I, K)
    # the -e1 users' answers do lie among the tiny items (positions 300..359)
    assert ((ref[0][:16] >= 300) & (ref[0][:16] < 360)).all() and (ref[1][:16, 0] > 0).all()
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4, dtype=dtype)
    fn = mips.topk if method == "bmm" else mips.topk_maximus
    idx, sc = fn(index, torch.from_numpy(U).cuda(), K)
    mips.sync(index)
    check_against_oracle(U, I, K, idx.cpu().numpy(), sc.cpu().numpy(), ref=ref)
    index.close()
