"""GPU checks of the Optimus selector (mips_select, Sec. IV): the result equals
the oracle whatever path it picks, the sample has the requested size (with
the two-waves-per-SM floor), the report's estimates follow the overhead
formula of Sec. IV (C_I + n Q_I against n M_I) and the choice is the smaller
estimate."""
import math

import numpy as np
import pytest

from paper_1706_01449_gb300 import mips, synth
from parity_util import check_against_oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", ["fp32", "bf16"])
def test_select_exact_and_report(dtype):
    U = synth.clustered_users(60000, 16, 4, n_dirs=8, noise=0.15)
    I = synth.gaussian_rows(5000, 16, 4, synth.S_ITEMS, synth.S_ITEM_NORMS, (0.0, 0.7))
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=8, dtype=dtype, sample_frac=0.01)
    idx, sc, rep = mips.select(index, torch.from_numpy(U).cuda(), 10)
    mips.sync(index)
    props = torch.cuda.get_device_properties(0)
    floor_users = 2 * props.multi_processor_count * 128
    assert rep["sample_users"] == min(U.shape[0], max(math.ceil(0.01 * U.shape[0]), floor_users))
    n = U.shape[0]
    assert rep["est_bmm"] == pytest.approx(n * rep["m_user"], rel=1e-9)
    assert rep["est_index"] == pytest.approx(rep["t_build"] + n * rep["q_user"], rel=1e-9)
    assert rep["choice"] == (1 if rep["est_index"] < rep["est_bmm"] else 0)
    assert rep["m_user"] > 0 and rep["q_user"] > 0 and rep["t_build"] > 0
    rows = synth.distinct_ids(n, 2000, 1, synth.S_SAMPLE)
    check_against_oracle(U, I, 10, idx.cpu().numpy(), sc.cpu().numpy(), rows=rows)
    index.close()


def test_select_small_input_all_sampled():
    """Fewer users than the sample floor: every user is in the sample."""
    W = synth.WORKLOADS["small-2048x1024-f32"]
    U, I = synth.make_users(W, 0), synth.make_items(W, 0)
    index = mips.build_index(torch.from_numpy(I).cuda(), clusters=4, dtype="bf16")
    idx, sc, rep = mips.select(index, torch.from_numpy(U).cuda(), 10)
    assert rep["sample_users"] == U.shape[0]
    check_against_oracle(U, I, 10, idx.cpu().numpy(), sc.cpu().numpy())
    index.close()
