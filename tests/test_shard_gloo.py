"""CPU, world_size 2 (gloo): the multi-rank path of the benchmark.  Each
rank scores its own users (seed = rank) with no data-path collective; the
only collective is the maximum of the ranks' times; the job throughput
counts every rank's users over the slowest time.  Results per rank equal
the single-process results on the same users (checked with the oracle)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORKLOAD = "small-2048x1024-f32"


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import oracle
    from paper_1706_01449_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = shard.dist_env()
    assert (w, r) == (world, rank)
    U = shard.rank_users(WORKLOAD, r, n=96)
    I = synth.make_items(synth.WORKLOADS[WORKLOAD], 0)
    idx, sc = oracle.topk(U, I, 10)
    fake_ms = 10.0 + 5.0 * r  # the ranks' step times differ
    slowest = shard.max_over_ranks(fake_ms)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), U=U, idx=idx, sc=sc, slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_weak_scaling(tmp_path):
    import oracle
    from paper_1706_01449_gb300 import shard, synth
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    I = synth.make_items(synth.WORKLOADS[WORKLOAD], 0)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    # rank r's users are the workload recipe with seed r: distinct per rank
    for r in range(world):
        assert np.array_equal(res[r]["U"], shard.rank_users(WORKLOAD, r, n=96))
        idx, sc = oracle.topk(res[r]["U"], I, 10)
        assert np.array_equal(res[r]["idx"], idx) and np.array_equal(res[r]["sc"], sc)
        assert float(res[r]["slowest"]) == 15.0
    assert not np.array_equal(res[0]["U"], res[1]["U"])
    assert shard.job_throughput(96, world, 15.0) == pytest.approx(2 * 96 / 0.015)
    assert shard.max_over_ranks(3.5) == 3.5  # no process group: the value itself
