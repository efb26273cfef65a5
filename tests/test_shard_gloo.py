"""CPU, world_size 2 (gloo): the multi-rank path.  One job user matrix is
split into contiguous row ranges, one per rank; each rank computes the top-K
of its own rows against the same items with no data-path collective (the CPU
oracle stands in for the GPU path here); the disjoint output slices are
gathered in rank order and must equal the single-process answer on the
whole matrix.  The slowest rank's time gives the job throughput."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

WORKLOAD = "small-2048x1024-f32"
N_PER_RANK = 48


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
    U = shard.rank_users(WORKLOAD, r, n=N_PER_RANK)
    I = synth.make_items(synth.WORKLOADS[WORKLOAD], 0)
    idx, sc = oracle.topk(U, I, 10)
    all_idx = shard.gather_rows(idx)
    all_sc = shard.gather_rows(sc)
    all_U = shard.gather_rows(U)
    fake_ms = 10.0 + 5.0 * r  # the ranks' step times differ
    slowest = shard.max_over_ranks(fake_ms)
    np.savez(os.path.join(out_dir, f"rank{r}.npz"), U=U, idx=all_idx, sc=all_sc, allU=all_U, slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_ranks_partition_and_gather(tmp_path):
    import oracle
    from paper_1706_01449_gb300 import shard, synth
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    spec = synth.WORKLOADS[WORKLOAD]
    I = synth.make_items(spec, 0)
    U_job = synth.make_users(spec, 0, n=world * N_PER_RANK)
    ref_idx, ref_sc = oracle.topk(U_job, I, 10)
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(world)]
    for r in range(world):
        lo, hi = shard.rank_range(N_PER_RANK, r)
        # rank r owns the contiguous rows [lo, hi) of the one job matrix
        assert np.array_equal(res[r]["U"], U_job[lo:hi])
        assert np.array_equal(res[r]["allU"], U_job)
        # the gathered disjoint slices are the single-process answer
        assert np.array_equal(res[r]["idx"], ref_idx)
        assert np.array_equal(res[r]["sc"], ref_sc)
        assert float(res[r]["slowest"]) == 15.0
    assert shard.job_throughput(N_PER_RANK, world, 15.0) == pytest.approx(2 * N_PER_RANK / 0.015)
    assert shard.max_over_ranks(3.5) == 3.5  # no process group: the value itself
    one = np.arange(6).reshape(3, 2)
    assert shard.gather_rows(one) is one


def test_rank_zero_is_the_workload():
    from paper_1706_01449_gb300 import shard, synth
    spec = synth.WORKLOADS[WORKLOAD]
    assert np.array_equal(shard.rank_users(WORKLOAD, 0, n=100), synth.make_users(spec, 0, n=100))
    assert shard.rank_range(100, 3) == (300, 400)
