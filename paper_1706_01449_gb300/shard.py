"""Multi-rank plumbing of the benchmark (one process per GPU).

Users are independent and the index is read-only (the paper partitions
users over index replicas), so ranks share no data: rank r scores its own
users (workload users drawn with seed r: weak scaling) against the same
items, and the only collectives are a barrier around the timed region and
the maximum of the ranks' times.  Works on any torch.distributed backend
(nccl on GPUs, gloo on CPU)."""
from __future__ import annotations

import os


def dist_env():
    """(world, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_users(workload: str, rank: int, f: int | None = None, n: int | None = None):
    """The users rank `rank` scores: the workload's user recipe with seed = rank."""
    from . import synth
    return synth.make_users(synth.WORKLOADS[workload], seed=rank, f=f, n=n)


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of x over all ranks (x itself without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, world: int, ms_per_step: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (ms_per_step / 1e3)
