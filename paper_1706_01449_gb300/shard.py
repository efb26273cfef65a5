"""Multi-rank plumbing (one process per GPU).

Users are independent and the index is read-only (the paper partitions
users over index replicas, Sec. V's multi-core runs), so the user matrix is
split into contiguous row ranges, one per rank; every rank holds the same
items and computes the exact top-K of its own rows with no collective on the
data path.  The only collectives are a barrier around a timed region, the
maximum of the ranks' times, and an optional final gather of the disjoint
output slices.  Works on any torch.distributed backend (nccl on GPUs, gloo
on CPU).
"""
from __future__ import annotations

import os


def dist_env():
    """(world, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_range(n_per_rank: int, rank: int) -> tuple[int, int]:
    """Rows [lo, hi) of the job's user matrix that rank `rank` owns."""
    return rank * n_per_rank, (rank + 1) * n_per_rank


def rank_users(workload: str, rank: int, f: int | None = None, n: int | None = None):
    """Rank `rank`'s slice of the job's user matrix: rows
    [rank * n, (rank + 1) * n) of the workload's user recipe (seed 0), n =
    the workload's user count unless given.  With one rank this is the
    workload itself; with N ranks the job scores N * n users, n per rank
    (weak scaling)."""
    from . import synth
    spec = synth.WORKLOADS[workload]
    n = spec["n_users"] if n is None else n
    lo, _ = rank_range(n, rank)
    return synth.make_users(spec, seed=0, n=n, f=f, offset=lo)


def gather_rows(local, world: int | None = None):
    """Concatenate every rank's equally sized slice (a torch tensor on the
    backend's device, or a numpy array) in rank order; every rank gets the
    whole.  Without a process group, the slice itself."""
    import numpy as np
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    is_np = isinstance(local, np.ndarray)
    t = torch.from_numpy(np.ascontiguousarray(local)) if is_np else local.contiguous()
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    out = torch.cat(parts, dim=0)
    return out.numpy() if is_np else out


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
