"""Host-side logic of running the solve on several GPUs of one node.

The benchmark's unit of work (one m-column block of right-hand sides) is
independent of every other block, so N ranks solve N blocks with no exchange on
the data path (weak scaling).  The ranks meet only to bracket the timed region
and to combine its results: the job time is the slowest rank's time and the
job's count is the sum over ranks.
"""
from __future__ import annotations

import os


def rank_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rhs_seed(rank: int) -> int:
    """Seed of rank `rank`'s right-hand-side block (rank 0 = the single-GPU block)."""
    return rank


def job_throughput(t_local_s: float, solved_local: int, dist=None, device=None):
    """Whole-job throughput: columns solved by all ranks / slowest rank's time.

    Returns (value, t_max_s, solved_all).  `dist` is torch.distributed (or None
    for one process); `device` is where the reduction tensors live ("cuda" with
    NCCL, "cpu" with gloo)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return solved_local / t_local_s, t_local_s, solved_local
    import torch
    t = torch.tensor([t_local_s], dtype=torch.float64, device=device)
    n = torch.tensor([float(solved_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    t_max, solved = float(t.item()), int(n.item())
    return solved / t_max, t_max, solved
