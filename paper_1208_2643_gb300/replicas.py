"""Host logic of multi-GPU runs: one independent instance per rank (the path has no
exchange step, so ranks never communicate on the data path), weak scaling, and the
job time taken as the maximum over ranks."""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment (1 process: 0, 1, 0)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def instance_seed(base: int, rank: int) -> int:
    """Seed of this rank's instance: distinct per rank, rank 0 keeps the base seed."""
    return base + rank


def job_time_ms(local_ms: float, device=None) -> float:
    """Maximum of the ranks' timed-region lengths (all ranks get it); identity for 1 rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(local_ms)
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(units_per_rank: float, world: int, job_ms: float) -> float:
    """Whole-job rate: the units all ranks processed divided by the job time."""
    return world * units_per_rank / (job_ms * 1e-3)
