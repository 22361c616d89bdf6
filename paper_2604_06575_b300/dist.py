"""Process-group helpers for runs with one process per GPU.

The path partitions into independent problems (points, polynomials), so ranks
share no data: each rank processes its own batch (weak scaling) and the only
collectives are the timing barrier and a max over ranks of the elapsed time.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_info():
    """(rank, world_size, local_rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def workload_seed_offset(rank: int) -> int:
    """Each rank draws its own batch of the same family."""
    return rank


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device="cpu") -> float:
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, steps: int, max_total_ms: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world * steps / (max_total_ms * 1e-3)
