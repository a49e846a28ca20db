"""Replica-parallel host logic (one process per GPU, no data-path collective).

A plan does not shard: a turn chain spans every heading plane and a straight
line spans a whole plane, so several GPUs serve independent plans.  Each
rank plans its own work; the only collectives are the timing barrier, the
maximum of the ranks' elapsed times and the sum of the units they
processed.  The functions take the process group's backend as it is (NCCL
on GPUs, gloo on the host), so the same code path is tested on CPU.
"""
from __future__ import annotations

import os
from typing import List, Tuple


def rank_env() -> Tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def deal(n_items: int, world: int, rank: int) -> List[int]:
    """Indices of the independent items (queries, requests) this rank plans:
    round robin, so every item goes to exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank")
    return list(range(rank, n_items, world))


def _tensor(value: float, device):
    import torch
    return torch.tensor([float(value)], dtype=torch.float64, device=device)


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int, device="cpu") -> float:
    """The largest value over all ranks (the job's elapsed time)."""
    if world == 1:
        return float(value)
    import torch.distributed as dist
    t = _tensor(value, device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, world: int, device="cpu") -> float:
    """The sum over all ranks (units processed by the whole job)."""
    if world == 1:
        return float(value)
    import torch.distributed as dist
    t = _tensor(value, device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units: float, seconds: float, world: int, device="cpu") -> Tuple[float, float, float]:
    """Whole-job throughput: (units of all ranks / slowest rank's time,
    total units, slowest time)."""
    total = sum_over_ranks(units, world, device)
    slowest = max_over_ranks(seconds, world, device)
    return total / slowest, total, slowest
