"""Rank helpers for running the walk on several processes (one GPU each).

The walks of different instances are independent problems, so N ranks run N
shares of the work with no data exchange (weak scaling); the only collectives
are the timing barrier and the maximum of the per-rank times.  The helpers
take an explicit process group and work with any torch.distributed backend
(NCCL for CUDA tensors, gloo for CPU tensors).

A single walk also partitions by row: T~^dag, P and T~ never change
(jc, j, b1), so a rank owning a set of rows advances them alone, and S -- which
sends a branch to row (kc, k, b2) -- is the one exchange per step.
``row_owner`` is that ownership map.
"""
from __future__ import annotations

import os


def env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(count: int, rank: int, world: int) -> range:
    """Contiguous block of ``count`` units owned by ``rank``; blocks cover all
    units once and differ in size by at most one."""
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def instance_seed_offset(rank: int, count: int) -> int:
    """Seed offset giving each rank its own independent instances."""
    return rank * count


def row_owner(j: int, world: int) -> int:
    """Rank that owns every row (jc, j, b1) of column index j."""
    return j % world


def max_over_ranks(value: float, group=None, device=None) -> float:
    """Maximum of a per-rank float over the group (identity without one)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def barrier(group=None) -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
