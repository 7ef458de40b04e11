"""Replica bookkeeping for running the path on several GPUs.

The problems the path is applied to are independent units (Krylov directions,
illuminations, finite-difference perturbations), so each rank runs its own
problems with its own context and no exchange happens while propagating.
The one reduction the method has is the sum of per-illumination gradients
(eq. fre: the gradient of eq. obj_couple is sum_q D^* Lambda_q (Lambda_q -
P-hat_q)), done once per outer iteration through ``sum_over_ranks``.
"""
from __future__ import annotations

import os
from typing import List


def world():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def assign(n_units: int, rank: int, world_size: int) -> List[int]:
    """Units (e.g. illuminations) of this rank: a contiguous, balanced block."""
    base, extra = divmod(n_units, world_size)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(t):
    """In-place sum of a tensor over ranks (the gradient sum over illuminations)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def throughput(units_per_rank: float, world_size: int, max_seconds: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / max_seconds
