"""Multi-process helpers: one process per GPU, no collective on the data path.

Poses are independent and so are decks, so the path shards without any
exchange: a rank either docks its own deck (weak scaling, what the benchmark
does) or a contiguous slice of one deck's poses.  The only collectives are
the benchmark's barrier and the max-over-ranks of its step time; they work
on any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def rank_seed(base: int, rank: int) -> int:
    """Seed of the deck a rank docks in the weak-scaling benchmark."""
    return base + rank


def shard_range(n: int, rank: int, world_size: int) -> tuple[int, int]:
    """Contiguous [lo, hi) slice of n poses owned by rank (sizes differ by <= 1)."""
    if world_size < 1 or not 0 <= rank < world_size or n < 0:
        raise ValueError("bad shard arguments")
    lo = n * rank // world_size
    hi = n * (rank + 1) // world_size
    return lo, hi


def max_over_ranks(value: float, device=None) -> float:
    """The largest value over all ranks (the slowest rank's step time)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, ms_per_step_max: float, world_size: int) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's step time."""
    if ms_per_step_max <= 0:
        raise ValueError("step time must be positive")
    return world_size * units_per_rank / (ms_per_step_max / 1e3)
