"""Multi-process helpers: one process per GPU, no collective on the data path.

Poses are independent and so are decks, so the path shards without any
exchange: a rank docks its own deck (weak scaling, what the benchmark does),
a contiguous slice of one deck's poses, or, for a batch of uneven decks, the
decks that a longest-processing-time-first assignment by pair count gives it.
The only collectives are the benchmark's barrier and the max-over-ranks of
its step time; they work on any torch.distributed backend (NCCL on GPUs,
gloo on CPU).
"""
from __future__ import annotations

import math
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


def deck_cost(n_lig: int, n_pro: int, n_poses: int) -> int:
    """Work of one deck: its ligand x protein x pose pair evaluations."""
    return int(n_lig) * int(n_pro) * int(n_poses)


def lpt_partition(costs, world_size: int) -> list[list[int]]:
    """Indices of the items (decks) each rank takes: longest processing time
    first, each item in turn (largest cost first, ties by index) to the rank
    with the least load so far (ties by rank).  Deterministic, so every rank
    computes the same assignment without an exchange; its largest load is at
    most (4/3 - 1/(3 world_size)) of the best possible (Graham, 1969)."""
    if world_size < 1:
        raise ValueError("world_size must be positive")
    costs = [float(c) for c in costs]
    if any(c < 0 for c in costs):
        raise ValueError("costs must be non-negative")
    loads = [0.0] * world_size
    parts: list[list[int]] = [[] for _ in range(world_size)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world_size), key=lambda q: (loads[q], q))
        parts[r].append(i)
        loads[r] += costs[i]
    return [sorted(p) for p in parts]


def split_and_partition(shapes, world_size: int) -> list[list[tuple[int, int, int]]]:
    """Work of each rank for a batch of uneven decks, as (deck, lo, hi) pose
    slices.  A deck whose pair count exceeds the per-rank average is cut into
    that many contiguous pose slices (rounded up, sizes within one pose of
    each other), so no single piece dominates a rank; the pieces then go to
    the ranks by lpt_partition.  shapes: (n_lig, n_pro, n_poses) per deck."""
    if world_size < 1:
        raise ValueError("world_size must be positive")
    costs = [deck_cost(*s) for s in shapes]
    avg = sum(costs) / world_size if costs else 0.0
    pieces: list[tuple[int, int, int]] = []
    piece_cost: list[float] = []
    for d, ((nl, npro, npo), c) in enumerate(zip(shapes, costs)):
        k = min(int(npo), math.ceil(c / avg)) if avg > 0 and c > avg else 1
        for r in range(k):
            lo, hi = shard_range(int(npo), r, k)
            pieces.append((d, lo, hi))
            piece_cost.append(float(deck_cost(nl, npro, hi - lo)))
    parts = lpt_partition(piece_cost, world_size)
    return [[pieces[i] for i in p] for p in parts]


SHARD_MODES = ("decks", "poses", "batch")


def shard_pieces(mode: str, rank: int, world_size: int, n_poses: int = 0, batch_shapes=None):
    """The work one rank evaluates, as (pieces, total_units, scaling).

    pieces are (deck, lo, hi) slices of a deck's poses:
      "decks"  each rank docks its own deck (deck index = rank), all its poses:
               independent problems, weak scaling;
      "poses"  one deck (index 0) whose n_poses are cut into contiguous slices,
               one per rank: strong scaling;
      "batch"  a batch of uneven decks (batch_shapes: (n_lig, n_pro, n_poses)
               per deck) split and assigned by split_and_partition: strong
               scaling.
    total_units is the number of poses all ranks evaluate together.  Every
    rank computes the same assignment, so nothing is exchanged."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad rank or world size")
    if mode == "decks":
        return [(rank, 0, int(n_poses))], world_size * int(n_poses), "weak"
    if mode == "poses":
        lo, hi = shard_range(int(n_poses), rank, world_size)
        return [(0, lo, hi)], int(n_poses), "strong"
    if mode == "batch":
        if not batch_shapes:
            raise ValueError("batch mode needs the decks' shapes")
        parts = split_and_partition(batch_shapes, world_size)
        return parts[rank], sum(int(s[2]) for s in batch_shapes), "strong"
    raise ValueError(f"unknown shard mode {mode!r}; one of {SHARD_MODES}")
