"""Replicas across GPUs.

The path has no exchange step: every rank renders and differentiates its own
scene with its own seeds and reads nothing from the other ranks.  A run on N
GPUs is N independent replicas; the only cross-rank operations are a barrier
and the maximum of the elapsed times, so the aggregate throughput is the
units of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import os


def rank_info() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def replica_seeds(scene_seed: int, adjoint_seed: int, rank: int) -> tuple[int, int]:
    """Seeds of rank's replica: distinct scenes and loss adjoints per rank."""
    return scene_seed + rank, adjoint_seed + rank


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """Maximum of x over all ranks (x itself without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Units per second of the whole job: world * units / slowest time."""
    if ms <= 0:
        raise ValueError("elapsed time must be positive")
    return world * float(units_per_rank) / (ms / 1e3)
