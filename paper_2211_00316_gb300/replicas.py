"""Multi-GPU replicas: one process per GPU, independent jobs, no data-path collective.

The update of one reconstruction job does not shard across GPUs here; independent jobs
(slices, patients, phantom seeds) do. Each rank runs its own jobs; the only collectives
are the timing barrier and a max over ranks of the elapsed time, so the reported
throughput is the units all ranks processed divided by the slowest rank's time (weak
scaling).
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass
class RankInfo:
    rank: int
    world: int
    local: int

    @staticmethod
    def from_env() -> "RankInfo":
        return RankInfo(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                        int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank: int, base: int = 0) -> int:
    """Phantom seed of this rank's replica job."""
    return base + rank


def assign_slices(n_slices: int, rank: int, world: int) -> list[int]:
    """Round-robin assignment of independent slices to ranks (a partition of range(n_slices))."""
    return list(range(rank, n_slices, world))


def max_over_ranks(value: float, device: str | torch.device = "cpu") -> float:
    """Largest value over all ranks (identity without an initialised process group)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device: str | torch.device = "cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_throughput(units_all_ranks: float, slowest_seconds: float) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    return units_all_ranks / slowest_seconds
