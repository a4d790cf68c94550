"""Replicas on several GPUs of one node.

The decode shards by queries with no exchange step (every query is independent,
Eq. 3): each rank decodes its own frame with its own copy of the textures and
weights, so a run on N GPUs is N replicas (weak scaling).  The only cross-rank
operations are the measurement's: a barrier around the timed region, the
slowest rank's time and the total work of all ranks.  Ranks come from the
launcher's environment (RANK, WORLD_SIZE, LOCAL_RANK).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_env() -> tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment; (0, 1, 0) without a launcher."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous query range [a, b) of `rank` when n queries are split over `world` ranks (strong scaling);
    the ranges cover [0, n) exactly, sizes differ by at most one."""
    q, r = divmod(n, world)
    a = rank * q + min(rank, r)
    return a, a + q + (1 if rank < r else 0)


def barrier() -> None:
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def aggregate(units: float, ms: float, device: str | torch.device = "cpu") -> tuple[float, float]:
    """(units of all ranks, slowest rank's milliseconds): the whole-job throughput is their ratio."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(units), float(ms)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())
