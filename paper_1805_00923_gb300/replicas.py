"""Multi-GPU as independent replicas (the single-graph path has no exchange step).

With N processes (one GPU each, launched by torchrun), every rank runs its own
copy of the workload or its own share of independent queries; the only
communication is host-side: a barrier before and after the timed region, the
maximum of the ranks' elapsed times, and gathering per-rank results.  These
helpers work with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the torchrun environment (1, 0, 0 if absent)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_items: int, rank: int, world_size: int) -> range:
    """Contiguous block of item indices owned by `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_items, world_size)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def shard_balanced(costs, rank: int, world_size: int) -> list[int]:
    """Item indices owned by `rank` when items of the given costs are dealt
    longest first to the rank with the least cost so far (ties to the lower
    rank): every item exactly once, deterministic on every rank."""
    load = [0.0] * world_size
    owner = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i)):
        r = min(range(world_size), key=lambda r: (load[r], r))
        owner[i] = r
        load[r] += float(costs[i])
    return [i for i in range(len(costs)) if owner[i] == rank]


def max_over_ranks(x: float, device: str = "cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device: str = "cpu") -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def gather_objects(obj):
    """List of every rank's `obj` (on all ranks)."""
    if not (dist.is_available() and dist.is_initialized()):
        return [obj]
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, obj)
    return out
