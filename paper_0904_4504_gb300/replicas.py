"""Replicas across ranks (one process per GPU).

The units of work of this method are independent: the instances of a tau*omega x AR sweep and the
requests of a serving stream each run a whole lattice on one GPU, and no step needs data of
another instance.  N ranks therefore share work with no collective on the data path (weak
scaling: each rank does the per-rank work of one GPU).  The only collectives are on the host side
of a measurement: a barrier around the timed region and the maximum of the ranks' times.  These
helpers run on any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import os


def env_rank():
    """(rank, world size, local rank) from the launcher's environment (1 process if unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_slice(items, rank: int, per_rank: int):
    """The rank's own block of a shared sequence: items [rank * per_rank, (rank + 1) * per_rank).
    Blocks of different ranks are disjoint and together are the first world * per_rank items."""
    if rank < 0 or per_rank < 0:
        raise ValueError("rank and per_rank must be >= 0")
    return items[rank * per_rank:(rank + 1) * per_rank]


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """Maximum of a host scalar over all ranks (the time of the slowest rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units all ranks processed per second of the slowest rank (weak scaling)."""
    if not seconds_max > 0:
        raise ValueError("need a positive time")
    return units_per_rank * world / seconds_max
