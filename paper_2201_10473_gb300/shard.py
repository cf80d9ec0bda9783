"""Multi-GPU sharding of independent products (weak scaling, no collective
on the data path).

Products are independent units: with one process per GPU, rank r multiplies
its own contiguous slice of the work; ranks meet only at a barrier around
the timed region and in one MAX reduction of the elapsed time.  Under the
nccl backend the reduction runs on a CUDA tensor, under gloo on the CPU.
"""
from __future__ import annotations

import os


def world_info():
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard_range(rank: int, world: int, per_rank: int) -> range:
    """Products of `rank` when every rank multiplies `per_rank` of them (weak scaling)."""
    if not 0 <= rank < world or per_rank < 0:
        raise ValueError("bad rank / world / per_rank")
    return range(rank * per_rank, (rank + 1) * per_rank)


def split_range(rank: int, world: int, total: int) -> range:
    """Contiguous near-equal slice of `total` products for `rank` (strong scaling)."""
    if not 0 <= rank < world or total < 0:
        raise ValueError("bad rank / world / total")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """MAX of `value` over all ranks (identity without an initialised group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def whole_job_rate(units_per_rank: int, world: int, seconds_max: float) -> float:
    """Units of all ranks divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max
