"""Multi-process helpers (one process per GPU, torch.distributed).

GP fitness evaluation partitions by programs: programs are independent, so
ranks evaluate disjoint shards and nothing is exchanged on the data path.
These helpers give each rank its shard and reduce timings and counts for
reporting (max of times over ranks, sum of work over ranks).  They work with
any backend (NCCL on GPUs, gloo on CPU for tests) and degrade to the
single-process identity when torch.distributed is not initialised.
"""
from __future__ import annotations


def world():
    """(rank, world size) of this process (0, 1 without torch.distributed)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard(n: int, rank: int, world_size: int):
    """Contiguous, balanced [begin, end) of n units for `rank` of `world_size`."""
    if world_size <= 0 or not 0 <= rank < world_size:
        raise ValueError("bad rank or world size")
    base, extra = divmod(n, world_size)
    begin = rank * base + min(rank, extra)
    return begin, begin + base + (1 if rank < extra else 0)


def population_seed(base_seed: int, rank: int) -> int:
    """Seed of the population a rank evaluates when each rank has its own."""
    return base_seed + 1000 * rank


def _reduce(value: float, op: str, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(value: float, device=None) -> float:
    return _reduce(value, "max", device)


def sum_over_ranks(value: float, device=None) -> float:
    return _reduce(value, "sum", device)
