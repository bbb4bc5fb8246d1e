"""Multi-process helpers for running the step on several GPUs of one node (one process per GPU).

The full-order and reduced-order steps do not exchange data between GPUs: a batch of independent
instances is split into contiguous ranges of whole instances (`shard_instances`), and the only
collective is the reduction of timings or error sums (`max_over_ranks`, `sum_over_ranks`).  The
functions work with any initialised torch.distributed process group (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch


def shard_instances(n_inst: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous range [lo, hi) of whole instances for `rank` out of `world`; sizes differ by at
    most one, every instance is owned by exactly one rank."""
    if world < 1 or not 0 <= rank < world or n_inst < 0:
        raise ValueError("bad shard request")
    q, rem = divmod(n_inst, world)
    lo = rank * q + min(rank, rem)
    return lo, lo + q + (1 if rank < rem else 0)


def _reduce(value: float, op, device) -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value: float, device="cpu") -> float:
    """The maximum of `value` over all ranks (the slowest rank's time)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.MAX, device)


def sum_over_ranks(value: float, device="cpu") -> float:
    """The sum of `value` over all ranks (e.g. error numerators and denominators)."""
    import torch.distributed as dist
    return _reduce(value, dist.ReduceOp.SUM, device)
