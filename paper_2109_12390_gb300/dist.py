"""Multi-process helpers for running the step on several GPUs of one node (one process per GPU).

The full-order and reduced-order steps do not exchange data between GPUs: a batch of independent
instances is split into contiguous ranges of whole instances (`shard_instances`), and the only
collective is the reduction of timings or error sums (`max_over_ranks`, `sum_over_ranks`).
Decoder training is data-parallel: each rank draws a contiguous range of the step's minibatch
(`shard_minibatch`), its gradients are normalised by the whole minibatch, and one sum over the
ranks (`allreduce_gradients`) of the decoder's and the latents' gradients precedes every update
(`train_data_parallel`).  The functions work with any initialised torch.distributed process group
(NCCL on GPUs, gloo on CPU).
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


def _world():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def shard_minibatch(global_batch: int, rank: int, world: int) -> tuple[int, int]:
    """(first draw, draws) of `rank`'s contiguous share of a minibatch of `global_batch` points:
    the trainer's shard_index / shard_count.  The minibatch must divide evenly."""
    if world < 1 or not 0 <= rank < world or global_batch < world or global_batch % world:
        raise ValueError("the minibatch must split evenly over the ranks")
    local = global_batch // world
    return rank * local, local


def allreduce_gradients(*tensors) -> None:
    """Sums each gradient tensor over all ranks in place (no-op on one rank)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)


def train_data_parallel(trainer, n_steps: int) -> None:
    """n_steps data-parallel optimisation steps of a Trainer created with this rank's
    shard_index / shard_count: each step computes this rank's gradients, sums them over the ranks,
    and applies the same Adam step on every rank (the replicas stay identical)."""
    g_params, g_second = trainer.gradient_buffers()
    for _ in range(n_steps):
        trainer.compute_gradients(g_params, g_second)
        allreduce_gradients(g_params, g_second)
        trainer.apply_gradients(g_params, g_second)
