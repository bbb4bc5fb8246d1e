"""Multi-process helpers for running the step on several GPUs of one node (one process per GPU).

The full-order and reduced-order steps do not exchange data between GPUs: a batch of independent
instances is split into contiguous ranges of whole instances (`shard_instances`, `scene_shard`),
and the only collective of a run is the reduction of timings or error sums (`max_over_ranks`,
`sum_over_ranks`).  Batched snapshot generation (`generate_snapshots_sharded`) steps each rank's
instances alone, then gathers the snapshot stores once so that every rank holds the whole store,
in instance order, for data-parallel training.
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


def scene_shard(scene, rank: int, world: int):
    """This rank's whole instances of a batched scene (a contiguous range, shard_instances): the
    sub-scene and its (lo, hi) instance range."""
    lo, hi = shard_instances(scene.n_inst, rank, world)
    return scene.subset_instances(range(lo, hi)), (lo, hi)


def gather_instance_rows(local: torch.Tensor) -> torch.Tensor:
    """All ranks' (J, P_rank, c) arrays of per-particle rows, concatenated along the particle axis
    in rank order (the instance order of scene_shard): one all-gather of arrays padded to the
    largest shard.  Returns `local` itself on one rank."""
    import torch.distributed as dist
    rank, world = _world()
    if world == 1:
        return local
    n = torch.tensor([local.shape[1]], dtype=torch.int64, device=local.device)
    sizes = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(sizes, n)
    sizes = [int(t.item()) for t in sizes]
    pmax = max(sizes)
    pad = torch.zeros((local.shape[0], pmax, local.shape[2]), dtype=local.dtype, device=local.device)
    pad[:, :local.shape[1]] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:, :m] for p, m in zip(parts, sizes)], dim=1)


def generate_snapshots_sharded(scene, n_steps: int, every: int, device="cuda"):
    """Batched snapshot generation over the ranks: each rank steps its own whole instances
    (scene_shard, no exchange while stepping), then x, v and F are gathered once
    (gather_instance_rows) so that every rank returns the store of the whole scene, in the layout
    of train.generate_snapshots.  The status word is OR-ed over the ranks."""
    import numpy as np
    import torch.distributed as dist
    from .train import generate_snapshots
    rank, world = _world()
    if world == 1:
        return generate_snapshots(scene, n_steps, every, device)
    sub, _ = scene_shard(scene, rank, world)
    part = generate_snapshots(sub, n_steps, every, device)
    J = n_steps // every + 1
    d = scene.dim
    full = {k: gather_instance_rows(part[k].reshape(J, -1, part[k].shape[-1])).reshape(-1, part[k].shape[-1])
            for k in ("x", "v", "F")}
    st = torch.tensor([int(part["status"])], dtype=torch.int64, device=part["x"].device)
    words = [torch.zeros_like(st) for _ in range(world)]
    dist.all_gather(words, st)
    status = 0
    for w in words:
        status |= int(w.item())
    n_inst = scene.n_inst
    S = J * n_inst
    snap_inst = np.array([s % n_inst for s in range(S)], np.int32)
    snap_next = np.array([s + n_inst if s + n_inst < S else -1 for s in range(S)], np.int32)
    return dict(dim=d, n_inst=n_inst, inst_offsets=np.ascontiguousarray(scene.inst_offsets, np.int64),
                X=torch.from_numpy(scene.x.astype(np.float32)).to(device), n_snap=S, snap_inst=snap_inst,
                snap_next=snap_next, x=full["x"], v=full["v"], F=full["F"], status=status,
                steps_between=every, dt_snap=part["dt_snap"])
