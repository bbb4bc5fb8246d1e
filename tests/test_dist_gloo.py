"""The multi-GPU path's host logic on CPU: two gloo ranks (world size 2) share a batch of
independent instances with no data exchange and reduce only their timings and error sums."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2109_12390_gb300.dist import max_over_ranks, shard_instances, sum_over_ranks


def test_shard_instances_partition():
    for n in (0, 1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            ranges = [shard_instances(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_instances(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = shard_instances(7, rank, world)
    owned = list(range(lo, hi))
    # each rank "times" its own instances and accumulates an error numerator over them
    t = 10.0 + rank
    num = float(sum(i * i for i in owned))
    q.put((rank, owned, max_over_ranks(t), sum_over_ranks(num)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_instances_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    owned = [o[1] for o in out]
    assert sorted(owned[0] + owned[1]) == list(range(7)) and not set(owned[0]) & set(owned[1])
    assert all(o[2] == 11.0 for o in out)                      # slowest rank's time on both
    assert all(o[3] == float(sum(i * i for i in range(7))) for o in out)


def test_shard_minibatch_partition():
    from paper_2109_12390_gb300.dist import shard_minibatch
    for world in (1, 2, 4):
        parts = [shard_minibatch(4096, r, world) for r in range(world)]
        assert parts[0][0] == 0 and sum(n for _, n in parts) == 4096
        assert all(a[0] + a[1] == b[0] for a, b in zip(parts, parts[1:]))
    with pytest.raises(ValueError):
        shard_minibatch(10, 0, 4)


def _dp_worker(rank, world, port, q):
    """One data-parallel rank on the CPU: the oracle's gradients of this rank's contiguous share of
    a minibatch, normalised by the whole minibatch (as the GPU trainer normalises a shard), summed
    over the ranks by the same helper the GPU path uses."""
    import numpy as np
    import oracle.decoder as OD
    import synth.scenes as S
    from paper_2109_12390_gb300.dist import allreduce_gradients, shard_minibatch
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    batch, latents, p = _dp_problem()
    n = len(batch["X"])
    lo, cnt = shard_minibatch(n, rank, world)
    mine = {k: v[lo:lo + cnt] for k, v in batch.items()}
    _, gW, gb, gl = OD.batch_loss_grads(p, latents, mine, 0.01, 3.0, 0.05)
    flat = np.concatenate([g.ravel() for g in gW + gb] + [gl.ravel()]) * (cnt / n)
    t = torch.from_numpy(flat)
    allreduce_gradients(t)
    q.put((rank, t.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _dp_problem():
    import numpy as np
    import oracle.decoder as OD
    import synth.scenes as S
    rng = np.random.default_rng(5)
    d, r, n_snap, n = 2, 4, 6, 64
    p = S.xavier_decoder(9, d, r, 16, 2, OD.ELU, X_min=np.zeros(d), X_range=np.ones(d), bias_scale=0.2)
    p.width = 16
    latents = rng.normal(size=(n_snap, r))
    snap = rng.integers(0, n_snap, size=n)
    nxt = np.where(snap + 1 < n_snap, snap + 1, -1)
    batch = dict(X=rng.uniform(size=(n, d)), snap=snap, next=nxt, x=rng.normal(size=(n, d)),
                 F=np.eye(d)[None] + 0.1 * rng.normal(size=(n, d, d)), v=rng.normal(size=(n, d)))
    return batch, latents, p


def test_two_gloo_ranks_data_parallel_gradients_equal_the_whole_minibatch():
    import numpy as np
    import oracle.decoder as OD
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dp_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=120) for _ in procs), key=lambda o: o[0])
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    batch, latents, p = _dp_problem()
    _, gW, gb, gl = OD.batch_loss_grads(p, latents, batch, 0.01, 3.0, 0.05)
    want = np.concatenate([g.ravel() for g in gW + gb] + [gl.ravel()])
    for _, got in out:
        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-14 * np.abs(want).max())


def _shard_worker(rank, world, port, q):
    import numpy as np
    import oracle.mpm as OM
    import synth.scenes as S
    from paper_2109_12390_gb300.dist import gather_instance_rows, scene_shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = S.batch_2d(seed=9, n_inst=5, count_range=(60, 200), n_grid=32, origin_y=0.1)
    sub, (lo, hi) = scene_shard(sc, rank, world)
    J = 3
    xs = []
    for j in range(J):
        if j:
            OM.step(sub, 4)
        xs.append(sub.x.copy())
    local = torch.from_numpy(np.stack(xs))                     # (J, P_rank, d)
    full = gather_instance_rows(local)
    q.put((rank, lo, hi, full.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_a_batched_run_and_gather_rows():
    """Instance sharding of a batched full-order run: two gloo ranks step their own whole instances
    with the FP64 oracle (no exchange while stepping) and gather the per-particle rows once; both
    ranks then hold exactly the rows of the unsharded run, in instance order."""
    import numpy as np
    import oracle.mpm as OM
    import synth.scenes as S
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=300) for _ in procs), key=lambda o: o[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    sc = S.batch_2d(seed=9, n_inst=5, count_range=(60, 200), n_grid=32, origin_y=0.1)
    ref = []
    for j in range(3):
        if j:
            OM.step(sc, 4)
        ref.append(sc.x.copy())
    ref = np.stack(ref)
    assert [(o[1], o[2]) for o in out] == [(0, 3), (3, 5)]
    for o in out:
        np.testing.assert_array_equal(o[3], ref)
