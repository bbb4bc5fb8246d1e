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
