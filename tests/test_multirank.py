"""World-size-2 gloo tests of the multi-GPU host logic on the CPU: the probe-point
partition and the coarse-array gather reproduce the single-process layout exactly."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2609_16408_gb300.shard import gather_coarse, probe_point_shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_probe_point_once():
    for P, nw, world in [(216, 8, 2), (17576, 10, 8), (5, 3, 4), (1, 1, 3)]:
        seen = np.zeros((nw, P), dtype=int)
        sizes = []
        for r in range(world):
            p, f = probe_point_shard(P, nw, r, world)
            seen[f, p] += 1
            sizes.append(len(p))
        assert np.all(seen == 1)
        assert max(sizes) - min(sizes) <= 1


def _fake_d(p, f):
    return -1e-3 * (1.0 + 0.1 * f) * np.cos(0.37 * p)


def _worker(rank, world, port, P, nw, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p, f = probe_point_shard(P, nw, rank, world)
    d = torch.from_numpy(_fake_d(p, f))
    full = gather_coarse(d, P, nw, rank, world)
    # the timed interval is max-reduced across ranks
    t = torch.tensor([float(rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, full.numpy(), float(t.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("P,nw", [(216, 8), (13, 3)])
def test_gather_reproduces_single_process_array(P, nw):
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, P, nw, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    ref = np.zeros((nw, P))
    for f in range(nw):
        ref[f] = _fake_d(np.arange(P), np.full(P, f))
    for rank, full, tmax in res:
        assert np.array_equal(full, ref)
        assert tmax == 2.0
