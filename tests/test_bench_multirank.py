"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
owns its own sequences (weak scaling, no data-path collective) and the job
time is the slowest rank's."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = bench.shard(rank, world, 5)
    wl = bench.make_workload("C2", rank, 5)
    t = bench.max_over_ranks(10.0 + rank, dist)
    q.put((rank, ids, wl.x0.tolist(), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ids0, x00, t0), (r1, ids1, x01, t1) = out
    assert ids0 == list(range(0, 5)) and ids1 == list(range(5, 10))
    assert not np.allclose(x00, x01)            # each rank simulates its own sequences
    assert t0 == t1 == 11.0                     # max over ranks
