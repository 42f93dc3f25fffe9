"""Host logic of the multi-rank bench on CPU: world_size-2 gloo ranks shard the energy
grid without overlap and the timing reduction takes the max over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    t = bench.max_over_ranks(world, 1.0 + rank)
    grid = np.linspace(0.0, 1.0, 1024)
    shard = bench.shard_energies(grid, 64, rank, world)
    bench.barrier(world)
    out.put((rank, t, shard.tolist()))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert res[0][1] == res[1][1] == 2.0              # max over ranks
    a, b = set(res[0][2]), set(res[1][2])
    assert len(a) == 64 and len(b) == 64 and not (a & b)


def test_single_rank_shard_spreads_over_grid():
    import bench
    grid = np.linspace(0.0, 1.0, 1024)
    s = bench.shard_energies(grid, 64, 0, 1)
    assert len(set(s.tolist())) == 64 and s.min() == 0.0 and s.max() > 0.9
