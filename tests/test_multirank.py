"""Host logic of the multi-GPU bench on CPU ranks (gloo, world size 2): each rank
advances its own replica, and rank 0 reports total units over the slowest rank."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, u = bench.reduce_over_ranks(1.0 + rank, 100.0 * (rank + 1), world)
    out[rank] = (t, u)
    dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        assert out[r] == (2.0, 300.0)   # max time, summed units


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(1.5, 7.0, 1) == (1.5, 7.0)
