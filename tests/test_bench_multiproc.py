"""The N > 1 path of bench.py (independent replicas; the slowest rank sets the
time) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    elapsed = 1.0 + rank  # rank 1 is the slower replica
    m = bench.max_over_ranks(elapsed, dist)
    v = bench.job_value(1000, world, m)
    dist.barrier()
    out[rank] = (m, v)
    dist.destroy_process_group()


def test_replicas_take_slowest_rank():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (2.0, 1000.0)


def test_single_rank_value():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.job_value(10, 1, 2.0) == 5.0
