"""The N > 1 host logic of bench.py on CPU: two gloo ranks aggregate their
replicas' times (max) and work (sum) the way the GPU run does over NCCL."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, total = bench.aggregate(torch, dist, 10.0 + 5.0 * rank, 1000.0 * (rank + 1))
    out[rank] = (ms, total)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregate():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (15.0, 3000.0)


def test_single_rank_identity():
    import bench

    assert bench.aggregate(None, None, 7.0, 42.0) == (7.0, 42.0)


def _worker_one_leaves(rank, world, port, out):
    import datetime

    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    import bench

    if rank == 1:
        out[rank] = "left"  # a replica that fails between steps and never reaches the aggregation
        return
    try:
        bench.aggregate(torch, dist, 10.0, 1000.0)
        out[rank] = "no error"
    except Exception as e:  # the collective ends with an error instead of waiting forever
        out[rank] = "error: " + type(e).__name__


def test_rank_that_leaves_ends_the_collective_with_an_error():
    """Failure detection on the host: when one replica leaves between steps,
    the others' next collective fails after the process group's timeout
    rather than hanging."""
    pytest.importorskip("torch")
    import time

    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        t0 = time.time()
        mp.spawn(_worker_one_leaves, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[1] == "left"
    assert res[0].startswith("error"), res[0]
    assert time.time() - t0 < 60
