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


def _worker_shard(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_1008_1685_gb300 as picrr

    scan = [bench.scan_desc(i) for i in range(256)]
    ranks, loads = bench.shard(picrr, scan, world)
    mine = [i for i, r in enumerate(ranks) if r == rank]
    reqs = bench.serve_requests(20.0, 4.0, 77)
    cfg = dict(bench.SERVE, window_s=4.0)
    stream = [d["seed"] for _, d in bench.my_requests(picrr, cfg, bench.SCAN, rank, world)]
    gathered = [None] * world
    dist.all_gather_object(gathered, (ranks, mine, stream, list(loads)))
    out[rank] = gathered
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_split_one_scan_and_one_stream():
    """The 256-run scan and a request stream are split over two gloo ranks by
    pic_shard_runs (host only): both ranks compute the same assignment with
    no exchange, every run and every request goes to exactly one rank, and
    the work is balanced."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp

    from paper_1008_1685_gb300 import build as b

    b.build()
    import bench

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker_shard, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    g0, g1 = res[0], res[1]
    assert g0 == g1  # both ranks saw the same gathered data
    (ranks0, mine0, stream0, loads0), (ranks1, mine1, stream1, loads1) = g0
    assert ranks0 == ranks1  # the same assignment, computed independently
    assert sorted(mine0 + mine1) == list(range(256)) and not set(mine0) & set(mine1)
    assert max(loads0) / min(loads0) < 1.02  # largest-first greedy balances 256 uneven runs
    seeds = [d["seed"] for _, d in bench.serve_requests(20.0, 4.0, 77)]
    assert sorted(stream0 + stream1) == sorted(seeds) and not set(stream0) & set(stream1)
    assert stream0 and stream1


def test_shard_runs_budget_and_order():
    """pic_shard_runs on the host: a budget that holds one run per rank
    spreads them, one that holds none fails with PIC_ERR_OOM, in_order keeps
    the arrival order of the greedy choice."""
    from paper_1008_1685_gb300 import build as b

    b.build()
    import paper_1008_1685_gb300 as picrr

    d = [picrr.run_desc(30.0, 10.0, 1.0, 100.0, 300.0, 0, 20.0, 1000, ppc=64, seed=i) for i in range(4)]
    ranks, work = picrr.shard_runs(d, 4, 500.0)
    assert sorted(ranks) == [0, 1, 2, 3] and len(set(work)) == 1
    big = [picrr.run_desc(30.0, 10.0, 1.0, 100.0, 300.0, 0, 20.0, 1000 * (i + 1), ppc=64, seed=i) for i in range(3)]
    ranks, _ = picrr.shard_runs(big, 2, 500.0, in_order=True)
    assert ranks == [0, 1, 0]  # run 2 goes where the least work is (rank 0 holds 1000 steps, rank 1 2000)
    ranks, _ = picrr.shard_runs(big, 2, 500.0)
    assert ranks == [1, 1, 0]  # largest first: run 2 to rank 0, run 1 to rank 1, run 0 to the lighter rank 1
    with pytest.raises(picrr.PicError) as e:
        picrr.shard_runs(d, 2, 500.0, budget_per_rank=1000)
    assert e.value.status == -3
