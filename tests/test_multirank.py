"""Host logic of the multi-rank bench on CPU: two gloo ranks (one process
each), the barrier and the max-over-ranks reduction bench.py uses for its
timing.  The rSVD itself is not sharded (every box has one GPU and the bench
runs N independent replicas), so no data-path collective is tested.  A rank
that leaves between steps is injected on the host (a process that exits
before the barrier) and the other rank must get an error, not hang."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        m = bench.max_over_ranks(world, 1.5 + rank, "cpu")
        out.put((rank, m))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_barrier_and_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_single_rank_helpers_are_identities():
    import bench
    bench.barrier(1)
    assert bench.max_over_ranks(1, 3.25, "cpu") == 3.25


def _worker_fails(rank, world, port, out):
    """Rank 1 dies between steps (before the barrier); rank 0 must see an
    error from the barrier within the process group's timeout, not hang."""
    import datetime

    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)  # an injected failure: the rank leaves without a word
    try:
        bench.barrier(world)
        out.put((rank, "no error"))
    except Exception as exc:  # the failure, detected on the host
        out.put((rank, "error: " + type(exc).__name__))
    finally:
        try:
            dist.destroy_process_group()
        except Exception:
            pass


def test_a_rank_that_leaves_is_detected_by_the_others():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_fails, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        rank, what = q.get(timeout=120)
    finally:
        for p in procs:
            p.join(30)
            if p.is_alive():
                p.kill()
                p.join(10)
    assert rank == 0 and what.startswith("error"), what
    assert procs[1].exitcode == 3
