"""Replica-parallel host logic on two gloo ranks (CPU): dealing covers every
item once, the job's time is the slowest rank's and its rate counts the
units of all ranks."""
import os
import socket
import time

import pytest
import torch.multiprocessing as mp

from paper_2306_01301_b300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = replicas.rank_env()
    mine = replicas.deal(10, w, r)
    replicas.barrier(w)
    t0 = time.perf_counter()
    time.sleep(0.05 * (r + 1))  # rank 1 is the slower one
    dt = time.perf_counter() - t0
    rate, total, slowest = replicas.job_rate(len(mine), dt, w)
    q.put((r, mine, dt, rate, total, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    items = sorted(i for _, mine, *_ in out for i in mine)
    assert items == list(range(10))
    slow = max(dt for _, _, dt, *_ in out)
    for _, _, _, rate, total, slowest in out:
        assert total == 10 and slowest == pytest.approx(slow)
        assert rate == pytest.approx(10 / slow)


def test_single_rank_and_bad_ranks():
    assert replicas.deal(5, 1, 0) == [0, 1, 2, 3, 4]
    assert replicas.job_rate(7, 2.0, 1) == (3.5, 7.0, 2.0)
    with pytest.raises(ValueError):
        replicas.deal(5, 2, 2)
