"""bench.py's multi-rank bookkeeping on the CPU: two gloo ranks (spawned
processes on 127.0.0.1) with unequal step times agree on the slowest rank's
time, and the whole-job value divides it by the units both ranks processed;
the reference arm does no work on ranks other than 0.  Every rank computes
its own C(n) (replicas), so no data moves between ranks."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q) -> None:
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 0.25 + 0.5 * rank      # rank 1 is the slow one
        t = bench.slowest_rank(local, dist)
        q.put((rank, t, bench.per_unit(t, 5, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [r for r, _, _ in got] == [0, 1]
    for _, t, v in got:
        assert t == pytest.approx(0.75)
        assert v == pytest.approx(0.75 / (5 * 2))   # 10 C(n) in 0.75 s
    assert all(p.exitcode == 0 for p in procs)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.slowest_rank(1.25) == 1.25
    assert bench.per_unit(1.25, 5, 1) == pytest.approx(0.25)


def test_reference_arm_skips_other_ranks():
    import bench

    class Args:
        n, steps, warmup, gpus = 1000, 1, 0, 2

    assert bench.run_reference(Args(), rank=1, world=2) is None
