"""The sharding plan (paper_2601_11621_gb300/shard.py) on the CPU: ranges of
the grouped primes balanced by bit weight, root bounds that hold the real
roots, a binomial combining schedule in which every rank sends once and only
after it has received everything, and the whole plan carried out by gloo
ranks (2 and 4 spawned processes on 127.0.0.1) whose subtree products come
from the CPU oracle inside the test: rank 0 ends with the product of all the
primes."""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from paper_2601_11621_gb300 import shard


def g1_primes(orc, n=20000):
    exps, offs, gp = orc.factor(orc.CATALAN, n)
    g = list(exps).index(1)
    return gp[int(offs[g]): int(offs[g + 1])]


@pytest.mark.parametrize("parts", [1, 2, 3, 4, 7, 8])
def test_ranges_balanced_by_bits(orc, parts):
    p = g1_primes(orc)
    b = shard.partition_by_bits(p, parts)
    assert b[0] == 0 and b[-1] == len(p) and all(x <= y for x, y in zip(b, b[1:]))
    w = [float(np.log2(p[b[r]:b[r + 1]].astype(np.float64)).sum()) for r in range(parts)]
    total = sum(w)
    for x in w:
        assert abs(x - total / parts) <= 33.0  # within one prime's bits of the mean


def test_root_bounds_hold_the_roots(orc):
    p = g1_primes(orc)
    P = shard.plan(p, 4)
    for rk in P["ranks"]:
        root = orc.product_tree(p[rk["lo"]:rk["hi"]])
        # each prime adds less than one bit beyond log2 p to the bound
        assert len(root) <= rk["root_limbs"] <= len(root) + (rk["hi"] - rk["lo"]) // 32 + 1
    whole = len(orc.product_tree(p))
    assert P["rounds"][-1][0]["product_limbs"] >= whole


@pytest.mark.parametrize("parts", [1, 2, 3, 5, 8, 16])
def test_schedule_sends_once_after_receiving(parts):
    rounds = shard.combine_schedule(parts)
    assert len(rounds) == (0 if parts == 1 else (parts - 1).bit_length())
    sent, received = {}, {r: [] for r in range(parts)}
    for k, pairs in enumerate(rounds):
        for dst, src in pairs:
            assert src not in sent and dst not in sent
            assert all(k2 < k for k2 in received[src])  # src is complete
            sent[src] = k
            received[dst].append(k)
    assert sorted(sent) == list(range(1, parts))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist

    import oracle as orc
    from paper_2601_11621_gb300 import shard as sh
    orc.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = g1_primes(orc)
        P = sh.plan(p, world)
        me = P["ranks"][rank]
        root = orc.product_tree(p[me["lo"]:me["hi"]])   # this rank's subtree
        for step in P["rounds"]:
            for pr in step:
                if pr["send"] == rank:
                    n = torch.tensor([len(root)], dtype=torch.int64)
                    dist.send(n, pr["recv"])
                    dist.send(torch.from_numpy(root.view(np.int32).copy()), pr["recv"])
                elif pr["recv"] == rank:
                    n = torch.zeros(1, dtype=torch.int64)
                    dist.recv(n, pr["send"])
                    assert int(n) <= pr["send_limbs"]
                    buf = torch.zeros(int(n), dtype=torch.int32)
                    dist.recv(buf, pr["send"])
                    root = orc.mul(root, buf.numpy().view(np.uint32))
                    assert len(root) <= pr["product_limbs"]
        if rank == 0:
            q.put(bool(np.array_equal(root, orc.product_tree(p))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_plan_carried_out_by_gloo_ranks(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    try:
        ok = q.get(timeout=180)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert ok
    assert all(p.exitcode == 0 for p in procs)
