"""The continuous-batching server (cat_server_*): every result is the same
as the request computed alone, whether it arrived in a burst, while other
batches were running, or alone; ticket bookkeeping and errors."""
import time

import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture
def server(cat_lib):
    from paper_2601_11621_gb300.server import Server
    sv = Server(0, hbm_budget_bytes=8 * 10**9, workers=2, max_batch=64)
    yield sv
    sv.close()


def alone(ctx, cat_lib, kind, n):
    return cat_lib.to_numpy(cat_lib.cat_exact(ctx, kind, n))


def test_burst_and_trickle_match_alone(ctx, cat_lib, orc, server):
    reqs = [(0, 10), (1, 7), (2, 12), (0, 200000), (2, 60000), (1, 150000), (0, 0), (2, 1),
            (0, 33333), (1, 4444), (2, 5555), (0, 999983)]
    tickets = [server.submit(k, n) for k, n in reqs[:6]]      # burst
    for k, n in reqs[6:]:                                      # trickle while running
        time.sleep(0.002)
        tickets.append(server.submit(k, n))
    for (k, n), t in zip(reqs, tickets):
        got = server.fetch_host(t)
        want = alone(ctx, cat_lib, k, n)
        assert got.shape == want.shape and (got == want).all(), (k, n)
        if n <= 5555:
            assert (got == orc.exact(k, n)).all()
        assert server.release(t) == 0
    q, total = server.pending()
    assert q == 0 and total == 0


def test_poisson_stream_matches_alone(ctx, cat_lib, server):
    from paper_2601_11621_gb300.server import replay_server
    stream = W.served_requests(48, rate=400.0, seed=7, lo=1e3, hi=3e5)
    lat, wall, results, nbatches = replay_server(server, stream, keep_results=True)
    assert len(results) == len(stream) and (lat > 0).all()
    for (a, k, n), got in zip(stream, results):
        want = alone(ctx, cat_lib, k, n)
        assert got.shape == want.shape and (got == want).all(), (k, n)


def test_ticket_errors(cat_lib, server):
    with pytest.raises(cat_lib.CatError):
        server.submit(0, 1 << 31)
    with pytest.raises(cat_lib.CatError):
        server.submit(9, 10)
    rc, _ = server.poll(123456789)
    assert rc == -1  # unknown ticket
    t = server.submit(0, 1000)
    r = server.wait(t)
    assert r.length > 0 and r.t_end_ns >= r.t_start_ns >= r.t_submit_ns
    assert server.release(t) == 0
    assert server.release(t) == -1  # already released


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_footprint_estimate_covers_measured_peak(cat_lib, kind):
    # admission's estimate (cat_batch_footprint) against the device bytes a
    # fresh context really holds at its peak, for single requests and batches
    for n in (0, 100, 1000, 10**4, 10**5, 10**6, 10**7):
        c = cat_lib.Context(0)
        try:
            cat_lib.cat_exact(c, kind, n)
            peak = c.memory()[1]
        finally:
            c.close()
        assert peak <= cat_lib.cat_batch_footprint([(kind, n)]), (kind, n, peak)
    reqs = [(k, n) for _, k, n in W.served_requests(24, 300.0, seed=kind, lo=1e3, hi=3e6)]
    c = cat_lib.Context(0)
    try:
        cat_lib.cat_exact_batch(c, reqs)
        peak = c.memory()[1]
    finally:
        c.close()
    assert peak <= cat_lib.cat_batch_footprint(reqs)


def test_server_budget_bounds_all_workers_together(cat_lib, ctx):
    # a mix whose estimates add up to over three times the budget: batches are
    # admitted only while they fit, the bytes all workers hold together never
    # pass the budget, and every result equals the request computed alone
    from paper_2601_11621_gb300.server import Server
    reqs = [(k, n) for _, k, n in W.served_requests(40, 300.0, seed=11, lo=1e5, hi=4e6)]
    budget = 3 * max(cat_lib.cat_batch_footprint([r]) for r in reqs) // 2
    assert cat_lib.cat_batch_footprint(reqs) > 3 * budget
    sv = Server(0, hbm_budget_bytes=budget, workers=3, max_batch=64)
    try:
        tickets = [sv.submit(k, n) for k, n in reqs]
        got = [sv.fetch_host(t) for t in tickets]
        _, peak = sv.memory()
        for t in tickets:
            sv.release(t)
    finally:
        sv.close()
    assert 0 < peak <= budget
    for (k, n), g in zip(reqs, got):
        assert np.array_equal(g, alone(ctx, cat_lib, k, n)), (k, n)
