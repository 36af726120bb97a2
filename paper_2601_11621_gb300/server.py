"""Serving: a thin binding of the native continuous-batching engine
(cat_server_* in include/catalan.h) and a driver that replays a seeded
arrival stream against it, or against one-at-a-time calls for comparison.

Latency of a request = completion time - its scheduled arrival time (both on
the monotonic clock), so queueing delay is included.
"""
from __future__ import annotations

import ctypes
import threading
import time

import numpy as np

from . import capi


class Server:
    """cat_server: `workers` threads, each with its own context and stream."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 120 * 10**9, workers: int = 2,
                 max_batch: int = 4096):
        L = capi.load()
        h = ctypes.c_void_p()
        rc = L.cat_server_create(device, int(hbm_budget_bytes), workers, max_batch,
                                 ctypes.byref(h))
        if rc != 0:
            raise capi.CatError(rc, "cat_server_create")
        self.h = h

    def submit(self, kind: int, n: int) -> int:
        t = ctypes.c_uint64()
        rc = capi.load().cat_server_submit(self.h, kind, n, ctypes.byref(t))
        if rc != 0:
            raise capi.CatError(rc, "cat_server_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 600_000) -> capi.ServerResult:
        r = capi.ServerResult()
        rc = capi.load().cat_server_wait(self.h, ticket, timeout_ms, ctypes.byref(r))
        if rc != 0:
            raise capi.CatError(rc, f"ticket {ticket}")
        return r

    def poll(self, ticket: int):
        r = capi.ServerResult()
        rc = capi.load().cat_server_poll(self.h, ticket, ctypes.byref(r))
        return rc, r

    def fetch_host(self, ticket: int) -> np.ndarray:
        r = self.wait(ticket)
        out = np.empty(max(1, r.length), dtype=np.uint32)
        n = ctypes.c_size_t()
        rc = capi.load().cat_server_fetch(self.h, ticket, out.ctypes.data_as(ctypes.c_void_p),
                                          out.size, 1, ctypes.byref(n))
        if rc != 0:
            raise capi.CatError(rc, "cat_server_fetch")
        return out[:n.value]

    def release(self, ticket: int) -> int:
        return capi.load().cat_server_release(self.h, ticket)

    def memory(self):
        """(bytes all workers hold now, their high-water mark)."""
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        rc = capi.load().cat_server_memory(self.h, ctypes.byref(a), ctypes.byref(b))
        if rc != 0:
            raise capi.CatError(rc, "cat_server_memory")
        return a.value, b.value

    def pending(self):
        q, t = ctypes.c_size_t(), ctypes.c_size_t()
        capi.load().cat_server_pending(self.h, ctypes.byref(q), ctypes.byref(t))
        return q.value, t.value

    def close(self):
        if getattr(self, "h", None):
            capi.load().cat_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _percentiles(lat):
    lat = np.asarray(lat)
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


def replay_server(server: Server, stream, keep_results: bool = False):
    """Submit each (arrival_s, kind, n) at its arrival time; return per-request
    latencies (s), wall time, and optionally the host results."""
    t0 = time.monotonic_ns() + 5_000_000
    tickets = [None] * len(stream)

    def submitter():
        for i, (a, kind, n) in enumerate(stream):
            target = t0 + int(a * 1e9)
            while True:
                d = target - time.monotonic_ns()
                if d <= 0:
                    break
                time.sleep(min(d / 1e9, 0.002))
            tickets[i] = server.submit(kind, n)

    th = threading.Thread(target=submitter)
    th.start()
    lat, results, batches = [], [], set()
    for i, (a, kind, n) in enumerate(stream):
        while tickets[i] is None:
            time.sleep(0.0005)
        r = server.wait(tickets[i])
        lat.append((r.t_end_ns - (t0 + int(a * 1e9))) / 1e9)
        batches.add(r.batch)
        if keep_results:
            results.append(server.fetch_host(tickets[i]))
        server.release(tickets[i])
    th.join()
    wall = (time.monotonic_ns() - t0) / 1e9
    return np.asarray(lat), wall, results, len(batches)


def replay_one_at_a_time(ctx: capi.Context, stream, keep_results: bool = False):
    """The same stream served by plain cat_exact calls, one at a time in
    arrival order."""
    import torch
    t0 = time.monotonic_ns() + 5_000_000
    lat, results = [], []
    for a, kind, n in stream:
        target = t0 + int(a * 1e9)
        while time.monotonic_ns() < target:
            time.sleep(0.0005)
        r = capi.cat_exact(ctx, kind, n)
        torch.cuda.current_stream().synchronize()
        lat.append((time.monotonic_ns() - target) / 1e9)
        if keep_results:
            results.append(capi.to_numpy(r))
        del r
    wall = (time.monotonic_ns() - t0) / 1e9
    return np.asarray(lat), wall, results


def summarize(lat, wall, count):
    p50, p99 = _percentiles(lat)
    return {"p50_s": p50, "p99_s": p99, "req_per_s": count / wall, "wall_s": wall}
