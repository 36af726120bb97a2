"""Benchmark: seconds per exact Catalan number at the paper's scale.

One step = one call of catalan_exact(n) through the C ABI: Phase 1 on the
device (segmented sieve of the primes <= 2n, Legendre exponents, grouping by
exponent) and Phase 2 (balanced product tree, Q_e^e, final product), leaving
the exact C(n) as uint32 limbs in device memory.  Default n = 2,050,572,903
(Table 1 of arXiv 2601.11621, 1,234,567,890 decimal digits).

Prints one JSON line (rank 0):
  value        device-timed seconds per C(n) over all ranks (replicas: each
               rank computes its own C(n)), the library's per-launch profiler
               off;
  e2e          the same through cat_exact_host into pinned host memory (the
               512 MB result copied back inside the timed region);
  roofline     the kernel with the largest device time in a separate profiled
               step: the algorithmic bytes of the products it completes (4 B
               per limb of each operand read and of each product written: for
               a tree level 8 B per limb of the level) over its launch time,
               against the measured HBM copy peak; the bytes of the pass
               itself and the ncu DRAM traffic beside them;
  cpu_baseline the CPU oracle (plain C) timed on all host cores at n = 10^6,
               10^7 and 5 * 10^7, extrapolated to the paper's n by a fitted
               growth exponent (single-threaded runs reported beside);
  mul_sweep    bigint_mul of seeded random operands at 2^10, 2^12, ..., 2^26
               uint64 limbs (ratios 1:1 and 1:4): GB/s of algorithmic bytes,
               each product checked modulo two primes;
  batched      4,096 seeded requests (C(n) / C(2n, n), n log-uniform in
               [10^3, 10^6]) in one cat_exact_batch call against one-at-a-time
               cat_exact calls, results compared;
  served       a seeded Poisson stream (300 req/s offered) through the serving
               engine against the same stream one request at a time: p50/p99
               latency, req/s, results compared; served_rates the same at 10,
               30, 100 and 1000 req/s;
  decimal      to_decimal of the C(n) just computed (its 1,234,567,890 digits at
               the paper's n).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PAPER_N = 2_050_572_903
METRIC = "sec per exact C(n) at n=2.05e9"
# Table 1: total wall time of the paper's own run (Phase 1 + Phase 2) on a
# Ryzen 9 4900HS laptop with Python and GMP; another machine, context only.
PAPER_SECONDS = 1549.14

NTT_SOURCES = ["paper_2601_11621_gb300/csrc/ntt.cu", "paper_2601_11621_gb300/csrc/ntt_kernels.cuh",
               "paper_2601_11621_gb300/csrc/cat_internal.cuh"]


def slowest_rank(seconds: float, dist=None, device: str = "cpu") -> float:
    """The largest of the ranks' timings, on every rank: the job takes as long
    as its slowest rank (one all-reduce MAX; the local value when alone)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_unit(seconds: float, units_per_rank: int, world: int) -> float:
    """Whole-job seconds per C(n): the slowest rank's time over the units that
    all ranks processed (every rank computes units_per_rank replicas)."""
    return seconds / (units_per_rank * world)


def sources_digest() -> str:
    h = hashlib.sha256()
    for f in NTT_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or
    None when there is none or the kernel sources changed since the capture."""
    import glob
    digest = sources_digest()
    for path in glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_traffic_*.md")):
        fields = {}
        for line in open(path):
            if ":" in line and not line.startswith(" "):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.strip()
        if fields.get("source_sha256_16") == digest and "traffic_bytes_per_launch" in fields:
            return float(fields["traffic_bytes_per_launch"])
    return None


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU baseline

def _oracle_point(oracle, n: int, threads: int):
    """(limbs, phase-1 seconds, total seconds) of the oracle's C(n): Phase 1
    alone (sieve, exponents, grouping) timed separately, then the whole
    computation (both phases) on `threads` threads."""
    t0 = time.perf_counter()
    oracle.factor(oracle.CATALAN, n)
    t_p1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.exact_mt(oracle.CATALAN, n, threads)
    t_all = time.perf_counter() - t0
    return len(r), t_p1, t_all


def _fit_exponent(points):
    """Least-squares slope of log(phase-2 seconds) against log(limbs)."""
    xs = [math.log(p[0]) for p in points]
    ys = [math.log(max(1e-6, p[2] - p[1])) for p in points]
    mx, my = sum(xs) / len(xs), sum(ys) / len(ys)
    sxx = sum((x - mx) ** 2 for x in xs)
    return sum((x - mx) * (y - my) for x, y in zip(xs, ys)) / sxx if sxx > 0 else 1.585


def _extrapolate(oracle, point, alpha: float, n_from: int, n_to: int) -> float:
    """Seconds per C(n_to) from a measured point at n_from: Phase 1 linear in
    n (the sieve range), Phase 2 as (limbs ratio)^alpha."""
    limbs, t_p1, t_all = point
    full = oracle.bound_limbs(oracle.CATALAN, n_to)
    return t_p1 * n_to / n_from + (t_all - t_p1) * (full / limbs) ** alpha


# The oracle's growth steepens with size (Karatsuba's exponent takes over from
# the schoolbook base cases and the sieve), so the exponent is fitted at the
# top of the measured range, where the extrapolation starts.
FIT_NS = (10**7, 2 * 10**7, 5 * 10**7)
ST_NS = (10**6, 10**7)


def oracle_baseline(n: int):
    """The CPU oracle timed on all host cores at n = 10^7, 2 * 10^7, 5 * 10^7
    and single-threaded at 10^6, 10^7; the all-core figure extrapolated to C(n)
    from the largest point with the growth exponent fitted to the three."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    pts = [_oracle_point(oracle, m, threads) for m in FIT_NS]
    alpha = _fit_exponent(pts)
    value = _extrapolate(oracle, pts[-1], alpha, FIT_NS[-1], n)
    st = [_oracle_point(oracle, m, 1) for m in ST_NS]
    alpha_st = _fit_exponent(st)
    value_st = _extrapolate(oracle, st[-1], alpha_st, ST_NS[-1], n)
    measured = {f"{m:.0e}": round(p[2], 3) for m, p in zip(FIT_NS, pts)}
    desc = (f"oracle (plain C, OpenMP tasks over product-tree halves and Karatsuba "
            f"sub-products, {threads} threads) timed end to end at n = 1e7, 2e7, 5e7 "
            f"({', '.join(f'{k}: {v} s' for k, v in measured.items())}); Phase 2 growth "
            f"exponent fitted = {alpha:.3f} (limbs); extrapolated from 5e7 to n = {n:,} "
            f"(Phase 1 linear in n); single-threaded: {st[0][2]:.2f} s at 1e6, "
            f"{st[1][2]:.2f} s at 1e7, extrapolated {value_st:.0f} s (exponent {alpha_st:.3f})")
    return {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
            "sample": desc, "extrapolated": True, "fitted_exponent": round(alpha, 4),
            "measured_s": measured, "config2_n5e7_measured_s": round(pts[-1][2], 3),
            "single_thread_extrapolated_s": round(value_st, 1)}


def run_reference(args, rank, world):
    """The oracle as the reference arm: the warm-up steps time it on all host
    cores at n = 10^7, 2 * 10^7, 5 * 10^7 in turn (every size at least once;
    the growth exponent is fitted from them), and each timed step is one
    all-core oracle run at n = 2 * 10^7, extrapolated to the bench's n with
    that exponent."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    fit = [_oracle_point(oracle, FIT_NS[i % len(FIT_NS)], threads)
           for i in range(max(len(FIT_NS), args.warmup))]
    alpha = _fit_exponent(fit)
    step_n = FIT_NS[1]
    vals, cpu_s = [], 0.0
    for _ in range(args.steps):
        p = _oracle_point(oracle, step_n, threads)
        cpu_s += p[2] + p[1]
        vals.append(_extrapolate(oracle, p, alpha, step_n, args.n))
    value = statistics.median(vals)
    desc = (f"oracle (plain C, {threads} threads) at n = 2e7 per step, extrapolated to "
            f"n = {args.n:,} with the Phase 2 exponent {alpha:.3f} fitted in the warm-up "
            f"steps (n = 1e7, 2e7, 5e7)")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * cpu_s / max(1, args.steps),
        "higher_is_better": False, "scaling": "weak",
        "vs_baseline": value / PAPER_SECONDS,
        "dtype": "u32", "data": "synthetic (the input is n itself)",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "s", "cores": threads, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def verify_result(n: int, limbs) -> dict:
    """The computed C(n) checked after timing: at the paper's n the result file
    (bytes 01 01, then the little-endian magnitude) must hash to Table 1's
    SHA-256 (tests/golden/paper_table1.txt); a mismatch stops the benchmark."""
    if n != PAPER_N:
        return {}
    want = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(None, 1)
            want[k] = v.strip()
    top = int(limbs[-1])
    bits = (len(limbs) - 1) * 32 + top.bit_length()
    nbytes = (bits + 7) // 8
    body = limbs.astype("<u4").tobytes()[:nbytes]
    sha = hashlib.sha256(bytes.fromhex(want["sha256_header_hex"]) + body).hexdigest()
    if sha != want["sha256"] or bits != int(want["bit_length"]):
        raise RuntimeError(f"C({n}) does not match Table 1: sha256 {sha}, {bits} bits")
    return {"bits": bits, "sha256_table1": True}


def workload_config(args):
    return {"workload": f"catalan_exact n={args.n:,} (Table 1 scale)" if args.n == PAPER_N
            else f"catalan_exact n={args.n:,}",
            "n": args.n, "kind": "catalan",
            "l2": "inputs larger than L2: each step streams multi-GB transforms through the "
                  "129 MB L2",
            "parallelism": f"replicas x{args.gpus}"}


# ------------------------------------------------- the other metric terms

def limbs_mod_dev(t, q: int) -> int:
    """A device limb tensor (int32 holding uint32 limbs) mod q < 2^31, with
    plain torch integer ops: sum_j limb_j 2^(32 j) mod q, the powers built by
    doubling.  Every product stays below 2^62."""
    import torch
    x = t.to(torch.int64) & 0xFFFFFFFF
    m = x.numel()
    pw = torch.ones(1, dtype=torch.int64, device=t.device)
    bk = (1 << 32) % q
    while pw.numel() < m:
        pw = torch.cat([pw, (pw * bk) % q])
        bk = bk * bk % q
    return int((((x % q) * pw[:m]) % q).sum().item()) % q


def range_prod_mod(lo: int, hi: int, q: int) -> int:
    """prod_{k=lo}^{hi} k mod q < 2^31 by pairwise products (numpy)."""
    import numpy as np
    if lo > hi:
        return 1 % q
    v = np.arange(lo, hi + 1, dtype=np.uint64) % np.uint64(q)
    while v.size > 1:
        if v.size & 1:
            v = np.append(v, np.uint64(1))
        v = (v[0::2] * v[1::2]) % np.uint64(q)
    return int(v[0])


def binomial_mod(kind: int, n: int, q: int) -> int:
    """C(n) (kind 0) or C(2n, n) (kind 1) mod a prime q > 2n from factorial
    products: prod_{k=n+2 (or n+1)}^{2n} k / n!."""
    num = range_prod_mod(n + 2 if kind == 0 else n + 1, 2 * n, q)
    return num * pow(range_prod_mod(1, n, q), q - 2, q) % q


CHECK_PRIMES = (2147483647, 2147483629)  # primes below 2^31, above every 2n used here


# bigint_mul sweep sizes (log2 of the uint64 limbs of the longer operand):
# every second power from 2^10 to 2^26; the 2^26 products (2^28 uint32
# limbs) are longer than one transform and go by pieces
SWEEP_LOGS = (10, 12, 14, 16, 18, 20, 22, 24, 26)


def mul_sweep(ctx, capi, W, dev):
    import torch
    out = []
    stream = torch.cuda.current_stream()
    for k in SWEEP_LOGS:
        for ratio in (1, 4):
            na64, nb64 = 1 << k, (1 << k) // ratio
            a = torch.from_numpy(W.random_limbs(na64, 100 + k).view("i4")).to(dev)
            b = torch.from_numpy(W.random_limbs(nb64, 200 + k + ratio).view("i4")).to(dev)
            r = capi.bigint_mul(ctx, a, b)
            for q in CHECK_PRIMES:
                if limbs_mod_dev(r, q) != limbs_mod_dev(a, q) * limbs_mod_dev(b, q) % q:
                    raise RuntimeError(f"mul_sweep check failed at 2^{k} 1:{ratio}")
            reps = 20 if k <= 16 else (5 if k < 24 else 3)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                capi.bigint_mul(ctx, a, b)
            e1.record(stream)
            torch.cuda.synchronize()
            s = e0.elapsed_time(e1) / 1000.0 / reps
            nbytes = 8.0 * (a.numel() + b.numel())  # operands read + product written
            out.append({"u64_limbs": [na64, nb64], "ms": round(1000 * s, 4),
                        "gbs": round(nbytes / s / 1e9, 2), "checked": "mod 2 primes"})
            del a, b, r
    return out


def batched(ctx, capi, W):
    import torch
    reqs = W.batched_requests(4096, seed=0)
    stream = torch.cuda.current_stream()
    res = capi.cat_exact_batch(ctx, reqs)
    torch.cuda.synchronize()
    reps = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        res = capi.cat_exact_batch(ctx, reqs)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1000.0 / reps
    out, offs, lens = res
    sub = 256
    singles = []
    e0.record(stream)
    for kind, n in reqs[:sub]:
        singles.append(capi.cat_exact(ctx, kind, n))
    e1.record(stream)
    torch.cuda.synchronize()
    t_one = e0.elapsed_time(e1) / 1000.0 / sub
    for i, r in enumerate(singles):
        got = out[int(offs[i]): int(offs[i]) + int(lens[i])]
        if got.numel() != r.numel() or not torch.equal(got, r):
            raise RuntimeError(f"batched result {i} differs from the one-at-a-time call")
    for i in range(0, 4096, 256):
        kind, n = reqs[i]
        got = out[int(offs[i]): int(offs[i]) + int(lens[i])]
        q = CHECK_PRIMES[i % 2]
        if limbs_mod_dev(got, q) != binomial_mod(kind, n, q):
            raise RuntimeError(f"batched result {i} fails its modular check")
    return {"requests": 4096, "batch_ms": round(1000 * t_batch, 3),
            "req_per_s": round(4096 / t_batch, 1),
            "one_at_a_time_req_per_s": round(1 / t_one, 1),
            "one_at_a_time_sample": sub,
            "speedup": round(t_one * 4096 / t_batch, 2),
            "checked": f"first {sub} equal to one-at-a-time results; 16 mod q"}


def decimal(ctx, capi, limbs, n):
    """to_decimal of the computed C(n) (the optional decimal output): median of
    two timed conversions after one warm-up; at the paper's n the digit count
    must be Table 1's 1,234,567,890."""
    import torch
    stream = torch.cuda.current_stream()
    out = torch.empty(capi.cat_decimal_bound(limbs.numel()), dtype=torch.uint8,
                      device=limbs.device)
    d = capi.to_decimal(ctx, limbs, out=out)
    ms = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d = capi.to_decimal(ctx, limbs, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    if n == PAPER_N and d.numel() != 1_234_567_890:
        raise RuntimeError(f"to_decimal gave {d.numel()} digits")
    return {"digits": int(d.numel()), "ms": round(min(ms), 2),
            "checked": "digit count (Table 1)" if n == PAPER_N else "none"}


# the other offered rates of the serving sweep (req/s, requests per stream),
# each stream a few seconds long at most
SERVED_RATES = ((10.0, 20), (30.0, 40), (100.0, 96), (1000.0, 192))


def served(ctx, capi, W, device, rate=300.0, count=96):
    from paper_2601_11621_gb300 import server
    stream = W.served_requests(count, rate, seed=1)
    sv = server.Server(device, hbm_budget_bytes=120 * 10**9, workers=3)
    try:
        lat, wall, res_s, nb = server.replay_server(sv, stream, keep_results=True)
    finally:
        sv.close()
    lat1, wall1, res_1 = server.replay_one_at_a_time(ctx, stream, keep_results=True)
    for i, (x, y) in enumerate(zip(res_s, res_1)):
        if x.shape != y.shape or not (x == y).all():
            raise RuntimeError(f"served result {i} differs from the one-at-a-time result")
    s, s1 = server.summarize(lat, wall, count), server.summarize(lat1, wall1, count)
    return {"rate_offered": rate, "requests": count, "batches": nb,
            "p50_ms": round(1000 * s["p50_s"], 2), "p99_ms": round(1000 * s["p99_s"], 2),
            "req_per_s": round(s["req_per_s"], 1),
            "one_at_a_time": {"p50_ms": round(1000 * s1["p50_s"], 2),
                              "p99_ms": round(1000 * s1["p99_s"], 2),
                              "req_per_s": round(s1["req_per_s"], 1)},
            "checked": "every served result equal to the one-at-a-time result",
            "mix": "kinds C(n), C(2n,n), n! uniform; n log-uniform in [1e4, 1e8]; "
                   "3 workers, 120 GB budget"}


# ------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=PAPER_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the mul sweep, batched and served measurements")
    ap.add_argument("--profile-json", default=None, help="also dump per-kernel totals here")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    from paper_2601_11621_gb300 import build, capi
    from paper_2601_11621_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dev = f"cuda:{local_rank}"
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    ctx = capi.Context(local_rank)
    # the library's autotuner picks the transform plans and the schoolbook
    # crossover for this device; its table goes next to the library, where
    # every context created later (the serving engine's too) reads it
    tune_path = os.path.join(os.path.dirname(capi.LIB_PATH), "autotune.txt")
    t0 = time.perf_counter()
    ctx.autotune(tune_path if rank == 0 else None)
    tune_s = time.perf_counter() - t0
    slot, rows = ctx.tuning()
    tuning = {"seconds": round(tune_s, 2), "comba_max_slot": slot,
              "row_log": {str(k): v for k, v in rows.items()}}
    n = args.n
    cap = capi.cat_bound_limbs(n, capi.CAT_CATALAN)
    out = torch.empty(cap, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    warmup = max(3, args.warmup)
    for _ in range(warmup):
        res = capi.catalan_exact(ctx, n, out=out)
    nlimbs = res.numel()

    # timed region: the library's profiler stays off
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = capi.cat_launch_count()
    ev0.record(stream)
    for _ in range(args.steps):
        capi.catalan_exact(ctx, n, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    timed_launches = capi.cat_launch_count() - launches0
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    ms = 1000.0 * slowest_rank(ms / 1000.0, dist, dev)
    value = per_unit(ms / 1000.0, args.steps, world)

    # one profiled step (CUDA events around every launch, on its stream)
    ctx.set_profiling(True)
    prof_steps = 2
    t0 = time.perf_counter()
    for _ in range(prof_steps):
        capi.catalan_exact(ctx, n, out=out)
    torch.cuda.synchronize()
    prof = ctx.profile()
    ctx.set_profiling(False)
    prof_ms = sum(v[1] for v in prof.values()) / prof_steps

    # end to end through the C ABI into pinned host memory
    host = torch.empty(cap, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    capi.cat_exact_host(ctx, capi.CAT_CATALAN, n, out=host)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        hres = capi.cat_exact_host(ctx, capi.CAT_CATALAN, n, out=host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s = slowest_rank(e2e_s, dist, dev)
    e2e_value = per_unit(e2e_s, e2e_steps, world)
    check = verify_result(n, hres)

    # dominant kernel by device time, against the measured HBM copy peak
    peak, peak_kind = read_peaks()
    launches_per_step = sum(v[0] for v in prof.values()) / prof_steps
    roof = None
    if prof:
        name, (cnt, kms, pass_bytes, unit_bytes) = max(prof.items(), key=lambda kv: kv[1][1])
        secs = kms / 1000.0
        alg = unit_bytes if unit_bytes > 0 else pass_bytes
        gbs = alg / secs / 1e9
        pass_gbs = pass_bytes / secs / 1e9
        traffic = captured_traffic(name)
        roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                "frac": round(gbs / peak, 4),
                "peak_source": f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy, read + write)",
                "traffic": traffic,
                "kernel": name, "launches": cnt, "avg_launch_ms": round(kms / cnt, 4),
                "algorithmic_bytes_per_launch": alg / cnt,
                "algorithmic": "operands read once + products written once, 4 B per limb "
                               "each (8 B per limb of a tree level)"
                               if unit_bytes > 0 else "pass bytes (no products completed)",
                "traffic_over_algorithmic": round(traffic / (alg / cnt), 2) if traffic else None,
                "pass_bytes_per_launch": pass_bytes / cnt,
                "pass_gbs": round(pass_gbs, 1), "pass_frac": round(pass_gbs / peak, 4),
                "share_of_step": round(kms / prof_steps / prof_ms, 4) if prof_ms else None,
                "timing": "CUDA events around each launch on its stream, separate profiled "
                          f"steps ({prof_steps})"}
    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as f:
            json.dump({k: {"launches": v[0], "ms": v[1], "pass_bytes": v[2], "unit_bytes": v[3]}
                       for k, v in prof.items()}, f, indent=1)

    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        extras["mul_sweep"] = mul_sweep(ctx, capi, W, dev)
        extras["batched"] = batched(ctx, capi, W)
        extras["served"] = served(ctx, capi, W, local_rank)
        extras["served_rates"] = [
            {k: v for k, v in served(ctx, capi, W, local_rank, rate, count).items()
             if k not in ("checked", "mix")}
            for rate, count in SERVED_RATES]
        extras["decimal"] = decimal(ctx, capi, out[:nlimbs], n)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = oracle_baseline(n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": value / PAPER_SECONDS,
            "vs_baseline_ref": "Table 1: 1549.14 s per C(2,050,572,903) on a Ryzen 9 4900HS "
                               "laptop (Python + GMP); another machine, context only",
            "dtype": "u32",
            "data": "synthetic (the input is n itself)",
            "config": workload_config(args),
            "result": {"limbs": int(nlimbs), "host_limbs": int(hres.size), **check},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(4 * hres.size)},
            "gpu_launches": int(timed_launches),
            "autotune": tuning,
            "roofline": roof,
            "cpu_baseline": cpu,
            **extras,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
