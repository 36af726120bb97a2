"""Benchmark: seconds per exact Catalan number at the paper's scale.

One step = one call of catalan_exact(n) through the C ABI: Phase 1 on the
device (segmented sieve of the primes <= 2n, Legendre exponents, grouping by
exponent) and Phase 2 (balanced product tree, Q_e^e, final product), leaving
the exact C(n) as uint32 limbs in device memory.  Default n = 2,050,572,903
(Table 1 of arXiv 2601.11621, 1,234,567,890 decimal digits).

Prints one JSON line (rank 0).  `value` = device-timed seconds per C(n) over
all ranks (replicas: each rank computes its own C(n)); `e2e` = the same through
cat_exact_host into pinned host memory (device-to-host copy of the result
inside the timed region).  `roofline` reports the kernel with the largest
device time, timed by CUDA events around each of its launches on its stream.
`cpu_baseline` (and `--impl reference`) time the CPU oracle on a bounded
slice of the same workload and scale it to one C(n) (see oracle_sample).
"""
from __future__ import annotations

import argparse
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
# Integer issue peak of one GB300: 152 SMs x 4 schedulers x 32 lanes, one
# instruction per scheduler per clock, at the 2,070 MHz maximum SM clock.
ALU_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


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


def captured_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from its committed ncu summary, or
    None when there is none or the kernel sources changed since the capture."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in NTT_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    digest = h.hexdigest()[:16]
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


def oracle_sample(n: int):
    """Time the CPU oracle on a bounded slice of C(n) and scale it to one C(n).

    Phase 1 slice: sieve of the 2^27 integers below 2n plus the Legendre
    exponents of the primes found; scaled by 2n / 2^27 (the sieve and the
    exponent loop are linear in the range).  Phase 2 slice: the oracle's
    product tree over the first 2^18 primes of that slice; scaled to the
    number of primes with e > 0 by (count / 2^18)^log2(3), the growth of a
    Karatsuba product tree.  Single-threaded (the oracle is)."""
    import oracle
    oracle.build()
    lim = 2 * n
    span = min(1 << 27, lim)
    t0 = time.perf_counter()
    pr = oracle.sieve_range(lim - span + 1, lim)
    e = oracle.exponents(oracle.CATALAN, n, pr)
    t1 = time.perf_counter() - t0
    m = min(1 << 18, len(pr))
    t0 = time.perf_counter()
    part = oracle.product_tree(pr[:m])
    t2 = time.perf_counter() - t0
    # Phase 2 scales with the result's size: limbs of C(n) (log-gamma) over
    # the limbs of the sampled product
    full_limbs = oracle.bound_limbs(oracle.CATALAN, n)
    ratio = max(1.0, full_limbs / max(1, len(part)))
    phase1 = t1 * lim / span
    phase2 = t2 * ratio ** math.log2(3)
    desc = (f"oracle (plain C, 1 thread): sieve+Legendre over the top 2^27 integers of "
            f"[2, 2n] ({t1:.2f} s, scaled x{lim / span:.1f}) and the product tree of 2^18 of "
            f"their primes ({t2:.2f} s, {len(part)} limbs, scaled by "
            f"({full_limbs}/{len(part)})^log2(3), Karatsuba growth); "
            f"estimate phase1={phase1:.0f} s + phase2={phase2:.0f} s")
    return phase1 + phase2, desc, t1 + t2


def run_reference(args, rank, world):
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(args.n)
    vals, descs, cpu_s = [], [], 0.0
    for _ in range(args.steps):
        v, d, s = oracle_sample(args.n)
        vals.append(v)
        descs.append(d)
        cpu_s += s
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * cpu_s / max(1, args.steps),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "u32", "data": "synthetic (the input is n itself)",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": descs[-1]},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"catalan_exact n={args.n:,} (Table 1 scale)" if args.n == PAPER_N
            else f"catalan_exact n={args.n:,}",
            "n": args.n, "kind": "catalan",
            "l2": "inputs larger than L2: each step streams multi-GB transforms through the "
                  "129 MB L2",
            "parallelism": f"replicas x{args.gpus}"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=PAPER_N)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    ctx = capi.Context(local_rank)
    n = args.n
    cap = capi.cat_bound_limbs(n, capi.CAT_CATALAN)
    out = torch.empty(cap, dtype=torch.int32, device=f"cuda:{local_rank}")
    stream = torch.cuda.current_stream()

    for _ in range(max(3, args.warmup)):
        res = capi.catalan_exact(ctx, n, out=out)
    nlimbs = res.numel()

    ctx.set_profiling(True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        capi.catalan_exact(ctx, n, out=out)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clk = clocks.stop()
    prof = ctx.profile()
    ctx.set_profiling(False)
    ms = 1000.0 * slowest_rank(ms / 1000.0, dist, f"cuda:{local_rank}")
    value = per_unit(ms / 1000.0, args.steps, world)

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
    e2e_s = slowest_rank(e2e_s, dist, f"cuda:{local_rank}")
    e2e_value = per_unit(e2e_s, e2e_steps, world)

    # dominant kernel by device time
    peak, peak_kind = read_peaks()
    launches = sum(v[0] for v in prof.values())
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = None
    if dom:
        name, (cnt, kms, kbytes, kops) = dom
        traffic = captured_traffic(name)
        secs = kms / 1000.0
        gbs = kbytes / secs / 1e9 if secs > 0 else 0.0
        tops = kops / secs / 1e12 if secs > 0 else 0.0
        common = {"kernel": name, "launches": cnt, "avg_launch_ms": round(kms / cnt, 4),
                  "algorithmic_bytes_per_launch": kbytes / cnt,
                  "algorithmic_ops_per_launch": kops / cnt,
                  "hbm_achieved_gbs": round(gbs, 1), "hbm_frac": round(gbs / peak, 4),
                  "share_of_step": round(kms / ms, 4) if ms > 0 else None}
        if kops > 0 and tops / ALU_PEAK_TOPS > gbs / peak:
            # compute-bound: 32-bit integer instruction issue (see ALU_PEAK_TOPS)
            roof = {"bound": "alu", "achieved": round(tops, 3), "peak": ALU_PEAK_TOPS,
                    "unit": "Tops/s", "frac": round(tops / ALU_PEAK_TOPS, 4),
                    "peak_source": "derived: 152 SMs x 128 lanes x 2.07 GHz",
                    "traffic": traffic, **common}
        else:
            roof = {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                    "frac": round(gbs / peak, 4), "peak_source": peak_kind, "traffic": traffic,
                    **common}
    if args.profile_json and rank == 0:
        with open(args.profile_json, "w") as f:
            json.dump({k: {"launches": v[0], "ms": v[1], "bytes": v[2], "ops": v[3]}
                       for k, v in prof.items()}, f, indent=1)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, d, _ = oracle_sample(n)
        cpu = {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": d}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup),
            "ms_per_step": ms / args.steps, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (the input is n itself)",
            "config": workload_config(args),
            "result": {"limbs": int(nlimbs), "host_limbs": int(hres.size)},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": "s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": int(4 * hres.size)},
            "gpu_launches": int(launches),
            "roofline": roof,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
