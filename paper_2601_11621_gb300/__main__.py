"""Command line for the library (everything runs through the C ABI on cuda:0).

    python -m paper_2601_11621_gb300 exact N [--kind catalan|central_binomial|factorial]
                                             [--repeat K] [--bin FILE] [--decimal FILE]
                                             [--factorization FILE] [--sha256]
        The exact quantity of n (C(n) by default), timed (K times), with the run's
        files as the paper describes them: the result file (bytes 01 01, then
        the little-endian magnitude), its decimal digits, and the grouped
        factorisation as text.

    python -m paper_2601_11621_gb300 ratio --num A1 A2 ... --den B1 B2 ...
        prod A_i! / prod B_j! (an integer, or CAT_ENOTINTEGRAL).

    python -m paper_2601_11621_gb300 mul LOG2A [LOG2B] [--repeat K]
        One product of two seeded random operands of 2^LOG2A and 2^LOG2B limbs
        (the product kernels at a chosen size).

    python -m paper_2601_11621_gb300 batch COUNT [--seed S] [--lo A] [--hi B] [--repeat K]
        COUNT seeded requests (C(n) or C(2n, n), n log-uniform in [A, B]) in one
        cat_exact_batch call, timed (K times).
"""
from __future__ import annotations

import argparse
import hashlib
import sys
import time


def _sync():
    import torch
    torch.cuda.synchronize()


def cmd_exact(a) -> int:
    from . import capi
    ctx = capi.Context(0)
    kind = capi.KINDS[a.kind]
    for _ in range(max(1, a.repeat)):
        _sync()
        t = time.perf_counter()
        r = capi.cat_exact(ctx, kind, a.n)
        _sync()
        dt = time.perf_counter() - t
        print(f"{a.kind}({a.n}): {r.numel()} limbs in {dt * 1e3:.1f} ms")
    if a.bin or a.sha256:
        data = capi.cat_binary(ctx, r).cpu().numpy().tobytes()
        if a.bin:
            with open(a.bin, "wb") as f:
                f.write(data)
            print(f"wrote {a.bin}: {len(data)} bytes")
        if a.sha256:
            print(f"sha256 of the result file: {hashlib.sha256(data).hexdigest()}")
    if a.decimal:
        for _ in range(max(1, a.repeat)):
            _sync()
            t = time.perf_counter()
            dd = capi.to_decimal(ctx, r)
            _sync()
            dt = time.perf_counter() - t
            print(f"to_decimal: {dd.numel()} digits in {dt * 1e3:.1f} ms")
        d = dd.cpu().numpy().tobytes()
        with open(a.decimal, "wb") as f:
            f.write(d)
        print(f"wrote {a.decimal}: {len(d)} digits")
    if a.factorization:
        names = {"catalan": "Catalan", "central_binomial": "CentralBinomial",
                 "factorial": "Factorial"}
        fr = capi.catalan_factor(ctx, a.n, kind)
        try:
            txt = capi.cat_factor_text(ctx, fr, f"{names[a.kind]}({a.n})").cpu().numpy()
        finally:
            fr.free()
        with open(a.factorization, "wb") as f:
            f.write(txt.tobytes())
        print(f"wrote {a.factorization}: {txt.size} bytes")
    return 0


def cmd_ratio(a) -> int:
    from . import capi
    ctx = capi.Context(0)
    r = capi.cat_ratio_exact(ctx, a.num, a.den)
    print(f"{r.numel()} limbs")
    if a.decimal:
        print(capi.to_decimal(ctx, r).cpu().numpy().tobytes().decode())
    return 0


def cmd_mul(a) -> int:
    from . import capi, workloads
    import numpy as np
    import torch
    ctx = capi.Context(0)
    lb = a.log2b if a.log2b is not None else a.log2a
    x = torch.from_numpy(workloads.random_limbs32(1 << a.log2a, 1).view(np.int32)).cuda()
    y = torch.from_numpy(workloads.random_limbs32(1 << lb, 2).view(np.int32)).cuda()
    for i in range(a.repeat):
        _sync()
        t = time.perf_counter()
        r = capi.bigint_mul(ctx, x, y)
        _sync()
        print(f"2^{a.log2a} x 2^{lb} limbs: {r.numel()} limbs in "
              f"{(time.perf_counter() - t) * 1e3:.2f} ms")
    return 0


def cmd_batch(a) -> int:
    from . import capi, workloads
    ctx = capi.Context(0)
    reqs = workloads.batched_requests(a.count, seed=a.seed, lo=a.lo, hi=a.hi)
    for _ in range(max(1, a.repeat)):
        _sync()
        t = time.perf_counter()
        out, offs, lens = capi.cat_exact_batch(ctx, reqs)
        _sync()
        dt = time.perf_counter() - t
        print(f"{a.count} requests: {int(lens.sum())} limbs in {dt * 1e3:.2f} ms")
    return 0


def main(argv=None) -> int:
    p = argparse.ArgumentParser(prog="python -m paper_2601_11621_gb300")
    sub = p.add_subparsers(dest="cmd", required=True)
    e = sub.add_parser("exact")
    e.add_argument("n", type=int)
    e.add_argument("--kind", default="catalan",
                   choices=["catalan", "central_binomial", "factorial"])
    e.add_argument("--bin")
    e.add_argument("--decimal")
    e.add_argument("--factorization")
    e.add_argument("--sha256", action="store_true")
    e.add_argument("--repeat", type=int, default=1)
    r = sub.add_parser("ratio")
    r.add_argument("--num", type=int, nargs="*", default=[])
    r.add_argument("--den", type=int, nargs="*", default=[])
    r.add_argument("--decimal", action="store_true")
    m = sub.add_parser("mul")
    m.add_argument("log2a", type=int)
    m.add_argument("log2b", type=int, nargs="?")
    m.add_argument("--repeat", type=int, default=1)
    b = sub.add_parser("batch")
    b.add_argument("count", type=int)
    b.add_argument("--seed", type=int, default=0)
    b.add_argument("--lo", type=float, default=1e3)
    b.add_argument("--hi", type=float, default=1e6)
    b.add_argument("--repeat", type=int, default=1)
    a = p.parse_args(argv)
    return {"exact": cmd_exact, "ratio": cmd_ratio, "mul": cmd_mul, "batch": cmd_batch}[a.cmd](a)


if __name__ == "__main__":
    sys.exit(main())
