"""Writes tests/golden/oracle_results.txt and tests/golden/oracle_groups_*.txt.

Every value in those files comes from the CPU oracle (``oracle/``) alone:
the SHA-256 of the exact result's little-endian uint32 limbs, its limb and
bit counts, and the Phase-1 group sizes.  The GPU tests compare the CUDA
path against these for sizes where running the oracle inside a test would
take minutes.

Usage:  python tests/golden/make_oracle_golden.py [--paper]
"""
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

CASES = [
    (oracle.CATALAN, 10**6),
    (oracle.CENTRAL_BINOMIAL, 10**6),
    (oracle.FACTORIAL, 10**6),
    (oracle.CATALAN, 10**7),
    (oracle.CATALAN, 50_000_000),
]
KIND_NAME = {oracle.CATALAN: "catalan", oracle.CENTRAL_BINOMIAL: "central_binomial",
             oracle.FACTORIAL: "factorial"}


def exact_line(kind, n):
    t = time.time()
    limbs = oracle.exact(kind, n)
    dt = time.time() - t
    sha = hashlib.sha256(limbs.astype("<u4").tobytes()).hexdigest()
    top = int(limbs[-1])
    bits = (len(limbs) - 1) * 32 + top.bit_length()
    print(f"{KIND_NAME[kind]} {n}: {len(limbs)} limbs, {dt:.1f} s", flush=True)
    return f"{KIND_NAME[kind]} {n} {len(limbs)} {bits} {sha}"


def groups_file(kind, n, path):
    t = time.time()
    pr = oracle.sieve(oracle.prime_limit(kind, n))
    e = oracle.exponents(kind, n, pr)
    exps, offs, gp = oracle.group(pr, e)
    h = hashlib.sha256(gp.astype("<u4").tobytes()).hexdigest()
    with open(path, "w") as f:
        f.write(f"# Phase-1 groups of {KIND_NAME[kind]}({n}) from the CPU oracle\n")
        f.write("# (make_oracle_golden.py): primes sieved, primes with e > 0,\n")
        f.write("# SHA-256 of the grouped primes (LE uint32), then 'exponent count' rows.\n")
        f.write(f"sieved {len(pr)}\n")
        f.write(f"positive {int(offs[-1])}\n")
        f.write(f"sha256 {h}\n")
        for g, ex in enumerate(exps):
            f.write(f"{int(ex)} {int(offs[g + 1] - offs[g])}\n")
    print(f"groups {KIND_NAME[kind]} {n}: {time.time() - t:.1f} s", flush=True)


def main():
    oracle.build()
    lines = ["# Exact results from the CPU oracle (make_oracle_golden.py):",
             "# kind n limbs bits sha256(LE uint32 limbs)"]
    for kind, n in CASES:
        lines.append(exact_line(kind, n))
    with open(os.path.join(HERE, "oracle_results.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    groups_file(oracle.CATALAN, 50_000_000, os.path.join(HERE, "oracle_groups_catalan_50000000.txt"))
    if "--paper" in sys.argv:
        groups_file(oracle.CATALAN, 2050572903,
                    os.path.join(HERE, "oracle_groups_catalan_2050572903.txt"))


if __name__ == "__main__":
    main()
