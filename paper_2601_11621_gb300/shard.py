"""Sharding plan for computing one C(n) on several GPUs (host logic only).

The product tree of Phase 2 (Sec. 3.2, Algorithm 2) splits over G devices
the way the paper's sieve splits over disjoint intervals (Sec. 3.1): rank r
takes a contiguous range of the grouped primes, multiplies it by its own
product tree, and the G roots are combined by a binomial tree of products,
ceil(log2 G) rounds of pairwise sends, after which rank 0 holds the product.
The ranges are balanced by bit weight (the sum of log2 p over a range is the
bit length of its product), so every rank's subtree, and every product of a
combining round, has about the same size.

Only the plan lives here: which primes each rank multiplies, how long each
root can be, and who sends to whom in which round.  Every machine this
library runs on has one GPU, so no multi-GPU execution path is built on it;
the plan's bookkeeping is tested with CPU ranks.
"""
from __future__ import annotations

import math

import numpy as np


def partition_by_bits(primes: np.ndarray, parts: int) -> list[int]:
    """Boundaries 0 = b_0 <= b_1 <= ... <= b_parts = len(primes): rank r
    multiplies primes[b_r : b_{r+1}], and the ranges' bit weights (sums of
    log2 p) are as equal as cuts between primes allow."""
    if parts < 1:
        raise ValueError("parts must be positive")
    p = np.asarray(primes, dtype=np.float64)
    if p.size == 0:
        return [0] * (parts + 1)
    cum = np.cumsum(np.log2(p))
    targets = cum[-1] * np.arange(1, parts) / parts
    cuts = np.searchsorted(cum, targets, side="left").tolist()
    return [0, *[int(c) for c in cuts], int(p.size)]


def root_limbs(primes: np.ndarray, lo: int, hi: int) -> int:
    """Limbs that always hold the product of primes[lo:hi]: every prime below
    2^32 adds at most bitlen(p) bits."""
    bits = sum(int(x).bit_length() for x in np.asarray(primes[lo:hi]).tolist())
    return max(1, (bits + 31) // 32)


def combine_schedule(parts: int) -> list[list[tuple[int, int]]]:
    """Rounds of (receiver, sender) pairs of a binomial tree over the ranks:
    in round k every rank r with r mod 2^(k+1) == 0 receives the root of rank
    r + 2^k (when it exists) and multiplies it into its own.  Rank 0 ends with
    the product of all roots, in rank order (receiver's root times sender's,
    the sender's primes being the larger ones)."""
    rounds = []
    step = 1
    while step < parts:
        rounds.append([(r, r + step) for r in range(0, parts, 2 * step) if r + step < parts])
        step *= 2
    return rounds


def plan(primes: np.ndarray, parts: int) -> dict:
    """The whole plan: per rank its prime range and root bound, and the
    combining rounds with the bound of every product they form."""
    b = partition_by_bits(primes, parts)
    ranks = [{"rank": r, "lo": b[r], "hi": b[r + 1], "root_limbs": root_limbs(primes, b[r], b[r + 1])}
             for r in range(parts)]
    held = {r: ranks[r]["root_limbs"] for r in range(parts)}
    rounds = []
    for pairs in combine_schedule(parts):
        step = []
        for dst, src in pairs:
            held[dst] += held[src]
            step.append({"recv": dst, "send": src, "send_limbs": held[src],
                         "product_limbs": held[dst]})
            del held[src]
        rounds.append(step)
    return {"parts": parts, "ranks": ranks, "rounds": rounds,
            "depth": math.ceil(math.log2(parts)) if parts > 1 else 0}
