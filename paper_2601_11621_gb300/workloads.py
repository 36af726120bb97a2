"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU
oracle checks.  Random draws only: nothing here computes any part of the
method.

The paper's workloads are single values of n (Table 1: n = 2,050,572,903;
Table 2: n = 10^6, 10^7, 10^8).  The other inputs below are the stand-ins
for the multiplication sweep (uniform random 64-bit words, read as pairs of
little-endian 32-bit limbs) and for the batched and served request streams
(n log-uniform over a range, kinds mixed, Poisson arrivals).
"""
from __future__ import annotations

import numpy as np

PAPER_N = 2_050_572_903


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def random_limbs(n_u64: int, seed: int) -> np.ndarray:
    """2 * n_u64 uint32 limbs from n_u64 uniform 64-bit words; top limb forced
    non-zero so the length is exact."""
    if n_u64 == 0:
        return np.zeros(0, dtype=np.uint32)
    w = rng(seed).integers(0, 1 << 64, size=n_u64, dtype=np.uint64, endpoint=False)
    limbs = w.view("<u4").astype(np.uint32)
    if limbs[-1] == 0:
        limbs[-1] = 1
    return limbs


def random_limbs32(n: int, seed: int, top_nonzero: bool = True) -> np.ndarray:
    if n == 0:
        return np.zeros(0, dtype=np.uint32)
    limbs = rng(seed).integers(0, 1 << 32, size=n, dtype=np.uint64).astype(np.uint32)
    if top_nonzero and limbs[-1] == 0:
        limbs[-1] = 1
    return limbs


def random_values(count: int, seed: int, lo: int = 1, hi: int = 1 << 32) -> np.ndarray:
    """count uint32 values uniform in [lo, hi)."""
    return rng(seed).integers(lo, hi, size=count, dtype=np.uint64).astype(np.uint32)


def batched_requests(count: int = 4096, seed: int = 0, lo: float = 1e3, hi: float = 1e6):
    """(kind, n) pairs: kind 0 (Catalan) or 1 (central binomial) with equal
    probability, n = floor(exp(U(ln lo, ln hi)))."""
    g = rng(seed)
    kinds = g.integers(0, 2, size=count)
    ns = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    return [(int(k), int(n)) for k, n in zip(kinds, ns)]


def served_requests(count: int, rate: float, seed: int = 0, lo: float = 1e4, hi: float = 1e8):
    """(arrival_time_s, kind, n) with Poisson arrivals at `rate` per second,
    kind uniform over {0, 1, 2} and n log-uniform in [lo, hi]."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    kinds = g.integers(0, 3, size=count)
    ns = np.floor(np.exp(g.uniform(np.log(lo), np.log(hi), size=count))).astype(np.int64)
    return [(float(a), int(k), int(n)) for a, k, n in zip(t, kinds, ns)]
