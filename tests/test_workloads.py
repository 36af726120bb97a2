"""The seeded input generators shared by the oracle checks, the GPU tests and
the benchmark: same seed, same inputs; the shapes and distributions stated
for each workload (limb layout, request mixes, Poisson arrivals)."""
import math

import numpy as np

from paper_2601_11621_gb300 import workloads


def test_same_seed_same_inputs():
    assert np.array_equal(workloads.random_limbs(1000, 5), workloads.random_limbs(1000, 5))
    assert not np.array_equal(workloads.random_limbs(1000, 5), workloads.random_limbs(1000, 6))
    assert workloads.batched_requests(64, 3) == workloads.batched_requests(64, 3)
    assert workloads.served_requests(64, 100.0, 3) == workloads.served_requests(64, 100.0, 3)


def test_limbs_are_little_endian_words_with_a_nonzero_top():
    a = workloads.random_limbs(257, 11)
    assert a.dtype == np.uint32 and a.size == 514 and a[-1] != 0
    w = workloads.rng(11).integers(0, 1 << 64, size=257, dtype=np.uint64, endpoint=False)
    lo = (w & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    hi = (w >> np.uint64(32)).astype(np.uint32)
    assert np.array_equal(a[0:-2:2], lo[:-1]) and np.array_equal(a[1:-2:2], hi[:-1])
    b = workloads.random_limbs32(1001, 2)
    assert b.dtype == np.uint32 and b.size == 1001 and b[-1] != 0
    assert workloads.random_limbs(0, 1).size == 0 and workloads.random_limbs32(0, 1).size == 0


def test_random_values_range():
    v = workloads.random_values(10000, 4, lo=2, hi=1000)
    assert v.min() >= 2 and v.max() < 1000


def test_batched_requests_mix():
    reqs = workloads.batched_requests(4096, 0)
    kinds = [k for k, _ in reqs]
    ns = np.array([n for _, n in reqs], dtype=float)
    assert set(kinds) == {0, 1} and abs(sum(kinds) / 4096 - 0.5) < 0.05
    assert ns.min() >= 1e3 and ns.max() < 1e6
    # log-uniform: the mean of ln n is the midpoint of [ln 1e3, ln 1e6]
    assert abs(np.log(ns).mean() - 0.5 * (math.log(1e3) + math.log(1e6))) < 0.1


def test_served_requests_arrivals():
    reqs = workloads.served_requests(5000, 300.0, 1)
    t = np.array([a for a, _, _ in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.diff(t).mean() - 1 / 300.0) < 0.1 / 300.0   # exponential gaps, mean 1/rate
    assert {k for _, k, _ in reqs} == {0, 1, 2}
    ns = np.array([n for _, _, n in reqs], dtype=float)
    assert ns.min() >= 1e4 and ns.max() < 1e8
