"""Reconstruction within an HBM budget below its in-core need (the paper's
chunked products and offloaded partial products, Sec. 3.2): the grouped
primes move to pinned host memory, chunks of primes are multiplied on the
device, their roots and the powers live in host memory, and products too
large for the budget run by pieces through a sliding device window.  The
integer must be the same, limb for limb, and the context's high-water mark
must stay within its budget."""
import hashlib
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def in_core_peak(cat_lib, kind, n):
    c = cat_lib.Context(0)
    try:
        cat_lib.cat_exact(c, kind, n)
        return c.memory()[1]
    finally:
        c.close()


@pytest.mark.parametrize("kind,n,budget", [
    (0, 200_000, 600_000),       # chunks of 4,096 primes; the top products by pieces
    (0, 150_001, 1_000_000),
    (1, 120_000, 700_000),
    (2, 40_000, 500_000),        # n!: hundreds of groups, every Q_e^e by host powering
    (0, 2, 300_000), (0, 0, 300_000), (2, 1, 300_000),
])
def test_budgeted_exact_matches_oracle(cat_lib, orc, kind, n, budget):
    # really out of core: the listed budget or 80 % of the measured in-core
    # peak, whichever is smaller
    if n >= 100:
        peak_in_core = in_core_peak(cat_lib, kind, n)
        budget = min(budget, peak_in_core * 4 // 5)
        assert peak_in_core > budget
    c = cat_lib.Context(0, hbm_budget_bytes=budget)
    try:
        got = host(cat_lib.cat_exact(c, kind, n))
        peak = c.memory()[1]
    finally:
        c.close()
    want = orc.exact(kind, n)
    assert got.shape == want.shape and np.array_equal(got, want)
    assert peak <= budget


def test_budgeted_exact_into_host_and_ratio(cat_lib, orc):
    c = cat_lib.Context(0, hbm_budget_bytes=800_000)
    try:
        got = cat_lib.cat_exact_host(c, 0, 180_000)
        assert np.array_equal(got, orc.catalan(180_000))
        r = host(cat_lib.cat_ratio_exact(c, [60_000], [20_000, 25_000, 15_000]))
        assert np.array_equal(r, orc.ratio_exact([60_000], [20_000, 25_000, 15_000]))
        assert c.memory()[1] <= 800_000
    finally:
        c.close()


@pytest.mark.slow
def test_catalan_5e7_within_a_small_budget(cat_lib):
    """C(5 * 10^7) (3,124,999 limbs; ~200 MB in core) within a budget of its
    Phase 1 peak plus 8 MB, against the oracle's stored SHA-256."""
    n = 50_000_000
    want = {}
    for line in open(os.path.join(GOLDEN, "oracle_results.txt")):
        if line.startswith("catalan 50000000 "):
            _, _, limbs, bits, sha = line.split()
            want = {"limbs": int(limbs), "sha": sha}
    c = cat_lib.Context(0)
    try:
        f = cat_lib.catalan_factor(c, n, 0)
        f.free()
        phase1 = c.memory()[1]
    finally:
        c.close()
    budget = phase1 + (8 << 20)
    assert in_core_peak(cat_lib, 0, n) > 4 * budget // 2
    c = cat_lib.Context(0, hbm_budget_bytes=budget)
    try:
        got = host(cat_lib.catalan_exact(c, n))
        peak = c.memory()[1]
    finally:
        c.close()
    assert len(got) == want["limbs"]
    assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == want["sha"]
    assert peak <= budget


def test_budgeted_reconstruct_keeps_the_callers_factorization(cat_lib, orc):
    # a factorisation made in one context, reconstructed in a small-budget one
    # twice (the caller still owns it afterwards)
    big = cat_lib.Context(0)
    small = cat_lib.Context(0, hbm_budget_bytes=700_000)
    try:
        f = cat_lib.catalan_factor(big, 160_000, 0)
        cap = cat_lib.cat_bound_limbs(160_000, 0)
        for _ in range(2):
            got = host(cat_lib.cat_reconstruct(small, f, cap))
            assert np.array_equal(got, orc.catalan(160_000))
        assert f.primes().numel() == f.num_primes
        f.free()
        assert small.memory()[1] <= 700_000
    finally:
        small.close()
        big.close()
