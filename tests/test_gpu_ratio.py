"""Factorial ratios prod a_i! / prod b_j! (Sec. 6.3) through the C ABI on the
GPU, against the oracle's two-phase computation."""
import math

import numpy as np
import pytest

from paper_2601_11621_gb300 import capi

pytestmark = pytest.mark.gpu

CASES = [
    ([10], [3, 7]),                         # C(10, 3)
    ([10**6], [3 * 10**5, 7 * 10**5]),      # C(10^6, 3 10^5)
    ([3 * 10**5], [10**5, 10**5, 10**5]),   # multinomial
    ([2 * 10**5], [10**5, 10**5 + 1]),      # C(10^5) in ratio form
    ([10**6], [10**6 - 17]),                # falling factorial
    ([60000, 50000], [50000, 40000, 20000]),  # C(60000, 20000), a term cancelling
    ([1234567], [617283, 617284]),          # odd split
    ([0, 1, 1], [0]),                       # ones
    ([], []),                               # empty product
]


@pytest.mark.parametrize("a,b", CASES)
def test_ratio_vs_oracle(orc, ctx, a, b):
    r = capi.to_numpy(capi.cat_ratio_exact(ctx, a, b))
    want = orc.ratio_exact(a, b)
    assert (r == want).all()
    assert capi.cat_ratio_bound_limbs(a, b) >= len(want)


def test_ratio_catalan_equals_kind(ctx):
    n = 123457
    r = capi.to_numpy(capi.cat_ratio_exact(ctx, [2 * n], [n, n + 1]))
    k = capi.to_numpy(capi.catalan_exact(ctx, n))
    assert (r == k).all()


def test_ratio_factorisation_vs_oracle(orc, ctx):
    a, b = [10**6, 3 * 10**5], [5 * 10**5, 2 * 10**5, 10**5]
    f = capi.cat_ratio_factor(ctx, a, b)
    try:
        primes = orc.sieve(10**6)
        e = orc.ratio_exponents(a, b, primes)
        exps, offs, gp = orc.group(primes, e)
        assert (f.exps == exps).all() and (f.offsets == offs).all()
        assert (capi.to_numpy(f.primes()) == gp).all()
    finally:
        f.free()


@pytest.mark.parametrize("a,b", [([5], [3, 3]), ([3], [4]), ([10**6], [10**6 + 1]),
                                 ([100], [60, 60]), ([50000, 50000], [40000, 60000])])
def test_ratio_not_integral(ctx, a, b):
    with pytest.raises(capi.CatError) as e:
        capi.cat_ratio_exact(ctx, a, b)
    assert e.value.code == capi.CAT_ENOTINTEGRAL


def test_ratio_limits(ctx):
    with pytest.raises(capi.CatError) as e:
        capi.cat_ratio_exact(ctx, [1] * 17, [])
    assert e.value.code == capi.CAT_EINVAL
    with pytest.raises(capi.CatError) as e:
        capi.cat_ratio_exact(ctx, [2**31, 2**31], [])   # numerator sum 2^32
    assert e.value.code == capi.CAT_EINVAL
    with pytest.raises(capi.CatError):
        capi.cat_ratio_bound_limbs([2**32], [])
