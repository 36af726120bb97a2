"""The C ABI's host-only size functions (no GPU needed): each bound covers the
exact size computed with Python integers and stays close to it, and invalid
arguments are rejected with CAT_EINVAL."""
import math
import random
import sys
from decimal import Decimal, getcontext
from fractions import Fraction

import pytest

if hasattr(sys, "set_int_max_str_digits"):
    sys.set_int_max_str_digits(0)


def _digits_of_all_ones(limbs: int) -> int:
    # decimal digits of 2^(32 limbs) - 1 = floor(32 limbs log10 2) + 1 (2^k is
    # never a power of ten, so 2^k - 1 has as many digits as 2^k)
    getcontext().prec = 60
    return int(Decimal(32 * limbs) * Decimal(2).log10()) + 1


@pytest.mark.parametrize("nl", list(range(1, 70)) + [100, 999, 4096, 10**4])
def test_decimal_bound_covers_every_value_small(cat_lib, nl):
    exact = len(str((1 << (32 * nl)) - 1))
    b = cat_lib.cat_decimal_bound(nl)
    assert exact <= b <= exact + 64


@pytest.mark.parametrize("nl", [10**5, 10**6, 128_160_805, 1 << 27, (1 << 30) + 7])
def test_decimal_bound_covers_every_value_large(cat_lib, nl):
    exact = _digits_of_all_ones(nl)
    b = cat_lib.cat_decimal_bound(nl)
    assert exact <= b <= exact + exact // 10**6 + 64


def _limbs(x: int) -> int:
    return max(1, (x.bit_length() + 31) // 32)


def test_ratio_bound_covers_binomials_and_multinomials(cat_lib):
    rng = random.Random(7)
    cases = [([10], [3, 7]), ([1000], [500, 500]), ([4000], [1, 3999]), ([5], [5]),
             ([0], []), ([2000, 3], [2001])]
    for _ in range(40):
        parts = [rng.randint(0, 600) for _ in range(rng.randint(1, 5))]
        cases.append(([sum(parts)], parts))
    for a, b in cases:
        q = Fraction(math.prod(math.factorial(x) for x in a),
                     math.prod(math.factorial(x) for x in b))
        bound = cat_lib.cat_ratio_bound_limbs(a, b)
        if q.denominator == 1:
            assert _limbs(int(q)) <= bound <= _limbs(int(q)) + 3, (a, b)


def test_ratio_bound_rejects_bad_terms(cat_lib):
    with pytest.raises(cat_lib.CatError) as e:
        cat_lib.cat_ratio_bound_limbs([1] * 17, [1])          # more than 16 terms
    assert e.value.code == cat_lib.CAT_EINVAL
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_ratio_bound_limbs([1 << 32], [1])         # a term of 33 bits
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_ratio_bound_limbs([1 << 31, 1 << 31], [1])  # numerators sum to 2^32


def test_batch_bound_is_the_sum_of_bounds(cat_lib):
    rng = random.Random(3)
    reqs = [(rng.randint(0, 2), rng.randint(0, 10**6)) for _ in range(200)]
    assert cat_lib.cat_batch_bound(reqs) == sum(cat_lib.cat_bound_limbs(n, k) for k, n in reqs)
    assert cat_lib.cat_batch_bound([]) == 0
    with pytest.raises(cat_lib.CatError) as e:
        cat_lib.cat_batch_bound([(0, 10), (0, 1 << 31)])
    assert e.value.code == cat_lib.CAT_EINVAL
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_batch_bound([(3, 10)])                    # unknown kind


def test_noalloc_size_check_on_the_host(cat_lib):
    # bigint_mul_noalloc rejects sizes beyond its static scratch before any
    # device work, including lengths whose sum would wrap around size_t (the
    # pointers are never dereferenced, so no GPU is needed)
    import ctypes
    L = cat_lib.load()
    n = ctypes.c_size_t()
    fake = ctypes.c_void_p(16)
    big = (1 << 64) - 1
    for na, nb in [(big, 2), (2, big), (cat_lib.NOALLOC_MAX_LIMBS + 1, 0),
                   (cat_lib.NOALLOC_MAX_LIMBS, 1), (1 << 63, 1 << 63)]:
        rc = L.bigint_mul_noalloc(fake, na, fake, nb, fake, big, ctypes.byref(n), None)
        assert rc == cat_lib.CAT_ENOMEM, (na, nb)
    rc = L.bigint_mul_noalloc(fake, 4, fake, 4, fake, 7, ctypes.byref(n), None)
    assert rc == cat_lib.CAT_ERANGE  # cap below na + nb, still before device work
