"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: textbook
prime counts, brute-force valuations, Kummer's theorem, de Polignac's digit-sum
form of Legendre's formula, CPython's own big integers (an independent bignum
implementation), the Catalan recurrence, and the figures the paper prints in
Table 1.  A plausible mistake (a dropped c_p term, a wrong Legendre bound, a
transposed Karatsuba operand, a lost carry) fails at least one of them.
"""
import math
import os
import random

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            rows[k] = v
    return rows


# ------------------------------------------------------------------ sieve

def test_prime_counts_textbook(orc):
    for x, pi in read_golden("prime_counts.txt").items():
        x, pi = int(x), int(pi)
        if x > 10**7:
            continue  # 10^8 runs in the slow variant below
        assert orc.prime_count(x) == pi, x


@pytest.mark.slow
def test_prime_count_1e8(orc):
    assert orc.prime_count(10**8) == int(read_golden("prime_counts.txt")["100000000"])


def _is_prime_trial(x):
    if x < 2:
        return False
    d = 2
    while d * d <= x:
        if x % d == 0:
            return False
        d += 1
    return True


def test_sieve_matches_trial_division(orc):
    for limit in (0, 1, 2, 3, 4, 10, 97, 100, 1009, 5000):
        got = orc.sieve(limit).tolist()
        want = [x for x in range(limit + 1) if _is_prime_trial(x)]
        assert got == want, limit


def test_sieve_block_boundary(orc):
    # the oracle sieves in blocks of 2^24 integers; primes straddling a block
    # edge must all be found
    lo = (1 << 24) - 200
    pr = orc.sieve((1 << 24) + 200)
    tail = [int(p) for p in pr if p >= lo]
    want = [x for x in range(lo, (1 << 24) + 201) if _is_prime_trial(x)]
    assert tail == want


def test_miller_rabin(orc):
    for x in range(0, 3000):
        assert orc.is_prime(x) == _is_prime_trial(x), x
    # Carmichael numbers and a strong pseudoprime to base 2
    for x in (561, 1105, 1729, 2047, 3215031751, 3825123056546413051):
        assert not orc.is_prime(x)
    assert orc.is_prime((1 << 61) - 1)          # Mersenne prime M61
    assert orc.is_prime(2305843009213693951)


# ---------------------------------------------------------------- Legendre

def _vp_brute(x, p):
    v = 0
    while x % p == 0:
        x //= p
        v += 1
    return v


def test_legendre_brute_force(orc):
    for p in (2, 3, 5, 7, 11, 13, 97):
        acc = 0
        for m in range(0, 600):
            if m > 0:
                acc += _vp_brute(m, p)
            assert orc.legendre(m, p) == acc, (m, p)


def test_legendre_digit_sum_form(orc):
    # de Polignac / Legendre: v_p(m!) = (m - s_p(m)) / (p - 1), s_p = base-p
    # digit sum.  A different formula, exact at every size; it also exercises
    # the p^k overflow guard near 2^64.
    rng = random.Random(7)
    primes = [2, 3, 5, 7, 65521, 4294967291, 4101145801]
    for _ in range(400):
        m = rng.randrange(0, 1 << rng.choice([8, 20, 32, 40, 62, 63]))
        p = rng.choice(primes)
        s, x = 0, m
        while x:
            s += x % p
            x //= p
        assert orc.legendre(m, p) == (m - s) // (p - 1), (m, p)


def _kummer_carries(a, b, p):
    carries, c = 0, 0
    while a or b or c:
        d = a % p + b % p + c
        c = 1 if d >= p else 0
        carries += c
        a //= p
        b //= p
    return carries


def test_catalan_exponents_kummer(orc):
    # Kummer's theorem: v_p(binom(2n, n)) = number of carries when adding
    # n + n in base p.  With v_p(n+1) this gives v_p(C(n)) independently of
    # Legendre's formula (Sec. 2 cites Kummer for integrality).
    rng = random.Random(11)
    ns = list(range(0, 60)) + [rng.randrange(60, 200000) for _ in range(40)]
    for n in ns:
        prs = orc.sieve(2 * n)
        e = orc.exponents(orc.CATALAN, n, prs)
        eb = orc.exponents(orc.CENTRAL_BINOMIAL, n, prs)
        for p, ep, ebp in zip(prs.tolist(), e.tolist(), eb.tolist()):
            k = _kummer_carries(n, n, p)
            assert ebp == k, (n, p)
            assert ep == k - _vp_brute(n + 1, p), (n, p)
            assert ep >= 0
    # the paper's n, on the seed primes and on primes near n and 2n
    n = 2050572903
    prs = np.concatenate([orc.sieve(64040),
                          np.array([orc.next_prime(n - 1000), orc.next_prime(n + 1),
                                    orc.next_prime(2 * n - 100)], dtype=np.uint32)])
    e = orc.exponents(orc.CATALAN, n, prs)
    for p, ep in zip(prs.tolist(), e.tolist()):
        assert ep == _kummer_carries(n, n, p) - _vp_brute(n + 1, p), p


def test_large_primes_exponent_is_0_or_1(orc):
    # Sec. 3.1: for primes p > sqrt(2n) only the first Legendre term survives,
    # so e_p in {0, 1} (minus v_p(n+1)).
    n = 123456
    pr = orc.sieve(2 * n)
    e = orc.exponents(orc.CENTRAL_BINOMIAL, n, pr)
    big = pr > math.isqrt(2 * n)
    assert set(np.unique(e[big]).tolist()) <= {0, 1}
    for p, ep in zip(pr[big].tolist(), e[big].tolist()):
        assert ep == (2 * n) // p - 2 * (n // p)


def test_factor_trial(orc):
    pr = orc.sieve(1 << 17)
    rng = random.Random(3)
    ms = [1, 2, 3, 4, 1 << 31, 2050572904, 4294967291, 600851475143 % (1 << 33)]
    ms += [rng.randrange(1, 1 << 32) for _ in range(300)]
    for m in ms:
        f = orc.factor_trial(m, pr)
        prod = 1
        for p, e in f:
            assert _is_prime_trial(p) if p < 10**7 else orc.is_prime(p)
            prod *= p ** e
        assert prod == m, m
        assert [p for p, _ in f] == sorted(p for p, _ in f)
    # n + 1 for the paper's n = 2,050,572,903
    assert orc.factor_trial(2050572904, pr) == [(2, 3), (347, 1), (691, 1), (1069, 1)]


def test_ratio_form_equals_algorithm_1(orc):
    # Sec. 6.3 generalisation with a = [2n], b = [n, n+1] is the Catalan number.
    for n in (1, 2, 10, 99, 1000, 54321):
        pr = orc.sieve(2 * n)
        e1 = orc.exponents(orc.CATALAN, n, pr)
        e2 = orc.ratio_exponents([2 * n], [n, n + 1], pr)
        assert (e1 == e2).all(), n


# ---------------------------------------------------------------- grouping

def test_group_csr(orc):
    rng = np.random.default_rng(5)
    pr = orc.sieve(50000)
    e = rng.integers(-1, 6, size=len(pr)).astype(np.int64)
    exps, offs, gp = orc.group(pr, e)
    assert list(exps) == sorted(set(int(x) for x in e if x > 0))
    for g, ex in enumerate(exps):
        members = gp[offs[g]:offs[g + 1]]
        want = pr[e == ex]
        assert (members == want).all()
    assert offs[-1] == (e > 0).sum()


# ---------------------------------------------------------------- bigints

def _rand_int(rng, nlimbs, kind="rand"):
    if nlimbs == 0:
        return 0
    if kind == "ones":
        return (1 << (32 * nlimbs)) - 1
    if kind == "pow2":
        return 1 << (32 * nlimbs - 1)
    return rng.getrandbits(32 * nlimbs) | (1 << (32 * nlimbs - 1))


def test_mul_vs_cpython(orc):
    rng = random.Random(17)
    sizes = [(1, 1), (1, 9), (2, 2), (31, 31), (32, 32), (33, 33), (31, 32),
             (63, 64), (64, 65), (100, 400), (400, 100), (1000, 999), (1024, 4096),
             (2047, 2049), (5000, 5000), (7000, 13), (3, 7000), (30000, 7500)]
    for na, nb in sizes:
        for kind in ("rand", "ones", "pow2"):
            a, b = _rand_int(rng, na, kind), _rand_int(rng, nb, kind)
            got = orc.limbs_to_int(orc.mul(orc.int_to_limbs(a), orc.int_to_limbs(b)))
            assert got == a * b, (na, nb, kind)
    assert orc.mul([], [5]).size == 0
    assert orc.mul([0, 0], [5]).size == 0


def test_product_tree_vs_cpython(orc):
    rng = random.Random(19)
    for count in (0, 1, 2, 3, 5, 64, 1000, 4097):
        v = [rng.randrange(1, 1 << 32) for _ in range(count)]
        got = orc.limbs_to_int(orc.product_tree(np.array(v, dtype=np.uint32)))
        assert got == math.prod(v), count


def test_pow_vs_cpython(orc):
    rng = random.Random(23)
    for nl, e in ((1, 0), (1, 1), (1, 2), (1, 31), (3, 17), (40, 13), (1, 1000),
                  (5, 257)):
        a = _rand_int(rng, nl)
        got = orc.limbs_to_int(orc.power(orc.int_to_limbs(a), e))
        assert got == a ** e, (nl, e)
    assert orc.limbs_to_int(orc.power([2], 100000)) == 1 << 100000


# ---------------------------------------------------------- exact results

def test_catalan_recurrence_small(orc):
    # C(0) = 1, C(n+1) = C(n) * 2(2n+1) / (n+2): brute force in CPython ints
    c = 1
    for n in range(0, 400):
        assert orc.limbs_to_int(orc.catalan(n)) == c, n
        assert c == math.factorial(2 * n) // (math.factorial(n) * math.factorial(n + 1))
        c = c * 2 * (2 * n + 1) // (n + 2)


def test_catalan_first_values(orc):
    # C(n) = (2n)! / (n! (n+1)!) for the first few n (Sec. 1 definition)
    first = [1, 1, 2, 5, 14, 42, 132, 429, 1430, 4862, 16796]
    assert [orc.limbs_to_int(orc.catalan(n)) for n in range(11)] == first


@pytest.mark.parametrize("n", [1000, 12345, 100000])
def test_three_kinds_vs_math(orc, n):
    assert orc.limbs_to_int(orc.exact(orc.CATALAN, n)) == math.comb(2 * n, n) // (n + 1)
    assert orc.limbs_to_int(orc.exact(orc.CENTRAL_BINOMIAL, n)) == math.comb(2 * n, n)
    assert orc.limbs_to_int(orc.exact(orc.FACTORIAL, n)) == math.factorial(n)


def test_digit_estimate(orc):
    # Algorithm 1 last step: floor(sum e_p log10 p) + 1 is the digit count
    for n in (10, 1000, 100000):
        pr = orc.sieve(2 * n)
        e = orc.exponents(orc.CATALAN, n, pr)
        est = orc.log10_estimate(pr, e)
        c = math.comb(2 * n, n) // (n + 1)
        d = math.floor(est) + 1
        assert 10 ** (d - 1) <= c < 10 ** d, n


def test_config_1_sizes(orc):
    # n = 10^5: 17,984 primes <= 2n; the result has 199,975 bits.
    n = 10**5
    pr = orc.sieve(2 * n)
    assert len(pr) == 17984
    c = orc.catalan(n)
    assert orc.limbs_to_int(c).bit_length() == 199975


# ------------------------------------------------------------ mod checks

def test_mulmod_montgomery(orc):
    rng = random.Random(29)
    for _ in range(500):
        q = orc.next_prime(rng.randrange(3, 1 << 63))
        if q >= 1 << 63:
            continue
        a, b = rng.randrange(0, 1 << 64), rng.randrange(0, 1 << 64)
        assert orc.mulmod_mont(a, b, q) == (a * b) % q
        assert orc.mulmod_plain(a, b, q) == (a * b) % q


def test_range_product_mod(orc):
    q = orc.next_prime(10**12)
    assert orc.range_product_mod(1, 1000, q) == math.factorial(1000) % q
    assert orc.range_product_mod(500, 499, q) == 1
    assert orc.range_product_mod(7, 7, q) == 7


def test_exact_mod_and_horner(orc):
    for n in (5, 1000, 30000):
        for q in orc.check_primes(seed=n, count=3, lower=2 * n, bits=62):
            c = math.comb(2 * n, n) // (n + 1)
            assert orc.exact_mod(orc.CATALAN, n, q) == c % q
            assert orc.exact_mod(orc.CENTRAL_BINOMIAL, n, q) == math.comb(2 * n, n) % q
            assert orc.exact_mod(orc.FACTORIAL, n, q) == math.factorial(n) % q
            assert orc.limbs_mod(orc.int_to_limbs(c), q) == c % q
    for q in orc.check_primes(seed=1, count=8, lower=2 * 10**5, bits=31):
        assert q < 1 << 31
        assert orc.limbs_mod(orc.catalan(10**5), q) == orc.exact_mod(orc.CATALAN, 10**5, q)


# --------------------------------------------------------- paper's Table 1

def _log_catalan_mp(n, base):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    lg = mpmath.loggamma(2 * n + 1) - mpmath.loggamma(n + 1) - mpmath.loggamma(n + 2)
    return lg / mpmath.log(base)


def test_paper_digits_and_bits_closed_form(orc):
    # Table 1: n = 2,050,572,903 gives 1,234,567,890 digits and
    # 4,101,145,759 bits.  Closed form: floor(log_b C) + 1 from log-gamma.
    t = read_golden("paper_table1.txt")
    n = int(t["n"])
    l10 = _log_catalan_mp(n, 10)
    l2 = _log_catalan_mp(n, 2)
    import mpmath
    assert int(mpmath.floor(l10)) + 1 == int(t["decimal_digits"])
    assert int(mpmath.floor(l2)) + 1 == int(t["bit_length"])
    assert (int(t["bit_length"]) + 7) // 8 == int(t["result_file_bytes"])
    # the oracle's limb bound covers it
    assert orc.bound_limbs(orc.CATALAN, n) * 32 >= int(t["bit_length"])


def test_paper_n_plus_1_and_seed_range(orc):
    # the seed primes of the paper's n: primes up to sqrt(2n) = 64,040
    n = 2050572903
    assert math.isqrt(2 * n) == 64040
    assert orc.prime_count(64040) == 6418


def test_sieve_range_is_a_slice_of_the_sieve(orc):
    full = orc.sieve((1 << 24) + 100)
    for lo, hi in [(0, 100), (2, 2), (90, 97), (1_000_000, 1_000_100),
                   ((1 << 24) - 50, (1 << 24) + 50), (2_999_000, 3_000_000)]:
        want = full[(full >= lo) & (full <= hi)]
        assert (orc.sieve_range(lo, hi) == want).all(), (lo, hi)


# ------------------------------------------------- decimal output (Sec. 3.2)

def _dec_special_values():
    vals = [0, 1, 9, 10, 999_999_999, 1_000_000_000, 2**32 - 1, 2**32, 2**64 - 1]
    for k in (9, 10, 17, 18, 19, 81, 154, 155, 1000):
        vals += [10**k - 1, 10**k, 10**k + 1]
    for w in (1, 2, 15, 16, 17, 100):
        vals += [2 ** (32 * w) - 1, 2 ** (32 * w)]
    return vals


def test_to_decimal_vs_cpython(orc):
    # the digits are unique; CPython's int -> str is an independent routine
    import sys
    if hasattr(sys, "set_int_max_str_digits"):
        sys.set_int_max_str_digits(0)
    rnd = random.Random(20260101)
    vals = _dec_special_values()
    for nl in (1, 2, 3, 7, 16, 33, 257, 2049):
        vals.append(rnd.getrandbits(32 * nl) | 1 << (32 * nl - 1))
    for v in vals:
        assert orc.to_decimal(orc.int_to_limbs(v)) == str(v).encode(), v
    # leading zero limbs are ignored
    limbs = np.concatenate([orc.int_to_limbs(12345), np.zeros(5, np.uint32)])
    assert orc.to_decimal(limbs) == b"12345"


def test_to_decimal_catalan_digit_count(orc):
    # C(10^5) has 60,199 digits (floor(log10 C) + 1 from log-gamma)
    d = orc.to_decimal(orc.catalan(10**5))
    assert len(d) == 60199
    lg = math.lgamma(2e5 + 1) - math.lgamma(1e5 + 1) - math.lgamma(1e5 + 2)
    assert len(d) == int(lg / math.log(10)) + 1
    # leading digits from the fractional part of log10 C
    frac = lg / math.log(10) - int(lg / math.log(10))
    assert d[:6] == str(int(10 ** (frac + 5))).encode()


# --------------------------------------- factorial ratios (Sec. 6.3)

def test_ratio_exact_vs_cpython(orc):
    f = math.factorial
    cases = [([10], [3, 7]), ([1000], [400, 600]), ([30], [10, 10, 10]),
             ([2 * 500], [500, 501]), ([200, 7], [100, 100]), ([12], [12]), ([], []),
             ([5000], [4999]), ([0], []), ([1, 1], [0])]
    for a, b in cases:
        want = 1
        for x in a:
            want *= f(x)
        for y in b:
            assert want % f(y) == 0
            want //= f(y)
        assert orc.limbs_to_int(orc.ratio_exact(a, b)) == want, (a, b)
    # C(n) through the ratio form equals Algorithm 1 (kind = Catalan)
    assert (orc.ratio_exact([2 * 3000], [3000, 3001]) == orc.catalan(3000)).all()


def test_ratio_not_integral(orc):
    # 5!/(3! 3!) = 10/3; 3!/4!; 7!/(2! 2! 2! 2!) = 315 is integral
    for a, b in [([5], [3, 3]), ([3], [4]), ([10], [11])]:
        with pytest.raises(ValueError):
            orc.ratio_exact(a, b)
    assert orc.limbs_to_int(orc.ratio_exact([7], [2, 2, 2, 2])) == 315


def test_exact_mt_matches_single_thread_and_cpython(orc):
    # the OpenMP variant (tree halves and Karatsuba sub-products as tasks)
    # computes the same integers: against CPython's math.comb / factorial at
    # small n, against the single-threaded oracle where the tasks really split
    for kind, n in [(0, 0), (0, 1), (0, 77), (1, 5000), (2, 3000), (0, 20000)]:
        want = {0: math.comb(2 * n, n) // (n + 1), 1: math.comb(2 * n, n),
                2: math.factorial(n)}[kind]
        assert orc.limbs_to_int(orc.exact_mt(kind, n, threads=4)) == want, (kind, n)
    for kind, n in [(0, 300_000), (2, 200_000)]:
        a = orc.exact(kind, n)
        for t in (1, 3, orc.max_threads()):
            assert np.array_equal(orc.exact_mt(kind, n, threads=t), a), (kind, n, t)
