"""GPU parity: Phase 1 (grouped factorisation) and the end-to-end exact
results, against the CPU oracle.  Integer work: bit-exact.

Sizes the oracle finishes in seconds are compared limb for limb (or group by
group); the larger ones against oracle results stored by
tests/golden/make_oracle_golden.py, plus modular checks against residues the
oracle computes from factorial products, and, at the paper's n, the digit
count, bit length, byte count and SHA-256 printed in Table 1."""
import hashlib
import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEG = 1 << 18  # odd numbers per sieve segment on the device


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def read_kv(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split(None, 1)
            rows[k] = v
    return rows


def oracle_results():
    out = {}
    for line in open(os.path.join(GOLDEN, "oracle_results.txt")):
        if line.startswith("#") or not line.strip():
            continue
        kind, n, limbs, bits, sha = line.split()
        out[(kind, int(n))] = (int(limbs), int(bits), sha)
    return out


KIND = {0: "catalan", 1: "central_binomial", 2: "factorial"}

# n chosen around sieve-segment edges (2n = 2 * 2^18 * k +- small) and tiny cases
FACTOR_NS = [0, 1, 2, 3, 4, 5, 10, 97, 1000, SEG, SEG + 1, 2 * SEG - 1, 3 * SEG + 7,
             100000, 999_983, 10**6]


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("n", FACTOR_NS)
def test_factor_matches_oracle(ctx, cat_lib, orc, kind, n):
    f = cat_lib.catalan_factor(ctx, n, kind)
    try:
        exps, offs, gp = orc.factor(kind, n)
        assert f.primes_sieved == orc.prime_count(orc.prime_limit(kind, n))
        assert f.exps.tolist() == exps.tolist()
        assert f.offsets.tolist() == offs.tolist()
        got = host(f.primes())
        assert got.shape == gp.shape and (got == gp).all()
    finally:
        f.free()


@pytest.mark.parametrize("kind", [0, 1])
def test_factor_small_sweep_binomial(ctx, cat_lib, orc, kind):
    # every n up to 300: n + 1 prime (Catalan exponent 0 above sqrt(2n)),
    # sqrt(2n) crossing a prime, the smallest cases of the binomial kinds
    for n in range(1, 301):
        f = cat_lib.catalan_factor(ctx, n, kind)
        try:
            exps, offs, gp = orc.factor(kind, n)
            assert f.exps.tolist() == exps.tolist(), n
            assert f.offsets.tolist() == offs.tolist(), n
            assert (host(f.primes()) == gp).all(), n
            assert f.primes_sieved == orc.prime_count(2 * n), n
        finally:
            f.free()


# (p^2 - 1)/2 for a prime p: sqrt(2n) lies just below p, so p is the smallest
# prime handled by the one-division exponent; 2^31 - 1 is the largest n taken
@pytest.mark.parametrize("n", [(1009**2 - 1) // 2, 12_345_679, 2**30 + 3,
                               (65521**2 - 1) // 2, 2**31 - 1])
@pytest.mark.parametrize("kind", [0, 1])
def test_factor_binomial_vs_ratio_path(ctx, cat_lib, kind, n):
    # C(n) = (2n)!/(n! (n+1)!) and C(2n, n) = (2n)!/(n! n!) as factorial
    # ratios take Legendre's formula for every prime and the radix grouping;
    # the binomial kinds take the one-division exponent above sqrt(2n).
    import torch
    b = [n, n + 1] if kind == 0 else [n, n]
    f = cat_lib.catalan_factor(ctx, n, kind)
    g = cat_lib.cat_ratio_factor(ctx, [2 * n], b)
    try:
        assert f.primes_sieved == g.primes_sieved
        assert f.num_primes == g.num_primes
        assert f.exps.tolist() == g.exps.tolist()
        assert f.offsets.tolist() == g.offsets.tolist()
        assert torch.equal(f.primes(), g.primes())
    finally:
        f.free()
        g.free()
        torch.cuda.empty_cache()


def test_factor_config1_counts(ctx, cat_lib):
    # n = 10^5: 17,984 primes <= 2n (pi(2*10^5), textbook value)
    f = cat_lib.catalan_factor(ctx, 100000, 0)
    assert f.primes_sieved == 17984
    f.free()


def test_factor_50m_vs_oracle_groups(ctx, cat_lib):
    g = read_kv("oracle_groups_catalan_50000000.txt")
    f = cat_lib.catalan_factor(ctx, 50_000_000, 0)
    try:
        assert f.primes_sieved == int(g["sieved"])
        assert f.num_primes == int(g["positive"])
        counts = {int(k): int(v) for k, v in g.items() if k.isdigit()}
        got = {int(e): int(f.offsets[i + 1] - f.offsets[i]) for i, e in enumerate(f.exps)}
        assert got == counts
        sha = hashlib.sha256(host(f.primes()).astype("<u4").tobytes()).hexdigest()
        assert sha == g["sha256"]
    finally:
        f.free()


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 10, 33, 100, 1000, 4097, 12345, 100000])
def test_exact_small(ctx, cat_lib, orc, kind, n):
    got = host(cat_lib.cat_exact(ctx, kind, n))
    want = orc.exact(kind, n)
    assert got.shape == want.shape and (got == want).all()


def test_catalan_config1_with_mod_checks(ctx, cat_lib, orc):
    n = 100000
    got = host(cat_lib.catalan_exact(ctx, n))
    want = orc.catalan(n)
    assert (got == want).all()
    # 8 seeded random 31-bit primes q > 2n
    for q in orc.check_primes(seed=2024, count=8, lower=2 * n, bits=31):
        assert orc.limbs_mod(got, q) == orc.exact_mod(orc.CATALAN, n, q)


def test_exact_host_buffer(ctx, cat_lib, orc):
    got = cat_lib.cat_exact_host(ctx, 0, 54321)
    assert (got == orc.catalan(54321)).all()


@pytest.mark.parametrize("shift", [0, 1, 2, 3])
@pytest.mark.parametrize("kind,n", [(0, 54321), (1, 7), (2, 3000), (0, 2 * 10**6)])
def test_exact_into_pinned_host(ctx, cat_lib, orc, shift, kind, n):
    # page-locked destinations take the store kernel: 16-byte aligned (shift 0)
    # or not (1..3 limbs in), lengths with and without a ragged last 1..3
    # limbs; limbs around the result stay untouched
    import torch
    cap = cat_lib.cat_bound_limbs(n, kind)
    pinned = torch.empty(cap + 8, dtype=torch.int32, pin_memory=True)
    buf = pinned.numpy().view(np.uint32)
    buf[:] = 0xDEADBEEF
    got = cat_lib.cat_exact_host(ctx, kind, n, out=buf[shift:shift + cap])
    want = cat_lib.to_numpy(cat_lib.cat_exact(ctx, kind, n))
    assert (got == want).all()
    if n <= 10**5:
        assert (got == orc.exact(kind, n)).all()
    assert (buf[:shift] == 0xDEADBEEF).all()
    assert (buf[shift + got.size:] == 0xDEADBEEF).all()


def test_exact_into_pageable_host(ctx, cat_lib):
    # pageable memory takes the copy-engine transfer
    n = 10**6
    cap = cat_lib.cat_bound_limbs(n, 0)
    buf = np.full(cap + 3, 0xDEADBEEF, dtype=np.uint32)
    got = cat_lib.cat_exact_host(ctx, 0, n, out=buf[1:1 + cap])
    want = cat_lib.to_numpy(cat_lib.catalan_exact(ctx, n))
    assert (got == want).all()
    assert buf[0] == 0xDEADBEEF and (buf[1 + got.size:] == 0xDEADBEEF).all()


@pytest.mark.parametrize("kind,n", [("catalan", 10**6), ("central_binomial", 10**6),
                                    ("factorial", 10**6), ("catalan", 10**7),
                                    ("catalan", 50_000_000)])
def test_exact_vs_stored_oracle(ctx, cat_lib, orc, kind, n):
    limbs, bits, sha = oracle_results()[(kind, n)]
    k = {v: k for k, v in KIND.items()}[kind]
    got = host(cat_lib.cat_exact(ctx, k, n))
    assert len(got) == limbs
    assert (len(got) - 1) * 32 + int(got[-1]).bit_length() == bits
    assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == sha
    if kind == "catalan" and n <= 10**7:
        for q in orc.check_primes(seed=n, count=4, lower=2 * n, bits=62):
            assert orc.limbs_mod(got, q) == orc.exact_mod(orc.CATALAN, n, q)


def _leading_digits(limbs, bits, ndig=12):
    top = int.from_bytes(np.asarray(limbs[-4:], dtype="<u4").tobytes(), "little")
    shift = (len(limbs) - 4) * 32
    # value ~ top * 2^shift; log10 of it
    return math.log10(top) + shift * math.log10(2)


@pytest.mark.slow
def test_paper_scale(ctx, cat_lib, orc):
    """n = 2,050,572,903 (Table 1): digits, bits, bytes, SHA-256, mod checks."""
    t = read_kv("paper_table1.txt")
    n = int(t["n"])
    got = host(cat_lib.catalan_exact(ctx, n))
    bits = (len(got) - 1) * 32 + int(got[-1]).bit_length()
    assert bits == int(t["bit_length"])
    nbytes = (bits + 7) // 8
    assert nbytes == int(t["result_file_bytes"])
    le = got.astype("<u4").tobytes()[:nbytes]
    header = bytes.fromhex(t["sha256_header_hex"])
    sha = hashlib.sha256(header + le).hexdigest()
    print("paper-scale SHA-256 (header + LE magnitude)", sha)
    # digits: floor(log10 C) + 1 from the top limbs (the fraction 0.981 is far
    # from an integer, so double precision decides it)
    l10 = _leading_digits(got, bits)
    assert math.floor(l10) + 1 == int(t["decimal_digits"])
    # modular checks against residues from factorial products (no sieve)
    qs = orc.check_primes(seed=20260101, count=16, lower=2 * n, bits=62)
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        want = list(ex.map(lambda q: orc.exact_mod(orc.CATALAN, n, q), qs))
        have = list(ex.map(lambda q: orc.limbs_mod(got, q), qs))
    assert have == want
    # Table 1's SHA-256 of the paper's own result file
    assert sha == t["sha256"]


def read_groups(name):
    """sieved / positive / sha256 rows and 'exponent count' rows of an
    oracle-written Phase-1 golden file."""
    head, groups = {}, []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, v = line.split()
        if k in ("sieved", "positive", "sha256"):
            head[k] = v
        else:
            groups.append((int(k), int(v)))
    return head, groups


@pytest.mark.slow
def test_paper_scale_factor_vs_oracle_groups(ctx, cat_lib):
    """Phase 1 at n = 2,050,572,903 (Algorithm 1 at Table 1's scale) against
    the oracle's grouping: the number of primes <= 2n, the number with
    e_p > 0, every group's exponent and size, and the SHA-256 of all grouped
    primes in CSR order (tests/golden/make_oracle_golden.py --paper)."""
    head, groups = read_groups("oracle_groups_catalan_2050572903.txt")
    f = cat_lib.catalan_factor(ctx, 2_050_572_903, 0)
    try:
        assert f.primes_sieved == int(head["sieved"])
        assert int(f.offsets[-1]) == int(head["positive"])
        assert f.exps.tolist() == [e for e, _ in groups]
        counts = np.diff(np.asarray(f.offsets.tolist(), dtype=np.int64)).tolist()
        assert counts == [c for _, c in groups]
        got = host(f.primes())
        assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == head["sha256"]
    finally:
        f.free()
