"""to_decimal (the optional decimal output, Sec. 3.2) and products longer than
one transform, through the C ABI on the GPU, against the oracle."""
import math
import random
import sys

import numpy as np
import pytest

from paper_2601_11621_gb300 import capi, workloads

pytestmark = pytest.mark.gpu

if hasattr(sys, "set_int_max_str_digits"):
    sys.set_int_max_str_digits(0)


def _gpu_decimal(ctx, limbs) -> bytes:
    return bytes(capi.to_decimal(ctx, limbs).cpu().numpy())


def _special_values():
    vals = [0, 1, 7, 10, 999_999_999, 10**9, 2**32 - 1, 2**32]
    for k in (9, 18, 27, 153, 154, 155, 156, 1000, 4815, 40000):
        vals += [10**k - 1, 10**k, 10**k + 1]
    for w in (1, 15, 16, 17, 31, 32, 33, 255, 256, 257, 4096, 5000):
        vals += [2 ** (32 * w) - 1, 2 ** (32 * w)]
    return vals


def test_decimal_special_values(orc, ctx):
    # carry chains of nines, exact powers of ten, all-ones limbs, leaf edges
    for v in _special_values():
        limbs = orc.int_to_limbs(v)
        assert _gpu_decimal(ctx, limbs) == orc.to_decimal(limbs), v


@pytest.mark.parametrize("nl", [1, 2, 15, 16, 17, 63, 64, 65, 255, 256, 257, 1000,
                                4095, 4096, 4097, 8192 + 3, 40000])
def test_decimal_random(orc, ctx, nl):
    # sizes across the 16-limb leaves, the one-block levels (<= 2^12 points)
    # and the multi-pass levels, with ragged tails
    limbs = workloads.random_limbs32(nl, seed=nl)
    assert _gpu_decimal(ctx, limbs) == orc.to_decimal(limbs)


def test_decimal_leading_zero_limbs_and_capacity(orc, ctx):
    import torch
    limbs = np.concatenate([orc.int_to_limbs(10**50 + 12345), np.zeros(9, np.uint32)])
    assert _gpu_decimal(ctx, limbs) == str(10**50 + 12345).encode()
    # too small a buffer: CAT_ERANGE
    small = torch.empty(10, dtype=torch.uint8, device="cuda")
    with pytest.raises(capi.CatError) as e:
        capi.to_decimal(ctx, orc.int_to_limbs(10**50), out=small)
    assert e.value.code == capi.CAT_ERANGE
    # the bound never undercuts
    for nl in (1, 2, 10, 1000, 10**6):
        assert capi.cat_decimal_bound(nl) >= math.floor(nl * 32 * math.log10(2)) + 1


def test_decimal_of_catalan(orc, ctx):
    # C(10^6) from the GPU, printed on the GPU, against CPython's int -> str
    import torch
    n = 10**6
    r = capi.catalan_exact(ctx, n)
    d = bytes(capi.to_decimal(ctx, r).cpu().numpy())
    want = str(orc.limbs_to_int(orc.catalan(n))).encode()
    assert d == want


def test_long_product_by_pieces(orc, ctx):
    # na + nb > 2^27: summed from piece products of at most 2^26 limbs.
    # Checked by eight residues mod seeded 62-bit primes, mod 2^32 - 1 and
    # the low limbs (mod 2^(32 k)) from the oracle's product of the low limbs.
    import torch
    na, nb = (1 << 26) + 1000, (1 << 26) + 517
    a = workloads.random_limbs32(na, seed=11)
    b = workloads.random_limbs32(nb, seed=12)
    r = capi.bigint_mul(ctx, a, b)
    assert r.numel() in (na + nb - 1, na + nb)
    h = capi.to_numpy(r)
    for q in orc.check_primes(seed=5, count=8, lower=1 << 61, bits=62):
        assert orc.limbs_mod(h, q) == (orc.limbs_mod(a, q) * orc.limbs_mod(b, q)) % q
    m = (1 << 32) - 1
    fold = lambda x: int(np.asarray(x, dtype=np.uint64).sum()) % m  # 2^32 = 1 mod 2^32 - 1
    assert fold(h) == fold(a) * fold(b) % m
    k = 4096
    low = orc.mul(a[:k], b[:k])[:k]
    assert (h[:k] == low).all()
    del r
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def small_transform_ctx(cat_lib):
    """A context whose single-transform limit is 2^13 points, so that products
    longer than 8192 limbs go through the piece path."""
    import os
    old = os.environ.get("CAT_MAX_TRANSFORM_LOG")
    os.environ["CAT_MAX_TRANSFORM_LOG"] = "13"
    try:
        c = capi.Context(0)
    finally:
        if old is None:
            del os.environ["CAT_MAX_TRANSFORM_LOG"]
        else:
            os.environ["CAT_MAX_TRANSFORM_LOG"] = old
    yield c
    c.close()


@pytest.mark.parametrize("na,nb", [(5000, 7000), (4096, 4097), (20000, 3), (9000, 9000)])
def test_products_by_pieces_small(orc, small_transform_ctx, na, nb):
    a = workloads.random_limbs32(na, seed=na)
    b = workloads.random_limbs32(nb, seed=nb + 1)
    r = capi.to_numpy(capi.bigint_mul(small_transform_ctx, a, b))
    assert (r == orc.mul(a, b)).all()


def test_products_by_pieces_carry_chains(orc, small_transform_ctx):
    # (2^(32 k) - 1)^2 and (2^(32 k) - 1) (2^(32 m) - 1): long carry chains
    # through the piece additions
    for k, m in [(6000, 6000), (9000, 300), (8191, 8193)]:
        a, b = 2 ** (32 * k) - 1, 2 ** (32 * m) - 1
        r = capi.to_numpy(capi.bigint_mul(small_transform_ctx, orc.int_to_limbs(a),
                                          orc.int_to_limbs(b)))
        assert orc.limbs_to_int(r) == a * b


@pytest.mark.parametrize("nl", [9000, 20000])
def test_decimal_by_pieces(orc, small_transform_ctx, nl):
    # the upper conversion levels exceed 2^13 points and go by pieces
    limbs = workloads.random_limbs32(nl, seed=3 * nl)
    assert _gpu_decimal(small_transform_ctx, limbs) == orc.to_decimal(limbs)
    nines = orc.int_to_limbs(10 ** (9 * nl) - 1)  # all nines: maximal carries
    assert _gpu_decimal(small_transform_ctx, nines) == b"9" * (9 * nl)


def test_catalan_tree_by_pieces(orc, small_transform_ctx):
    # a product tree whose upper levels exceed 2^13 points
    n = 200000
    r = capi.to_numpy(capi.catalan_exact(small_transform_ctx, n))
    assert (r == orc.catalan(n)).all()


@pytest.mark.slow
def test_paper_scale_decimal(ctx):
    # Table 1: C(2,050,572,903) has 1,234,567,890 digits.  Leading digits from
    # the closed form log10 C = (ln (2n)! - ln n! - ln (n+1)!) / ln 10 by
    # Stirling's series in 40-digit decimal arithmetic; trailing digits from
    # the binary limbs mod 10^18.
    import decimal
    import torch
    n = 2050572903
    r = capi.catalan_exact(ctx, n)
    d = capi.to_decimal(ctx, r)
    assert d.numel() == 1234567890
    head = bytes(d[:12].cpu().numpy())
    tail = bytes(d[-18:].cpu().numpy())
    decimal.getcontext().prec = 40
    D = decimal.Decimal

    pi_digits = D("3.141592653589793238462643383279502884197")

    def ln_fact40(m):  # ln m! = ln Gamma(m + 1) by Stirling's series (m > 10^9)
        x = D(m) + 1
        return ((x - D("0.5")) * x.ln() - x + (2 * pi_digits).ln() / 2
                + 1 / (12 * x) - 1 / (360 * x ** 3) + 1 / (1260 * x ** 5))

    l10 = (ln_fact40(2 * n) - ln_fact40(n) - ln_fact40(n + 1)) / D(10).ln()
    frac = l10 - int(l10)
    lead = int(D(10) ** (frac + 11))
    assert int(l10) + 1 == 1234567890
    assert head == str(lead).encode()
    h = capi.to_numpy(r)
    x = int.from_bytes(h.astype("<u4").tobytes(), "little")
    assert tail == str(x % 10**18).zfill(18).encode()
    # every digit: the decimal string mod four seeded 31-bit primes (plain
    # torch integer arithmetic, independent of the conversion) against the
    # oracle's residues of the binary limbs
    for q in orc_check_primes(4):
        assert _decimal_mod(d, q) == _orc().limbs_mod(h, q), q
    del d, r
    torch.cuda.empty_cache()


def _orc():
    import oracle
    oracle.build()
    return oracle


def orc_check_primes(count):
    return _orc().check_primes(seed=1234567890, count=count, lower=1 << 30, bits=31)


def _decimal_mod(d, q: int) -> int:
    """The value of the ASCII digit string d (a device tensor, most
    significant digit first) mod q < 2^31: nine-digit chunks c_i (leading
    zeros prepended so that the count divides by nine), then
    sum_i c_i B^(m-1-i) mod q with B = 10^9, the powers B^j mod q built by
    doubling (B^(j+k) = B^j B^k).  Every product is below 2^61 in int64."""
    import torch
    dev = d.device
    nd = d.numel()
    pad = (-nd) % 9
    digits = torch.cat([torch.full((pad,), 48, dtype=torch.uint8, device=dev), d.view(-1)])
    p10 = torch.tensor([10 ** (8 - k) for k in range(9)], dtype=torch.int64, device=dev)
    m = digits.numel() // 9
    chunks = torch.zeros(m, dtype=torch.int64, device=dev)
    step = 1 << 24
    for i in range(0, m, step):
        part = digits[9 * i: 9 * min(m, i + step)].view(-1, 9).to(torch.int64) - 48
        chunks[i: i + part.shape[0]] = (part * p10).sum(dim=1)
    pw = torch.ones(1, dtype=torch.int64, device=dev)  # B^0
    bk = 10 ** 9 % q                                    # B^k for k = len(pw)
    while pw.numel() < m:
        pw = torch.cat([pw, (pw * bk) % q])
        bk = bk * bk % q
    pw = pw[:m].flip(0)                                 # chunk i weighs B^(m-1-i)
    acc = 0
    for i in range(0, m, step):
        acc += int((((chunks[i: i + step] % q) * pw[i: i + step]) % q).sum().item())
    return acc % q
