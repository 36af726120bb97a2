"""The run's files (Sec. 3.1 factorisation text, Algorithm 2's binary result
file) through the C ABI on the GPU, against the oracle's grouping and limbs."""
import hashlib
import os

import numpy as np
import pytest

from paper_2601_11621_gb300 import capi

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _expected_text(orc, name, primes, e):
    exps, offs, gp = orc.group(primes, e)
    lines = [f"# Prime factorization of {name}"]
    for g in range(len(exps)):
        grp = gp[int(offs[g]):int(offs[g + 1])]
        lines.append(f"# exponent={int(exps[g])} count={len(grp)}")
        lines.append(" ".join(str(int(p)) for p in grp))
    return ("\n".join(lines) + "\n").encode()


@pytest.mark.parametrize("kind,n,name", [(0, 10**5, "Catalan(100000)"),
                                         (1, 3 * 10**4, "CentralBinomial(30000)"),
                                         (2, 20000, "Factorial(20000)"),
                                         (0, 1, "Catalan(1)")])
def test_factor_text_vs_oracle(orc, ctx, kind, n, name):
    f = capi.catalan_factor(ctx, n, kind)
    try:
        got = bytes(capi.cat_factor_text(ctx, f, name).cpu().numpy())
    finally:
        f.free()
    limit = n if kind == orc.FACTORIAL else 2 * n
    primes = orc.sieve(limit) if limit >= 2 else np.zeros(0, np.uint32)
    e = orc.exponents(kind, n, primes)
    assert got == _expected_text(orc, name, primes, e)


def test_ratio_factor_text(orc, ctx):
    a, b = [10**5], [4 * 10**4, 6 * 10**4]
    f = capi.cat_ratio_factor(ctx, a, b)
    try:
        got = bytes(capi.cat_factor_text(ctx, f, "C(100000,40000)").cpu().numpy())
    finally:
        f.free()
    primes = orc.sieve(10**5)
    assert got == _expected_text(orc, "C(100000,40000)", primes,
                                 orc.ratio_exponents(a, b, primes))


@pytest.mark.parametrize("v", [0, 1, 255, 256, 2**32 - 1, 2**32, 10**100])
def test_binary_small(orc, ctx, v):
    got = bytes(capi.cat_binary(ctx, orc.int_to_limbs(v)).cpu().numpy())
    assert got == b"\x01\x01" + v.to_bytes((v.bit_length() + 7) // 8, "little")


def test_binary_of_catalan(orc, ctx):
    n = 10**5
    got = bytes(capi.cat_binary(ctx, capi.catalan_exact(ctx, n)).cpu().numpy())
    c = orc.limbs_to_int(orc.catalan(n))
    assert got == b"\x01\x01" + c.to_bytes((c.bit_length() + 7) // 8, "little")


@pytest.mark.slow
def test_paper_scale_binary_sha256(ctx):
    # Table 1's SHA-256 of the result file, from the file bytes cat_binary writes
    fields = {}
    for line in open(os.path.join(GOLDEN, "paper_table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(None, 1)
            fields[k] = v.strip()
    r = capi.catalan_exact(ctx, int(fields["n"]))
    data = capi.cat_binary(ctx, r).cpu().numpy()
    assert len(data) == int(fields["result_file_bytes"]) + 2
    assert hashlib.sha256(data.tobytes()).hexdigest() == fields["sha256"]
