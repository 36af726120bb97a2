"""GPU parity: multiplication, powering and the product tree through the C ABI,
limb for limb against the CPU oracle (and CPython integers for the large
operands the oracle would take long on).  Integer work: bit-exact."""
import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def as_int(limbs):
    return int.from_bytes(np.asarray(limbs, dtype="<u4").tobytes(), "little")


def ones(n):
    return np.full(n, 0xFFFFFFFF, dtype=np.uint32)


MUL_SIZES = [
    (1, 1), (1, 7), (2, 2), (3, 5), (31, 33), (100, 100), (1000, 24),
    (2047, 2049),          # one-block transform, L = 4096 exactly
    (2048, 2049),          # first multi-pass size, L = 8192
    (4096, 4096), (5000, 3), (3, 20000), (12345, 54321),
    (1 << 16, 1 << 16),    # L = 2^17 (two passes)
    (1 << 18, 1 << 14),    # unequal lengths
    (1 << 21, 1 << 21),    # L = 2^22
]


@pytest.mark.parametrize("na,nb", MUL_SIZES)
def test_mul_random(ctx, cat_lib, orc, na, nb):
    a = W.random_limbs32(na, seed=na * 7 + 1)
    b = W.random_limbs32(nb, seed=nb * 13 + 2)
    got = host(cat_lib.bigint_mul(ctx, a, b))
    if na + nb <= 1 << 16:
        want = orc.mul(a, b)
        assert got.shape == want.shape and (got == want).all()
    else:
        assert as_int(got) == as_int(a) * as_int(b)


@pytest.mark.parametrize("na,nb", [(1, 1), (7, 9), (2048, 2048), (2049, 2047),
                                   (40000, 40000), (1 << 20, 1 << 20), (1 << 22, 3)])
def test_mul_all_ones_carry_chains(ctx, cat_lib, na, nb):
    # (2^32a - 1)(2^32b - 1): maximal coefficients and long carry chains
    a, b = ones(na), ones(nb)
    got = host(cat_lib.bigint_mul(ctx, a, b))
    assert as_int(got) == as_int(a) * as_int(b)


def test_mul_carry_through_whole_tiles(ctx, cat_lib):
    # a = 2^(32k) - 1, b = 2^(32k) + 1: product 2^(64k) - 1 is all ones
    for k in (1000, 4096, 50000, 300000):
        a = ones(k)
        b = np.zeros(k + 1, dtype=np.uint32)
        b[0] = 1
        b[k] = 1
        got = host(cat_lib.bigint_mul(ctx, a, b))
        assert got.shape == (2 * k,) and (got == 0xFFFFFFFF).all()


def test_mul_edge_cases(ctx, cat_lib):
    z = np.zeros(0, dtype=np.uint32)
    assert host(cat_lib.bigint_mul(ctx, z, np.array([5], np.uint32))).size == 0
    assert host(cat_lib.bigint_mul(ctx, np.array([0, 0], np.uint32),
                                   np.array([5], np.uint32))).size == 0
    got = host(cat_lib.bigint_mul(ctx, np.array([3, 0, 0], np.uint32),
                                  np.array([5, 0], np.uint32)))
    assert got.tolist() == [15]


@pytest.mark.parametrize("na,nb", [(3000, 2000), (40000, 30000)])
def test_mul_output_overlapping_an_operand(ctx, cat_lib, orc, na, nb):
    """The C ABI's out may overlap an operand (here out starts at a): the
    product then goes through scratch; a disjoint out takes it directly."""
    import ctypes
    import torch
    a = W.random_limbs32(na, seed=na + 11)
    b = W.random_limbs32(nb, seed=nb + 12)
    want = orc.mul(a, b)
    buf = torch.zeros(na + nb, dtype=torch.int32, device="cuda")
    buf[:na] = torch.from_numpy(a.view(np.int32)).cuda()
    tb = torch.from_numpy(b.view(np.int32)).cuda()
    n = ctypes.c_size_t()
    rc = cat_lib.load().bigint_mul(ctx.handle, cat_lib._ptr(buf), na, cat_lib._ptr(tb), nb,
                                   cat_lib._ptr(buf), na + nb, ctypes.byref(n),
                                   cat_lib._stream(None))
    assert rc == 0
    assert n.value == want.size and (host(buf[:n.value]) == want).all()
    out = torch.zeros(na + nb, dtype=torch.int32, device="cuda")
    ta = torch.from_numpy(a.view(np.int32)).cuda()
    rc = cat_lib.load().bigint_mul(ctx.handle, cat_lib._ptr(tb), nb, cat_lib._ptr(ta), na,
                                   cat_lib._ptr(out), na + nb, ctypes.byref(n),
                                   cat_lib._stream(None))
    assert rc == 0
    assert n.value == want.size and (host(out[:n.value]) == want).all()


@pytest.mark.parametrize("n", [1, 5, 2048, 2049, 70000, 1 << 20])
def test_square(ctx, cat_lib, n):
    import torch
    a = torch.from_numpy(W.random_limbs32(n, seed=n).view(np.int32)).cuda()
    got = host(cat_lib.bigint_mul(ctx, a, a))  # same pointer: the squaring path
    x = as_int(host(a))
    assert as_int(got) == x * x


@pytest.mark.parametrize("nl,e", [(1, 0), (1, 1), (1, 2), (3, 17), (40, 13), (1, 1000),
                                  (1, 100000), (500, 9)])
def test_pow(ctx, cat_lib, orc, nl, e):
    a = W.random_limbs32(nl, seed=nl + e)
    got = host(cat_lib.bigint_pow(ctx, a, e))
    want = orc.power(a, e)
    assert got.shape == want.shape and (got == want).all()


@pytest.mark.parametrize("count", [0, 1, 2, 7, 8, 9, 17, 100, 1000, 4097, 100003])
def test_product_tree_random(ctx, cat_lib, orc, count):
    v = W.random_values(count, seed=count)
    got = host(cat_lib.product_tree(ctx, v))
    want = orc.product_tree(v)
    assert got.shape == want.shape and (got == want).all()


def test_product_tree_max_values_all_levels(ctx, cat_lib, orc):
    # 2^17 + 5 values of 0xFFFFFFFF: every level (leaves, schoolbook, one-block
    # and multi-pass transforms) sees maximal limbs and an odd tail
    count = (1 << 17) + 5
    v = np.full(count, 0xFFFFFFFF, dtype=np.uint32)
    got = host(cat_lib.product_tree(ctx, v))
    assert as_int(got) == (2**32 - 1) ** count


def test_product_tree_primes(ctx, cat_lib, orc):
    pr = orc.sieve(3_000_000)
    got = host(cat_lib.product_tree(ctx, pr))
    want = orc.product_tree(pr)
    assert (got == want).all()


@pytest.fixture(scope="module")
def computed_twiddle_ctx(cat_lib):
    """A context whose column passes compute their inter-pass twiddles (no
    tables), as budgeted contexts and the no-allocation multiply do."""
    import os
    old = os.environ.get("CAT_COL_TWIDDLE_TABLES")
    os.environ["CAT_COL_TWIDDLE_TABLES"] = "0"
    try:
        c = cat_lib.Context(0)
    finally:
        if old is None:
            del os.environ["CAT_COL_TWIDDLE_TABLES"]
        else:
            os.environ["CAT_COL_TWIDDLE_TABLES"] = old
    yield c
    c.close()


@pytest.mark.parametrize("na,nb", [(5000, 4000), (40000, 30000), (1 << 20, 1 << 20),
                                   (1 << 24, 1 << 22), (3 << 23, 1 << 25), (1 << 26, 3 << 24)])
def test_twiddle_tables_match_computed_twiddles(ctx, computed_twiddle_ctx, cat_lib, orc, na, nb):
    """Column passes with twiddle tables (the default) and with computed
    twiddles give the same limbs, across the prime sets (products of 2^14 to
    2^27 points); the smaller sizes also against the oracle."""
    a = W.random_limbs32(na, seed=na + 3)
    b = W.random_limbs32(nb, seed=nb + 4)
    got = host(cat_lib.bigint_mul(ctx, a, b))
    ref = host(cat_lib.bigint_mul(computed_twiddle_ctx, a, b))
    assert got.shape == ref.shape and (got == ref).all()
    if na + nb <= 70000:
        assert (got == orc.mul(a, b)).all()


@pytest.mark.parametrize("na,nb", [(5001, 4000), (40000, 30001)])
def test_mul_unaligned_operands(ctx, cat_lib, orc, na, nb):
    """Operands starting one limb into a buffer (4-byte but not 8-byte
    aligned) are read word by word; aligned ones two words at a time: both
    give the oracle's product."""
    import torch
    a = W.random_limbs32(na, seed=na + 21)
    b = W.random_limbs32(nb, seed=nb + 22)
    want = orc.mul(a, b)
    ba = torch.zeros(na + 1, dtype=torch.int32, device="cuda")
    bb = torch.zeros(nb + 1, dtype=torch.int32, device="cuda")
    ba[1:] = torch.from_numpy(a.view(np.int32)).cuda()
    bb[1:] = torch.from_numpy(b.view(np.int32)).cuda()
    got = host(cat_lib.bigint_mul(ctx, ba[1:], bb[1:]))
    assert got.shape == want.shape and (got == want).all()
    got = host(cat_lib.bigint_mul(ctx, ba[1:], torch.from_numpy(b.view(np.int32)).cuda()))
    assert got.shape == want.shape and (got == want).all()


def test_launch_count_grows_with_work(ctx, cat_lib):
    """cat_launch_count counts the library's kernel launches: a multi-pass
    product launches several kernels, a call that fails its argument check
    launches none."""
    a = W.random_limbs32(20000, seed=31)
    n0 = cat_lib.cat_launch_count()
    cat_lib.bigint_mul(ctx, a, a)
    n1 = cat_lib.cat_launch_count()
    assert n1 - n0 >= 5
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_exact_batch(ctx, [(5, 10)])  # unknown kind
    assert cat_lib.cat_launch_count() == n1
