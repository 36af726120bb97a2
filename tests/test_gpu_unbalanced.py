"""Unbalanced products (a long operand times a short one) through bigint_mul:
chunks of the long operand against the short one, overlap-added."""
import numpy as np
import pytest

from paper_2601_11621_gb300 import capi, workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("na,nb", [(5000, 2000), (100000, 1), (100000, 3), (200000, 3000),
                                   ((1 << 20) + 7, 4099), (300001, 70000), (9000, 4097)])
def test_unbalanced_vs_oracle(orc, ctx, na, nb):
    a = workloads.random_limbs32(na, seed=na % 1000 + 1)
    b = workloads.random_limbs32(nb, seed=nb % 1000 + 2)
    r = capi.to_numpy(capi.bigint_mul(ctx, a, b))
    assert (r == orc.mul(a, b)).all()
    r2 = capi.to_numpy(capi.bigint_mul(ctx, b, a))  # operand order does not matter
    assert (r2 == r).all()


def test_unbalanced_carry_chains(orc, ctx):
    # (2^(32 k) - 1)(2^(32 m) - 1): every chunk product's overlap carries
    for k, m in [(50000, 300), (120000, 4096), (70001, 1)]:
        x, y = 2 ** (32 * k) - 1, 2 ** (32 * m) - 1
        r = capi.to_numpy(capi.bigint_mul(ctx, orc.int_to_limbs(x), orc.int_to_limbs(y)))
        assert orc.limbs_to_int(r) == x * y


def test_unbalanced_takes_the_chunk_path(orc, ctx):
    a = workloads.random_limbs32(1 << 20, seed=5)
    b = workloads.random_limbs32(1000, seed=6)
    ctx.set_profiling(True)
    try:
        r = capi.to_numpy(capi.bigint_mul(ctx, a, b))
        prof = ctx.profile()
    finally:
        ctx.set_profiling(False)
    assert prof.get("overlap_tiles", (0,))[0] >= 1
    assert (r == orc.mul(a, b)).all()
