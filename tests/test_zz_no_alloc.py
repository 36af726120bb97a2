"""bigint_mul_noalloc: the multiplication entry point that allocates no
device memory (for callers that cannot call cudaMalloc; its scratch is a
fixed __device__ array inside the library).

Checked through the C ABI against the context-based bigint_mul, bit-exact,
on two calls in a row (the second call reuses the scratch the first left
behind).  Collected last so that a failure here comes after every other
test has run."""
import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


# sizes on both sides of the one-block limit (4096 limbs) and at the maximum
SIZES = [(1, 1), (37, 1000), (2048, 2048), (2049, 2048), (20000, 13000),
         (1 << 15, 1 << 15)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_noalloc_matches_bigint_mul_twice(cat_lib, ctx, na, nb):
    import torch
    for call, seed in enumerate((na * 3 + 1, nb * 5 + 2)):
        a = torch.from_numpy(W.random_limbs32(na, seed).view(np.int32)).cuda()
        b = torch.from_numpy(W.random_limbs32(nb, seed + 7).view(np.int32)).cuda()
        want = host(cat_lib.bigint_mul(ctx, a, b))
        got = host(cat_lib.bigint_mul_noalloc(a, b))
        assert got.shape == want.shape, (call, got.shape, want.shape)
        assert np.array_equal(got, want), call


def test_noalloc_all_ones_twice(cat_lib, ctx):
    import torch
    for n in (40000, 30000):
        a = torch.full((n,), -1, dtype=torch.int32, device="cuda")  # 0xFFFFFFFF limbs
        want = host(cat_lib.bigint_mul(ctx, a, a[: n // 2]))
        got = host(cat_lib.bigint_mul_noalloc(a, a[: n // 2]))
        assert np.array_equal(got, want)


def test_noalloc_rejects_too_large(cat_lib):
    import torch
    n = cat_lib.NOALLOC_MAX_LIMBS // 2 + 1
    a = torch.ones(n, dtype=torch.int32, device="cuda")
    with pytest.raises(cat_lib.CatError) as e:
        cat_lib.bigint_mul_noalloc(a, a)
    assert e.value.code == -2  # CAT_ENOMEM: beyond the static scratch
