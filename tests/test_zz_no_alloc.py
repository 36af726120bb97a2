"""bigint_mul_noalloc: the multiplication entry point that allocates no
device memory, for callers that cannot call cudaMalloc (an application whose
own allocator holds the device's memory, or code that must not take
cudaMalloc's device-wide synchronisation).  Its scratch is a fixed __device__
array inside the library.

Checked through the C ABI against the CPU oracle's product, limb for limb, on
two calls in a row with different operands (the second call reuses the
scratch the first left behind); one case on a non-default stream; and the
device's free memory and torch's allocation are unchanged across a call.
Collected last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32).view(np.int32)).cuda()


# sizes on both sides of the one-block limit (4096 limbs) and at the maximum
SIZES = [(1, 1), (37, 1000), (2048, 2048), (2049, 2048), (20000, 13000),
         (1 << 15, 1 << 15)]


@pytest.mark.parametrize("na,nb", SIZES)
def test_noalloc_matches_oracle_twice(cat_lib, orc, na, nb):
    for call, seed in enumerate((na * 3 + 1, nb * 5 + 2)):
        a = W.random_limbs32(na, seed)
        b = W.random_limbs32(nb, seed + 7)
        got = host(cat_lib.bigint_mul_noalloc(dev(a), dev(b)))
        want = orc.mul(a, b)
        assert got.shape == want.shape, (call, got.shape, want.shape)
        assert np.array_equal(got, want), call


def test_noalloc_all_ones_twice(cat_lib, orc):
    # (2^(32 n) - 1)(2^(16 n) - 1): carries through every limb
    for n in (40000, 30000):
        a = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
        got = host(cat_lib.bigint_mul_noalloc(dev(a), dev(a[: n // 2])))
        assert np.array_equal(got, orc.mul(a, a[: n // 2]))


def test_noalloc_on_a_side_stream(cat_lib, orc):
    import torch
    a = W.random_limbs32(30001, 11)
    b = W.random_limbs32(25000, 12)
    ta, tb = dev(a), dev(b)
    out = torch.empty(a.size + b.size, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        r = cat_lib.bigint_mul_noalloc(ta, tb, out=out, stream=s)
    s.synchronize()
    assert np.array_equal(host(r), orc.mul(a, b))


def test_noalloc_allocates_nothing(cat_lib, orc):
    import torch
    a = W.random_limbs32(40000, 21)
    b = W.random_limbs32(20000, 22)
    ta, tb = dev(a), dev(b)
    out = torch.empty(a.size + b.size, dtype=torch.int32, device="cuda")
    cat_lib.bigint_mul_noalloc(ta, tb, out=out)  # warm: per-device set-up done
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    r = cat_lib.bigint_mul_noalloc(ta, tb, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(host(r), orc.mul(a, b))


def test_noalloc_rejects_too_large(cat_lib):
    import torch
    n = cat_lib.NOALLOC_MAX_LIMBS // 2 + 1
    a = torch.ones(n, dtype=torch.int32, device="cuda")
    with pytest.raises(cat_lib.CatError) as e:
        cat_lib.bigint_mul_noalloc(a, a)
    assert e.value.code == -2  # CAT_ENOMEM: beyond the static scratch
