"""GPU parity of the batched solver (cat_exact_batch): every request of a
batch, bit-exact against the CPU oracle, and the same whether computed alone
or in the mix."""
import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def split(out, offs, lens):
    h = host(out)
    return [h[int(o):int(o) + int(n)] for o, n in zip(offs, lens)]


MIXED = [(0, 0), (0, 1), (1, 0), (2, 0), (2, 1), (2, 2), (0, 2), (0, 5), (1, 7), (2, 10),
         (0, 100), (1, 1000), (2, 500), (0, 54321), (1, 12345), (2, 3000), (0, 262144),
         (0, 262145), (1, 99991)]


def test_mixed_batch_vs_oracle(ctx, cat_lib, orc):
    out, offs, lens = cat_lib.cat_exact_batch(ctx, MIXED)
    for (kind, n), got in zip(MIXED, split(out, offs, lens)):
        want = orc.exact(kind, n)
        assert got.shape == want.shape and (got == want).all(), (kind, n)


def test_single_request_batches(ctx, cat_lib, orc):
    for kind, n in [(0, 0), (1, 1), (2, 3), (0, 70000)]:
        out, offs, lens = cat_lib.cat_exact_batch(ctx, [(kind, n)])
        got = split(out, offs, lens)[0]
        assert (got == orc.exact(kind, n)).all()


def test_batch_errors(ctx, cat_lib):
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_exact_batch(ctx, [(0, 1 << 31)])
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_exact_batch(ctx, [(5, 10)])
    import torch
    small = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(cat_lib.CatError) as e:
        cat_lib.cat_exact_batch(ctx, [(0, 1000)], out=small)
    assert e.value.code == -3


def test_config3_batch(ctx, cat_lib, orc):
    """4,096 requests, half Catalan, half central binomial, n log-uniform in
    [1e3, 1e6]: every result checked modulo a seeded 62-bit prime against the
    oracle's factorial-product residue; a sample against the full oracle;
    a sample against the same request computed alone."""
    reqs = W.batched_requests(4096, seed=0)
    out, offs, lens = cat_lib.cat_exact_batch(ctx, reqs)
    res = split(out, offs, lens)
    q = orc.check_primes(seed=3, count=1, lower=2 * 10**6, bits=62)[0]
    for (kind, n), got in zip(reqs, res):
        assert orc.limbs_mod(got, q) == orc.exact_mod(kind, n, q), (kind, n)
    rng = np.random.default_rng(1)
    for i in rng.choice(len(reqs), size=24, replace=False):
        kind, n = reqs[i]
        assert (res[i] == orc.exact(kind, n)).all(), (kind, n)
    for i in rng.choice(len(reqs), size=64, replace=False):
        kind, n = reqs[i]
        alone = host(cat_lib.cat_exact(ctx, kind, n))
        assert alone.shape == res[i].shape and (alone == res[i]).all(), (kind, n)


@pytest.fixture(scope="module")
def small_transform_ctx(cat_lib):
    """A context whose single-transform limit is 2^13 points: tree nodes
    above 4,096 limbs are multiplied by pieces."""
    import os
    old = os.environ.get("CAT_MAX_TRANSFORM_LOG")
    os.environ["CAT_MAX_TRANSFORM_LOG"] = "13"
    try:
        c = cat_lib.Context(0)
    finally:
        if old is None:
            del os.environ["CAT_MAX_TRANSFORM_LOG"]
        else:
            os.environ["CAT_MAX_TRANSFORM_LOG"] = old
    yield c
    c.close()


def test_batch_with_products_by_pieces(small_transform_ctx, cat_lib, orc):
    """The batched tree's top levels through the piece path (each product
    placed by the host copy of its level's index table), beside small
    requests that finish early; 40000! goes through the bit-decomposed
    reconstruction, whose segmented tree takes the same path."""
    reqs = [(0, 262144), (1, 5), (2, 40000), (0, 3), (1, 99991), (0, 0)]
    out, offs, lens = cat_lib.cat_exact_batch(small_transform_ctx, reqs)
    for (kind, n), got in zip(reqs, split(out, offs, lens)):
        want = orc.exact(kind, n)
        assert got.shape == want.shape and (got == want).all(), (kind, n)
