"""The autotuner (cat_autotune): every multi-pass plan it may choose gives
exact products (against the CPU oracle, or, at sizes where the oracle would
take minutes, against the default plan's product and residues modulo two
primes from the oracle), its table round-trips through a file, a context that
loads it computes C(10^6) exactly, and a table made on another kind of device
is refused."""
import hashlib
import os

import numpy as np
import pytest

from paper_2601_11621_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def plan_ok(n, r):
    # the rule of the library's plan_row_ok: rows of 2^9 .. 2^12 points, at
    # most two column passes of at least 2 rows each (2^4 rows for n > 23)
    if n > 27 or r < 9 or r > 12:
        return False
    rem = n - r
    ncol = (rem + 9) // 10
    return rem >= 2 and ncol <= 2 and rem // ncol >= (2 if n <= 23 else 4)


def device_tag():
    import torch
    p = torch.cuda.get_device_properties(0)
    return f"{p.name.replace(' ', '_')} {p.multi_processor_count}"


def write_table(path, slot, rows):
    with open(path, "w") as f:
        f.write(f"device {device_tag()}\ncomba_max_slot {slot}\n")
        for n, r in rows.items():
            f.write(f"row_log {n} {r}\n")


def golden_sha(kind, n):
    for line in open(os.path.join(GOLDEN, "oracle_results.txt")):
        parts = line.split()
        if len(parts) == 5 and parts[0] == kind and parts[1] == str(n):
            return parts[4]


@pytest.mark.parametrize("n", list(range(13, 28)))
def test_every_tunable_plan_is_exact(cat_lib, orc, ctx, n, tmp_path):
    a = W.random_limbs32(1 << (n - 1), seed=n)
    b = W.random_limbs32((1 << (n - 1)) - 3, seed=n + 100)
    ref = host(cat_lib.bigint_mul(ctx, a, b))            # default plan
    if n <= 17:
        assert np.array_equal(ref, orc.mul(a, b))
    qs = orc.check_primes(seed=n, count=2, lower=1 << 40, bits=62)
    for r in range(9, 13):
        if not plan_ok(n, r):
            continue
        path = str(tmp_path / f"t{n}_{r}.txt")
        write_table(path, 128, {n: r})
        c = cat_lib.Context(0)
        try:
            c.load_tuning(path)
            assert c.tuning()[1] == {n: r}
            got = host(cat_lib.bigint_mul(c, a, b))
        finally:
            c.close()
        assert np.array_equal(got, ref), (n, r)
    for q in qs:
        assert orc.limbs_mod(ref, q) == orc.limbs_mod(a, q) * orc.limbs_mod(b, q) % q


def test_autotune_round_trip_and_exact_catalan(cat_lib, tmp_path):
    path = str(tmp_path / "autotune.txt")
    c = cat_lib.Context(0)
    try:
        c.autotune(path)
        slot, rows = c.tuning()
    finally:
        c.close()
    assert slot in (16, 32, 64, 128, 256)
    assert set(rows) == set(range(13, 28)) and all(plan_ok(n, r) for n, r in rows.items())
    assert open(path).read().count("row_log") == 15
    c = cat_lib.Context(0)
    try:
        c.load_tuning(path)
        assert c.tuning() == (slot, rows)
        got = host(cat_lib.catalan_exact(c, 10**6))
    finally:
        c.close()
    assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == golden_sha("catalan", 10**6)


def test_tuned_crossover_and_plans_in_the_tree(cat_lib, orc, tmp_path):
    # the extreme choices at once: schoolbook up to 256-limb slots, the
    # smallest row passes; a product tree and C(n) still come out exact
    path = str(tmp_path / "t.txt")
    write_table(path, 256, {n: 9 for n in range(13, 28)})
    c = cat_lib.Context(0)
    try:
        c.load_tuning(path)
        v = W.random_values(70_001, seed=9)
        assert np.array_equal(host(cat_lib.product_tree(c, v)), orc.product_tree(v))
        got = host(cat_lib.catalan_exact(c, 10**6))
    finally:
        c.close()
    assert hashlib.sha256(got.astype("<u4").tobytes()).hexdigest() == golden_sha("catalan", 10**6)


def test_table_from_another_device_is_refused(cat_lib, tmp_path):
    path = str(tmp_path / "other.txt")
    with open(path, "w") as f:
        f.write("device Some_Other_GPU 7\ncomba_max_slot 64\nrow_log 20 10\n")
    c = cat_lib.Context(0)
    try:
        before = c.tuning()
        with pytest.raises(cat_lib.CatError) as e:
            c.load_tuning(path)
        assert e.value.code == cat_lib.CAT_EINVAL
        assert c.tuning() == before
    finally:
        c.close()


@pytest.mark.slow
def test_paper_scale_with_tuned_plans(cat_lib, tmp_path):
    """C(2,050,572,903) with the plans the autotuner picks on this device (the
    configuration bench.py times) against Table 1's SHA-256."""
    t = {}
    for line in open(os.path.join(GOLDEN, "paper_table1.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split(None, 1)
            t[k] = v.strip()
    path = str(tmp_path / "autotune.txt")
    c = cat_lib.Context(0)
    try:
        c.autotune(path)
        got = host(cat_lib.catalan_exact(c, int(t["n"])))
    finally:
        c.close()
    bits = (len(got) - 1) * 32 + int(got[-1]).bit_length()
    assert bits == int(t["bit_length"])
    body = got.astype("<u4").tobytes()[:(bits + 7) // 8]
    sha = hashlib.sha256(bytes.fromhex(t["sha256_header_hex"]) + body).hexdigest()
    assert sha == t["sha256"]
