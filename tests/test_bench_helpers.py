"""bench.py's host-side helpers on the CPU: the modular checks it applies
before printing the mul sweep and batched numbers (against CPython integers
and math.comb), and the CPU-baseline growth fit and extrapolation (against
exact power laws)."""
import json
import math
import random
import subprocess
import sys

import numpy as np
import pytest

import bench


def test_limbs_mod_matches_python_ints():
    import torch
    rng = random.Random(5)
    for nl in (1, 2, 3, 31, 32, 33, 1000, 4099):
        limbs = np.array([rng.getrandbits(32) for _ in range(nl)], dtype=np.uint32)
        x = int.from_bytes(limbs.astype("<u4").tobytes(), "little")
        t = torch.from_numpy(limbs.view(np.int32))
        for q in bench.CHECK_PRIMES + (1000003,):
            assert bench.limbs_mod_dev(t, q) == x % q, (nl, q)


def test_binomial_mod_matches_math_comb():
    for n in (1, 2, 3, 10, 99, 1000, 4321):
        for q in bench.CHECK_PRIMES:
            assert bench.binomial_mod(0, n, q) == (math.comb(2 * n, n) // (n + 1)) % q
            assert bench.binomial_mod(1, n, q) == math.comb(2 * n, n) % q
    assert bench.range_prod_mod(5, 4, 7) == 1


def test_fit_and_extrapolation_recover_a_power_law():
    class FakeOracle:
        CATALAN = 0

        @staticmethod
        def bound_limbs(kind, n):
            return n // 10

    alpha = 1.57
    pts = [(m // 10, 0.001 * m / 1e6, 0.001 * m / 1e6 + 2e-9 * (m // 10) ** alpha)
           for m in (10**6, 10**7, 5 * 10**7)]
    assert bench._fit_exponent(pts) == pytest.approx(alpha, rel=1e-9)
    v = bench._extrapolate(FakeOracle, pts[-1], alpha, 5 * 10**7, 2 * 10**9)
    want = 0.001 * 2000 + 2e-9 * (2 * 10**8) ** alpha
    assert v == pytest.approx(want, rel=1e-9)


def test_reference_arm_prints_one_line(monkeypatch, capsys):
    # small sizes in place of 10^6 / 10^7 so that the arm runs in seconds
    monkeypatch.setattr(bench, "FIT_NS", (2000, 20000, 50000))
    monkeypatch.setattr(bench, "ST_NS", (2000, 20000))

    class Args:
        n, steps, warmup, gpus = 10**6, 2, 2, 1

    bench.run_reference(Args(), rank=0, world=1)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "s"
    assert line["value"] > 0 and line["higher_is_better"] is False
    assert line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0
