"""CPU oracle for the exact Catalan / central-binomial / factorial path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It wraps the plain C
implementation in ``oracle.c`` (compiled with gcc into ``liboracle.so`` next
to it) and shares nothing with the CUDA library.

Big integers are little-endian ``uint32`` limb arrays (numpy), normalised so
that the top limb is non-zero; zero is the empty array.

Paper citations (arXiv 2601.11621):
  * Legendre's formula and the Catalan valuation: Sec. 2.
  * Sieve, n+1 trial division, exponent loop, grouping, digit estimate:
    Sec. 3.1, Algorithm 1.
  * Q_e = BalancedProductTree(G_e), P_e = Q_e^e, final product: Sec. 3.2,
    Algorithm 2.
  * Factorial-ratio exponents: Sec. 6.3.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

CATALAN, CENTRAL_BINOMIAL, FACTORIAL = 0, 1, 2
_U64_MAX = (1 << 64) - 1


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` with gcc (plain -O2; with
    OpenMP when the compiler has it, which only ``exact_mt`` uses)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC]
    try:
        subprocess.check_call(base + ["-fopenmp", "-lm"], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + ["-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u64, u32p, u64p, i64p = (ctypes.c_uint64, ctypes.POINTER(ctypes.c_uint32),
                                 ctypes.POINTER(ctypes.c_uint64),
                                 ctypes.POINTER(ctypes.c_int64))
        L.orc_sieve.argtypes = [u64, u32p, u64]
        L.orc_sieve.restype = u64
        L.orc_sieve_range.argtypes = [u64, u64, u32p, u64]
        L.orc_sieve_range.restype = u64
        L.orc_legendre.argtypes = [u64, u64]
        L.orc_legendre.restype = u64
        L.orc_factor_trial.argtypes = [u64, u32p, u64, u64p, u64p, ctypes.c_int]
        L.orc_factor_trial.restype = ctypes.c_int
        L.orc_prime_limit.argtypes = [ctypes.c_int, u64]
        L.orc_prime_limit.restype = u64
        L.orc_exponents.argtypes = [ctypes.c_int, u64, u32p, u64, i64p]
        L.orc_exponents.restype = ctypes.c_int
        L.orc_ratio_exponents.argtypes = [u64p, ctypes.c_int, u64p, ctypes.c_int,
                                          u32p, u64, i64p]
        L.orc_ratio_exponents.restype = None
        L.orc_group.argtypes = [u32p, i64p, u64, u64p, u64p, u32p]
        L.orc_group.restype = u64
        L.orc_log10_estimate.argtypes = [u32p, i64p, u64]
        L.orc_log10_estimate.restype = ctypes.c_longdouble
        L.orc_mul.argtypes = [u32p, u64, u32p, u64, u32p]
        L.orc_mul.restype = u64
        L.orc_product_tree.argtypes = [u32p, u64, u32p, u64]
        L.orc_product_tree.restype = u64
        L.orc_pow.argtypes = [u32p, u64, u64, u32p, u64]
        L.orc_pow.restype = u64
        L.orc_reconstruct.argtypes = [u64, u64p, u64p, u32p, u32p, u64]
        L.orc_reconstruct.restype = u64
        L.orc_exact.argtypes = [ctypes.c_int, u64, u32p, u64]
        L.orc_exact.restype = u64
        L.orc_exact_mt.argtypes = [ctypes.c_int, u64, u32p, u64, ctypes.c_int]
        L.orc_exact_mt.restype = u64
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_mulmod_plain.argtypes = [u64, u64, u64]
        L.orc_mulmod_plain.restype = u64
        L.orc_mulmod_mont.argtypes = [u64, u64, u64]
        L.orc_mulmod_mont.restype = u64
        L.orc_range_product_mod.argtypes = [u64, u64, u64]
        L.orc_range_product_mod.restype = u64
        L.orc_exact_mod.argtypes = [ctypes.c_int, u64, u64]
        L.orc_exact_mod.restype = u64
        L.orc_limbs_mod.argtypes = [u32p, u64, u64]
        L.orc_limbs_mod.restype = u64
        L.orc_is_prime.argtypes = [u64]
        L.orc_is_prime.restype = ctypes.c_int
        L.orc_next_prime.argtypes = [u64]
        L.orc_next_prime.restype = u64
        L.orc_to_decimal.argtypes = [u32p, u64, ctypes.c_char_p, u64]
        L.orc_to_decimal.restype = u64
        _lib = L
    return _lib


def _p32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _p64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _pi64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _limbs(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint32))


# ---------------------------------------------------------------- Phase 1

def sieve(limit: int) -> np.ndarray:
    """All primes <= limit, ascending (Algorithm 1 step 1)."""
    L = lib()
    count = L.orc_sieve(limit, None, 0)
    out = np.empty(count, dtype=np.uint32)
    L.orc_sieve(limit, _p32(out), count)
    return out


def sieve_range(lo: int, hi: int) -> np.ndarray:
    """The primes in [lo, hi], ascending."""
    L = lib()
    count = L.orc_sieve_range(lo, hi, None, 0)
    out = np.empty(count, dtype=np.uint32)
    L.orc_sieve_range(lo, hi, _p32(out), count)
    return out


def prime_count(limit: int) -> int:
    return int(lib().orc_sieve(limit, None, 0))


def legendre(m: int, p: int) -> int:
    """v_p(m!) by Legendre's formula (Sec. 2)."""
    return int(lib().orc_legendre(m, p))


def factor_trial(m: int, primes: np.ndarray) -> list[tuple[int, int]]:
    """Trial-division factorisation of m (Algorithm 1 step 2)."""
    primes = _limbs(primes)
    fp = np.zeros(64, dtype=np.uint64)
    fe = np.zeros(64, dtype=np.uint64)
    k = lib().orc_factor_trial(m, _p32(primes), len(primes), _p64(fp), _p64(fe), 64)
    return [(int(fp[i]), int(fe[i])) for i in range(min(k, 64))]


def prime_limit(kind: int, n: int) -> int:
    return int(lib().orc_prime_limit(kind, n))


def exponents(kind: int, n: int, primes: np.ndarray) -> np.ndarray:
    """Signed e_p for each prime (Algorithm 1 steps 3-9)."""
    primes = _limbs(primes)
    e = np.empty(len(primes), dtype=np.int64)
    rc = lib().orc_exponents(kind, n, _p32(primes), len(primes), _pi64(e))
    if rc != 0:
        raise RuntimeError("n+1 has too many prime factors")
    return e


def ratio_exponents(a: list[int], b: list[int], primes: np.ndarray) -> np.ndarray:
    """v_p(prod a_i! / prod b_j!) for each prime (Sec. 6.3)."""
    primes = _limbs(primes)
    aa = np.asarray(a, dtype=np.uint64)
    bb = np.asarray(b, dtype=np.uint64)
    e = np.empty(len(primes), dtype=np.int64)
    lib().orc_ratio_exponents(_p64(aa), len(aa), _p64(bb), len(bb),
                              _p32(primes), len(primes), _pi64(e))
    return e


def group(primes: np.ndarray, e: np.ndarray):
    """Group primes with e > 0 by exponent (Algorithm 1 steps 10-14).

    Returns (exps, offsets, grouped_primes): CSR with ascending exponents and
    ascending primes within each group."""
    primes = _limbs(primes)
    e = np.ascontiguousarray(e, dtype=np.int64)
    n = len(primes)
    exps = np.zeros(n + 2, dtype=np.uint64)
    offs = np.zeros(n + 2, dtype=np.uint64)
    gp = np.zeros(n + 1, dtype=np.uint32)
    ng = lib().orc_group(_p32(primes), _pi64(e), n, _p64(exps), _p64(offs), _p32(gp))
    ng = int(ng)
    return exps[:ng].copy(), offs[:ng + 1].copy(), gp[:int(offs[ng])].copy()


def factor(kind: int, n: int):
    """Phase 1 end to end: (exps, offsets, grouped_primes)."""
    pr = sieve(prime_limit(kind, n))
    e = exponents(kind, n, pr)
    if (e < 0).any():
        raise ValueError("negative exponent: quantity is not integral")
    return group(pr, e)


def log10_estimate(primes: np.ndarray, e: np.ndarray) -> float:
    """sum e_p log10 p (Algorithm 1, digit-count estimate)."""
    primes = _limbs(primes)
    e = np.ascontiguousarray(e, dtype=np.int64)
    return float(lib().orc_log10_estimate(_p32(primes), _pi64(e), len(primes)))


# ---------------------------------------------------------------- Phase 2

def mul(a, b) -> np.ndarray:
    """Exact product of two limb arrays (schoolbook / Karatsuba)."""
    a, b = _limbs(a), _limbs(b)
    out = np.zeros(len(a) + len(b) + 1, dtype=np.uint32)
    n = lib().orc_mul(_p32(a), len(a), _p32(b), len(b), _p32(out))
    return out[:n].copy()


def product_tree(values) -> np.ndarray:
    """BalancedProductTree over 32-bit values (Sec. 3.2)."""
    v = _limbs(values)
    cap = len(v) + 1
    out = np.zeros(cap, dtype=np.uint32)
    n = lib().orc_product_tree(_p32(v), len(v), _p32(out), cap)
    return out[:n].copy()


def power(a, e: int) -> np.ndarray:
    """a**e by left-to-right binary exponentiation (Algorithm 2 'fast pow')."""
    a = _limbs(a)
    na = len(a)
    while na and a[na - 1] == 0:
        na -= 1
    if e == 0:
        return np.ones(1, dtype=np.uint32)
    if na == 0:
        return np.zeros(0, dtype=np.uint32)
    top_bits = (na - 1) * 32 + int(a[na - 1]).bit_length()
    cap = (top_bits * e) // 32 + 2
    out = np.zeros(cap, dtype=np.uint32)
    n = lib().orc_pow(_p32(a), na, e, _p32(out), cap)
    return out[:n].copy()


def reconstruct(exps, offsets, gprimes, cap: int) -> np.ndarray:
    """Algorithm 2: prod_e (prod_{p in G_e} p)^e."""
    exps = np.ascontiguousarray(exps, dtype=np.uint64)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    gprimes = _limbs(gprimes)
    out = np.zeros(cap, dtype=np.uint32)
    n = lib().orc_reconstruct(len(exps), _p64(exps), _p64(offsets), _p32(gprimes),
                              _p32(out), cap)
    if n > cap:
        raise ValueError("cap too small")
    return out[:n].copy()


def bound_limbs(kind: int, n: int) -> int:
    """A safe upper bound on the limb count: every prime power p^e dividing
    the quantity contributes at most e * bitlen(p) bits."""
    import math
    if kind == FACTORIAL:
        bits = math.lgamma(n + 1) / math.log(2)
    elif kind == CENTRAL_BINOMIAL:
        bits = (math.lgamma(2 * n + 1) - 2 * math.lgamma(n + 1)) / math.log(2)
    else:
        bits = (math.lgamma(2 * n + 1) - math.lgamma(n + 1) - math.lgamma(n + 2)) / math.log(2)
    return int(bits // 32) + 3


def exact(kind: int, n: int) -> np.ndarray:
    """Algorithms 1 and 2 end to end: the exact integer as limbs."""
    cap = bound_limbs(kind, n)
    out = np.zeros(cap, dtype=np.uint32)
    m = lib().orc_exact(kind, n, _p32(out), cap)
    if m == _U64_MAX:
        raise ValueError("not integral")
    if m > cap:
        raise ValueError("cap too small")
    return out[:m].copy()


def exact_mt(kind: int, n: int, threads: int | None = None) -> np.ndarray:
    """``exact`` on several host threads (product-tree halves and large
    Karatsuba sub-products as OpenMP tasks); the same integer."""
    cap = bound_limbs(kind, n)
    out = np.zeros(cap, dtype=np.uint32)
    t = max_threads() if threads is None else int(threads)
    m = lib().orc_exact_mt(kind, n, _p32(out), cap, t)
    if m == _U64_MAX:
        raise ValueError("not integral")
    if m > cap:
        raise ValueError("cap too small")
    return out[:m].copy()


def max_threads() -> int:
    """Host threads ``exact_mt`` can use (1 when built without OpenMP)."""
    return int(lib().orc_max_threads())


def catalan(n: int) -> np.ndarray:
    return exact(CATALAN, n)


def ratio_exact(a: list[int], b: list[int]) -> np.ndarray:
    """prod a_i! / prod b_j! (Sec. 6.3) by the same two phases: sieve to the
    largest term, exponents by the ratio form of Legendre's formula, grouping,
    Algorithm 2.  Raises ValueError when some exponent is negative (the ratio
    is not an integer)."""
    limit = max(list(a) + list(b) + [0])
    primes = sieve(limit) if limit >= 2 else np.zeros(0, dtype=np.uint32)
    e = ratio_exponents(a, b, primes)
    if (e < 0).any():
        raise ValueError("not integral")
    exps, offs, gp = group(primes, e)
    # bits: sum e_p * bitlen(p)
    bits = int(sum(int(x) * int(p).bit_length() for x, p in zip(e, primes) if x > 0))
    return reconstruct(exps, offs, gp, bits // 32 + 2)


# ---------------------------------------------------------------- checks

def exact_mod(kind: int, n: int, q: int) -> int:
    """The quantity mod a prime q from factorial products (no sieve)."""
    r = lib().orc_exact_mod(kind, n, q)
    if r == _U64_MAX:
        raise ValueError("q too small for this kind")
    return int(r)


def limbs_mod(limbs, q: int) -> int:
    """Limb array reduced mod q by Horner's rule from the top limb."""
    a = _limbs(limbs)
    return int(lib().orc_limbs_mod(_p32(a), len(a), q))


def to_decimal(limbs) -> bytes:
    """Decimal digits of a limb array (schoolbook division by 10^9)."""
    a = _limbs(limbs)
    cap = int(len(a) * 32 * 0.30103) + 2
    buf = ctypes.create_string_buffer(max(cap, 1))
    n = lib().orc_to_decimal(_p32(a), len(a), buf, cap)
    if n == _U64_MAX:
        raise ValueError("decimal buffer too small")
    return buf.raw[:n]


def mulmod_plain(a: int, b: int, q: int) -> int:
    return int(lib().orc_mulmod_plain(a, b, q))


def mulmod_mont(a: int, b: int, q: int) -> int:
    return int(lib().orc_mulmod_mont(a, b, q))


def range_product_mod(lo: int, hi: int, q: int) -> int:
    return int(lib().orc_range_product_mod(lo, hi, q))


def is_prime(x: int) -> bool:
    return bool(lib().orc_is_prime(x))


def next_prime(x: int) -> int:
    return int(lib().orc_next_prime(x))


def check_primes(seed: int, count: int, lower: int, bits: int = 62) -> list[int]:
    """`count` distinct primes q > lower drawn from a seeded stream: each is the
    next prime after a seeded random start in [lower, 2^bits)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out: list[int] = []
    hi = 1 << bits
    while len(out) < count:
        start = int(rng.integers(lower + 1, hi, dtype=np.uint64))
        q = next_prime(start)
        if q < hi and q > lower and q not in out:
            out.append(q)
    return out


def limbs_to_int(limbs) -> int:
    a = _limbs(limbs)
    return int.from_bytes(a.astype("<u4").tobytes(), "little")


def int_to_limbs(x: int) -> np.ndarray:
    if x == 0:
        return np.zeros(0, dtype=np.uint32)
    nbytes = (x.bit_length() + 31) // 32 * 4
    return np.frombuffer(x.to_bytes(nbytes, "little"), dtype="<u4").astype(np.uint32)
