"""ctypes binding of libcatalan (include/catalan.h).

Same names as the C entry points; each function only converts arguments
(torch tensors to device pointers, the current torch stream to a
cudaStream_t) and status codes to exceptions.  Big integers are 1-D int32
torch tensors holding little-endian uint32 limbs (torch has no general
uint32 arithmetic; the bits are the same).  There is no CPU fallback: if the
library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libcatalan.so")

CAT_CATALAN, CAT_CENTRAL_BINOMIAL, CAT_FACTORIAL = 0, 1, 2
KINDS = {"catalan": CAT_CATALAN, "central_binomial": CAT_CENTRAL_BINOMIAL,
         "factorial": CAT_FACTORIAL}

STATUS = {0: "CAT_OK", -1: "CAT_EINVAL", -2: "CAT_ENOMEM", -3: "CAT_ERANGE",
          -4: "CAT_ENOTINTEGRAL", -5: "CAT_ETIMEOUT", -6: "CAT_ECUDA", -7: "CAT_EBUSY"}
CAT_OK, CAT_EINVAL, CAT_ENOMEM, CAT_ERANGE = 0, -1, -2, -3
CAT_ENOTINTEGRAL, CAT_ETIMEOUT, CAT_ECUDA, CAT_EBUSY = -4, -5, -6, -7

EXPORTED = ["cat_ctx_create", "cat_ctx_destroy", "cat_last_error", "cat_ctx_memory",
            "cat_launch_count",
            "cat_autotune", "cat_ctx_load_tuning", "cat_ctx_tuning",
            "cat_ctx_set_profiling", "cat_ctx_profile",
            "catalan_factor", "cat_factor_free", "cat_factor_copy_primes", "bigint_mul",
            "bigint_mul_noalloc", "bigint_pow",
            "product_tree", "cat_reconstruct", "cat_bound_limbs", "cat_exact",
            "catalan_exact", "cat_exact_host", "cat_batch_bound", "cat_exact_batch",
            "cat_server_create", "cat_server_submit", "cat_server_poll", "cat_server_wait",
            "cat_server_fetch", "cat_server_release", "cat_server_pending",
            "cat_server_destroy", "cat_server_memory", "cat_batch_footprint",
            "cat_decimal_bound", "to_decimal",
            "cat_ratio_bound_limbs", "cat_ratio_factor", "cat_ratio_exact",
            "cat_factor_text", "cat_binary"]


class CatError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class Factorization(ctypes.Structure):
    _fields_ = [("num_groups", ctypes.c_uint64), ("num_primes", ctypes.c_uint64),
                ("primes_sieved", ctypes.c_uint64),
                ("exps", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("primes", ctypes.c_void_p),
                ("host_exps", ctypes.POINTER(ctypes.c_uint64)),
                ("host_offsets", ctypes.POINTER(ctypes.c_uint64))]


class Request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_uint64)]


class ServerResult(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("n", ctypes.c_uint64), ("limbs", ctypes.c_void_p),
                ("length", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64),
                ("t_start_ns", ctypes.c_uint64), ("t_end_ns", ctypes.c_uint64),
                ("batch", ctypes.c_uint64)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libcatalan.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"libcatalan.so not built at {path}; run paper_2601_11621_gb300.build")
    L = ctypes.CDLL(path)
    vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
    szp = ctypes.POINTER(ctypes.c_size_t)
    L.cat_ctx_create.argtypes = [i32, sz, ctypes.POINTER(vp)]
    L.cat_ctx_create.restype = i32
    L.cat_ctx_destroy.argtypes = [vp]
    L.cat_ctx_destroy.restype = None
    L.cat_last_error.argtypes = [vp]
    L.cat_last_error.restype = ctypes.c_char_p
    L.cat_autotune.argtypes = [vp, ctypes.c_char_p, vp]
    L.cat_autotune.restype = i32
    L.cat_ctx_load_tuning.argtypes = [vp, ctypes.c_char_p]
    L.cat_ctx_load_tuning.restype = i32
    L.cat_ctx_tuning.argtypes = [vp, szp, ctypes.POINTER(i32), sz]
    L.cat_ctx_tuning.restype = i32
    L.cat_ctx_memory.argtypes = [vp, szp, szp]
    L.cat_ctx_memory.restype = i32
    L.cat_launch_count.argtypes = []
    L.cat_launch_count.restype = ctypes.c_ulonglong
    L.cat_ctx_set_profiling.argtypes = [vp, i32]
    L.cat_ctx_set_profiling.restype = i32
    L.cat_ctx_profile.argtypes = [vp, sz, ctypes.POINTER(ctypes.c_char_p),
                                  ctypes.POINTER(ctypes.c_uint64),
                                  ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    L.cat_ctx_profile.restype = i32
    L.catalan_factor.argtypes = [vp, u64, i32, ctypes.POINTER(Factorization), vp]
    L.catalan_factor.restype = i32
    L.cat_factor_free.argtypes = [vp, ctypes.POINTER(Factorization)]
    L.cat_factor_free.restype = None
    L.cat_factor_copy_primes.argtypes = [vp, ctypes.POINTER(Factorization), vp, sz, vp]
    L.cat_factor_copy_primes.restype = i32
    L.bigint_mul.argtypes = [vp, vp, sz, vp, sz, vp, sz, szp, vp]
    L.bigint_mul.restype = i32
    L.bigint_mul_noalloc.argtypes = [vp, sz, vp, sz, vp, sz, szp, vp]
    L.bigint_mul_noalloc.restype = i32
    u64a = ctypes.POINTER(ctypes.c_uint64)
    L.cat_ratio_bound_limbs.argtypes = [u64a, i32, u64a, i32, szp]
    L.cat_ratio_bound_limbs.restype = i32
    L.cat_ratio_factor.argtypes = [vp, u64a, i32, u64a, i32, ctypes.POINTER(Factorization), vp]
    L.cat_ratio_factor.restype = i32
    L.cat_ratio_exact.argtypes = [vp, u64a, i32, u64a, i32, vp, sz, szp, vp]
    L.cat_ratio_exact.restype = i32
    L.cat_factor_text.argtypes = [vp, ctypes.POINTER(Factorization), ctypes.c_char_p, vp, sz,
                                  szp, vp]
    L.cat_factor_text.restype = i32
    L.cat_binary.argtypes = [vp, vp, sz, vp, sz, szp, vp]
    L.cat_binary.restype = i32
    L.cat_decimal_bound.argtypes = [sz]
    L.cat_decimal_bound.restype = sz
    L.to_decimal.argtypes = [vp, vp, sz, vp, sz, szp, vp]
    L.to_decimal.restype = i32
    L.bigint_pow.argtypes = [vp, vp, sz, u64, vp, sz, szp, vp]
    L.bigint_pow.restype = i32
    L.product_tree.argtypes = [vp, vp, sz, vp, sz, szp, vp]
    L.product_tree.restype = i32
    L.cat_reconstruct.argtypes = [vp, ctypes.POINTER(Factorization), vp, sz, szp, vp]
    L.cat_reconstruct.restype = i32
    L.cat_bound_limbs.argtypes = [u64, i32, szp]
    L.cat_bound_limbs.restype = i32
    L.cat_exact.argtypes = [vp, i32, u64, vp, sz, szp, vp]
    L.cat_exact.restype = i32
    L.catalan_exact.argtypes = [vp, u64, vp, sz, szp, vp]
    L.catalan_exact.restype = i32
    L.cat_exact_host.argtypes = [vp, i32, u64, vp, sz, szp, vp]
    L.cat_exact_host.restype = i32
    u64p = ctypes.POINTER(ctypes.c_uint64)
    L.cat_batch_bound.argtypes = [ctypes.POINTER(Request), sz, szp]
    L.cat_batch_footprint.argtypes = [ctypes.POINTER(Request), sz, szp]
    L.cat_server_memory.argtypes = [vp, szp, szp]
    L.cat_server_memory.restype = i32
    L.cat_batch_footprint.restype = i32
    L.cat_batch_bound.restype = i32
    L.cat_exact_batch.argtypes = [vp, ctypes.POINTER(Request), sz, vp, sz, u64p, u64p, vp]
    L.cat_exact_batch.restype = i32
    resp = ctypes.POINTER(ServerResult)
    L.cat_server_create.argtypes = [i32, sz, i32, sz, ctypes.POINTER(vp)]
    L.cat_server_create.restype = i32
    L.cat_server_submit.argtypes = [vp, i32, u64, u64p]
    L.cat_server_submit.restype = i32
    L.cat_server_poll.argtypes = [vp, u64, resp]
    L.cat_server_poll.restype = i32
    L.cat_server_wait.argtypes = [vp, u64, u64, resp]
    L.cat_server_wait.restype = i32
    L.cat_server_fetch.argtypes = [vp, u64, vp, sz, i32, szp]
    L.cat_server_fetch.restype = i32
    L.cat_server_release.argtypes = [vp, u64]
    L.cat_server_release.restype = i32
    L.cat_server_pending.argtypes = [vp, szp, szp]
    L.cat_server_pending.restype = i32
    L.cat_server_destroy.argtypes = [vp]
    L.cat_server_destroy.restype = None
    _lib = L
    return L


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() else ctypes.c_void_p(0)


class Context:
    """A libcatalan context on one CUDA device (twiddle tables + scratch pool)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        L = load()
        h = ctypes.c_void_p()
        rc = L.cat_ctx_create(device, hbm_budget_bytes, ctypes.byref(h))
        if rc != 0:
            raise CatError(rc, "cat_ctx_create failed")
        self.handle = h
        self.device = device

    def check(self, rc: int):
        if rc != 0:
            msg = load().cat_last_error(self.handle) or b""
            raise CatError(rc, msg.decode(errors="replace"))

    def memory(self) -> tuple[int, int]:
        a, b = ctypes.c_size_t(), ctypes.c_size_t()
        self.check(load().cat_ctx_memory(self.handle, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def autotune(self, path: str | None = None, stream=None):
        """cat_autotune: measure, apply and (with path) save the tuned choices."""
        self.check(load().cat_autotune(self.handle, path.encode() if path else None,
                                       _stream(stream)))

    def load_tuning(self, path: str):
        """cat_ctx_load_tuning."""
        self.check(load().cat_ctx_load_tuning(self.handle, path.encode()))

    def tuning(self) -> tuple[int, dict]:
        """(crossover slot, {n: row-pass log2 size} for the tuned sizes)."""
        slot = ctypes.c_size_t()
        rows = (ctypes.c_int * 28)()
        self.check(load().cat_ctx_tuning(self.handle, ctypes.byref(slot), rows, 28))
        return slot.value, {n: rows[n] for n in range(28) if rows[n]}

    def set_profiling(self, on: bool):
        self.check(load().cat_ctx_set_profiling(self.handle, 1 if on else 0))

    def profile(self) -> dict:
        """{kernel name: (launches, total ms, total pass bytes, total unit bytes)}
        (cat_ctx_profile)."""
        out = {}
        i = 0
        while True:
            name = ctypes.c_char_p()
            n, ms, b, o = ctypes.c_uint64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
            rc = load().cat_ctx_profile(self.handle, i, ctypes.byref(name), ctypes.byref(n),
                                        ctypes.byref(ms), ctypes.byref(b), ctypes.byref(o))
            if rc != 0:
                break
            out[name.value.decode()] = (n.value, ms.value, b.value, o.value)
            i += 1
        return out

    def close(self):
        if getattr(self, "handle", None):
            load().cat_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _limbs_tensor(x, device):
    """Accept a torch tensor (int32/uint32 limbs on the device) or a numpy array."""
    import torch
    if isinstance(x, torch.Tensor):
        if x.dtype not in (torch.int32,) and str(x.dtype) != "torch.uint32":
            raise TypeError("limb tensors must be int32 (uint32 bits)")
        return x.contiguous().view(torch.int32)
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint32)).view(np.int32)
    return torch.from_numpy(a.copy()).to(device)


def _empty(n, device):
    import torch
    return torch.empty(max(n, 1), dtype=torch.int32, device=device)


def cat_launch_count() -> int:
    """Kernels the library has launched in this process so far."""
    return int(load().cat_launch_count())


def cat_bound_limbs(n: int, kind: int = CAT_CATALAN) -> int:
    out = ctypes.c_size_t()
    rc = load().cat_bound_limbs(n, kind, ctypes.byref(out))
    if rc != 0:
        raise CatError(rc, "cat_bound_limbs")
    return out.value


def bigint_mul(ctx: Context, a, b, stream=None):
    dev = f"cuda:{ctx.device}"
    ta, tb = _limbs_tensor(a, dev), _limbs_tensor(b, dev)
    cap = ta.numel() + tb.numel()
    out = _empty(cap, dev)
    n = ctypes.c_size_t()
    ctx.check(load().bigint_mul(ctx.handle, _ptr(ta), ta.numel(), _ptr(tb), tb.numel(),
                                _ptr(out), cap, ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def _u64_array(v):
    arr = (ctypes.c_uint64 * max(len(v), 1))(*[int(x) for x in v])
    return arr, len(v)


def cat_ratio_bound_limbs(a, b) -> int:
    """Limb bound of prod a_i! / prod b_j! (Sec. 6.3)."""
    (pa, ka), (pb, kb) = _u64_array(a), _u64_array(b)
    out = ctypes.c_size_t()
    rc = load().cat_ratio_bound_limbs(pa, ka, pb, kb, ctypes.byref(out))
    if rc != 0:
        raise CatError(rc, "cat_ratio_bound_limbs")
    return out.value


def cat_ratio_factor(ctx: Context, a, b, stream=None) -> "FactorResult":
    """Grouped factorisation of prod a_i! / prod b_j! (device arrays)."""
    (pa, ka), (pb, kb) = _u64_array(a), _u64_array(b)
    f = Factorization()
    ctx.check(load().cat_ratio_factor(ctx.handle, pa, ka, pb, kb, ctypes.byref(f),
                                      _stream(stream)))
    return FactorResult(ctx, f)


def cat_ratio_exact(ctx: Context, a, b, out=None, stream=None):
    """prod a_i! / prod b_j! as a device limb tensor (CAT_ENOTINTEGRAL when it is
    not an integer)."""
    dev = f"cuda:{ctx.device}"
    (pa, ka), (pb, kb) = _u64_array(a), _u64_array(b)
    if out is None:
        out = _empty(cat_ratio_bound_limbs(a, b), dev)
    n = ctypes.c_size_t()
    ctx.check(load().cat_ratio_exact(ctx.handle, pa, ka, pb, kb, _ptr(out), out.numel(),
                                     ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def cat_factor_text(ctx: Context, fr: "FactorResult", name: str, stream=None):
    """The factorisation in the text layout of Sec. 3.1 (uint8 device tensor)."""
    import torch
    dev = f"cuda:{ctx.device}"
    n = ctypes.c_size_t()
    rc = load().cat_factor_text(ctx.handle, ctypes.byref(fr.f), name.encode(), None, 0,
                                ctypes.byref(n), _stream(stream))
    if rc not in (0, CAT_ERANGE):
        ctx.check(rc)
    out = torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)
    ctx.check(load().cat_factor_text(ctx.handle, ctypes.byref(fr.f), name.encode(), _ptr(out),
                                     out.numel(), ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def cat_binary(ctx: Context, limbs, stream=None):
    """The result file bytes (01 01, then the little-endian magnitude) as a
    uint8 device tensor."""
    import torch
    dev = f"cuda:{ctx.device}"
    t = _limbs_tensor(limbs, dev)
    out = torch.empty(4 * t.numel() + 2, dtype=torch.uint8, device=dev)
    n = ctypes.c_size_t()
    ctx.check(load().cat_binary(ctx.handle, _ptr(t), t.numel(), _ptr(out), out.numel(),
                                ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def cat_decimal_bound(n_limbs: int) -> int:
    """Upper bound on the decimal digit count of an n-limb number."""
    return load().cat_decimal_bound(n_limbs)


def to_decimal(ctx: Context, limbs, out=None, stream=None):
    """Decimal digits of a little-endian uint32 number (device tensor or numpy
    array) through to_decimal: a uint8 device tensor of ASCII digits, most
    significant first ("0" for zero).  `out` may be a preallocated uint8
    device tensor of at least cat_decimal_bound(len(limbs)) bytes."""
    import torch
    dev = f"cuda:{ctx.device}"
    t = _limbs_tensor(limbs, dev)
    if out is None:
        out = torch.empty(max(cat_decimal_bound(t.numel()), 1), dtype=torch.uint8, device=dev)
    n = ctypes.c_size_t()
    ctx.check(load().to_decimal(ctx.handle, _ptr(t), t.numel(), _ptr(out), out.numel(),
                                ctypes.byref(n), _stream(stream)))
    return out[:n.value]


NOALLOC_MAX_LIMBS = 1 << 16


def bigint_mul_noalloc(a, b, out=None, stream=None, device: int = 0):
    """a * b through bigint_mul_noalloc (no context, no device allocation in
    the library).  `out` may be a preallocated int32 device tensor of at
    least len(a) + len(b) limbs; the result is a view of it."""
    dev = f"cuda:{device}"
    ta, tb = _limbs_tensor(a, dev), _limbs_tensor(b, dev)
    cap = ta.numel() + tb.numel()
    if out is None:
        out = _empty(cap, dev)
    n = ctypes.c_size_t()
    rc = load().bigint_mul_noalloc(_ptr(ta), ta.numel(), _ptr(tb), tb.numel(), _ptr(out),
                                   out.numel(), ctypes.byref(n), _stream(stream))
    if rc != 0:
        raise CatError(rc, "bigint_mul_noalloc")
    return out[:n.value]


def bigint_pow(ctx: Context, a, e: int, stream=None):
    dev = f"cuda:{ctx.device}"
    ta = _limbs_tensor(a, dev)
    na = ta.numel()
    bits = na * 32
    cap = max(1, (bits * e) // 32 + 2) if e else 1
    out = _empty(cap, dev)
    n = ctypes.c_size_t()
    ctx.check(load().bigint_pow(ctx.handle, _ptr(ta), na, e, _ptr(out), cap,
                                ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def product_tree(ctx: Context, values, stream=None):
    dev = f"cuda:{ctx.device}"
    tv = _limbs_tensor(values, dev)
    cap = max(1, tv.numel())
    out = _empty(cap, dev)
    n = ctypes.c_size_t()
    ctx.check(load().product_tree(ctx.handle, _ptr(tv), tv.numel(), _ptr(out), cap,
                                  ctypes.byref(n), _stream(stream)))
    return out[:n.value]


class FactorResult:
    """Grouped factorisation (CSR) returned by catalan_factor; owns the
    device arrays until free() (or garbage collection)."""

    def __init__(self, ctx: Context, f: Factorization):
        self.ctx = ctx
        self.f = f
        ng = f.num_groups
        self.exps = np.array([f.host_exps[i] for i in range(ng)], dtype=np.uint64)
        self.offsets = np.array([f.host_offsets[i] for i in range(ng + 1)], dtype=np.uint64)
        self.num_primes = f.num_primes
        self.primes_sieved = f.primes_sieved

    def primes(self):
        """Device copy of the grouped primes as an int32 tensor (uint32 bits)."""
        out = _empty(self.num_primes, f"cuda:{self.ctx.device}")
        self.ctx.check(load().cat_factor_copy_primes(self.ctx.handle, ctypes.byref(self.f),
                                                     _ptr(out), self.num_primes,
                                                     _stream(None)))
        return out[:self.num_primes]

    def free(self):
        if self.f is not None and self.ctx.handle:
            load().cat_factor_free(self.ctx.handle, ctypes.byref(self.f))
        self.f = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def catalan_factor(ctx: Context, n: int, kind: int = CAT_CATALAN, stream=None) -> FactorResult:
    f = Factorization()
    ctx.check(load().catalan_factor(ctx.handle, n, kind, ctypes.byref(f), _stream(stream)))
    return FactorResult(ctx, f)


def cat_reconstruct(ctx: Context, fact: FactorResult, cap: int, stream=None):
    out = _empty(cap, f"cuda:{ctx.device}")
    n = ctypes.c_size_t()
    ctx.check(load().cat_reconstruct(ctx.handle, ctypes.byref(fact.f), _ptr(out), cap,
                                     ctypes.byref(n), _stream(stream)))
    return out[:n.value]


def cat_exact(ctx: Context, kind: int, n: int, out=None, stream=None):
    """The exact quantity as an int32 device tensor of uint32 limbs.  `out`
    may be a preallocated int32 device tensor of at least cat_bound_limbs."""
    if out is None:
        out = _empty(cat_bound_limbs(n, kind), f"cuda:{ctx.device}")
    m = ctypes.c_size_t()
    ctx.check(load().cat_exact(ctx.handle, kind, n, _ptr(out), out.numel(),
                               ctypes.byref(m), _stream(stream)))
    return out[:m.value]


def catalan_exact(ctx: Context, n: int, out=None, stream=None):
    return cat_exact(ctx, CAT_CATALAN, n, out=out, stream=stream)


def cat_exact_host(ctx: Context, kind: int, n: int, out: np.ndarray | None = None,
                   stream=None) -> np.ndarray:
    """The exact quantity copied into a host uint32 array (pinned if given)."""
    if out is None:
        out = np.empty(cat_bound_limbs(n, kind), dtype=np.uint32)
    m = ctypes.c_size_t()
    ctx.check(load().cat_exact_host(ctx.handle, kind, n,
                                    out.ctypes.data_as(ctypes.c_void_p), out.size,
                                    ctypes.byref(m), _stream(stream)))
    return out[:m.value]


_REQUEST_DTYPE = np.dtype({"names": ["kind", "n"], "formats": [np.int32, np.uint64],
                           "offsets": [Request.kind.offset, Request.n.offset],
                           "itemsize": ctypes.sizeof(Request)})


def _requests(reqs):
    """(kind, n) pairs as a numpy-backed array of cat_request (at least one
    element); pass it through _request_ptr and keep it alive for the call."""
    v = np.asarray(reqs, dtype=np.int64).reshape(-1, 2)
    arr = np.zeros(max(1, len(v)), dtype=_REQUEST_DTYPE)
    arr["kind"][:len(v)] = v[:, 0]
    arr["n"][:len(v)] = v[:, 1].astype(np.uint64)
    return arr


def _request_ptr(arr):
    return arr.ctypes.data_as(ctypes.POINTER(Request))


def cat_batch_bound(reqs) -> int:
    """Total limbs a batch of (kind, n) requests needs."""
    total = ctypes.c_size_t()
    arr = _requests(reqs)
    rc = load().cat_batch_bound(_request_ptr(arr), len(reqs), ctypes.byref(total))
    if rc != 0:
        raise CatError(rc, "cat_batch_bound")
    return total.value


def cat_batch_footprint(reqs) -> int:
    """The serving engine's device-byte estimate for a batch of (kind, n)."""
    total = ctypes.c_size_t()
    arr = _requests(reqs)
    rc = load().cat_batch_footprint(_request_ptr(arr), len(reqs), ctypes.byref(total))
    if rc != 0:
        raise CatError(rc, "cat_batch_footprint")
    return total.value


def cat_exact_batch(ctx: Context, reqs, out=None, stream=None):
    """All (kind, n) requests computed together.  Returns (out, offsets,
    lengths): request r's limbs are out[offsets[r] : offsets[r] + lengths[r]]
    (out an int32 device tensor of uint32 limbs)."""
    count = len(reqs)
    arr = _requests(reqs)
    total = ctypes.c_size_t()
    rc = load().cat_batch_bound(_request_ptr(arr), count, ctypes.byref(total))
    if rc != 0:
        raise CatError(rc, "cat_batch_bound")
    if out is None:
        out = _empty(total.value, f"cuda:{ctx.device}")
    offs = np.zeros(max(1, count), dtype=np.uint64)
    lens = np.zeros(max(1, count), dtype=np.uint64)
    u64p = ctypes.POINTER(ctypes.c_uint64)
    ctx.check(load().cat_exact_batch(ctx.handle, _request_ptr(arr), count, _ptr(out), out.numel(),
                                     offs.ctypes.data_as(u64p), lens.ctypes.data_as(u64p),
                                     _stream(stream)))
    return out, offs[:count], lens[:count]


def to_numpy(t) -> np.ndarray:
    """Device limb tensor -> host uint32 numpy array."""
    return t.detach().cpu().numpy().view(np.uint32)
