"""GB300 (sm_103a) library for exact Catalan numbers, central binomials and
factorials by the two-phase prime-exponent method of arXiv 2601.11621.

The computation runs in ``lib/libcatalan.so`` (CUDA, built from ``csrc/`` by
``build.py``) behind the C ABI of ``include/catalan.h``.  ``capi`` is the thin
ctypes binding with the same function names; it only marshals arguments.
Importing this package does not load the CUDA library; the first call does,
and raises if the library is missing.
"""

__all__ = ["capi", "build", "workloads"]
