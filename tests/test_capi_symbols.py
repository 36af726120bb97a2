"""The C-ABI library builds, loads and exports every function the header
declares (no GPU needed: nothing here launches device work)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "catalan.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:int|void|size_t|unsigned\s+long\s+long|const\s+char\s*\*)"
                       r"\s*\*?\s*(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("catalan_factor", "bigint_mul", "bigint_pow", "product_tree",
                 "catalan_exact", "cat_bound_limbs", "cat_exact", "to_decimal"):
        assert must in names


def test_library_exports_every_declared_symbol(cat_lib):
    lib = ctypes.CDLL(cat_lib.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", cat_lib.LIB_PATH],
                         capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(declared_functions()) <= exported
    assert set(cat_lib.EXPORTED) <= exported


def test_binding_covers_the_header(cat_lib):
    assert set(declared_functions()) == set(cat_lib.EXPORTED)


def test_bound_limbs_host_only(cat_lib, orc):
    # cat_bound_limbs is host arithmetic: it must cover the exact length
    for kind, n in [(0, 0), (0, 1), (0, 2), (0, 10), (0, 1000), (1, 1000), (2, 1000),
                    (0, 100000), (2, 12345)]:
        exact = orc.exact(kind, n)
        assert cat_lib.cat_bound_limbs(n, kind) >= len(exact)
        assert cat_lib.cat_bound_limbs(n, kind) <= len(exact) + 3
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_bound_limbs(1 << 31, 0)
    with pytest.raises(cat_lib.CatError):
        cat_lib.cat_bound_limbs(10, 7)


def test_library_fails_loudly_without_build(cat_lib, tmp_path):
    import importlib
    mod = importlib.import_module("paper_2601_11621_gb300.capi")
    with pytest.raises(OSError):
        mod._lib_saved = mod._lib
        try:
            mod._lib = None
            mod.load(str(tmp_path / "missing.so"))
        finally:
            mod._lib = mod._lib_saved
