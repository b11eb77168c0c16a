"""The C-ABI library builds, loads and exports every entry point include/lfem.h
declares; host-side argument checks answer without a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lfem.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lfem_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_14035_gb300 import build as b

    return b.build()


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2605_14035_gb300 import lfem

    assert sorted(lfem.EXPORTS) == declared_functions()


def test_host_side_errors_without_gpu(libpath):
    lib = ctypes.CDLL(libpath)
    lib.lfem_pattern.restype = ctypes.c_int
    lib.lfem_pattern.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_void_p, ctypes.c_void_p]
    lib.lfem_last_error.restype = ctypes.c_char_p
    lib.lfem_status_string.restype = ctypes.c_char_p
    assert lib.lfem_pattern(None, 10, 10, 2, 1, None, None) == 1          # out is NULL
    h = ctypes.c_void_p()
    assert lib.lfem_pattern(None, 10, 10, 2, 1, None, ctypes.byref(h)) == 1  # conn is NULL
    assert b"conn" in lib.lfem_last_error()
    assert lib.lfem_pattern(None, 0, 10, 4, 1, None, ctypes.byref(h)) == 3   # dim 4 unsupported
    assert lib.lfem_pattern(None, 1 << 28, 10, 2, 1, None, ctypes.byref(h)) in (1, 4)
    assert lib.lfem_status_string(7) == b"degenerate element"
    lib.lfem_assemble.restype = ctypes.c_int
    assert lib.lfem_assemble(None, None, 3, None, None, 0, 1, 0, None, None, None, None) == 1
    lib.lfem_set_mixed_kappa.argtypes = [ctypes.c_void_p, ctypes.c_double]
    assert lib.lfem_set_mixed_kappa(None, 2.0) == 1


def declared_arities():
    """Number of parameters of every entry point the header declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(lfem_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", text, flags=re.S):
        args = m.group(2).strip()
        out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_arities_match_header():
    """Every argtypes list in the Python binding has the header's parameter count."""
    from paper_2605_14035_gb300 import lfem

    ar = declared_arities()
    assert len(ar) >= 15
    lib = lfem.lib()
    bad = {}
    for n in lfem.EXPORTS:
        t = getattr(lib, n).argtypes
        if t is not None and n in ar and len(t) != ar[n]:
            bad[n] = (len(t), ar[n])
    assert not bad, bad
