"""The C-ABI library builds (nvcc cross-compiles sm_103a without a GPU),
loads, and exports every entry point declared in include/*.h.  No compute
call is made here."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sphfsi_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_all_declared_symbols():
    from paper_1911_13255_gb300 import _build
    path = _build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_argument_checks_without_gpu():
    """Entry points that touch no device reject bad arguments."""
    import paper_1911_13255_gb300 as pkg
    L = pkg.lib()
    assert L.sphfsi_strerror(0) == b"ok"
    assert L.sphfsi_strerror(-6).startswith(b"bounded")
    p = pkg.Params()
    p.dim = 4
    h = ctypes.c_void_p()
    assert L.sphfsi_create(ctypes.byref(h), ctypes.byref(p), None) == -1
    assert L.sphfsi_step(None, 1.0) == -1
    assert L.sphfsi_set_substeps(None, 2) == -1
