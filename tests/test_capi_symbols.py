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


def test_batch_creation_checks_without_gpu():
    """sphfsi_create_batch validates its arguments; sphfsi_select its index."""
    import paper_1911_13255_gb300 as pkg
    L = pkg.lib()
    ps = (pkg.Params * 3)()
    for k in range(3):
        ps[k].dim = 2
        for d in range(2):
            ps[k].domain_lo[d], ps[k].domain_hi[d] = 0.0, 1.0
    h = ctypes.c_void_p()
    assert L.sphfsi_create_batch(ctypes.byref(h), 0, ps, None) == -1
    ps[2].dim = 3
    assert L.sphfsi_create_batch(ctypes.byref(h), 3, ps, None) == -1
    ps[2].dim = 2
    ps[1].domain_hi[0] = -1.0
    assert L.sphfsi_create_batch(ctypes.byref(h), 3, ps, None) == -1
    ps[1].domain_hi[0] = 1.0
    assert L.sphfsi_create_batch(ctypes.byref(h), 3, ps, None) == 0
    assert L.sphfsi_select(h, 2) == 0
    assert L.sphfsi_select(h, 3) == -1
    assert L.sphfsi_select(h, -1) == -1
    assert L.sphfsi_select(None, 0) == -1
    assert L.sphfsi_step(h, 1.0) == -4      # not finalized
    L.sphfsi_destroy(h)


def test_time_stepping_and_inflow_checks_without_gpu():
    """The single-time-step modes and the inflow profiles (Womersley needs
    its period and number) are validated on the host."""
    import paper_1911_13255_gb300 as pkg
    L = pkg.lib()
    p = pkg.Params()
    p.dim = 2
    for d in range(2):
        p.domain_lo[d], p.domain_hi[d] = 0.0, 1.0
    h = ctypes.c_void_p()
    assert L.sphfsi_create(ctypes.byref(h), ctypes.byref(p), None) == 0
    assert L.sphfsi_set_time_stepping(None, 1) == -1
    for mode, rc in ((0, 0), (1, 0), (2, 0), (3, -1), (-1, -1)):
        assert L.sphfsi_set_time_stepping(h, mode) == rc, mode
    assert L.sphfsi_set_substeps(h, 4) == 0
    cases = [((1, 2, 0.1, 0.0, 1.0, 2.5, 0.0, 0.6, 5.0), 0),
             ((1, 2, 0.1, 0.0, 1.0, 2.5, 0.0, 0.0, 5.0), -1),    # no period
             ((1, 2, 0.1, 0.0, 1.0, 2.5, 0.0, 0.6, 0.0), -1),    # no Womersley number
             ((1, 2, 0.1, 0.0, 0.0, 2.5, 0.0, 0.6, 5.0), -1),    # no channel height
             ((1, 4, 0.1, 0.0, 1.0, 2.5, 0.0, 0.0, 0.0), -1),    # unknown profile
             ((1, 3, 0.1, 0.0, 1.0, 2.5, 0.0, 0.0, 0.0, 0.0, 1.0), 0),         # duct
             ((1, 3, 0.1, 0.0, 1.0, 2.5, 0.0, 0.0, 0.0, 0.0, 0.0), -1),        # duct without its z extent
             ((1, 3, 0.1, 0.0, 1.0, 2.5, 0.0, 0.0, 0.0, float("nan"), 1.0), -1),  # non-finite z0
             ((1, 3, 0.1, 0.0, 0.0, 2.5, 0.0, 0.0, 0.0, 0.0, 1.0), -1),        # duct without its height
             ((1, 0, 0.0, 0.0, 1.0, 1.0, 0.0, 0.0, 0.0), -1),    # no buffer
             ((1, 1, 0.1, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0), 0),     # uniform: no height needed
             ((0, 7, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0), 0)]     # off: not checked
    for vals, rc in cases:
        f = pkg.Inflow(*vals)
        assert L.sphfsi_set_inflow(h, ctypes.byref(f)) == rc, vals
    L.sphfsi_destroy(h)


def test_new_entry_points_check_their_state_without_gpu():
    """The asynchronous position read, the advection cadence (0 = automatic)
    and the wait limit refuse a NULL context, and a context that is not
    finalized yet (SPHFSI_E_STATE), before touching any device; the strings
    of the two stop conditions name them."""
    import paper_1911_13255_gb300 as pkg
    L = pkg.lib()
    buf = (ctypes.c_double * 4)()
    assert L.sphfsi_get_solid_positions_async(None, buf) == -1
    assert L.sphfsi_set_advection_cadence(None, 0) == -1
    assert L.sphfsi_set_wait_limit(None, 0) == -1
    p = pkg.Params()
    p.dim = 2
    for d in range(2):
        p.domain_lo[d], p.domain_hi[d] = 0.0, 1.0
    h = ctypes.c_void_p()
    assert L.sphfsi_create(ctypes.byref(h), ctypes.byref(p), None) == 0
    assert L.sphfsi_get_solid_positions_async(h, buf) == -4
    assert L.sphfsi_set_advection_cadence(h, 0) == -4
    assert L.sphfsi_set_advection_cadence(h, 3) == -4
    assert L.sphfsi_step(h, 1.0) == -4
    L.sphfsi_destroy(h)
    assert b"run-away" in L.sphfsi_strerror(-5)
    assert L.sphfsi_strerror(-6).startswith(b"bounded")
