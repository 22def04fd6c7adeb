"""The C-ABI library builds, loads, and exports every entry point declared in
include/hodlr2d.h; argument checks that need no GPU return their codes."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hodlr2d.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(hodlr2d_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hodlr2d_build", "hodlr2d_matvec", "hodlr2d_gmres", "hodlr2d_free",
                 "hodlr2d_get_stats", "hodlr2d_strerror", "hodlr2d_import_factors"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2204_05536_gb300 import _lib
    lib = _lib.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares exactly the header's entry points
    assert sorted(_lib.SIGNATURES) == _declared()


def test_strerror_and_defaults_without_gpu():
    from paper_2204_05536_gb300 import _lib
    lib = _lib.load()
    assert lib.hodlr2d_strerror(0) == b"ok"
    assert lib.hodlr2d_strerror(-1) == b"invalid argument"
    o = _lib.Opts()
    lib.hodlr2d_default_opts(C.byref(o))
    assert (o.levels, o.compress, o.max_rank, o.mode) == (-1, 1, 256, 0)


def test_argument_checks_without_gpu():
    """Invalid arguments are rejected before any device work."""
    from paper_2204_05536_gb300 import _lib, kernel
    lib = _lib.load()
    h = C.c_void_p()
    import numpy as np
    pts = np.zeros((4, 2))
    p = C.c_void_p(pts.ctypes.data)
    k = kernel("imq", a=0.1)
    assert lib.hodlr2d_build(None, 4, k, 8, 1e-8, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 0, k, 8, 1e-8, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 4, k, 0, 1e-8, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 4, k, 8, 0.0, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 4, k, 8, float("nan"), C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 4, kernel("imq", a=0.0), 8, 1e-8, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_build(p, 4, kernel("phi1", a=1.0), 8, 1e-8, C.byref(h)) == _lib.ERR_ARG
    bad = _lib.Kernel(9, 0.1, 0, 0.0)
    assert lib.hodlr2d_build(p, 4, bad, 8, 1e-8, C.byref(h)) == _lib.ERR_ARG
    assert lib.hodlr2d_matvec(None, p, p, 1) == _lib.ERR_ARG
    assert lib.hodlr2d_gmres(None, p, p, 1e-8) == _lib.ERR_ARG
    assert lib.hodlr2d_get_stats(None, None) == _lib.ERR_ARG
    lib.hodlr2d_free(None)  # no-op


def test_batch_argument_checks_without_gpu():
    """The batch entry points reject null handles and out-of-range settings
    before any device work."""
    from paper_2204_05536_gb300 import _lib
    lib = _lib.load()
    out = C.c_void_p()
    assert lib.hodlr2d_batch_create(None, 1, C.byref(out)) == _lib.ERR_ARG
    arr = (C.c_void_p * 1)(None)
    assert lib.hodlr2d_batch_create(arr, 0, C.byref(out)) == _lib.ERR_ARG
    assert lib.hodlr2d_batch_create(arr, 1, C.byref(out)) == _lib.ERR_ARG  # a null handle
    for call in (lambda: lib.hodlr2d_batch_set_form(None, 0),
                 lambda: lib.hodlr2d_batch_set_wait_limit(None, 1),
                 lambda: lib.hodlr2d_batch_set_shapes(None, 384, 64),
                 lambda: lib.hodlr2d_batch_set_blocks_per_sm(None, 3),
                 lambda: lib.hodlr2d_batch_set_placement(None, 0),
                 lambda: lib.hodlr2d_batch_check(None),
                 lambda: lib.hodlr2d_batch_persistent_recorded(None),
                 lambda: lib.hodlr2d_batch_matvec(None, None, None, None, 0),
                 lambda: lib.hodlr2d_batch_autotune(None, None, None, None, 0, 1, None),
                 lambda: lib.hodlr2d_batch_phase_ms(None, None)):
        assert call() == _lib.ERR_ARG
    assert lib.hodlr2d_batch_last_form(None) == -1
    lib.hodlr2d_batch_free(None)  # no-op
