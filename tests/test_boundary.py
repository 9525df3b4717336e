"""The C-ABI library builds, loads and exports every symbol that include/gwas.h declares."""
import ctypes
import os
import re

import pytest

from paper_1210_7683_gb300 import build as gbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return gbuild.build()


def declared_functions():
    with open(os.path.join(ROOT, "include", "gwas.h")) as f:
        src = f.read()
    return re.findall(r"GWAS_API\s+[\w\s\*]+?\b(gwas_\w+)\s*\(", src)


def test_header_declares_the_api():
    names = declared_functions()
    for need in ("gwas_setup", "gwas_load_snps", "gwas_solve", "gwas_last_error", "gwas_destroy"):
        assert need in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_names_match_the_header():
    import paper_1210_7683_gb300 as g
    for name in declared_functions():
        assert callable(getattr(g, name)), name


def test_status_codes_parsed():
    import paper_1210_7683_gb300 as g
    assert g.GWAS_OK == 0 and g.GWAS_ERR_SINGULAR_PAIRS == 6 and g.GWAS_MIXED == 1


def test_argument_errors_without_gpu(libpath):
    # argument checks run before any device work, so they answer on a CPU-only host too
    lib = ctypes.CDLL(libpath)
    ctx = ctypes.c_void_p()
    rc = lib.gwas_setup(ctypes.byref(ctx), 0, 3, None, None, 1, None, None)
    assert rc == 1  # GWAS_ERR_ARG
    lib.gwas_last_error.restype = ctypes.c_char_p
    assert b"n = 0" in lib.gwas_last_error(None)
    rc = lib.gwas_setup(ctypes.byref(ctx), 100, 20, None, None, 1, None, None)
    assert rc == 8  # GWAS_ERR_UNSUPPORTED: p = 21 is above the paper's range 2 <= p <= 20
    assert b"[0, 19]" in lib.gwas_last_error(None)
    rc = lib.gwas_solve(None, None, 0, 0, None)
    assert rc == 1
    # the streaming entry points reject a missing context before any device work
    lib.gwas_solve_ooc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gwas_solve_ooc(None, 10, None, 0, None, 1, None, None, None, None) == 1
    lib.gwas_solve_stream.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gwas_solve_stream(None, None, 0, 0, 1, None, None, None, None) == 1

    # the autotuner and the introspection calls too
    lib.gwas_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    assert lib.gwas_autotune(None, None, 0, 0, None) == 1
    shape = (ctypes.c_int * 5)()
    lib.gwas_tune_shape.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gwas_tune_shape(None, shape) == 1
    lib.gwas_serve_stats.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert lib.gwas_serve_stats(None, None, None) == 1


def test_binding_refuses_arrays_too_small_for_the_call(monkeypatch):
    # the binding records each context's n, p, t and output mode at setup and refuses an array
    # smaller than what a call reads or writes, before the C call (which trusts pointers)
    import numpy as np
    import paper_1210_7683_gb300 as g
    fake = 0x5EED
    n, p, t = 100, 4, 7
    monkeypatch.setitem(g._CTX, fake, (n, p, t, g.GWAS_OUT_LAST_SE))
    Y = np.zeros((t, n))
    cases = [
        lambda: g.gwas_solve(fake, Y, 0, 10, np.zeros((2, t, 9), np.float32)),      # one SNP short
        lambda: g.gwas_solve(fake, Y[:6], 0, 10, np.zeros((2, t, 10), np.float32)),  # one trait short
        lambda: g.gwas_solve(fake, Y, 5, 20, np.zeros((2, t, 10), np.float32)),     # range wider than out
        lambda: g.gwas_load_snps(fake, 50, np.zeros((49, n), np.int8)),
        lambda: g.gwas_submit(fake, np.zeros((3, n)), 4, np.zeros(4), 0, 8, np.zeros((2, 4, 8), np.float32)),
        lambda: g.gwas_submit(fake, np.zeros((4, n)), 4, np.zeros(4), 0, 8, np.zeros((2, 4, 7), np.float32)),
    ]
    for call in cases:
        with pytest.raises(ValueError):
            call()
    # full coefficient vectors: p doubles per pair, so a float32 array of the LAST_SE size is short
    monkeypatch.setitem(g._CTX, fake, (n, p, t, g.GWAS_OUT_FULL_B))
    with pytest.raises(ValueError):
        g.gwas_solve(fake, Y, 0, 10, np.zeros((2, t, 10), np.float32))
    with pytest.raises(ValueError):
        g.gwas_solve(fake, Y, 0, 10, np.zeros((t, 10, p - 1)))
