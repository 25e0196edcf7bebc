"""C ABI checks that need no GPU: the library loads, exports every function
that include/*.h declares, validates arguments on the host and documents its
layout; the product package does not reach the oracle."""
import ctypes
import os
import re

import pytest

from paper_1008_2801_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_exports_every_declared_symbol():
    L = _lib.load()
    declared = _lib.header_symbols()
    assert len(declared) >= 25
    for name in sorted(declared):
        assert hasattr(L, name), name
    # and the binding declares a signature for each
    assert declared == set(_lib._SIGS)


def test_default_opts_and_error_strings():
    L = _lib.load()
    o = _lib.mg_opts()
    L.mg_default_opts(ctypes.byref(o))
    assert (o.precision, o.nu1, o.nu2, o.max_cycles, o.use_graph, o.smoother) == (0, 2, 2, 100, 1, 0)
    for code, name in _lib.STATUS_NAMES.items():
        assert L.mg_error_string(code)
    assert L.mg_error_string(99) == b"unknown status"


def test_host_side_argument_checks():
    L = _lib.load()
    n = _lib.c_int3(8, 8, 8)
    assert L.mg_create(None, n, 0.1, 0, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_set_beta(None, None, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_solve(None, None, None, 1e-10, None, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_adjoint(None, 1, None, None, None, None, 1e-10, None, None) == \
        _lib.MG_ERR_INVALID_ARG
    assert L.mg_solve_batched(None, None, None, 1e-10, None, None) == _lib.MG_ERR_INVALID_ARG
    bad = _lib.c_int3(0, 8, 8)
    P = ctypes.c_longlong()
    assert L.mg_layout(bad, ctypes.byref(P), None, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_op_rbgs_pass(0, n, None, None, None, None, None, None, 0, None) == \
        _lib.MG_ERR_INVALID_ARG
    assert L.mg_op_rbgs_pass(5, n, *([ctypes.c_void_p(16)] * 6), 0, None) == \
        _lib.MG_ERR_INVALID_ARG
    assert L.mg_last_error()
    # wall masks outside 0..511, or periodic axes with a Neumann bit, are
    # rejected before any device work
    h = ctypes.c_void_p()
    for bc in (-1, 512, 1000, 64 | 1, 128 | 8, 256 | 48):
        assert L.mg_create(ctypes.byref(h), n, 0.1, bc, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_bc_lift(None, None, None, None, None) == _lib.MG_ERR_INVALID_ARG
    assert L.mg_op_face_weights(n, 0.1, 64, *([ctypes.c_void_p(16)] * 4), None) == \
        _lib.MG_ERR_INVALID_ARG


def test_wall_mask_parsing():
    from paper_1008_2801_gb300.solver import bc_mask, wall_shapes
    assert bc_mask(0) == 0 and bc_mask("DDDDDD") == 0
    assert bc_mask("NNNNNN") == 63
    assert bc_mask("NDDDDN") == 1 | 32
    assert bc_mask("dndndn") == 2 | 8 | 32
    assert bc_mask("PPDNPP") == 64 | 8 | 256
    for bad in ("DDDDD", "DDDDDX", "PDDDDD", 512, -1, 64 | 2):
        with pytest.raises(ValueError):
            bc_mask(bad)
    assert wall_shapes((4, 5, 6)) == [(4, 5), (4, 5), (4, 6), (4, 6), (5, 6), (5, 6)]


@pytest.mark.parametrize("n", [(1, 1, 1), (7, 5, 3), (64, 64, 64), (48, 128, 96)])
def test_layout_formula(n):
    L = _lib.load()
    P, Q, E = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    assert L.mg_layout(_lib.c_int3(*n), ctypes.byref(P), ctypes.byref(Q), ctypes.byref(E)) == 0
    nx, ny, nz = n
    assert P.value == (nx + 1 + 7) // 8 * 8
    assert Q.value == P.value * (ny + 1)
    assert E.value == Q.value * (nz + 2)


def test_product_never_reaches_the_oracle():
    pkg = os.path.join(ROOT, "paper_1008_2801_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, fn)).read()
                hit = re.search(r"(import\s+oracle|from\s+oracle|liboracle|oracle\.\w+\(|oracle/)", txt)
                assert not hit, os.path.join(dirpath, fn)


def test_oracle_shares_no_code_with_the_product():
    for fn in os.listdir(os.path.join(ROOT, "oracle")):
        if fn.endswith((".py", ".c", ".h")):
            txt = open(os.path.join(ROOT, "oracle", fn)).read()
            assert "paper_1008_2801_gb300" not in txt
            assert "mg.h" not in txt
