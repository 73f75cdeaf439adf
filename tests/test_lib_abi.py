"""The C-ABI library builds, loads and exports every entry point declared in
include/mpspt.h (no compute calls: this runs without a GPU)."""
import ctypes
import os

import pytest


def _lib():
    from paper_1408_5092_gb300 import _lib as L
    if not os.path.exists(L.LIB_PATH):
        from paper_1408_5092_gb300.build import build
        build()
    return L


def test_every_declared_symbol_is_exported():
    L = _lib()
    lib = L.load()
    declared = L.declared_symbols()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name


def test_default_options_are_host_only():
    L = _lib()
    o = L.mpspt_default_options()
    assert o.prec == L.MPSPT_FP64
    assert o.max_sweeps == 30
    assert o.cg_tol == 1e-10 and o.e_tol == 1e-10
    assert o.seed == 1408


def test_status_strings():
    L = _lib()
    for st in range(-7, 1):
        assert isinstance(L.mpspt_status_string(st), str)
