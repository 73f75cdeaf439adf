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


def test_invalid_options_are_rejected_before_any_device_call():
    L = _lib()
    for field, bad in (("max_sweeps", 0), ("cg_max_iter", 0), ("cg_tol", 0.0), ("e_tol", -1.0)):
        o = L.mpspt_default_options()
        setattr(o, field, bad)
        with pytest.raises(L.MpsptError) as ei:
            L.mpspt_create(o)
        assert ei.value.status == L.MPSPT_ERR_INVALID, field


def test_null_arguments_are_rejected():
    L = _lib()
    lib = L.load()
    inv = L.MPSPT_ERR_INVALID
    n1 = (ctypes.c_int * 1)(4)
    assert lib.mpspt_create(None, None) == inv
    assert lib.mpspt_set_integrals(None, 2, 2, 2, None, None, 1) == inv
    assert lib.mpspt_set_reference_ci(None, None, 0) == inv
    assert lib.mpspt_set_reference(None, 0, None, None, None) == inv
    assert lib.mpspt_ground_state(None, 16, 0.0, None, None, None) == inv
    assert lib.mpspt_minimize_hylleraas(None, 0, 16, None, None, None) == inv
    assert lib.mpspt_minimize_partitioned(None, 0, 1, None, None, 1, None, None, None) == inv
    assert lib.mpspt_third_order(None, 0, None, None) == inv
    assert lib.mpspt_third_order_partitioned(None, 0, 1, None, None, 1, None, None, None,
                                             None, None, None, None) == inv
    assert lib.mpspt_local_apply(None, 0, None, 0, 0, None, None) == inv
    assert lib.mpspt_mps_shape(None, None, None) == inv
    assert lib.mpspt_mps_export(None, None, None) == inv
    assert lib.mpspt_mps_import(None, 1, None, None, None, None) == inv
    for f in (lib.mpspt_eigh_batched, lib.mpspt_eigh_batched_noalloc):
        assert f(0, None, 0, n1, None, None, None) == inv          # batch < 1
        assert f(0, None, 1, None, None, None, None) == inv        # no sizes
    assert lib.mpspt_eigh_batched_ex(0, None, 1, n1, None, None, None, 1) == inv
    out = ctypes.c_void_p()
    assert lib.mpspt_mlp_create(0, 0, 1, ctypes.byref(out)) == inv  # width < 1
    assert lib.mpspt_mlp_forward(None, 1, None, None) == inv
    assert lib.mpspt_mlp_train(None, 1, None, None, 1, 1, ctypes.c_float(1e-3), None) == inv
    assert lib.mpspt_harvest(None, 0, 16, 1, None, None, None) == inv
    assert lib.mpspt_set_preconditioner(None, None) == inv


def test_no_host_fallback_without_a_gpu():
    """Without a usable GPU the library reports a CUDA error; it never
    computes on the host instead."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = _lib()
    with pytest.raises(L.MpsptError) as ei:
        L.mpspt_create(L.mpspt_default_options())
    assert ei.value.status == L.MPSPT_ERR_CUDA
    lib = L.load()
    n1 = (ctypes.c_int * 1)(2)
    buf = (ctypes.c_double * 4)()
    st = lib.mpspt_eigh_batched(0, None, 1, n1, ctypes.cast(buf, ctypes.c_void_p),
                                ctypes.cast(buf, ctypes.c_void_p), ctypes.cast(buf, ctypes.c_void_p))
    assert st == L.MPSPT_ERR_CUDA


def test_status_constants_match_the_header():
    import re
    L = _lib()
    hdr = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mpspt.h")).read()
    vals = dict((k, int(v)) for k, v in re.findall(r"(MPSPT_(?:OK|ERR_[A-Z_]+))\s*=\s*(-?\d+)", hdr))
    assert len(vals) == 8
    for k, v in vals.items():
        assert getattr(L, k) == v, k


def test_shell_driver_fails_loudly_without_a_gpu():
    import subprocess
    import sys
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    _lib()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-m", "paper_1408_5092_gb300.cli", "--config", "tiny", "--M", "16"],
                       cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and r.stdout == ""
    assert "MpsptError" in r.stderr and "(CUDA)" in r.stderr
    bad = subprocess.run([sys.executable, "-m", "paper_1408_5092_gb300.cli", "--prec", "fp16"],
                         cwd=root, capture_output=True, text=True, timeout=300)
    assert bad.returncode == 2 and "invalid choice" in bad.stderr
