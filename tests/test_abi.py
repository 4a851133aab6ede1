"""The C-ABI library builds, loads and exports every entry point that
include/mppi.h declares (no device work: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mppi.h")


@pytest.fixture(scope="module")
def lib_path():
    from paper_2509_14726_gb300 import _build
    return _build.build()


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mppi_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("mppi_create", "mppi_solve", "mppi_solve_batch", "mppi_solve_async", "mppi_destroy"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(mppi_[a-z0-9_]+)$", out, flags=re.M))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(lib_path)
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_binding_struct_layout_matches_the_library(lib_path):
    from paper_2509_14726_gb300 import mppi
    L = mppi.load()
    sizes = (ctypes.c_size_t * 3)()
    assert L.mppi_abi_sizes(sizes) == 0
    assert list(sizes) == [ctypes.sizeof(mppi.Model), ctypes.sizeof(mppi.Params), ctypes.sizeof(mppi.TrackC)]


def test_library_defaults_match_the_python_defaults(lib_path):
    from paper_2509_14726_gb300 import mppi, workloads as W
    L = mppi.load()
    m = mppi.Model()
    p = mppi.Params()
    assert L.mppi_default_model(ctypes.byref(m)) == 0
    assert L.mppi_default_params(ctypes.byref(p), 0, 256, 20, 0.05) == 0
    mref = mppi.make_model(W.ModelConfig())
    pref = mppi.make_params(W.SolveConfig())
    for name, _ in mppi.Model._fields_:
        np.testing.assert_allclose(np.array(getattr(m, name)).ravel() if not isinstance(getattr(m, name), (int, float)) else getattr(m, name),
                                   np.array(getattr(mref, name)).ravel() if not isinstance(getattr(mref, name), (int, float)) else getattr(mref, name), rtol=1e-6)
    for name, _ in mppi.Params._fields_:
        a, b = getattr(p, name), getattr(pref, name)
        a = list(a) if hasattr(a, "__len__") else a
        b = list(b) if hasattr(b, "__len__") else b
        np.testing.assert_allclose(a, b, rtol=1e-6, err_msg=name)


def test_error_paths_need_no_device(lib_path):
    from paper_2509_14726_gb300 import mppi
    L = mppi.load()
    assert L.mppi_create(None, None, None, None) == mppi.MPPI_ERR_ARG
    h = ctypes.c_void_p()
    m, p = mppi.Model(), mppi.Params()
    L.mppi_default_model(ctypes.byref(m))
    L.mppi_default_params(ctypes.byref(p), 0, 0, 20, 0.05)  # K = 0
    t = mppi.TrackC()
    assert L.mppi_create(ctypes.byref(m), ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == mppi.MPPI_ERR_ARG
    assert b"K=0" in L.mppi_last_error()
    m.kind = 1
    L.mppi_default_params(ctypes.byref(p), 0, 16, 20, 0.05)
    assert L.mppi_create(ctypes.byref(m), ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == mppi.MPPI_ERR_ARG
    m.kind = 0
    p.samples_per_thread = 9
    assert L.mppi_create(ctypes.byref(m), ctypes.byref(p), ctypes.byref(t), ctypes.byref(h)) == mppi.MPPI_ERR_ARG
    assert b"samples_per_thread" in L.mppi_last_error()
    assert L.mppi_solve(None, None, 0.0, None, None) == mppi.MPPI_ERR_ARG
    assert L.mppi_destroy(None) == 0
    # empty and malformed batches are refused before any device work
    b = ctypes.c_void_p()
    hs = (ctypes.c_void_p * 2)()
    assert L.mppi_batch_create(0, hs, 1, ctypes.byref(b)) == mppi.MPPI_ERR_ARG
    assert L.mppi_batch_create(2, hs, 1, ctypes.byref(b)) == mppi.MPPI_ERR_ARG  # null handles
    assert b"null handle" in L.mppi_last_error()
    x = (ctypes.c_float * 13)()
    t = (ctypes.c_double * 1)()
    u = (ctypes.c_float * 5)()
    assert L.mppi_solve_batch(0, hs, x, t, None, u) == mppi.MPPI_ERR_ARG
    assert L.mppi_batch_destroy(None) == 0


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2509_14726_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.replace("Oracle", "oracle").split("#")[0] or f == "workloads.py" or \
                    "import oracle" not in txt and "from oracle" not in txt, f
