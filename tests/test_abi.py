"""The C-ABI library loads and exports every function include/fraclap.h
declares (no GPU needed: nothing is called but the error-string getter and
argument checks that fail before touching the device)."""

import ctypes
import os
import re

import pytest

from paper_1802_03770_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(fl_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1802_03770_gb300 import build
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header():
    assert sorted(_lib.SIGNATURES) == declared_functions()


def test_invalid_arguments_fail_before_the_device(lib):
    n = (ctypes.c_int64 * 2)(8, 8)
    h = ctypes.c_void_p()
    assert lib.fl_plan_create(4, n, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    assert "d must be" in _lib.last_error()
    assert lib.fl_plan_create(2, n, 0.1, 2.5, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    assert lib.fl_plan_create(2, n, -1.0, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    bad = (ctypes.c_int64 * 2)(0, 8)
    assert lib.fl_plan_create(2, bad, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    assert lib.fl_apply(None, None, None) == _lib.FL_INVALID_ARG
    assert lib.fl_plan_destroy(None) == _lib.FL_OK
    # d = 0 and the bounds of a 1D plan
    assert lib.fl_plan_create(0, n, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    for v in (0, 4097):
        one = (ctypes.c_int64 * 1)(v)
        assert lib.fl_plan_create(1, one, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
        assert "n_i must be" in _lib.last_error()
    two = (ctypes.c_int64 * 2)(4097, 8)
    assert lib.fl_plan_create(2, two, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    three = (ctypes.c_int64 * 3)(8, 1025, 8)
    assert lib.fl_plan_create(3, three, 0.1, 1.0, None, None, ctypes.byref(h)) == _lib.FL_INVALID_ARG
    assert "d = 3" in _lib.last_error()
    # the calls added for preconditioner parameters and column tiles
    out = ctypes.c_double()
    assert lib.fl_precond_params(None, 0, 0.0, 1.0, ctypes.byref(out), ctypes.byref(out)) \
        == _lib.FL_INVALID_ARG
    tiles = (ctypes.c_int * 6)()
    assert lib.fl_plan_set_tiles(None, tiles) == _lib.FL_INVALID_ARG
    assert lib.fl_plan_autotune(None, tiles) == _lib.FL_INVALID_ARG
    assert lib.fl_net_get_tensor(None, 0, 0, None, 0) == _lib.FL_INVALID_ARG
    flags = (ctypes.c_uint8 * 2)(1, 0)
    assert lib.fl_net_set_alpha_gate(None, 0.3, 1.8, 2, flags) == _lib.FL_INVALID_ARG


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load()
