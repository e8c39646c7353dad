"""The C ABI library builds, loads and exports every symbol include/pct.h declares.

CPU only: no call here touches a GPU.
"""
import ctypes
import os
import re

import pytest

import paper_1802_01070_b300 as pct
from paper_1802_01070_b300 import build as pct_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pct_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    pct_build.build()
    return pct.load_library()


def test_header_declares_the_binding_surface():
    assert set(_declared()) == set(pct.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(pct.LIB_PATH)
    for name in _declared():
        assert hasattr(raw, name), name


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument checks run before any CUDA call
    assert lib.pct_create(None, None, None, 0, None) == pct.PCT_ERR_ARG
    assert b"null" in lib.pct_last_error(None)
    assert lib.pct_solve(None, 1, 0.5, 10, None) == pct.PCT_ERR_ARG
    assert lib.pct_synchronize(None) == pct.PCT_ERR_ARG
    lib.pct_destroy(None)


def test_invalid_grid_is_rejected(lib):
    h = ctypes.c_void_p()
    g = pct.pct_grid(0, 4, 4, 1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.pct_create(ctypes.byref(h), ctypes.byref(g), None, 0, None) == pct.PCT_ERR_ARG
    g = pct.pct_grid(4, 4, 4, -1.0, 1.0, 1.0, 0.0, 0.0, 0.0)
    assert lib.pct_create(ctypes.byref(h), ctypes.byref(g), None, 0, None) == pct.PCT_ERR_ARG
    assert not h.value
