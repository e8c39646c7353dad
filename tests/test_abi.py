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


def test_binding_constants_match_the_header():
    """Every PCT_* constant the binding defines has the header's value, and
    every option and statistic the header defines is in the binding."""
    src = open(os.path.join(ROOT, "include", "pct.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    header = {k: int(v) for k, v in re.findall(r"\b(PCT_[A-Z0-9_]+)\s*=\s*(-?\d+)", src)}
    header.update({k: int(v) for k, v in re.findall(r"#define\s+(PCT_[A-Z0-9_]+)\s+(-?\d+)", src)})
    # implicitly numbered enumerators (status codes) follow their predecessor
    for body in re.findall(r"enum\s*\w*\s*\{(.*?)\}", src, flags=re.S):
        value = -1
        for item in body.split(","):
            m = re.match(r"\s*(PCT_[A-Z0-9_]+)\s*(?:=\s*(-?\d+))?\s*$", item)
            if not m:
                continue
            value = int(m.group(2)) if m.group(2) is not None else value + 1
            header[m.group(1)] = value
    binding = {k: v for k, v in vars(pct).items() if k.startswith("PCT_") and isinstance(v, int)}
    assert binding, "no constants in the binding"
    for k, v in binding.items():
        assert k in header, k
        assert header[k] == v, (k, header[k], v)
    for k in header:
        if k.startswith(("PCT_OPT_", "PCT_STAT_")):
            assert k in binding, k
