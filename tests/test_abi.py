"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/gs.h declares; the Python binding wraps exactly those names."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2604_02120_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_hot_path_calls():
    names = _declared()
    for n in ("gs_project", "gs_bin_sort", "gs_blend_forward", "gs_blend_backward"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2604_02120_gb300 import gs
    assert sorted(gs.ABI_FUNCTIONS) == _declared()


def test_host_only_calls_without_gpu(lib):
    lib.gs_status_string.restype = ctypes.c_char_p
    assert lib.gs_status_string(4) == b"device wait timed out"
    lib.gs_version.restype = ctypes.c_int32
    assert lib.gs_version() >= 100
    size = ctypes.c_size_t(0)
    lib.gs_bin_sort_workspace_size.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                               ctypes.POINTER(ctypes.c_size_t)]
    assert lib.gs_bin_sort_workspace_size(1000, 5000, 64, 48, ctypes.byref(size)) == 0
    assert size.value > 5000 * 16
    assert lib.gs_bin_sort_workspace_size(-1, 5000, 64, 48, ctypes.byref(size)) == 1
    assert lib.gs_bin_sort_workspace_size(10, 1 << 32, 64, 48, ctypes.byref(size)) == 1
