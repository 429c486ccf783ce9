"""The C ABI library: it builds, loads, exports every declared entry point,
and rejects invalid shapes before touching a GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "firls.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(firls_[a-z_A-Z0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1411_5057_gb300 import build as B
    if not os.path.exists(B.LIB) and not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("nvcc not available to build libfirls.so")
    B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("firls_create", "firls_set_operator", "firls_solve", "firls_destroy", "firls_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1411_5057_gb300 import binding
    assert sorted(binding.EXPORTED) == declared_functions()


def test_supported_sizes(lib):
    lib.firls_size_supported.restype = ctypes.c_int
    ok = [n for n in range(8, 600) if lib.firls_size_supported(n)]
    assert ok == [16, 32, 48, 64, 80, 96, 128, 160, 192, 256, 320, 384, 512]


def test_invalid_shapes_rejected_without_device_work(lib):
    h = ctypes.c_void_p()
    f = lib.firls_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    assert f(ctypes.byref(h), 100, 100, 1, 0, None) == 2      # FIRLS_E_SHAPE: no FFT plan
    assert f(ctypes.byref(h), 64, 128, 1, 0, None) == 2       # not square
    assert f(ctypes.byref(h), 64, 64, 0, 0, None) == 1        # empty batch
    assert f(None, 64, 64, 1, 0, None) == 1
    assert h.value is None


def test_dense_shapes_rejected_without_device_work(lib):
    """firls_dense_create checks its shape before any CUDA call: N a multiple
    of 4 in [4, 8192], M >= 1, 1 <= problems <= 65535 and P M int-sized."""
    h = ctypes.c_void_p()
    f = lib.firls_dense_create
    f.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_void_p]
    f.restype = ctypes.c_int
    for M, N, P in ((0, 8, 1), (10, 6, 1), (10, 0, 1), (10, 8196, 1), (10, 8, 0), (10, 8, 65536),
                    (40000, 8, 60000)):
        assert f(ctypes.byref(h), M, N, P, 1, None) == 2, (M, N, P)      # FIRLS_E_SHAPE
        assert h.value is None
    assert f(None, 10, 8, 1, 0, None) == 1                              # FIRLS_E_INVALID_ARG
