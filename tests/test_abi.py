"""CPU checks of the C-ABI boundary: the library loads, exports every entry point
declared in include/*.h, and the product package is independent of the oracle."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2411_09859_gb300")


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(skew_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2411_09859_gb300 import build
    build.build()
    from paper_2411_09859_gb300 import _native
    return _native.lib()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("skew_ltlt", "skew_pfaffian", "skew_rank2k", "skew_tridiag_rankk",
                     "skew_pfaffian_from_factors", "skew_ltlt_host"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    from paper_2411_09859_gb300 import _native
    assert set(_native.SIGNATURES) == set(declared_functions())


def test_host_only_queries(lib):
    assert lib.skew_version() >= 100
    assert lib.skew_default_nb(16384) in (16, 32, 64, 128)
    ws = lib.skew_workspace_bytes(16384, 64, 0)
    assert ws >= 16384 * 64 * 8
    assert lib.skew_workspace_bytes(16384, 64, 1) < ws


def test_argument_errors_before_any_device_work(lib):
    # invalid arguments are rejected before the device is touched
    assert lib.skew_ltlt(-1, None, 1, None, 1, None, None, None, 0, None, 0, None) == -1
    assert lib.skew_ltlt(4, None, 4, None, 4, None, None, None, 0, None, 0, None) == -2
    assert lib.skew_ltlt(4, 8, 3, 8, 4, 8, 8, None, 0, None, 0, None) == -3
    assert lib.skew_ltlt(4, 8, 4, 8, 4, 8, 8, None, 999, None, 0, None) == -9
    assert lib.skew_rank2k(4, 2, 1.0, None, 4, None, 4, 1.0, None, 4, None) == -4


def test_fails_loudly_without_gpu(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    # no device: the call returns SKEW_ERR_NODEVICE without touching the pointers
    st = lib.skew_ltlt(4, 8, 4, 8, 4, 8, 8, None, 0, None, 0, None)
    assert st == -104


def test_product_package_never_touches_oracle():
    for path in glob.glob(os.path.join(PKG, "**", "*"), recursive=True):
        if os.path.isfile(path) and path.endswith((".py", ".cu", ".cuh", ".h", ".c")):
            text = open(path).read()
            assert re.search(r"\b(import|from)\s+oracle\b", text) is None, path
            assert "liboracle" not in text and "skew_oracle" not in text, path


def test_oracle_never_touches_product():
    for path in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if path.endswith((".py", ".c")):
            text = open(path).read()
            assert "paper_2411_09859_gb300" not in text and "skewltlt" not in text, path
