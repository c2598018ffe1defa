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


def declared_arity():
    """Number of parameters of each prototype in include/*.h (comments removed)."""
    arity = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(skew_\w+)\s*\(([^;{]*?)\)\s*;", text):
            args = m.group(2).strip()
            arity[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return arity


def test_binding_argument_counts_match_the_header():
    from paper_2411_09859_gb300 import _native
    arity = declared_arity()
    assert set(arity) == set(_native.SIGNATURES)
    wrong = {name: (len(_native.SIGNATURES[name][0]), n) for name, n in arity.items()
             if len(_native.SIGNATURES[name][0]) != n}
    assert not wrong, wrong


def test_host_only_queries(lib):
    assert lib.skew_version() >= 100
    assert lib.skew_default_nb(16384) in (16, 32, 48, 64, 96, 128)
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


def test_nb_table_install_and_reset():
    """The panel-width table of the autotuner (host-only functions, no device work)."""
    import paper_2411_09859_gb300 as skew
    lib = skew.lib()
    before = [skew.default_nb(n) for n in (100, 1000, 5000, 20000)]
    try:
        skew.set_nb_table([(1000, 24), (8000, 48), (16384, 96)])
        assert [skew.default_nb(n) for n in (100, 1000, 1001, 8000, 9000, 16384, 50000)] == \
            [24, 24, 48, 48, 96, 96, 96]
        with pytest.raises(skew.SkewError):
            skew.set_nb_table([(1000, 24), (900, 48)])       # not increasing
        with pytest.raises(skew.SkewError):
            skew.set_nb_table([(1000, 0)])                   # bad width
        skew.set_nb_table([])
        assert [skew.default_nb(n) for n in (100, 1000, 5000)] == [16, 32, 64]
        skew.set_nb_table([(1000, 24, 0), (8000, 48, 1), (16384, 64, -1)])
        assert [skew.default_nb(n) for n in (100, 5000, 9000)] == [24, 48, 64]
        with pytest.raises(skew.SkewError):
            skew.set_nb_table([(1000, 24, 2)])                # bad path choice
        skew.set_nb_table([])
    finally:
        from paper_2411_09859_gb300 import autotune
        if not autotune.load():
            skew.set_nb_table([])
    assert [skew.default_nb(n) for n in (100, 1000, 5000, 20000)] == before
    assert lib.skew_set_nb_table(-1, None, None) == -1


def test_autotune_pick_rule():
    from paper_2411_09859_gb300 import autotune
    assert autotune.pick({"32": 10.0, "64": 9.99, "96": 9.98}) == 32      # all within 0.5 %
    assert autotune.pick({"32": 10.0, "64": 9.0, "96": 8.99}) == 64
    assert autotune.table_from_ms({"4096": {"32": 1.0, "64": 2.0}, "512": {"16": 3.0, "32": 1.0}}) == \
        [(512, 32, 0), (4096, 32, 0)]
    # the look-ahead is taken only when it is faster by more than the tie margin
    assert autotune.pick_path({"32": 10.0, "32+la": 9.99, "64": 10.2}) == (32, 0)
    assert autotune.pick_path({"32": 10.0, "32+la": 9.0, "64+la": 8.99, "64": 9.5}) == (32, 1)
    assert autotune.pick_path({"32": 10.0, "64+la": 8.0, "64": 9.5}) == (64, 1)


def test_batched_nb_table():
    import paper_2411_09859_gb300 as skew
    from paper_2411_09859_gb300 import autotune
    try:
        skew.set_batched_nb_table([(64, 8), (256, 16), (512, 32)])
        assert [skew.batched_nb(n) for n in (10, 64, 65, 256, 300, 600)] == [8, 8, 16, 16, 32, 32]
        with pytest.raises(skew.SkewError):
            skew.set_batched_nb_table([(64, 12)])
        skew.set_batched_nb_table([])
        assert skew.batched_nb(100) == 16 and skew.batched_warp_tile(100) == 32
        skew.set_batched_nb_table([(64, 8, 16), (256, 16, 32), (512, 32, 16)])
        assert [skew.batched_warp_tile(n) for n in (10, 65, 300, 600)] == [16, 32, 16, 16]
        assert [skew.batched_nb(n) for n in (10, 65, 300)] == [8, 16, 32]
        with pytest.raises(skew.SkewError):
            skew.set_batched_nb_table([(64, 8, 24)])
    finally:
        if not autotune.load():
            skew.set_batched_nb_table([])
