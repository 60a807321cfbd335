"""The C-ABI library builds, loads and exports every symbol include/tblr.h declares.

Host-only entry points (sizes, workspace queries, argument validation) are
exercised too; nothing here launches a kernel, so it runs without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tblr.h")


@pytest.fixture(scope="module")
def tb():
    from paper_2501_05528_gb300 import build
    build.build()
    from paper_2501_05528_gb300 import tblr
    return tblr


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(tblr_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tblr_tessellate", "tblr_test_matrices", "tblr_sketch", "tblr_decode",
                     "tblr_combine", "tblr_col", "tblr_coupling", "tblr_nearfield",
                     "tblr_compress", "tblr_compress_host", "tblr_apply"):
        assert required in names


def test_library_exports_every_declared_symbol(tb):
    handle = ctypes.CDLL(tb.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(handle, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(tb._SIGNATURES), "binding lacks a signature"


def test_sizes_and_validation_on_host(tb):
    prob = tb.make_problem(2, "laplace2d", 65536, (16, 16), (0, 0), (1, 1), k=32, p=10, e=3)
    sz = tb.tblr_sizes_of(prob)
    assert (sz.b, sz.ell, sz.r, sz.s3, sz.sketch_cols) == (256, 13, 42, 9, 2 * 13 * 42)
    prob3 = tb.make_problem(3, "laplace3d", 262144, (8, 8, 8), (0,) * 3, (1,) * 3, k=64)
    sz3 = tb.tblr_sizes_of(prob3)
    assert (sz3.b, sz3.ell, sz3.r, sz3.sketch_cols) == (512, 31, 74, 2 * 31 * 74)
    bad = tb.make_problem(2, "laplace3d", 100, (4, 4), (0, 0), (1, 1), k=4)
    with pytest.raises(tb.TblrError) as ei:
        tb.tblr_sizes_of(bad)
    assert ei.value.status == tb.TBLR_EINVAL
    assert b"laplace3d" in tb.lib().tblr_last_error()
    flat = tb.make_problem(2, "laplace2d", 100, (4, 4), (0, 0), (0, 1), k=4)
    with pytest.raises(tb.TblrError):
        tb.tblr_sizes_of(flat)
    assert tb.lib().tblr_tessellate_workspace(ctypes.byref(prob)) > 0
    assert tb.lib().tblr_compress_workspace(ctypes.byref(prob), 320) > 0
    assert tb.lib().tblr_status_string(-4) == b"workspace or capacity too small"


def test_null_arguments_are_rejected_before_any_launch(tb):
    prob = tb.make_problem(2, "laplace2d", 1000, (4, 4), (0, 0), (1, 1), k=4)
    st = tb.lib().tblr_tessellate(ctypes.byref(prob), None, None, None, 0, None)
    assert st == tb.TBLR_EINVAL
    st = tb.lib().tblr_decode(ctypes.byref(prob), None, None, None, None, None, None)
    assert st == tb.TBLR_EINVAL


def test_tile_width_tuner_validation_on_host(tb):
    """The tuner refuses non-mixed problems and missing arguments before any launch; the
    per-process width table is host state (empty: width 0, the built-in rule)."""
    lib = tb.lib()
    lib.tblr_tune_clear()
    mixed = tb.make_problem(3, "laplace3d", 2900, (3, 3, 2), (0,) * 3, (1,) * 3, k=50,
                            precision=tb.MIXED, sketch=tb.SKETCH_TAGGED)
    w = ctypes.c_int32(-1)
    assert lib.tblr_tuned_width(ctypes.byref(mixed), ctypes.byref(w)) == tb.TBLR_OK
    assert w.value == 0
    assert lib.tblr_tuned_width(ctypes.byref(mixed), None) == tb.TBLR_EINVAL
    empty = tb.LayoutStruct()
    st = lib.tblr_tune_tagged_sketch(ctypes.byref(mixed), ctypes.byref(empty), None, None, None,
                                     None, None, None, 0, ctypes.byref(w), None)
    assert st == tb.TBLR_EINVAL
    fp64 = tb.make_problem(3, "laplace3d", 2900, (3, 3, 2), (0,) * 3, (1,) * 3, k=50,
                           sketch=tb.SKETCH_TAGGED)
    st = lib.tblr_tune_tagged_sketch(ctypes.byref(fp64), ctypes.byref(empty), None, None, None,
                                     None, None, None, 0, ctypes.byref(w), None)
    assert st == tb.TBLR_EINVAL
