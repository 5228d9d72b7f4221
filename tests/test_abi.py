"""The C-ABI library builds, loads and exports every function include/*.h
declares (no compute call: this runs without a GPU)."""

import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"DPD_API\s+[\w\s\*]*?\b(dpd_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1911_04712_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("dpd_create", "dpd_set_state", "dpd_step", "dpd_get_state", "dpd_get_forces",
                 "dpd_get_stats", "dpd_debug_rng", "dpd_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_error_text_without_gpu(lib):
    lib.dpd_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.dpd_version()
    lib.dpd_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.dpd_last_error(), bytes)


def test_argument_errors_need_no_gpu(lib):
    """Invalid boxes are rejected before any device call."""
    import paper_1911_04712_gb300.dpd as dpd
    ctx = ctypes.c_void_p()
    bad = (ctypes.c_double * 3)(2.5, 8.0, 8.0)   # edge < 3 rc
    rc = dpd.lib().dpd_create(ctypes.byref(ctx), bad, 25.0, 4.5, 1.0, 1.0, 0.005, 0)
    assert rc == dpd.ERR_ARG
    assert b"3 rc" in dpd.lib().dpd_last_error()
    neg = (ctypes.c_double * 3)(8.0, 8.0, 8.0)
    assert dpd.lib().dpd_create(ctypes.byref(ctx), neg, -1.0, 4.5, 1.0, 1.0, 0.005, 0) == dpd.ERR_ARG
    assert dpd.lib().dpd_create(ctypes.byref(ctx), neg, 25.0, 4.5, 1.0, 1.0, 0.0, 0) == dpd.ERR_ARG
    assert dpd.lib().dpd_create(None, neg, 25.0, 4.5, 1.0, 1.0, 0.005, 0) == dpd.ERR_ARG
    # a box whose cell list (2 x-slices per cell) exceeds one scan's 2^26 - 1 entries
    huge = (ctypes.c_double * 3)(400.0, 400.0, 400.0)
    assert dpd.lib().dpd_create(ctypes.byref(ctx), huge, 25.0, 4.5, 1.0, 1.0, 0.005, 0) == dpd.ERR_ARG
    assert b"too many cells" in dpd.lib().dpd_last_error()
    fits = (ctypes.c_double * 3)(300.0, 300.0, 300.0)   # 5.4e7 entries
    rc = dpd.lib().dpd_create(ctypes.byref(ctx), fits, 25.0, 4.5, 1.0, 1.0, 0.005, 0)
    assert rc != dpd.ERR_ARG
    if rc == dpd.OK:
        dpd.lib().dpd_destroy(ctx)


def test_product_path_refuses_without_library(tmp_path, monkeypatch):
    """No CPU fallback: a missing library is an import-time error."""
    import paper_1911_04712_gb300.dpd as dpd
    monkeypatch.setattr(dpd, "_lib", None)
    monkeypatch.setattr(dpd, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        dpd.lib()


def test_tuning_tables_need_no_gpu(lib):
    """Four tables (stencil x single/packed), set and read back on the host;
    setting one leaves the others alone; bad tables are rejected."""
    import paper_1911_04712_gb300.batch as B
    import paper_1911_04712_gb300.dpd as dpd
    saved = [B.tuning_get(t) for t in range(4)]
    try:
        B.tuning_set(3, [4.0, 1e9], [12, 2])
        B.tuning_set(1, [1e9], [5])
        assert B.tuning_get(3) == ([4.0, 1e9], [12, 2])
        assert B.tuning_get(1) == ([1e9], [5])
        for bad in ((4, [1e9], [0]), (1, [2.0, 1.0], [0, 0]), (0, [1e9], [B.NUM_FORCE_VARIANTS])):
            with pytest.raises(dpd.DPDError) as ei:
                B.tuning_set(*bad)
            assert ei.value.code == dpd.ERR_ARG
    finally:
        for t, (up, var) in enumerate(saved):
            B.tuning_set(t, up, var)


def test_default_library_is_philox_r10(lib):
    lib.dpd_philox_rounds.restype = ctypes.c_int
    assert lib.dpd_philox_rounds() == 10
    lib.dpd_version.restype = ctypes.c_char_p
    assert b"Philox-4x32-10" in lib.dpd_version()

