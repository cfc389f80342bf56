"""The C ABI library builds, loads, and exports every entry point include/lfmm.h declares.

CPU only: nothing here launches a kernel."""
import ctypes
import re

import numpy as np

import pytest

from paper_1105_3505_gb300 import build, lfmm


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lfmm.load()


def _declared_symbols():
    text = open(lfmm.HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lfmm_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_core_api():
    names = _declared_symbols()
    for required in ["lfmm_plan_create", "lfmm_eval", "lfmm_plan_destroy", "lfmm_eval_parts",
                     "lfmm_plan_get_info", "lfmm_status_string", "lfmm_last_error", "lfmm_opts_default"]:
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_defaults(lib):
    assert lfmm.lfmm_status_string(0) == "ok"
    assert lfmm.lfmm_status_string(lfmm.LFMM_EINVAL) == "invalid argument"
    o = lfmm.lfmm_opts_default()
    assert (o.precision, o.p, o.leaf_size, o.max_leaf_side, o.proxies_per_edge, o.tc_min_level) == \
        (lfmm.LFMM_MIXED, 8, 64, 32, 64, 0)
    assert (o.m2l_tile, o.m2l_stages, o.m2l_split, o.reserved) == (0, 0, 0, 0)
    assert ctypes.sizeof(lfmm.lfmm_opts) == 48


def test_invalid_arguments_rejected_without_gpu(lib):
    h = ctypes.c_void_p(123)
    # NULL coordinates are rejected before any CUDA call
    st = lib.lfmm_plan_create(ctypes.byref(h), None, 4, None, 4, None, None)
    assert st == lfmm.LFMM_EINVAL and h.value is None
    assert "NULL" in lfmm.lfmm_last_error()
    assert lib.lfmm_plan_destroy(None) == lfmm.LFMM_OK
    with pytest.raises(lfmm.LfmmError):
        lfmm.lfmm_phi_table(0)


def test_forest_offsets_validated_without_gpu(lib):
    h = ctypes.c_void_p(123)
    pts = np.zeros((4, 2), dtype=np.int32)
    so = np.array([0, 2, 2, 4], dtype=np.int64)  # problem 1 has no sources
    to = np.array([0, 1, 2, 4], dtype=np.int64)
    st = lib.lfmm_forest_create(ctypes.byref(h), pts.ctypes.data, so.ctypes.data, pts.ctypes.data,
                                to.ctypes.data, 3, None, None)
    assert st == lfmm.LFMM_EINVAL and h.value is None
    assert "problem 1" in lfmm.lfmm_last_error()
    so = np.array([1, 2, 4], dtype=np.int64)  # does not start at 0
    st = lib.lfmm_forest_create(ctypes.byref(h), pts.ctypes.data, so.ctypes.data, pts.ctypes.data,
                                to.ctypes.data, 2, None, None)
    assert st == lfmm.LFMM_EINVAL
    o = lfmm.make_opts(tree=7)
    st = lib.lfmm_plan_create(ctypes.byref(h), pts.ctypes.data, 4, pts.ctypes.data, 4, ctypes.byref(o), None)
    assert st == lfmm.LFMM_EINVAL and "opts.tree" in lfmm.lfmm_last_error()


def test_opts_flags_validated_without_gpu(lib):
    h = ctypes.c_void_p(123)
    pts = np.zeros((4, 2), dtype=np.int32)
    o = lfmm.make_opts()
    o.flags = 8  # unknown bit
    st = lib.lfmm_plan_create(ctypes.byref(h), pts.ctypes.data, 4, pts.ctypes.data, 4, ctypes.byref(o), None)
    assert st == lfmm.LFMM_EINVAL and "flags" in lfmm.lfmm_last_error()
    assert lfmm.make_opts(graph=True).flags == lfmm.LFMM_FLAG_GRAPH
    # the M2L tiling fields are validated too
    for field, bad in (("m2l_tile", 48), ("m2l_stages", 5), ("m2l_split", 10), ("reserved", 1)):
        o = lfmm.make_opts()
        setattr(o, field, bad)
        st = lib.lfmm_plan_create(ctypes.byref(h), pts.ctypes.data, 4, pts.ctypes.data, 4, ctypes.byref(o), None)
        assert st == lfmm.LFMM_EINVAL and field in lfmm.lfmm_last_error()


def test_autotune_arguments_validated_without_gpu(lib):
    pts = np.zeros((4, 2), dtype=np.int32)
    r = lfmm.lfmm_tune_result()
    for tol in (0.0, 1e-14, 0.5, float("nan")):
        st = lib.lfmm_autotune(pts.ctypes.data, 4, None, pts.ctypes.data, 4, None, 1, tol, None, ctypes.byref(r), None)
        assert st == lfmm.LFMM_EINVAL and "tol" in lfmm.lfmm_last_error()
    so = np.array([0, 4], dtype=np.int64)
    st = lib.lfmm_autotune(pts.ctypes.data, 4, so.ctypes.data, pts.ctypes.data, 4, None, 1, 1e-6, None,
                           ctypes.byref(r), None)
    assert st == lfmm.LFMM_EINVAL


def test_tune_cache_roundtrip_without_gpu(lib, tmp_path):
    lfmm.tune_cache_clear()
    good = tmp_path / "tune.txt"
    good.write_text("lfmm-tune-2 1 -6 20 20 0 0 7 64 7 2.500000e-07 4.100000e-01 32 4 0\n"
                    "lfmm-tune-2 2 -10 17 15 0 0 14 128 0 3.000000e-12 2.000000e+00 0 0 3\n")
    lfmm.tune_cache_load(str(good))
    out = tmp_path / "out.txt"
    lfmm.tune_cache_save(str(out))
    lines = sorted(out.read_text().splitlines())
    assert lines == sorted(good.read_text().splitlines())
    # a version-1 line (no M2L tiling) loads with the library's tiling rules
    old = tmp_path / "old.txt"
    old.write_text("lfmm-tune-1 1 -6 22 22 0 0 8 64 7 2.500000e-07 4.100000e-01\n")
    lfmm.tune_cache_clear()
    lfmm.tune_cache_load(str(old))
    lfmm.tune_cache_save(str(out))
    assert out.read_text().split() == "lfmm-tune-2 1 -6 22 22 0 0 8 64 7 2.500000e-07 4.100000e-01 0 0 0".split()
    for line in ["lfmm-tune-1 1 -6 20 20 0 0 99 64 7 1e-7 1.0\n",  # p out of range
                 "lfmm-tune-2 1 -6 20 20 0 0 7 64 7 1e-7 1.0 48 0 0\n",  # tile width not allowed
                 "lfmm-tune-2 1 -6 20 20 0 0 7 64 7 1e-7 1.0 0 5 0\n"]:  # ring depth out of range
        bad = tmp_path / "bad.txt"
        bad.write_text(line)
        with pytest.raises(lfmm.LfmmError, match="line 1"):
            lfmm.tune_cache_load(str(bad))
    lfmm.tune_cache_clear()
    lfmm.tune_cache_save(str(out))
    assert out.read_text() == ""


def test_phi_quadrature_arguments_validated_without_gpu(lib):
    for offsets, weights, R in [([[2, 0], [0, 2]], [1.0, 1.0], 4),   # does not connect the lattice
                                ([[1, 0], [0, 1]], [1.0, -1.0], 4),  # negative conductivity
                                ([[1, 0], [0, 1]], [1.0, 1.0], 65),  # radius out of range
                                ([[0, 0], [0, 1]], [1.0, 1.0], 4),   # zero offset
                                ([[1, 0], [0, 1]], [1.0, 1000.0], 4)]:  # too anisotropic
        with pytest.raises(lfmm.LfmmError):
            lfmm.lfmm_phi_quadrature(offsets, weights, R)
