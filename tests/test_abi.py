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
    assert ctypes.sizeof(lfmm.lfmm_opts) == 32


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
