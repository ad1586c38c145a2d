"""The C-ABI library loads and exports every entry point declared in include/sfc.h (no GPU
needed: only symbol lookup and host-only calls)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "sfc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sfc_[a-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libsfc():
    from paper_2508_19891_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["sfc_build", "sfc_query_batch", "sfc_update", "sfc_query_count",
                     "sfc_query_write", "sfc_train_model", "sfc_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libsfc):
    missing = [n for n in declared_functions() if not hasattr(libsfc, n)]
    assert not missing, missing


def test_host_only_calls(libsfc):
    import paper_2508_19891_gb300 as sfc
    assert sfc.sfc_status_string(0) == "SFC_OK"
    assert sfc.sfc_status_string(-4) == "SFC_ERR_NOT_FOUND"
    o = sfc.sfc_default_options()
    assert o.leaves == 4096 and o.bounds == 0
    assert sfc.sfc_model_hidden() == 16
    # invalid arguments are rejected on the host before anything touches a device
    L = sfc.lib()
    assert L.sfc_build(None, None, 0, 0, None, None) == sfc.SFC_ERR_INVALID
    h = ctypes.c_void_p()
    assert L.sfc_build(ctypes.byref(h), None, 5, 0, None, None) == sfc.SFC_ERR_INVALID
    assert L.sfc_build(ctypes.byref(h), None, 0, 7, None, None) == sfc.SFC_ERR_INVALID
    assert L.sfc_query_count(None, None, None, 0, None, None) == sfc.SFC_ERR_INVALID
