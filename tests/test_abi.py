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
    assert L.sfc_build(None, None, 0, 0, None, None, None) == sfc.SFC_ERR_INVALID
    h = ctypes.c_void_p()
    assert L.sfc_build(ctypes.byref(h), None, 5, 0, None, None, None) == sfc.SFC_ERR_INVALID
    assert L.sfc_build(ctypes.byref(h), None, 0, 7, None, None, None) == sfc.SFC_ERR_INVALID
    assert L.sfc_query_count(None, None, None, 0, None, None) == sfc.SFC_ERR_INVALID
    assert L.sfc_set_tuning(None, 1024, 4, 8) == sfc.SFC_ERR_INVALID
    # an allocator must bring both callbacks (checked before any device work)
    half = sfc.sfc_allocator()
    half.alloc = sfc.SFC_ALLOC_FN(lambda n, s, c: None)
    assert L.sfc_build(ctypes.byref(h), None, 0, 0, None, ctypes.byref(half), None) == sfc.SFC_ERR_INVALID
    assert L.sfc_build_host(ctypes.byref(h), None, 0, 0, None, ctypes.byref(half), None) == sfc.SFC_ERR_INVALID
    assert L.sfc_build3(ctypes.byref(h), None, 0, None, ctypes.byref(half), None) == sfc.SFC_ERR_INVALID


def test_build_signatures_take_an_allocator():
    """sfc_build, sfc_build_host, sfc_build3 and sfc_build3_host take a const sfc_allocator*
    before the stream, and the header declares the allocator's two callbacks and context."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for name in ("sfc_build", "sfc_build_host", "sfc_build3", "sfc_build3_host"):
        m = re.search(name + r"\s*\(([^;]*)\);", text)
        assert m, name
        args = [a.strip() for a in m.group(1).split(",")]
        assert args[-2].startswith("const sfc_allocator*") and args[-1].startswith("void* stream"), (name, args)
    assert re.search(r"void\*\s*\(\*alloc\)\(size_t bytes, void\* stream, void\* ctx\)", text)
    assert re.search(r"void\s*\(\*free\)\(void\* ptr, void\* stream, void\* ctx\)", text)
