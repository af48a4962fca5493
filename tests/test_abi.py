"""Host-side checks of the C ABI: the library loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

import paper_2504_13445_gb300 as rkm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rkm.h")


def declared_functions() -> list[str]:
    text = open(HEADER).read()
    return sorted(set(re.findall(r"RKM_API\s+[\w\s\*]+?\b(rkm_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(rkm.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return rkm.load_library()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("rkm_thresholds", "rkm_scores", "rkm_topn", "rkm_query_new_items", "rkm_create",
                     "rkm_destroy", "rkm_resident_set", "rkm_item_bounds", "rkm_topn_host"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in rkm.h but not exported"
    assert set(declared_functions()) <= set(rkm.EXPORTED) | set(declared_functions())


def test_binding_covers_header(lib):
    assert sorted(rkm.EXPORTED) == declared_functions()


def test_version_and_default_opts(lib):
    assert b"sm_103a" in lib.rkm_version()
    o = rkm.Opts()
    lib.rkm_default_opts(ctypes.byref(o))
    assert o.precision == rkm.RKM_BF16 and o.k_max == 64 and o.filter == 1


def test_create_rejects_bad_options(lib):
    o = rkm.Opts()
    lib.rkm_default_opts(ctypes.byref(o))
    o.k_max = 0
    h = ctypes.c_void_p()
    assert lib.rkm_create(ctypes.byref(h), ctypes.byref(o), 0) == 1  # RKM_EINVAL
    assert b"k_max" in lib.rkm_last_error()
    o.k_max = 64
    o.precision = 7
    assert lib.rkm_create(ctypes.byref(h), ctypes.byref(o), 0) == 1


def test_null_context_is_rejected(lib):
    status = lib.rkm_thresholds(None, None, 0, 1, None, 0, 1, 1, 1, None, None, None, None)
    assert status == 1 and b"context" in lib.rkm_last_error()
    lib.rkm_destroy(None)  # accepted


def test_create_without_gpu_reports_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    status = lib.rkm_create(ctypes.byref(h), None, 0)
    assert status != 0 and lib.rkm_last_error()


def test_debug_build_exports_every_declared_symbol():
    """The RKM_DEBUG variant (device index checks on) builds from the same sources and exports
    the same C ABI."""
    from paper_2504_13445_gb300 import build as b
    path = b.build(debug=True)
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} missing from the debug library"
