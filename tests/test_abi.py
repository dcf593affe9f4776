"""The C ABI library builds, loads and exports every entry point declared in
include/dem.h (no compute call is made: this runs without a GPU)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2307_03445_gb300 import build

    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("dem_create", "dem_load_clump_templates", "dem_add_clumps", "dem_step",
                     "dem_get_state", "dem_destroy", "dem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert missing == []


def test_binding_declares_every_symbol():
    from paper_2307_03445_gb300 import capi

    assert sorted(capi.SIGNATURES) == _declared_functions()


def test_binding_refuses_missing_library(tmp_path):
    from paper_2307_03445_gb300 import capi

    with pytest.raises(RuntimeError, match="must be built"):
        capi.load(str(tmp_path / "nope.so"))


def test_create_rejects_bad_parameters_before_touching_a_device(lib):
    from paper_2307_03445_gb300 import capi

    capi._lib = None
    L = capi.load()
    p = capi.DemParams()
    p.dt = -1.0
    ctx = C.c_void_p()
    assert L.dem_create(C.byref(p), C.byref(ctx)) == -1
    assert b"dt" in L.dem_last_error(None)
    assert not ctx.value
    assert L.dem_create(None, C.byref(ctx)) == -1
