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


def _params_with_walls(capi, walls, keep):
    import numpy as np

    from paper_2307_03445_gb300 import walls_to_c

    p = capi.DemParams()
    p.dt = 1e-6
    for k in range(3):
        p.domain_lo[k], p.domain_hi[k] = -0.1, 0.1
    p.rebuild_interval, p.v_bound, p.guard = 10, 0.5, 1
    mats = [np.array([v]) for v in (1e8, 0.3, 0.5, 0.5)]
    keep += mats
    p.n_materials = 1
    p.E, p.nu, p.mu, p.cor = (m.ctypes.data_as(C.POINTER(C.c_double)) for m in mats)
    warr = walls_to_c(walls)
    keep.append(warr)
    p.n_walls = len(walls)
    p.walls = C.cast(warr, C.POINTER(capi.DemWall))
    return p


def test_create_checks_mesh_facets(lib):
    """A facet must be a real triangle whose normal is (b - p) x (c - p)
    normalised; a valid one passes to the device lookup."""
    from paper_2307_03445_gb300 import capi, scenes

    capi._lib = None
    L = capi.load()
    good = scenes.triangle((0, 0, 0), (0.01, 0, 0), (0, 0.01, 0))
    flipped = dict(good, n=(0.0, 0.0, -1.0))
    flat = dict(good, c=(0.02, 0.0, 0.0))
    for wall, msg in ((flat, b"degenerate triangle"), (flipped, b"triangle normal")):
        keep = []
        ctx = C.c_void_p()
        assert L.dem_create(C.byref(_params_with_walls(capi, [wall], keep)), C.byref(ctx)) == -1
        assert msg in L.dem_last_error(None) and not ctx.value
    keep = []
    ctx = C.c_void_p()
    rc = L.dem_create(C.byref(_params_with_walls(capi, [good], keep)), C.byref(ctx))
    if rc == 0:  # a device is present: the context was made
        L.dem_destroy(ctx)
    else:
        assert b"no CUDA device" in L.dem_last_error(None)


def test_binding_structures_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    the C compiler gives the header's struct (a C program built with gcc
    prints them; nothing runs on a device)."""
    import shutil
    import subprocess

    from paper_2307_03445_gb300 import capi

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"dem_wall": capi.DemWall, "dem_params": capi.DemParams, "dem_stats": capi.DemStats,
             "dem_learned_params": capi.DemLearnedParams, "dem_tiles": capi.DemTiles}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "dem.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
