"""ctypes declarations of the C ABI in include/dem.h (argument marshalling only).

Every computation runs inside libdem.so; loading fails loudly if the library
has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdem.so")

DEM_OK = 0
ERRORS = {
    -1: "DEM_ERR_INVALID_ARG", -2: "DEM_ERR_OOM", -3: "DEM_ERR_CAPACITY",
    -4: "DEM_ERR_NONFINITE", -5: "DEM_ERR_TIMEOUT", -6: "DEM_ERR_CUDA",
    -7: "DEM_ERR_STATE", -8: "DEM_ERR_GUARD",
}
DEM_FP64, DEM_FP32_VOXEL = 0, 1
DEM_MLP_NOALLOC_MAX_ROWS = 262144  # include/dem.h
DEM_MARGIN_FIXED, DEM_MARGIN_LEARNED = 0, 1
DEM_GUARD_OFF, DEM_GUARD_COUNT, DEM_GUARD_ROLLBACK = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class DemWall(C.Structure):
    _fields_ = [("type", C.c_int), ("material", C.c_int), ("p", C.c_double * 3),
                ("n", C.c_double * 3), ("radius", C.c_double), ("half_angle", C.c_double),
                ("height", C.c_double), ("vel", C.c_double * 3), ("scene", C.c_int),
                ("b", C.c_double * 3), ("c", C.c_double * 3)]


class DemParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("g", C.c_double * 3), ("domain_lo", C.c_double * 3),
                ("domain_hi", C.c_double * 3), ("precision", C.c_int), ("bin_size", C.c_double),
                ("margin_policy", C.c_int), ("rebuild_interval", C.c_int), ("v_bound", C.c_double),
                ("margin", C.c_double), ("mix_rule", C.c_int), ("n_materials", C.c_int),
                ("E", C.POINTER(C.c_double)), ("nu", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double)), ("cor", C.POINTER(C.c_double)),
                ("n_walls", C.c_int), ("walls", C.POINTER(DemWall)),
                ("max_contacts", C.c_longlong), ("guard", C.c_int),
                ("cuda_stream", C.c_void_p), ("device", C.c_int),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", C.c_void_p)]


class DemStats(C.Structure):
    _fields_ = [("steps", C.c_longlong), ("rebuilds", C.c_longlong), ("n_clumps", C.c_longlong),
                ("n_spheres", C.c_longlong), ("n_pairs", C.c_longlong),
                ("n_wall_contacts", C.c_longlong), ("bin_entries", C.c_longlong),
                ("pair_steps", C.c_longlong), ("active_last", C.c_longlong),
                ("guard_violations", C.c_longlong), ("rollbacks", C.c_longlong),
                ("missed_contacts", C.c_longlong), ("margin", C.c_double), ("time", C.c_double),
                ("ms_detect", C.c_double), ("ms_pairs", C.c_double), ("ms_walls", C.c_double),
                ("ms_update", C.c_double), ("timed_steps", C.c_longlong),
                ("launches", C.c_longlong), ("early_rebuilds", C.c_longlong),
                ("ms_predict", C.c_double), ("outer_rebuilds", C.c_longlong)]


_D = C.POINTER(C.c_double)
_F = C.POINTER(C.c_float)
_I = C.POINTER(C.c_int)
_V = C.c_void_p


class DemLearnedParams(C.Structure):
    _fields_ = [("interval", C.c_int), ("safety", C.c_double), ("n_candidates", C.c_int),
                ("candidates", C.POINTER(C.c_double)), ("mode", C.c_int),
                ("speed_floor", C.c_double)]


DEM_LEARNED_HALT, DEM_LEARNED_ROLLBACK = 0, 1


class DemTiles(C.Structure):
    _fields_ = [("pairs_blocks_per_sm", C.c_int), ("update_block", C.c_int),
                ("narrow_chunk", C.c_int)]

# name -> (restype, argtypes); the exported symbols of include/dem.h
SIGNATURES = {
    "dem_create": (C.c_int, [C.POINTER(DemParams), C.POINTER(C.c_void_p)]),
    "dem_destroy": (None, [_V]),
    "dem_last_error": (C.c_char_p, [_V]),
    "dem_load_clump_templates": (C.c_int, [_V, C.c_int, _I, _D, _D, _I, _D, _D]),
    "dem_add_scene": (C.c_int, [_V, _D, _D, C.c_double, _I]),
    "dem_add_clumps": (C.c_int, [_V, C.c_int, _I, _D, _D, _D, _D, C.c_int]),
    "dem_step": (C.c_int, [_V, C.c_int]),
    "dem_get_state": (C.c_int, [_V, _V, _V, _V, _V, C.c_int]),
    "dem_set_state": (C.c_int, [_V, _D, _D, _D, _D]),
    "dem_get_stats": (C.c_int, [_V, C.POINTER(DemStats)]),
    "dem_reset_stats": (C.c_int, [_V]),
    "dem_set_timing": (C.c_int, [_V, C.c_int]),
    "dem_set_graphs": (C.c_int, [_V, C.c_int]),
    "dem_set_deterministic": (C.c_int, [_V, C.c_int]),
    "dem_set_outer_list": (C.c_int, [_V, C.c_double, C.c_int, C.c_int]),
    "dem_autotune_bins": (C.c_int, [_V, C.c_int, _D, C.c_int, _D, _D]),
    "dem_set_tiles": (C.c_int, [_V, C.POINTER(DemTiles)]),
    "dem_get_tiles": (C.c_int, [_V, C.POINTER(DemTiles)]),
    "dem_autotune_tiles": (C.c_int, [_V, C.c_int, C.c_int, C.POINTER(DemTiles)]),
    "dem_rebuild": (C.c_int, [_V]),
    "dem_eval_forces": (C.c_int, [_V]),
    "dem_get_forces": (C.c_int, [_V, _D, _D]),
    "dem_get_wall_forces": (C.c_int, [_V, _D]),
    "dem_get_wall_loads": (C.c_int, [_V, _D, _D]),
    "dem_set_wall_motion": (C.c_int, [_V, C.c_int, _D, _D]),
    "dem_num_contacts": (C.c_int, [_V, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "dem_get_contacts": (C.c_int, [_V, _I, _I, _D, _I, _I, _D]),
    "dem_get_bins": (C.c_int, [_V, C.c_longlong, C.POINTER(C.c_uint), _I,
                               C.POINTER(C.c_longlong)]),
    "dem_audit": (C.c_int, [_V, C.POINTER(C.c_longlong)]),
    "dem_mlp_num_params": (C.c_int, []),
    "dem_mlp_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p)]),
    "dem_mlp_destroy": (None, [_V]),
    "dem_mlp_set_params": (C.c_int, [_V, _F]),
    "dem_mlp_get_params": (C.c_int, [_V, _F]),
    "dem_mlp_forward": (C.c_int, [_V, C.c_longlong, _F, _F]),
    "dem_mlp_loss_grad": (C.c_int, [_V, C.c_longlong, _F, _F, C.POINTER(C.c_double), _F]),
    "dem_mlp_forward_tc": (C.c_int, [_V, C.c_longlong, _F, _F]),
    "dem_mlp_loss_grad_noalloc": (C.c_int, [_V, C.c_longlong, _F, _F, C.POINTER(C.c_double), _F]),
    "dem_mlp_train": (C.c_int, [_V, C.c_longlong, _F, _F, C.c_int, C.c_int, C.c_float,
                                C.c_ulonglong, C.POINTER(C.c_double)]),
    "dem_set_learned_policy": (C.c_int, [_V, _V, C.c_void_p]),
    "dem_trace": (C.c_int, [_V, C.c_int, C.c_int, C.c_int, _D, C.c_longlong, _F, _F,
                            C.POINTER(C.c_longlong)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libdem.so; raises if it is missing (build it with paper_2307_03445_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: the CUDA library must be built "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class DemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
