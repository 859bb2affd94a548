"""ctypes loader for libpcdf.so (the C ABI of include/pcdf.h).

The library is built in-tree by ``build.build_library()``.  There is no
fallback: if the shared library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None
_lib_checked = None
_use_checked = False


class PcdfGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("vox", ctypes.c_float), ("origin", ctypes.c_float * 3)]


class PcdfEnv(ctypes.Structure):
    _fields_ = [("grid", PcdfGrid), ("T", ctypes.c_int32), ("H", ctypes.c_int32), ("caps", ctypes.c_void_p),
                ("occ", ctypes.c_void_p), ("comp_sq", ctypes.c_void_p)]


class PcdfBatchTiles(ctypes.Structure):
    _fields_ = [("row_rows", ctypes.c_int32), ("dyn_slices", ctypes.c_int32), ("comp_t", ctypes.c_int32)]


EXPORTS = (
    "pcdf_last_error", "pcdf_version", "pcdf_bounds_check",
    "pcdf_static_workspace_bytes", "pcdf_build_static_sdf", "pcdf_build_static_sdf_noalloc",
    "pcdf_composite_workspace_bytes", "pcdf_build_predicted_composite",
    "pcdf_composite_prepare", "pcdf_composite_finish", "pcdf_composite_finish_range", "pcdf_composite_slab",
    "pcdf_filter_voxels", "pcdf_collapse_2d", "pcdf_update_workspace_bytes", "pcdf_update_fields",
    "pcdf_scratch_workspace_bytes", "pcdf_build_from_scratch",
    "pcdf_field_max", "pcdf_template_radius", "pcdf_lattice_placements", "pcdf_template_box", "pcdf_template_workspace_bytes", "pcdf_build_template", "pcdf_composite_translated",
    "pcdf_query_cost", "pcdf_query_cost_backward",
    "pcdf_batch_create", "pcdf_batch_destroy", "pcdf_batch_workspace_bytes", "pcdf_batch_tiles_used",
    "pcdf_batch_upload", "pcdf_batch_run", "pcdf_batch_error", "pcdf_batch_block_stage", "pcdf_batch_autotune_workspace_bytes",
    "pcdf_batch_autotune",
    "pcdf_create", "pcdf_destroy", "pcdf_scratch_bytes", "pcdf_ctx_reserve", "pcdf_ctx_build_static_sdf",
    "pcdf_ctx_build_predicted_composite", "pcdf_ctx_build_from_scratch", "pcdf_ctx_query_cost",
    "pcdf_ctx_query_cost_backward", "pcdf_build_batched",
    "pcdf_mlp_state_bytes", "pcdf_mlp_workspace_bytes", "pcdf_mlp_init", "pcdf_mlp_forward", "pcdf_mlp_infer", "pcdf_mlp_infer_tc", "pcdf_mlp_infer_tc_count",
    "pcdf_mlp_backward",
    "pcdf_mlp_adam", "pcdf_surrogate_samples", "pcdf_surrogate_features", "pcdf_surrogate_finish_workspace_bytes",
    "pcdf_surrogate_finish", "pcdf_surrogate_finish_slab", "pcdf_surrogate_select",
)


def _declare(lib):
    P, I32, I64, F32, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_size_t
    G = ctypes.POINTER(PcdfGrid)
    SZP = ctypes.POINTER(ctypes.c_size_t)
    lib.pcdf_last_error.restype = ctypes.c_char_p
    lib.pcdf_last_error.argtypes = []
    lib.pcdf_version.restype = ctypes.c_int
    sig = {
        "pcdf_bounds_check": [P, P, I32],
        "pcdf_static_workspace_bytes": [G, SZP],
        "pcdf_build_static_sdf": [G, P, P, P, P, SZ, P],
        "pcdf_build_static_sdf_noalloc": [G, P, P, P, P],
        "pcdf_composite_workspace_bytes": [G, I32, I32, P, SZP],
        "pcdf_build_predicted_composite": [G, P, P, I32, I32, P, P, P, P, SZ, P],
        "pcdf_composite_prepare": [G, I32, I32, P, P, SZ, P],
        "pcdf_composite_slab": [G, I32, I32, P, ctypes.POINTER(I32), ctypes.POINTER(I32)],
        "pcdf_composite_finish": [G, P, P, I32, I32, P, P, P, P, SZ, P],
        "pcdf_composite_finish_range": [G, P, P, I32, I32, P, I32, I32, P, P, P, SZ, P],
        "pcdf_filter_voxels": [G, P, I32, P, P],
        "pcdf_update_workspace_bytes": [G, I32, I32, P, SZP],
        "pcdf_update_fields": [G, P, I32, I32, P, P, P, P, P, P, SZ, P, P],
        "pcdf_collapse_2d": [G, P, I32, I32, P, P],
        "pcdf_scratch_workspace_bytes": [G, I32, I32, SZP],
        "pcdf_build_from_scratch": [G, P, I32, I32, P, P, P, P, SZ, P],
        "pcdf_field_max": [P, I64, P, P],
        "pcdf_template_radius": [I32, P],
        "pcdf_lattice_placements": [P, I32, I32, P, P, P],
        "pcdf_template_box": [P, I32, P, P],
        "pcdf_template_workspace_bytes": [P, I32, SZP],
        "pcdf_build_template": [P, I32, P, P, SZ, P],
        "pcdf_composite_translated": [G, P, P, I32, I32, P, P, I32, P, P, P, P],
        "pcdf_query_cost": [G, P, I32, P, P, I64, F32, P, P, P],
        "pcdf_query_cost_backward": [G, P, I32, P, P, I64, F32, P, P, P, P],
    }
    E = ctypes.POINTER(PcdfEnv)
    TL = ctypes.POINTER(PcdfBatchTiles)
    PP = ctypes.POINTER(ctypes.c_void_p)
    sig.update({
        "pcdf_batch_create": [E, I32, TL, PP],
        "pcdf_batch_workspace_bytes": [P, SZP],
        "pcdf_batch_tiles_used": [P, TL],
        "pcdf_batch_upload": [P, P, SZ, P],
        "pcdf_batch_run": [P, P, P],
        "pcdf_batch_error": [P, P, P, ctypes.POINTER(I32)],
        "pcdf_batch_block_stage": [P, I32, I32],
        "pcdf_batch_autotune_workspace_bytes": [E, I32, SZP],
        "pcdf_batch_autotune": [E, I32, P, SZ, P, I32, TL, ctypes.POINTER(ctypes.c_float)],
    })
    U64, F32 = ctypes.c_uint64, ctypes.c_float
    sig.update({
        "pcdf_mlp_state_bytes": [SZP],
        "pcdf_mlp_workspace_bytes": [I64, SZP],
        "pcdf_mlp_init": [P, U64, P],
        "pcdf_mlp_forward": [P, P, I64, P, P, SZ, P],
        "pcdf_mlp_infer": [P, P, I64, P, P],
        "pcdf_mlp_infer_tc": [P, P, I64, P, P],
        "pcdf_mlp_infer_tc_count": [P, P, I64, P, P, P],
        "pcdf_mlp_backward": [P, P, P, I64, P, P, P, SZ, P],
        "pcdf_mlp_adam": [P, F32, F32, F32, F32, I32, P],
        "pcdf_surrogate_samples": [G, P, P, P, I32, I32, I64, U64, F32, P, P, P],
        "pcdf_surrogate_features": [G, P, P, I64, I32, I32, P, P, P],
        "pcdf_surrogate_finish_workspace_bytes": [I32, I32, I64, SZP],
        "pcdf_surrogate_finish": [G, P, P, P, P, I64, I32, I32, P, P, P, P, F32, F32, P, P, P, P, SZ, P],
        "pcdf_surrogate_finish_slab": [G, P, P, P, P, I64, I32, I32, P, P, SZ, P, P, P, F32, F32, P, P, P, P, SZ,
                                       P],
        "pcdf_surrogate_select": [G, P, P, P, I64, I32, I32, P, F32, I32, P, P, P, P, P],
    })
    sig.update({
        "pcdf_create": [PP, I32, P],
        "pcdf_scratch_bytes": [G, I32, I32, SZP],
        "pcdf_ctx_reserve": [P, SZ],
        "pcdf_ctx_build_static_sdf": [P, G, P, P, P],
        "pcdf_ctx_build_predicted_composite": [P, G, P, P, I32, I32, P, P, P],
        "pcdf_ctx_build_from_scratch": [P, G, P, I32, I32, P, P, P],
        "pcdf_ctx_query_cost": [P, G, P, I32, P, P, I64, F32, P, P],
        "pcdf_ctx_query_cost_backward": [P, G, P, I32, P, P, I64, F32, P, P, P],
        "pcdf_build_batched": [P, E, I32, I32],
    })
    lib.pcdf_batch_destroy.argtypes = [P]
    lib.pcdf_batch_destroy.restype = None
    lib.pcdf_destroy.argtypes = [P]
    lib.pcdf_destroy.restype = None
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int


def lib_path() -> str:
    return _build.LIB


def use_checked(flag: bool):
    """Route every later load() (so every call of the package) to the
    bounds-checked debug library, libpcdf_checked.so, or back."""
    global _use_checked
    _use_checked = bool(flag)


def load(build_if_missing: bool = True, checked: bool = None):
    """Load libpcdf.so, or the bounds-checked libpcdf_checked.so (checked, or
    use_checked(True)), building it first if allowed and needed."""
    global _lib, _lib_checked
    checked = _use_checked if checked is None else checked
    path = _build.LIB_CHECKED if checked else _build.LIB
    with _lock:
        if (_lib_checked if checked else _lib) is None:
            if build_if_missing and not _build.up_to_date(checked):
                _build.build_library(checked=checked)
            if not os.path.exists(path):
                raise RuntimeError(f"libpcdf is not built ({path} missing); run build_library()")
            lib = ctypes.CDLL(path)
            _declare(lib)
            if checked:
                _lib_checked = lib
            else:
                _lib = lib
    return _lib_checked if checked else _lib


def check(rc: int, what: str):
    if rc != 0:
        msg = load().pcdf_last_error().decode(errors="replace")
        raise RuntimeError(f"{what} failed ({rc}): {msg}")
