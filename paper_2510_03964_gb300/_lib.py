"""ctypes declarations of libwrs (include/wrs.h). Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

from . import build as _build

WRS_OK, WRS_ERR_ARG, WRS_ERR_CUDA, WRS_ERR_BUDGET, WRS_ERR_TIMEOUT, WRS_ERR_STATE, WRS_ERR_CHECK = range(7)
WRS_MAX_K = 16
WRS_MAX_BATCH = 64
WRS_RULE_KEYS, WRS_RULE_LITERAL = 0, 1
WRS_EMPTY_SLOT = 0xFFFFFFFF
HEADER = os.path.join(_build.INCLUDE, "wrs.h")


class WrsConfig(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("K", C.c_int32),
                ("fovea_radius_px", C.c_float), ("deg_per_px", C.c_float), ("seed", C.c_uint64),
                ("stream_id", C.c_uint32), ("color_fp16", C.c_int32), ("temporal_bias", C.c_int32),
                ("update_rule", C.c_int32)]


class WrsLayout(C.Structure):
    _fields_ = [("plane_px", C.c_int64), ("plane_bytes4", C.c_int64), ("plane_bytes_col", C.c_int64),
                ("plane_bytes_wt", C.c_int64), ("status_off", C.c_int64), ("W_off", C.c_int64), ("P_off", C.c_int64),
                ("key_off", C.c_int64), ("idx_off", C.c_int64), ("wt_off", C.c_int64),
                ("col_off", C.c_int64), ("map_off", C.c_int64), ("map_frames", C.c_int64),
                ("total_bytes", C.c_int64)]


WRS_MAX_MIP_LEVELS = 6
WRS_FILTER_BOX, WRS_FILTER_BILINEAR = 0, 1


class WrsFovSource(C.Structure):
    _fields_ = [("d_img", C.c_void_p), ("img_pitch_elems", C.c_int64), ("d_mip", C.c_void_p),
                ("mip_bytes", C.c_size_t), ("nradii", C.c_int32),
                ("radii", C.c_float * (WRS_MAX_MIP_LEVELS - 1))]


class WrsMipLayout(C.Structure):
    _fields_ = [("levels", C.c_int32), ("width", C.c_int32 * WRS_MAX_MIP_LEVELS),
                ("height", C.c_int32 * WRS_MAX_MIP_LEVELS), ("offset", C.c_int64 * WRS_MAX_MIP_LEVELS),
                ("total_bytes", C.c_int64)]


_V = C.c_void_p
_I = C.c_int
SIGNATURES = {
    "wrs_state_bytes": (C.c_size_t, [C.POINTER(WrsConfig)]),
    "wrs_state_layout": (_I, [C.POINTER(WrsConfig), C.POINTER(WrsLayout)]),
    "wrs_create": (_I, [C.POINTER(WrsConfig), _V, C.c_size_t, _V, C.POINTER(_V)]),
    "wrs_push_frame": (_I, [_V, _V, C.c_int64, C.c_float, C.c_float, _V, _V, _V]),
    "wrs_resolve": (_I, [_V, _V, _V]),
    "wrs_destroy": (_I, [_V]),
    "wrs_push_frame_host": (_I, [_V, _V, C.c_float, C.c_float, _V, _V, _V, _V, _V, _V]),
    "wrs_export_state": (_I, [_V, _V, C.c_size_t, _V]),
    "wrs_import_state": (_I, [_V, _V, C.c_size_t, C.c_uint32, _V]),
    "wrs_frame_index": (C.c_uint32, [_V]),
    "wrs_set_launch": (_I, [_V, _I, _I]),
    "wrs_get_launch": (_I, [_V, C.POINTER(_I), C.POINTER(_I)]),
    "wrs_set_pipeline": (_I, [_V, _I, _I, _I, _I]),
    "wrs_get_pipeline": (_I, [_V, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "wrs_set_wait_limit": (_I, [_V, C.c_uint64, C.c_uint32]),
    "wrs_check_status": (_I, [_V, _V]),
    "wrs_batch_create": (_I, [_I, C.POINTER(_V)]),
    "wrs_batch_destroy": (_I, [_V]),
    "wrs_batch_set_launch": (_I, [_V, _I, _I, _I, _I]),
    "wrs_batch_get_launch": (_I, [_V, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "wrs_push_batch": (_I, [_V, _I, _V, _V, _V, _V, _V, _V]),
    "wrs_push_batch_foveated": (_I, [_V, _I, _V, _V, C.c_int32, _V, _V, _V, _V]),
    "wrs_get_stats": (_I, [_V, C.POINTER(C.c_uint64), _V]),
    "wrs_set_reprojection_buffer": (_I, [_V, _V, C.c_size_t, _V]),
    "wrs_push_frame_reproject": (_I, [_V, _V, C.c_int64, C.c_float, C.c_float, _V, _V, _V, C.c_float,
                                      _V, _V, _V]),
    "wrs_mip_layout_get": (_I, [C.c_int32, C.c_int32, C.c_int32, C.POINTER(WrsMipLayout)]),
    "wrs_mip_build": (_I, [_V, C.c_int64, C.c_int32, C.c_int32, C.c_int32, _V, C.c_size_t, _V]),
    "wrs_foveate": (_I, [_V, C.c_int64, _V, C.c_size_t, C.c_int32, C.c_int32, C.c_int32, _V,
                         C.c_float, C.c_float, C.c_int32, _V, C.c_int64, _V, _V]),
    "wrs_push_foveated": (_I, [_V, _V, C.c_int64, _V, C.c_size_t, C.c_int32, _V, C.c_int32, C.c_float,
                               C.c_float, _V, _V, _V]),
    "wrs_push_frame_host_noalloc": (_I, [_V, _V, C.c_float, C.c_float, _V, _V, _V]),
    "wrs_host_pipe_stage_bytes": (C.c_size_t, [_V, _I]),
    "wrs_host_pipe_create": (_I, [_V, _V, C.c_size_t, _I, C.POINTER(_V)]),
    "wrs_host_pipe_push": (_I, [_V, _V, C.c_float, C.c_float, _V, _V]),
    "wrs_host_pipe_finish": (_I, [_V]),
    "wrs_host_pipe_destroy": (_I, [_V]),
    "wrs_checked_build": (_I, []),
    "wrs_last_error": (C.c_char_p, []),
}

_lock = threading.Lock()
_lib = None


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions include/wrs.h declares."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wrs_[a-z0-9_]+)\s*\(", text)))


def library_path() -> str:
    """libwrs.so, or the checked build libwrs_checked.so when the environment
    sets WRS_CHECKED=1."""
    return _build.LIB_CHECKED if os.environ.get("WRS_CHECKED") == "1" else _build.LIB


def load(build_if_missing: bool = True):
    """Loads libwrs.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if build_if_missing and _build.is_stale(path):
                _build.build(libs=(path,))
            if not os.path.exists(path):
                raise RuntimeError(f"libwrs is not built ({path}); run paper_2510_03964_gb300.build.build()")
            lib = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class WrsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libwrs error {code}: {msg}")
        self.code = code


def check(rc: int):
    if rc != WRS_OK:
        raise WrsError(rc, load().wrs_last_error().decode())
    return rc
