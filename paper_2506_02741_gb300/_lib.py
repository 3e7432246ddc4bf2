"""ctypes declarations of the vtsplat C ABI (include/vtsplat.h).

Loading fails loudly when the compiled library is missing: there is no
fallback path.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

VT_OK, VT_ERR_INVALID_ARG, VT_ERR_OOM, VT_ERR_CUDA, VT_ERR_CAPACITY, VT_ERR_TIMEOUT, \
    VT_ERR_STATE = range(7)
VT_F32, VT_F16 = 0, 1
VT_GRAD_ATTR, VT_GRAD_POSE, VT_GRAD_VIEWS = 1, 2, 4

STATUS_NAMES = {0: "VT_OK", 1: "VT_ERR_INVALID_ARG", 2: "VT_ERR_OOM", 3: "VT_ERR_CUDA",
                4: "VT_ERR_CAPACITY", 5: "VT_ERR_TIMEOUT", 6: "VT_ERR_STATE"}


class Intrinsics(C.Structure):
    _fields_ = [("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float), ("cy", C.c_float)]


class SectionC(C.Structure):
    _fields_ = [("n_views", C.c_int32), ("W", C.c_int32), ("H", C.c_int32), ("K", Intrinsics),
                ("poses", C.c_void_p), ("depth", C.c_void_p), ("n", C.c_int64),
                ("src", C.c_void_p), ("prec", C.c_int), ("colour", C.c_void_p),
                ("opacity", C.c_void_p), ("radius", C.c_void_p), ("scale", C.c_void_p),
                ("rot", C.c_void_p)]


class GradsC(C.Structure):
    _fields_ = [("d_colour", C.c_void_p), ("d_opacity", C.c_void_p), ("d_radius", C.c_void_p),
                ("d_view_twist", C.c_void_p), ("d_view_mat", C.c_void_p),
                ("d_depth", C.c_void_p), ("d_scale", C.c_void_p), ("d_rot", C.c_void_p)]


class ViewC(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("W", C.c_int32), ("H", C.c_int32), ("K", Intrinsics),
                ("pose12", C.c_void_p)]


class BatchItemC(C.Structure):
    _fields_ = [("section", C.c_int32), ("track", C.c_int32), ("W", C.c_int32), ("H", C.c_int32),
                ("K", Intrinsics), ("pose12", C.c_void_p), ("image", C.c_void_p),
                ("obs", C.c_void_p), ("result", C.c_void_p)]


class L1WeightsC(C.Structure):
    _fields_ = [("w_rgb", C.c_double), ("w_depth", C.c_double), ("sil_min", C.c_float),
                ("rgb_needs_depth", C.c_int32)]


class AdamParamsC(C.Structure):
    _fields_ = [("lr", C.c_float * 5), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float)]


class ShapeAdamParamsC(C.Structure):
    _fields_ = [("lr_scale", C.c_float), ("lr_rot", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float)]


MAX_VIS_VIEWS = 8


class VTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None
_P = C.c_void_p


def _declare(L):
    sig = {
        "vt_ctx_create": (C.c_int, [C.POINTER(_P)]),
        "vt_ctx_destroy": (None, [_P]),
        "vt_ctx_reserve": (C.c_int, [_P, C.c_int64, C.c_int32, C.c_int32, C.c_int64, _P]),
        "vt_workspace_bytes": (C.c_size_t, [C.c_int64, C.c_int32, C.c_int32, C.c_int64]),
        "vt_ctx_sync_status": (C.c_int, [_P, _P, C.POINTER(C.c_int64)]),
        "vt_backproject": (C.c_int, [_P, C.c_int32, C.c_int32, Intrinsics, _P, _P, _P, C.c_int64,
                                     _P, _P]),
        "vt_backproject_noalloc": (C.c_int, [_P, C.c_int32, C.c_int32, Intrinsics, _P, _P, _P,
                                             C.c_int64, _P, _P]),
        "vt_section_init": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.c_int32, Intrinsics, C.c_int,
                                      _P, _P, _P, _P, C.c_int64, _P, _P]),
        "vt_render": (C.c_int, [_P, C.POINTER(SectionC), C.c_int32, _P, Intrinsics, C.c_int32,
                                C.c_int32, _P, _P, _P, _P]),
        "vt_render_backward": (C.c_int, [_P, _P, _P, _P, C.c_int32, C.POINTER(GradsC), _P, _P,
                                         _P]),
        "vt_visibility": (C.c_int, [_P, C.c_int32, C.c_int32, Intrinsics, _P, C.POINTER(ViewC),
                                    C.c_int32, C.c_double, _P, _P]),
        "vt_masked_l1": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, _P, _P, _P, _P, L1WeightsC,
                                   _P, _P, _P, _P]),
        "vt_pose_adam": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_double), C.c_double,
                                   C.c_double, C.c_double, _P]),
        "vt_attr_adam": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P,
                                   _P, AdamParamsC, _P]),
        "vt_shape_adam": (C.c_int, [_P, C.c_int64, _P, _P, _P, _P, _P, _P, C.c_int, _P, _P,
                                    ShapeAdamParamsC, _P]),
        "vt_section_complement": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32, Intrinsics,
                                            C.c_float, C.c_int32, C.c_int, _P, _P, _P, _P,
                                            C.c_int64, _P, _P]),
        "vt_visibility_counts": (C.c_int, [_P, C.c_int32, C.c_int32, Intrinsics, _P,
                                           C.POINTER(ViewC), C.c_int32, C.c_double, _P, _P,
                                           _P]),
        "vt_ssim": (C.c_int, [_P, C.c_int32, C.c_int32, _P, _P, C.c_double, _P, _P, _P]),
        "vt_ctx_set_timing": (C.c_int, [_P, C.c_int32]),
        "vt_ctx_timing": (C.c_int32, [_P, _P, C.POINTER(C.c_char_p), C.POINTER(C.c_int64),
                                      C.POINTER(C.c_double), C.c_int32, C.c_int32]),
        "vt_ctx_launch_count": (C.c_int64, [_P]),
        "vt_ctx_set_list_capacity": (C.c_int, [_P, C.c_int32]),
        "vt_ctx_set_workspace_budget": (C.c_int, [_P, C.c_size_t]),
        "vt_ctx_workspace_bytes": (C.c_size_t, [_P]),
        "vt_ctx_used_lists": (C.c_int32, [_P]),
        "vt_ctx_debug_copy": (C.c_int64, [_P, C.c_int32, _P, C.c_int64, _P]),
        "vt_ctx_debug_pixel_lists": (C.c_int, [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                               C.c_int32, _P, _P, _P, C.POINTER(C.c_int32),
                                               _P]),
        "vt_batch_workspace_bytes": (C.c_size_t, [C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                                  C.c_int64, C.c_int64, C.c_int32]),
        "vt_batch_reserve": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int64, C.c_int64,
                                       C.c_int64, C.c_int64, _P]),
        "vt_batch_set": (C.c_int, [_P, C.POINTER(SectionC), C.c_int32, C.POINTER(BatchItemC),
                                   C.c_int32, L1WeightsC]),
        "vt_batch_launch": (C.c_int, [_P, _P, _P]),
        "vt_adam_init": (C.c_int, [_P, C.c_int64, C.c_int, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                   _P]),
        "vt_last_error": (C.c_char_p, []),
        "vt_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


# Every symbol include/vtsplat.h declares (checked by the CPU test-suite).
EXPORTS = ["vt_ctx_create", "vt_ctx_destroy", "vt_ctx_reserve", "vt_workspace_bytes",
           "vt_ctx_sync_status", "vt_backproject", "vt_section_init", "vt_render",
           "vt_render_backward", "vt_ctx_set_timing", "vt_ctx_timing", "vt_ctx_launch_count",
           "vt_ctx_debug_copy", "vt_last_error", "vt_version", "vt_ctx_set_list_capacity",
           "vt_ctx_set_workspace_budget", "vt_ctx_workspace_bytes", "vt_ctx_used_lists",
           "vt_backproject_noalloc", "vt_visibility", "vt_masked_l1", "vt_pose_adam",
           "vt_attr_adam", "vt_section_complement", "vt_ssim",
           "vt_visibility_counts", "vt_shape_adam", "vt_ctx_debug_pixel_lists",
           "vt_batch_workspace_bytes", "vt_batch_reserve", "vt_batch_set", "vt_batch_launch",
           "vt_adam_init"]


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load the compiled library (building it first if sources changed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or os.environ.get("VTSPLAT_REBUILD"):
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("vtsplat CUDA library is missing; run build()")
            _lib = _declare(C.CDLL(path))
    return _lib


def check(status: int, what: str = "") -> None:
    if status != VT_OK:
        msg = lib().vt_last_error().decode()
        raise VTError(status, f"{what}: {msg}" if what else msg)
