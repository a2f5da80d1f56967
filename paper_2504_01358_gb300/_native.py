"""ctypes declarations of libssgi.so (include/ssgi.h).  Argument marshalling only.

Loading fails loudly: there is no CPU fallback for any entry point.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libssgi.so")

SSGI_MAX_VIEWS = 32
BACKWARD_NOALLOC_MAX_BYTES = 32 << 20
OK, INVALID_ARG, UNSUPPORTED, CUDA_ERR, OOM, BUDGET, QUEUE_FULL, TIMEOUT, NOT_READY, CANCELLED = range(10)
HIT_MISS, HIT_INVALID, HIT_BACKGROUND = -1, -2, -3
DIFFUSE_INDIRECT = 1
BRUTE_FORCE = 2
PATHWISE = 4
SRGB_LOSS = 8
SRGB_FINAL = 16

STATUS = {
    0: "SSGI_OK", 1: "SSGI_ERR_INVALID_ARG", 2: "SSGI_ERR_UNSUPPORTED", 3: "SSGI_ERR_CUDA", 4: "SSGI_ERR_OOM",
    5: "SSGI_ERR_BUDGET", 6: "SSGI_ERR_QUEUE_FULL", 7: "SSGI_ERR_TIMEOUT", 8: "SSGI_ERR_NOT_READY",
    9: "SSGI_ERR_CANCELLED",
}


class SSGIError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__(f"{fn} returned {STATUS.get(code, code)}")
        self.code = code


class Dims(C.Structure):
    _fields_ = [("views", C.c_int32), ("height", C.c_int32), ("width", C.c_int32)]


class Camera(C.Structure):
    _fields_ = [("cam_to_world", C.c_float * 12), ("fov_y_rad", C.c_float), ("z_near", C.c_float)]


class GBuffer(C.Structure):
    _fields_ = [("depth", C.c_void_p), ("normal", C.c_void_p), ("albedo", C.c_void_p), ("rough", C.c_void_p),
                ("metal", C.c_void_p), ("d", Dims)]


class EnvMap(C.Structure):
    _fields_ = [("mips", C.c_void_p), ("h", C.c_int32), ("w", C.c_int32), ("levels", C.c_int32)]


class TraceParams(C.Structure):
    _fields_ = [("spp", C.c_int32), ("max_steps", C.c_int32), ("hiz_levels", C.c_int32), ("thickness", C.c_float),
                ("max_distance", C.c_float), ("seed", C.c_uint64), ("flags", C.c_uint32)]


class ServeConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_slots", C.c_int32), ("queue_capacity", C.c_int32),
                ("lut_n", C.c_int32), ("lut_samples", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("scene", C.c_int64), ("d", Dims), ("depth", C.c_void_p), ("normal", C.c_void_p),
                ("albedo", C.c_void_p), ("rough", C.c_void_p), ("metal", C.c_void_p), ("cams", C.c_void_p),
                ("env", C.c_void_p), ("env_h", C.c_int32), ("env_w", C.c_int32), ("params", TraceParams),
                ("final_out", C.c_void_p)]


class ServeStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("cancelled", C.c_uint64), ("rejected", C.c_uint64), ("queued", C.c_int32),
                ("in_flight", C.c_int32), ("resident_scenes", C.c_int32), ("pad_", C.c_int32),
                ("arena_bytes_in_use", C.c_size_t), ("arena_bytes_peak", C.c_size_t)]


_lock = threading.Lock()
_lib = None

VP, I32, I64, SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t

_SIGS = {
    "ssgi_status_string": (C.c_char_p, [C.c_int]),
    "ssgi_version": (C.c_char_p, []),
    "ssgi_env_levels": (I32, [I32, I32]),
    "ssgi_env_mip_floats": (SZ, [I32, I32]),
    "ssgi_hiz_floats": (SZ, [Dims, I32]),
    "ssgi_backward_workspace_bytes": (SZ, [Dims, I32, I32]),
    "ssgi_build_brdf_lut": (C.c_int, [I32, I32, VP, VP]),
    "ssgi_build_env_mips": (C.c_int, [VP, I32, I32, VP, VP]),
    "ssgi_build_hiz": (C.c_int, [VP, Dims, I32, VP, VP]),
    "ssgi_shade_direct": (C.c_int, [C.POINTER(GBuffer), C.POINTER(Camera), C.POINTER(EnvMap), VP, I32, VP, VP, VP,
                                    VP]),
    "ssgi_trace_indirect": (C.c_int, [C.POINTER(GBuffer), C.POINTER(Camera), VP, VP, VP, C.POINTER(EnvMap),
                                      C.POINTER(TraceParams), VP, VP, VP, VP, VP, VP]),
    "ssgi_l2_loss": (C.c_int, [VP, VP, I64, VP, VP, VP]),
    "ssgi_backward": (C.c_int, [VP, C.POINTER(GBuffer), C.POINTER(Camera), VP, C.POINTER(EnvMap), VP, I32, VP,
                                C.POINTER(TraceParams), VP, VP, VP, VP, VP, VP, SZ, VP]),
    "ssgi_backward_noalloc": (C.c_int, [VP, C.POINTER(GBuffer), C.POINTER(Camera), VP, C.POINTER(EnvMap), VP, I32,
                                        VP, C.POINTER(TraceParams), VP, VP, VP, VP, VP, VP]),
    "ssgi_step_fused_workspace_bytes": (SZ, [Dims, I32, I32, I32]),
    "ssgi_step_fused": (C.c_int, [C.POINTER(GBuffer), C.POINTER(Camera), VP, I32, I32, VP, I32, VP,
                                  C.POINTER(TraceParams), VP, VP, VP, VP, VP, VP, VP, VP, VP, SZ, VP]),
    "ssgi_step_fused_check": (C.c_int, [VP, C.POINTER(I32)]),
    "ssgi_step_fused_set_wait_limit": (C.c_int, [I64]),
    "ssgi_step_fused_phase_ns": (C.c_int, [VP, C.POINTER(C.c_uint64)]),
    "ssgi_read_bandwidth_probe": (C.c_int, [VP, SZ, I32, VP, VP]),
    "ssgi_depth_normals": (C.c_int, [VP, Dims, C.POINTER(Camera), VP, VP]),
    "ssgi_build_hiz_normals": (C.c_int, [VP, Dims, C.POINTER(Camera), I32, VP, VP, VP]),
    "ssgi_tonemap_srgb": (C.c_int, [VP, VP, I64, VP]),
    "ssgi_l2_loss_srgb": (C.c_int, [VP, VP, I64, VP, VP, VP]),
    "ssgi_env_keyframe_lerp": (C.c_int, [VP, VP, C.c_float, I32, I32, VP, VP]),
    "ssgi_env_keyframe_lerp_backward": (C.c_int, [VP, C.c_float, I32, I32, VP, VP, I32, VP]),
    "ssgi_keyframe_of": (C.c_int, [I64, I32, C.POINTER(I64), C.POINTER(C.c_float)]),
    "ssgi_composite_gbuffer": (C.c_int, [C.POINTER(GBuffer), C.POINTER(GBuffer), VP, VP, VP, VP, VP, VP, VP]),
    "ssgi_serve_create": (C.c_int, [C.POINTER(ServeConfig), C.POINTER(VP)]),
    "ssgi_serve_scene_add": (C.c_int, [VP, Dims, VP, VP, VP, VP, VP, VP, I32, C.POINTER(I64)]),
    "ssgi_serve_scene_remove": (C.c_int, [VP, I64]),
    "ssgi_serve_submit": (C.c_int, [VP, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    "ssgi_serve_poll": (C.c_int, [VP, C.c_uint64, C.POINTER(C.c_double)]),
    "ssgi_serve_wait": (C.c_int, [VP, C.c_uint64, C.c_uint32, C.POINTER(C.c_double)]),
    "ssgi_serve_cancel": (C.c_int, [VP, C.c_uint64]),
    "ssgi_serve_stats_get": (C.c_int, [VP, C.POINTER(ServeStats)]),
    "ssgi_serve_destroy": (C.c_int, [VP, C.c_uint32]),
    "ssgi_serve_request_bytes": (SZ, [Dims, I32, I32, I32, I32]),
}

# every symbol include/ssgi.h declares (checked by the CPU tests)
EXPORTED = tuple(_SIGS.keys())


def lib():
    """Load libssgi.so (building it first if the sources are newer).  Raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            if not os.path.exists(LIB_PATH) or _build._stale(LIB_PATH, _build.sources()):
                _build.build()
            L = C.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def check(fn: str, code: int) -> None:
    if code != 0:
        raise SSGIError(fn, code)


def call(name: str, *args) -> None:
    check(name, getattr(lib(), name)(*args))
