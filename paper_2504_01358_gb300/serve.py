"""Binding of the SSGI serving loop (ssgi_serve_* in include/ssgi.h).

`Server` wraps one C server: device arena = HBM budget, `slots` concurrent requests on their own
CUDA streams, resident scenes for re-rendering.  Request inputs are host arrays (numpy or CPU
torch tensors; pinned memory lets copies overlap other requests' kernels) that the wrapper
keeps alive until the request is collected.  Every call is argument marshalling around the C
functions of the same name.
"""
from __future__ import annotations

import ctypes as C
from typing import Dict, Optional

import numpy as np

from . import _native as N


def _ptr(a) -> int:
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError("serving inputs are host arrays")
        if not a.is_contiguous():
            raise ValueError("host arrays must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return a.ctypes.data


def _cams(cams) -> C.Array:
    a = np.ascontiguousarray(np.asarray(cams, dtype=np.float32)).reshape(-1, 14)
    arr = (N.Camera * len(a))()
    for i, rec in enumerate(a):
        arr[i].cam_to_world[:] = rec[:12].tolist()
        arr[i].fov_y_rad = float(rec[12])
        arr[i].z_near = float(rec[13])
    return arr


def ssgi_serve_request_bytes(dims, env_h: int, env_w: int, hiz_levels: int, resident: bool) -> int:
    V, H, W = dims
    return N.lib().ssgi_serve_request_bytes(N.Dims(V, H, W), env_h, env_w, hiz_levels, int(resident))


class Server:
    def __init__(self, hbm_budget_bytes: int, max_slots: int = 4, queue_capacity: int = 1024, lut_n: int = 64,
                 lut_samples: int = 4096):
        cfg = N.ServeConfig(hbm_budget_bytes, max_slots, queue_capacity, lut_n, lut_samples)
        h = C.c_void_p()
        N.call("ssgi_serve_create", C.byref(cfg), C.byref(h))
        self._h = h
        self._keep: Dict[int, tuple] = {}

    # -- scenes ---------------------------------------------------------------------------------
    def scene_add(self, depth, normal, albedo, rough, metal, cams, hiz_levels: int = 8) -> int:
        V, H, W = depth.shape
        sid = C.c_int64()
        cam = _cams(cams)
        N.call("ssgi_serve_scene_add", self._h, N.Dims(V, H, W), _ptr(depth), _ptr(normal), _ptr(albedo), _ptr(rough),
               _ptr(metal), C.cast(cam, C.c_void_p), hiz_levels, C.byref(sid))
        return sid.value

    def scene_remove(self, scene: int) -> int:
        return N.lib().ssgi_serve_scene_remove(self._h, scene)

    # -- requests -------------------------------------------------------------------------------
    def submit(self, final_out, env, params, scene: int = -1, depth=None, normal=None, albedo=None, rough=None,
               metal=None, cams=None) -> tuple:
        """Queue one request; returns (status, ticket).  final_out: host [V,H,W,3] float32."""
        p = params.c_struct() if hasattr(params, "c_struct") else params
        if scene >= 0:
            dims = N.Dims(0, 0, 0)
            cam = None
        else:
            V, H, W = depth.shape
            dims = N.Dims(V, H, W)
            cam = _cams(cams)
        req = N.Request(scene, dims, _ptr(depth), _ptr(normal), _ptr(albedo), _ptr(rough), _ptr(metal),
                        C.cast(cam, C.c_void_p) if cam is not None else None, _ptr(env), int(env.shape[0]),
                        int(env.shape[1]), p, _ptr(final_out))
        t = C.c_uint64()
        rc = N.lib().ssgi_serve_submit(self._h, C.byref(req), C.byref(t))
        if rc == N.OK:
            self._keep[t.value] = (final_out, env, depth, normal, albedo, rough, metal, cam)
        return rc, t.value

    def poll(self, ticket: int) -> tuple:
        lat = C.c_double()
        rc = N.lib().ssgi_serve_poll(self._h, ticket, C.byref(lat))
        if rc not in (N.NOT_READY, N.INVALID_ARG):
            self._keep.pop(ticket, None)
        return rc, lat.value

    def wait(self, ticket: int, timeout_ms: int) -> tuple:
        lat = C.c_double()
        rc = N.lib().ssgi_serve_wait(self._h, ticket, timeout_ms, C.byref(lat))
        if rc not in (N.NOT_READY, N.INVALID_ARG, N.TIMEOUT):
            self._keep.pop(ticket, None)
        return rc, lat.value

    def cancel(self, ticket: int) -> int:
        return N.lib().ssgi_serve_cancel(self._h, ticket)

    def stats(self) -> dict:
        st = N.ServeStats()
        N.call("ssgi_serve_stats_get", self._h, C.byref(st))
        return {k: getattr(st, k) for k, _ in N.ServeStats._fields_ if k != "pad_"}

    def close(self, timeout_ms: int = 60000) -> int:
        if self._h:
            rc = N.lib().ssgi_serve_destroy(self._h, timeout_ms)
            if rc == N.OK:
                self._h = C.c_void_p()
                self._keep.clear()
            return rc
        return N.OK

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
