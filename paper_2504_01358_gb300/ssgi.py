"""Python binding of the SSGI library: the C-ABI entry points under the same names, taking
torch CUDA tensors (argument marshalling only -- every step runs in libssgi.so's kernels),
plus a torch.autograd.Function and a preallocated frame pipeline built from those calls.

PyTorch provides device memory and streams; nothing here computes on the CPU.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N
from ._native import BRUTE_FORCE, DIFFUSE_INDIRECT, HIT_BACKGROUND, HIT_INVALID, HIT_MISS, SSGIError  # noqa: F401

LUT_N = 64
LUT_SAMPLES = 4096


# ------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------
def _stream(stream: Optional[torch.cuda.Stream] = None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _dev(t: Optional[torch.Tensor], name: str, dtype=torch.float32) -> int:
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def cameras(cams) -> C.Array:
    """Host camera array from a [V,14] float array/tensor (cam_to_world 3x4, fov_y, z_near)."""
    a = cams.detach().cpu().numpy() if isinstance(cams, torch.Tensor) else np.asarray(cams)
    a = np.ascontiguousarray(a, dtype=np.float32).reshape(-1, 14)
    arr = (N.Camera * len(a))()
    for i, rec in enumerate(a):
        arr[i].cam_to_world[:] = rec[:12].tolist()
        arr[i].fov_y_rad = float(rec[12])
        arr[i].z_near = float(rec[13])
    return arr


@dataclasses.dataclass
class GBuffer:
    """Device G-buffer planes (Sec. 3.2, eq:g-buffer): depth [V,H,W], normal [V,H,W,3],
    albedo [V,H,W,3], rough [V,H,W], metal [V,H,W]; all float32, contiguous, on one GPU."""
    depth: torch.Tensor
    normal: torch.Tensor
    albedo: torch.Tensor
    rough: torch.Tensor
    metal: torch.Tensor

    @property
    def dims(self):
        return tuple(self.depth.shape)

    def c_struct(self) -> N.GBuffer:
        V, H, W = self.depth.shape
        for name, t, shape in (("normal", self.normal, (V, H, W, 3)), ("albedo", self.albedo, (V, H, W, 3)),
                               ("rough", self.rough, (V, H, W)), ("metal", self.metal, (V, H, W))):
            if tuple(t.shape) != shape:
                raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {shape}")
        return N.GBuffer(_dev(self.depth, "depth"), _dev(self.normal, "normal"), _dev(self.albedo, "albedo"),
                         _dev(self.rough, "rough"), _dev(self.metal, "metal"), N.Dims(V, H, W))


@dataclasses.dataclass
class EnvMap:
    """Packed device mip chain of an h x w lat-long RGB map."""
    mips: torch.Tensor
    h: int
    w: int

    @property
    def levels(self) -> int:
        return ssgi_env_levels(self.h, self.w)

    def c_struct(self) -> N.EnvMap:
        return N.EnvMap(_dev(self.mips, "env mips"), self.h, self.w, self.levels)


@dataclasses.dataclass
class TraceParams:
    spp: int
    max_steps: int
    hiz_levels: int = 8
    thickness: float = 0.05
    max_distance: float = 100.0
    seed: int = 0
    flags: int = 0

    def c_struct(self) -> N.TraceParams:
        return N.TraceParams(self.spp, self.max_steps, self.hiz_levels, self.thickness, self.max_distance,
                             self.seed & 0xFFFFFFFFFFFFFFFF, self.flags)


# ------------------------------------------------------------------------------------------
# sizes
# ------------------------------------------------------------------------------------------
def ssgi_env_levels(h: int, w: int) -> int:
    return N.lib().ssgi_env_levels(h, w)


def ssgi_env_mip_floats(h: int, w: int) -> int:
    return N.lib().ssgi_env_mip_floats(h, w)


def ssgi_hiz_floats(dims, levels: int) -> int:
    V, H, W = dims
    return N.lib().ssgi_hiz_floats(N.Dims(V, H, W), levels)


def ssgi_backward_workspace_bytes(dims, env_h: int, env_w: int) -> int:
    V, H, W = dims
    return N.lib().ssgi_backward_workspace_bytes(N.Dims(V, H, W), env_h, env_w)


def ssgi_version() -> str:
    return N.lib().ssgi_version().decode()


def ssgi_status_string(code: int) -> str:
    return N.lib().ssgi_status_string(code).decode()


# ------------------------------------------------------------------------------------------
# entry points
# ------------------------------------------------------------------------------------------
def ssgi_build_brdf_lut(n: int = LUT_N, samples: int = LUT_SAMPLES, out: Optional[torch.Tensor] = None,
                        stream=None) -> torch.Tensor:
    out = torch.empty((n, n, 2), device="cuda", dtype=torch.float32) if out is None else out
    N.call("ssgi_build_brdf_lut", n, samples, _dev(out, "lut_out"), _stream(stream))
    return out


def ssgi_build_env_mips(env: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> EnvMap:
    h, w = int(env.shape[0]), int(env.shape[1])
    nf = ssgi_env_mip_floats(h, w)
    if nf == 0:
        raise ValueError("environment sides must be powers of two with width >= height")
    out = torch.empty(nf, device=env.device, dtype=torch.float32) if out is None else out
    N.call("ssgi_build_env_mips", _dev(env, "env"), h, w, _dev(out, "mips_out"), _stream(stream))
    return EnvMap(out, h, w)


def ssgi_build_hiz(depth: torch.Tensor, levels: int, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    V, H, W = depth.shape
    nf = max(ssgi_hiz_floats((V, H, W), levels), 1)
    out = torch.empty(nf, device=depth.device, dtype=torch.float32) if out is None else out
    N.call("ssgi_build_hiz", _dev(depth, "depth"), N.Dims(V, H, W), levels, _dev(out, "hiz_out"), _stream(stream))
    return out


def ssgi_shade_direct(g: GBuffer, cams, env: EnvMap, lut: torch.Tensor, c_d=None, c_s=None, c1=None,
                      want_cs: bool = False, stream=None):
    V, H, W = g.dims
    mk = lambda: torch.empty((V, H, W, 3), device=g.depth.device, dtype=torch.float32)  # noqa: E731
    c_d = mk() if c_d is None else c_d
    c1 = mk() if c1 is None else c1
    if c_s is None and want_cs:
        c_s = mk()
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    gs, es = g.c_struct(), env.c_struct()
    N.call("ssgi_shade_direct", C.byref(gs), cam, C.byref(es), _dev(lut, "lut"), int(lut.shape[0]),
           _dev(c_d, "c_d"), _dev(c_s, "c_s"), _dev(c1, "c1"), _stream(stream))
    return c_d, c_s, c1


def ssgi_trace_indirect(g: GBuffer, cams, hiz: Optional[torch.Tensor], c1: torch.Tensor, c_d: torch.Tensor,
                        env: EnvMap, params: TraceParams, c_s_mc=None, c_id=None, final=None, hit_idx=None,
                        want_hits: bool = False, want_parts: bool = False, step_count=None, stream=None):
    V, H, W = g.dims
    dev = g.depth.device
    final = torch.empty((V, H, W, 3), device=dev, dtype=torch.float32) if final is None else final
    if want_parts:
        c_s_mc = torch.empty((V, H, W, 3), device=dev, dtype=torch.float32) if c_s_mc is None else c_s_mc
        c_id = torch.empty((V, H, W, 3), device=dev, dtype=torch.float32) if c_id is None else c_id
    if want_hits and hit_idx is None:
        hit_idx = torch.empty((V, H, W, params.spp), device=dev, dtype=torch.int32)
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    gs, es, ps = g.c_struct(), env.c_struct(), params.c_struct()
    N.call("ssgi_trace_indirect", C.byref(gs), cam, _dev(hiz, "hiz"), _dev(c1, "c1"), _dev(c_d, "c_d"), C.byref(es),
           C.byref(ps), _dev(c_s_mc, "c_s_mc"), _dev(c_id, "c_id"), _dev(final, "final"),
           _dev(hit_idx, "hit_idx", torch.int32), _dev(step_count, "step_count", torch.int64), _stream(stream))
    return {"final": final, "c_s_mc": c_s_mc, "c_id": c_id, "hit_idx": hit_idx}


def ssgi_l2_loss(final: torch.Tensor, target: torch.Tensor, g_final=None, loss=None, stream=None):
    g_final = torch.empty_like(final) if g_final is None else g_final
    loss = torch.empty(1, device=final.device, dtype=torch.float32) if loss is None else loss
    N.call("ssgi_l2_loss", _dev(final, "final"), _dev(target, "target"), final.numel(), _dev(g_final, "g_final"),
           _dev(loss, "loss"), _stream(stream))
    return g_final, loss


def ssgi_backward(g_final: torch.Tensor, g: GBuffer, cams, c1: torch.Tensor, env: EnvMap, lut: torch.Tensor,
                  hit_idx: torch.Tensor, params: TraceParams, out: Optional[dict] = None,
                  workspace: Optional[torch.Tensor] = None, stream=None) -> dict:
    V, H, W = g.dims
    dev = g.depth.device
    if out is None:
        out = {"albedo": torch.empty((V, H, W, 3), device=dev), "rough": torch.empty((V, H, W), device=dev),
               "metal": torch.empty((V, H, W), device=dev), "normal": torch.empty((V, H, W, 3), device=dev),
               "env": torch.empty((env.h, env.w, 3), device=dev)}
    nbytes = ssgi_backward_workspace_bytes((V, H, W), env.h, env.w)
    if workspace is None:
        workspace = torch.empty(nbytes, device=dev, dtype=torch.uint8)
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    gs, es, ps = g.c_struct(), env.c_struct(), params.c_struct()
    N.call("ssgi_backward", _dev(g_final, "g_final"), C.byref(gs), cam, _dev(c1, "c1"), C.byref(es),
           _dev(lut, "lut"), int(lut.shape[0]), _dev(hit_idx, "hit_idx", torch.int32), C.byref(ps),
           _dev(out["albedo"], "g_albedo"), _dev(out["rough"], "g_rough"), _dev(out["metal"], "g_metal"),
           _dev(out["normal"], "g_normal"), _dev(out["env"], "g_env"), _dev(workspace, "workspace", torch.uint8),
           workspace.numel(), _stream(stream))
    return out


def ssgi_backward_noalloc(g_final: torch.Tensor, g: GBuffer, cams, c1: torch.Tensor, env: EnvMap,
                          lut: torch.Tensor, hit_idx: torch.Tensor, params: TraceParams, out: dict,
                          stream=None) -> dict:
    """ssgi_backward without a workspace argument: the library's built-in scratch array is used,
    for callers that cannot allocate device memory (outputs in `out` are still the caller's)."""
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    gs, es, ps = g.c_struct(), env.c_struct(), params.c_struct()
    N.call("ssgi_backward_noalloc", _dev(g_final, "g_final"), C.byref(gs), cam, _dev(c1, "c1"), C.byref(es),
           _dev(lut, "lut"), int(lut.shape[0]), _dev(hit_idx, "hit_idx", torch.int32), C.byref(ps),
           _dev(out["albedo"], "g_albedo"), _dev(out["rough"], "g_rough"), _dev(out["metal"], "g_metal"),
           _dev(out["normal"], "g_normal"), _dev(out["env"], "g_env"), _stream(stream))
    return out


def ssgi_step_fused_workspace_bytes(dims, env_h: int, env_w: int, hiz_levels: int) -> int:
    V, H, W = dims
    return N.lib().ssgi_step_fused_workspace_bytes(N.Dims(V, H, W), env_h, env_w, hiz_levels)


def ssgi_step_fused(g: GBuffer, cams, env: torch.Tensor, lut: torch.Tensor, target: torch.Tensor,
                    params: TraceParams, out: Optional[dict] = None, workspace: Optional[torch.Tensor] = None,
                    stream=None) -> dict:
    """One fused forward + L2 loss + backward launch over all views (outputs in a dict)."""
    V, H, W = g.dims
    dev = g.depth.device
    he, we = int(env.shape[0]), int(env.shape[1])
    if out is None:
        out = {"final": torch.empty((V, H, W, 3), device=dev), "hit_idx": torch.empty((V, H, W, params.spp),
               device=dev, dtype=torch.int32), "loss": torch.empty(1, device=dev),
               "albedo": torch.empty((V, H, W, 3), device=dev), "rough": torch.empty((V, H, W), device=dev),
               "metal": torch.empty((V, H, W), device=dev), "normal": torch.empty((V, H, W, 3), device=dev),
               "env": torch.empty((he, we, 3), device=dev)}
    nbytes = ssgi_step_fused_workspace_bytes((V, H, W), he, we, params.hiz_levels)
    if workspace is None:
        workspace = torch.empty(nbytes, device=dev, dtype=torch.uint8)
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    gs, ps = g.c_struct(), params.c_struct()
    N.call("ssgi_step_fused", C.byref(gs), cam, _dev(env, "env"), he, we, _dev(lut, "lut"), int(lut.shape[0]),
           _dev(target, "target"), C.byref(ps), _dev(out["final"], "final"), _dev(out["hit_idx"], "hit_idx", torch.int32),
           _dev(out["loss"], "loss"), _dev(out["albedo"], "g_albedo"), _dev(out["rough"], "g_rough"),
           _dev(out["metal"], "g_metal"), _dev(out["normal"], "g_normal"), _dev(out["env"], "g_env"),
           _dev(workspace, "workspace", torch.uint8), workspace.numel(), _stream(stream))
    out["_workspace"] = workspace
    return out


def ssgi_step_fused_check(workspace: torch.Tensor) -> bool:
    """True if a block of the last fused step on this workspace gave up waiting (synchronous)."""
    f = C.c_int32()
    N.call("ssgi_step_fused_check", _dev(workspace, "workspace", torch.uint8), C.byref(f))
    return bool(f.value)


def ssgi_step_fused_set_wait_limit(polls: int) -> None:
    """Polls (~100 ns each) a fused-step block waits for the previous phase before giving up; < 0: default."""
    N.call("ssgi_step_fused_set_wait_limit", int(polls))


FUSED_PHASES = ("pyramids", "shade", "trace_loss_mc", "bwd_direct", "bwd_env")


def ssgi_step_fused_phase_ns(workspace: torch.Tensor) -> dict:
    """Phase durations (ns) of the last fused step on this workspace, as seen by its first block."""
    a = (C.c_uint64 * len(FUSED_PHASES))()
    N.call("ssgi_step_fused_phase_ns", _dev(workspace, "workspace", torch.uint8), a)
    return dict(zip(FUSED_PHASES, (int(x) for x in a)))


def ssgi_tonemap_srgb(linear: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """sRGB image: clamp to [0, 1], then the sRGB transfer function (tone mapping + gamma)."""
    out = torch.empty_like(linear) if out is None else out
    N.call("ssgi_tonemap_srgb", _dev(linear, "linear"), _dev(out, "srgb"), linear.numel(), _stream(stream))
    return out


def ssgi_l2_loss_srgb(final: torch.Tensor, target: torch.Tensor, g_final=None, loss=None, stream=None):
    """loss = mean((tonemap_srgb(final) - target)^2) and its gradient with respect to final."""
    g_final = torch.empty_like(final) if g_final is None else g_final
    loss = torch.empty(1, device=final.device, dtype=torch.float32) if loss is None else loss
    N.call("ssgi_l2_loss_srgb", _dev(final, "final"), _dev(target, "target"), final.numel(),
           _dev(g_final, "g_final"), _dev(loss, "loss"), _stream(stream))
    return g_final, loss


def ssgi_env_keyframe_lerp(env_a: torch.Tensor, env_b: torch.Tensor, alpha: float,
                           out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """(1 - alpha) env_a + alpha env_b for two [h, w, 3] keyframe maps."""
    h, w = int(env_a.shape[0]), int(env_a.shape[1])
    out = torch.empty_like(env_a) if out is None else out
    N.call("ssgi_env_keyframe_lerp", _dev(env_a, "env_a"), _dev(env_b, "env_b"), float(alpha), h, w,
           _dev(out, "env_out"), _stream(stream))
    return out


def ssgi_env_keyframe_lerp_backward(g_env: torch.Tensor, alpha: float, g_a: torch.Tensor, g_b: torch.Tensor,
                                    accumulate: bool = True, stream=None) -> None:
    h, w = int(g_env.shape[0]), int(g_env.shape[1])
    N.call("ssgi_env_keyframe_lerp_backward", _dev(g_env, "g_env"), float(alpha), h, w, _dev(g_a, "g_a"),
           _dev(g_b, "g_b"), 1 if accumulate else 0, _stream(stream))


def ssgi_keyframe_of(frame: int, period: int = 10):
    """(keyframe k, alpha): env(frame) = (1 - alpha) env_k + alpha env_{k+1}."""
    k, a = C.c_int64(), C.c_float()
    N.call("ssgi_keyframe_of", int(frame), int(period), C.byref(k), C.byref(a))
    return int(k.value), float(a.value)


def ssgi_composite_gbuffer(scene: GBuffer, obj: GBuffer, out: Optional[GBuffer] = None, mask: bool = False,
                           stream=None):
    """Object insertion: merge `obj` into `scene` by depth (in place when `out` is None or `scene`).
    Returns (out G-buffer, mask [V,H,W] uint8 or None)."""
    out = scene if out is None else out
    m = torch.empty(scene.dims, device=scene.depth.device, dtype=torch.uint8) if mask else None
    gs, go = scene.c_struct(), obj.c_struct()
    N.call("ssgi_composite_gbuffer", C.byref(gs), C.byref(go), _dev(out.depth, "depth"), _dev(out.normal, "normal"),
           _dev(out.albedo, "albedo"), _dev(out.rough, "rough"), _dev(out.metal, "metal"),
           _dev(m, "mask", torch.uint8), _stream(stream))
    return out, m


def ssgi_depth_normals(depth: torch.Tensor, cams, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """World-space normals [V,H,W,3] from a depth buffer [V,H,W] by finite differences."""
    V, H, W = depth.shape
    if out is None:
        out = torch.empty((V, H, W, 3), device=depth.device, dtype=torch.float32)
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    N.call("ssgi_depth_normals", _dev(depth, "depth"), N.Dims(V, H, W), cam, _dev(out, "normal_out"), _stream(stream))
    return out


def ssgi_build_hiz_normals(depth: torch.Tensor, cams, levels: int, hiz: Optional[torch.Tensor] = None,
                           normals: Optional[torch.Tensor] = None, stream=None):
    """(pyramid, normals) from one pass over depth: ssgi_build_hiz and ssgi_depth_normals fused."""
    V, H, W = depth.shape
    if hiz is None and levels > 1:
        hiz = torch.empty(max(ssgi_hiz_floats((V, H, W), levels), 1), device=depth.device, dtype=torch.float32)
    if normals is None:
        normals = torch.empty((V, H, W, 3), device=depth.device, dtype=torch.float32)
    cam = cams if isinstance(cams, C.Array) else cameras(cams)
    N.call("ssgi_build_hiz_normals", _dev(depth, "depth"), N.Dims(V, H, W), cam, levels, _dev(hiz, "hiz_out"),
           _dev(normals, "normal_out"), _stream(stream))
    return hiz, normals


def ssgi_read_bandwidth_probe(buf: torch.Tensor, reps: int, sink: Optional[torch.Tensor] = None,
                              stream=None) -> None:
    """Streams the bytes of `buf` (a contiguous CUDA tensor) `reps` times through L2."""
    if not (buf.is_cuda and buf.is_contiguous()):
        raise ValueError("buf: contiguous CUDA tensor expected")
    if sink is None:
        sink = torch.zeros(1, device=buf.device, dtype=torch.int32)
    N.call("ssgi_read_bandwidth_probe", C.c_void_p(buf.data_ptr()), buf.numel() * buf.element_size(), int(reps),
           _dev(sink, "sink", torch.int32), _stream(stream))


# ------------------------------------------------------------------------------------------
# autograd
# ------------------------------------------------------------------------------------------
class SSGIFunction(torch.autograd.Function):
    """final = SSGI(depth, normal, albedo, rough, metal, env) for fixed cameras and params.

    Forward runs build_env_mips -> build_hiz -> shade_direct -> trace_indirect and stores the
    hit indices; backward runs ssgi_backward (no re-march).  depth gets no gradient."""

    @staticmethod
    def forward(ctx, depth, normal, albedo, rough, metal, env, cams, params: TraceParams, lut):
        g = GBuffer(depth.contiguous(), normal.contiguous(), albedo.contiguous(), rough.contiguous(),
                    metal.contiguous())
        cam = cameras(cams)
        em = ssgi_build_env_mips(env.contiguous())
        hiz = ssgi_build_hiz(g.depth, params.hiz_levels) if params.hiz_levels > 1 else None
        c_d, _, c1 = ssgi_shade_direct(g, cam, em, lut)
        tr = ssgi_trace_indirect(g, cam, hiz, c1, c_d, em, params, want_hits=True)
        ctx.params, ctx.cam, ctx.em, ctx.lut = params, cam, em, lut
        ctx.save_for_backward(depth, normal, albedo, rough, metal, c1, tr["hit_idx"])
        return tr["final"]

    @staticmethod
    def backward(ctx, g_final):
        depth, normal, albedo, rough, metal, c1, hit_idx = ctx.saved_tensors
        g = GBuffer(depth.contiguous(), normal.contiguous(), albedo.contiguous(), rough.contiguous(),
                    metal.contiguous())
        gr = ssgi_backward(g_final.contiguous(), g, ctx.cam, c1, ctx.em, ctx.lut, hit_idx, ctx.params)
        return None, gr["normal"], gr["albedo"], gr["rough"], gr["metal"], gr["env"], None, None, None


def ssgi_render(depth, normal, albedo, rough, metal, env, cams, params: TraceParams, lut) -> torch.Tensor:
    return SSGIFunction.apply(depth, normal, albedo, rough, metal, env, cams, params, lut)


# ------------------------------------------------------------------------------------------
# preallocated frame pipeline (one forward + loss + backward with no allocation per step)
# ------------------------------------------------------------------------------------------
class FramePipeline:
    """All device buffers of one inverse-rendering step at fixed sizes.

    step() = env mips -> Hi-Z -> direct shading -> trace (hits stored) -> L2 loss ->
    backward, each a libssgi.so call on the current stream."""

    def __init__(self, dims, env_hw, params: TraceParams, cams, lut: Optional[torch.Tensor] = None,
                 device: str = "cuda"):
        V, H, W = dims
        self.dims, self.params = (V, H, W), params
        self.cam = cameras(cams)
        he, we = env_hw
        f = lambda *s: torch.empty(s, device=device, dtype=torch.float32)  # noqa: E731
        self.g = GBuffer(f(V, H, W), f(V, H, W, 3), f(V, H, W, 3), f(V, H, W), f(V, H, W))
        self.env = f(he, we, 3)
        self.target = f(V, H, W, 3)
        self.em = EnvMap(f(ssgi_env_mip_floats(he, we)), he, we)
        self.hiz = f(max(ssgi_hiz_floats((V, H, W), params.hiz_levels), 1))
        self.lut = ssgi_build_brdf_lut() if lut is None else lut
        self.c_d, self.c1, self.final, self.g_final = f(V, H, W, 3), f(V, H, W, 3), f(V, H, W, 3), f(V, H, W, 3)
        self.loss = f(1)
        self.hit_idx = torch.empty((V, H, W, params.spp), device=device, dtype=torch.int32)
        self.grads = {"albedo": f(V, H, W, 3), "rough": f(V, H, W), "metal": f(V, H, W), "normal": f(V, H, W, 3),
                      "env": f(he, we, 3)}
        self.ws = torch.empty(ssgi_backward_workspace_bytes((V, H, W), he, we), device=device, dtype=torch.uint8)

    def load(self, wl) -> None:
        """Copy a workload's host arrays (ssgi_inputs.Workload) into the device buffers."""
        for name in ("depth", "normal", "albedo", "rough", "metal"):
            getattr(self.g, name).copy_(torch.from_numpy(np.ascontiguousarray(getattr(wl, name))))
        self.env.copy_(torch.from_numpy(np.ascontiguousarray(wl.env)))
        if wl.target is not None:
            self.target.copy_(torch.from_numpy(np.ascontiguousarray(wl.target)))

    # -- the stages of one step, each one C-ABI call ------------------------------------------
    def env_mips(self, stream=None) -> None:
        ssgi_build_env_mips(self.env, out=self.em.mips, stream=stream)

    def hiz_build(self, stream=None) -> None:
        if self.params.hiz_levels > 1:
            ssgi_build_hiz(self.g.depth, self.params.hiz_levels, out=self.hiz, stream=stream)

    def shade(self, stream=None) -> None:
        ssgi_shade_direct(self.g, self.cam, self.em, self.lut, c_d=self.c_d, c1=self.c1, stream=stream)

    def trace(self, stream=None, step_count=None) -> None:
        ssgi_trace_indirect(self.g, self.cam, self.hiz, self.c1, self.c_d, self.em, self.params, final=self.final,
                            hit_idx=self.hit_idx, step_count=step_count, stream=stream)

    def loss_grad(self, stream=None) -> None:
        loss = ssgi_l2_loss_srgb if self.params.flags & N.SRGB_LOSS else ssgi_l2_loss
        loss(self.final, self.target, g_final=self.g_final, loss=self.loss, stream=stream)

    def adjoint(self, stream=None) -> None:
        ssgi_backward(self.g_final, self.g, self.cam, self.c1, self.em, self.lut, self.hit_idx, self.params,
                      out=self.grads, workspace=self.ws, stream=stream)

    def stages(self):
        return [("env_mips", self.env_mips), ("hiz", self.hiz_build), ("shade", self.shade), ("trace", self.trace),
                ("loss", self.loss_grad), ("backward", self.adjoint)]

    def forward(self, stream=None) -> None:
        self.env_mips(stream)
        self.hiz_build(stream)
        self.shade(stream)
        self.trace(stream)

    def backward(self, stream=None) -> None:
        self.loss_grad(stream)
        self.adjoint(stream)

    def step(self, stream=None) -> None:
        self.forward(stream)
        self.backward(stream)

    def kernels_per_step(self) -> int:
        """Kernel launches of libssgi.so in one step (as issued by the .cu entry points):
        env mips 1 (+1 above 6 levels), Hi-Z 1 (+1 above 6 levels; none for 1 level), shade 1,
        trace 1, loss 1, backward 3."""
        env = 1 + (1 if self.em.levels > 6 else 0)
        hz = 0 if self.params.hiz_levels <= 1 else 1 + (1 if self.params.hiz_levels > 6 else 0)
        return env + hz + 1 + 1 + 1 + 3

    def h2d_bytes(self) -> int:
        ts = [self.g.depth, self.g.normal, self.g.albedo, self.g.rough, self.g.metal, self.env, self.target]
        return sum(t.numel() * t.element_size() for t in ts)


def to_device_workload(wl, device: str = "cuda"):
    """(GBuffer, env tensor, cams array, target or None) of an ssgi_inputs.Workload."""
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device)  # noqa: E731
    g = GBuffer(t(wl.depth), t(wl.normal), t(wl.albedo), t(wl.rough), t(wl.metal))
    return g, t(wl.env), wl.cams, (t(wl.target) if wl.target is not None else None)


def params_of(wl_params) -> TraceParams:
    p = wl_params
    return TraceParams(p.spp, p.max_steps, p.hiz_levels, p.thickness, p.max_distance, p.seed, p.flags)


def exported_symbols() -> Sequence[str]:
    return N.EXPORTED
