"""ctypes + numpy wrapper of the FP64 C oracle (ssgi_oracle.c).  Test infrastructure only.

Every array handed to the C side is promoted to float64 (exact for FP32 inputs).  Functions
mirror the steps of the method (Sec. 3.2 direct shading, Sec. 3.3 trace and Monte-Carlo sum,
and the replay-mode adjoint); see the C file for the definitions and citations.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

__all__ = [
    "build", "lib", "philox4x32_10", "ggx_D", "ggx_G1", "fresnel", "ggx_sample_h", "env_levels",
    "build_env_mips", "env_lookup", "build_lut", "lut_sample", "hiz_floats_per_view", "build_hiz",
    "shade_direct", "depth_normals", "composite_gbuffer", "GBUFFER_KEYS", "srgb_oetf", "tonemap_srgb",
    "tonemap_srgb_grad", "l2_loss_srgb", "keyframe_of", "keyframe_lerp", "trace", "replay_final", "backward", "set_threads", "set_pathwise_step", "max_threads", "FLAG_DIFFUSE_INDIRECT",
    "FLAG_BRUTE_FORCE", "FLAG_PATHWISE", "MISS", "INVALID", "BACKGROUND", "forward", "hiz_levels_split", "LUT_N", "LUT_SAMPLES",
]

FLAG_DIFFUSE_INDIRECT = 1
FLAG_BRUTE_FORCE = 2
FLAG_PATHWISE = 4
MISS, INVALID, BACKGROUND = -1, -2, -3
LUT_N = 64          # table resolution used by the presets
LUT_SAMPLES = 4096  # Hammersley samples per table entry

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssgi_oracle.c")
_SO = os.path.join(_HERE, "libssgi_oracle.so")
_lock = threading.Lock()
_lib = None

D = C.c_double
I32 = C.c_int32
I64 = C.c_int64
PD = C.POINTER(C.c_double)
PI32 = C.POINTER(C.c_int32)
PI64 = C.POINTER(C.c_int64)
PU32 = C.POINTER(C.c_uint32)


def build(force: bool = False) -> str:
    """Compile ssgi_oracle.c into libssgi_oracle.so with gcc (-O2, OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_SO)
            L.orc_philox4x32_10.argtypes = [PU32, PU32, PU32]
            L.orc_ggx_D.restype = D
            L.orc_ggx_D.argtypes = [D, D]
            L.orc_ggx_G1.restype = D
            L.orc_ggx_G1.argtypes = [D, D]
            L.orc_fresnel.restype = D
            L.orc_fresnel.argtypes = [D, D]
            L.orc_ggx_sample_h.argtypes = [PD, D, D, D, PD]
            L.orc_env_levels.argtypes = [C.c_int, C.c_int]
            L.orc_env_mip_doubles.restype = C.c_long
            L.orc_env_mip_doubles.argtypes = [C.c_int, C.c_int]
            L.orc_build_env_mips.argtypes = [PD, C.c_int, C.c_int, PD]
            L.orc_env_lookup.argtypes = [PD, C.c_int, C.c_int, PD, D, PD]
            L.orc_build_lut.argtypes = [C.c_int, C.c_int, PD]
            L.orc_lut_sample.argtypes = [PD, C.c_int, D, D, PD]
            L.orc_hiz_floats_per_view.restype = C.c_long
            L.orc_hiz_floats_per_view.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_build_hiz.argtypes = [PD, C.c_int, C.c_int, C.c_int, C.c_int, PD]
            L.orc_shade_direct.argtypes = [C.c_int] * 3 + [PD] * 7 + [C.c_int, C.c_int, PD, C.c_int, PD, PD, PD]
            L.orc_trace.restype = C.c_int
            L.orc_trace.argtypes = ([C.c_int] * 3 + [PD] * 7 + [C.c_int, C.c_int] + [PD] * 3 +
                                    [C.c_int, C.c_int, C.c_int, D, D, C.c_uint64, C.c_uint32, PI64, C.c_long,
                                     PD, PD, PD, PI32, PI32, PD])
            L.orc_replay_final.restype = C.c_int
            L.orc_replay_final.argtypes = ([C.c_int] * 3 + [PD, PD, C.c_int, C.c_int, PD, C.c_int, C.c_int,
                                           C.c_uint64, C.c_uint32] + [PD] * 7 + [PI32, PD])
            L.orc_backward.restype = C.c_int
            L.orc_backward.argtypes = ([C.c_int] * 3 + [PD] * 7 + [C.c_int, C.c_int, PD, C.c_int, PD, PI32, PD,
                                       C.c_int, C.c_uint64, C.c_uint32] + [PD] * 5)
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_depth_normals.argtypes = [C.c_int] * 3 + [PD, PD, PD]
            L.orc_set_pathwise_step.argtypes = [D, C.c_int]
            L.orc_max_threads.restype = C.c_int
            _lib = L
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _p(a, t=PD):
    return None if a is None else a.ctypes.data_as(t)


# ---------------------------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c, PU32), _p(k, PU32), _p(o, PU32))
    return o


def ggx_D(nh: float, rho: float) -> float:
    return lib().orc_ggx_D(nh, rho)


def ggx_G1(z: float, rho: float) -> float:
    return lib().orc_ggx_G1(z, rho)


def fresnel(F0: float, vh: float) -> float:
    return lib().orc_fresnel(F0, vh)


def ggx_sample_h(n, rho, xi0, xi1) -> np.ndarray:
    nn = _d(n)
    h = np.zeros(3)
    lib().orc_ggx_sample_h(_p(nn), rho, xi0, xi1, _p(h))
    return h


def env_levels(He: int, We: int) -> int:
    return lib().orc_env_levels(He, We)


def build_env_mips(env) -> np.ndarray:
    env = _d(env)
    He, We = env.shape[:2]
    n = lib().orc_env_mip_doubles(He, We)
    if n < 0:
        raise ValueError("environment sides must be powers of two with width >= height")
    out = np.zeros(n)
    lib().orc_build_env_mips(_p(env), He, We, _p(out))
    return out


def env_lookup(mips, He, We, d, lam) -> np.ndarray:
    m = _d(mips)
    dd = _d(d)
    out = np.zeros(3)
    lib().orc_env_lookup(_p(m), He, We, _p(dd), lam, _p(out))
    return out


def build_lut(N: int = LUT_N, M: int = LUT_SAMPLES) -> np.ndarray:
    out = np.zeros((N, N, 2))
    lib().orc_build_lut(N, M, _p(out))
    return out


def lut_sample(lut, rho, mu):
    t = _d(lut)
    out = np.zeros(2)
    lib().orc_lut_sample(_p(t), t.shape[0], rho, mu, _p(out))
    return out


def hiz_floats_per_view(H, W, levels) -> int:
    return lib().orc_hiz_floats_per_view(H, W, levels)


def build_hiz(depth, levels: int) -> np.ndarray:
    """depth [V,H,W] -> packed levels 1..levels-1 per view, [V, per_view] float64."""
    dep = _d(depth)
    V, H, W = dep.shape
    per = hiz_floats_per_view(H, W, levels)
    out = np.zeros((V, max(per, 0)))
    lib().orc_build_hiz(_p(dep), V, H, W, levels, _p(out))
    return out


def hiz_levels_split(hiz_view: np.ndarray, H: int, W: int, levels: int):
    """Unpack one view's packed pyramid into a list of 2-D arrays (levels 1..levels-1)."""
    out, off = [], 0
    for l in range(1, levels):
        hl, wl = -(-H // (1 << l)), -(-W // (1 << l))
        out.append(hiz_view[off:off + hl * wl].reshape(hl, wl))
        off += hl * wl
    return out


# ---------------------------------------------------------------------------------------------
# the method
# ---------------------------------------------------------------------------------------------
def shade_direct(depth, normal, albedo, rough, metal, cams, mips, He, We, lut):
    dep = _d(depth)
    V, H, W = dep.shape
    nrm, alb, rgh, met, cm, mp, lt = map(_d, (normal, albedo, rough, metal, cams, mips, lut))
    cd = np.zeros((V, H, W, 3))
    cs = np.zeros((V, H, W, 3))
    c1 = np.zeros((V, H, W, 3))
    lib().orc_shade_direct(V, H, W, _p(dep), _p(nrm), _p(alb), _p(rgh), _p(met), _p(cm), _p(mp), He, We, _p(lt),
                           lt.shape[0], _p(cd), _p(cs), _p(c1))
    return cd, cs, c1


def trace(depth, normal, albedo, rough, metal, cams, mips, He, We, hiz, c1, cd, spp, max_steps, hiz_levels,
          thickness, max_distance, seed, flags=0, pix_list=None):
    """Returns dict(cs_mc, final, cid, hit_idx, iters, margin).  With `pix_list` (linear indices
    into [V,H,W]) only those pixels are traced and outputs are indexed by list position."""
    dep = _d(depth)
    V, H, W = dep.shape
    nrm, alb, rgh, met, cm, mp, c1d, cdd = map(_d, (normal, albedo, rough, metal, cams, mips, c1, cd))
    hz = None if hiz is None else _d(hiz)
    if pix_list is not None:
        pl = np.ascontiguousarray(np.asarray(pix_list, dtype=np.int64))
        n = len(pl)
        shape = (n,)
    else:
        pl, n, shape = None, 0, (V, H, W)
    out = {
        "cs_mc": np.zeros(shape + (3,)), "final": np.zeros(shape + (3,)), "cid": np.zeros(shape + (3,)),
        "hit_idx": np.zeros(shape + (spp,), np.int32), "iters": np.zeros(shape + (spp,), np.int32),
        "margin": np.zeros(shape + (spp,)),
    }
    rc = lib().orc_trace(V, H, W, _p(dep), _p(nrm), _p(alb), _p(rgh), _p(met), _p(cm), _p(mp), He, We, _p(hz),
                         _p(c1d), _p(cdd), spp, max_steps, hiz_levels, thickness, max_distance, seed, flags,
                         _p(pl, PI64), n, _p(out["cs_mc"]), _p(out["final"]), _p(out["cid"]),
                         _p(out["hit_idx"], PI32), _p(out["iters"], PI32), _p(out["margin"]))
    if rc != 0:
        raise ValueError("orc_trace rejected its arguments")
    return out


def replay_final(depth, cams, He, We, lut, spp, seed, flags, normal_b, rough_b, normal_e, albedo_e, rough_e,
                 metal_e, env_e, hit_idx):
    dep = _d(depth)
    V, H, W = dep.shape
    cm, lt, nb, rb, ne, ae, re_, me, ee = map(_d, (cams, lut, normal_b, rough_b, normal_e, albedo_e, rough_e,
                                                  metal_e, env_e))
    hi = np.ascontiguousarray(np.asarray(hit_idx, dtype=np.int32))
    out = np.zeros((V, H, W, 3))
    rc = lib().orc_replay_final(V, H, W, _p(dep), _p(cm), He, We, _p(lt), lt.shape[0], spp, seed, flags, _p(nb),
                                _p(rb), _p(ne), _p(ae), _p(re_), _p(me), _p(ee), _p(hi, PI32), _p(out))
    if rc != 0:
        raise ValueError("orc_replay_final rejected its arguments")
    return out


def backward(depth, normal, albedo, rough, metal, cams, mips, He, We, lut, c1, hit_idx, g_final, spp, seed,
             flags=0):
    dep = _d(depth)
    V, H, W = dep.shape
    nrm, alb, rgh, met, cm, mp, lt, c1d, gf = map(_d, (normal, albedo, rough, metal, cams, mips, lut, c1, g_final))
    hi = np.ascontiguousarray(np.asarray(hit_idx, dtype=np.int32))
    ga = np.zeros((V, H, W, 3))
    gr = np.zeros((V, H, W))
    gm = np.zeros((V, H, W))
    gn = np.zeros((V, H, W, 3))
    ge = np.zeros((He, We, 3))
    rc = lib().orc_backward(V, H, W, _p(dep), _p(nrm), _p(alb), _p(rgh), _p(met), _p(cm), _p(mp), He, We, _p(lt),
                            lt.shape[0], _p(c1d), _p(hi, PI32), _p(gf), spp, seed, flags, _p(ga), _p(gr), _p(gm),
                            _p(gn), _p(ge))
    if rc != 0:
        raise ValueError("orc_backward rejected its arguments")
    return {"albedo": ga, "rough": gr, "metal": gm, "normal": gn, "env": ge}


# ---- output transform and keyframe lighting (Sec. 3.3 composite sentence; Sec. 4 implementation) ----
def srgb_oetf(x):
    """The sRGB transfer function (IEC 61966-2-1) on [0, 1]: 12.92 x up to 0.0031308, then
    1.055 x^(1/2.4) - 0.055."""
    x = np.asarray(x, np.float64)
    return np.where(x <= 0.0031308, 12.92 * x, 1.055 * np.power(np.maximum(x, 0.0031308), 1.0 / 2.4) - 0.055)


def tonemap_srgb(linear):
    """Tone mapping and gamma correction to sRGB after the composite: clamp to [0, 1], then the
    sRGB transfer function."""
    return srgb_oetf(np.clip(np.asarray(linear, np.float64), 0.0, 1.0))


def tonemap_srgb_grad(linear):
    """d tonemap_srgb / d linear: 0 outside [0, 1], the transfer function's slope inside."""
    x = np.asarray(linear, np.float64)
    inside = (x >= 0.0) & (x <= 1.0)
    slope = np.where(x <= 0.0031308, 12.92, 1.055 / 2.4 * np.power(np.maximum(x, 0.0031308), 1.0 / 2.4 - 1.0))
    return np.where(inside, slope, 0.0)


def l2_loss_srgb(final, target):
    """loss = mean((tonemap_srgb(final) - target)^2) and its gradient with respect to final."""
    f = np.asarray(final, np.float64)
    r = tonemap_srgb(f) - np.asarray(target, np.float64)
    return float(np.mean(r * r)), 2.0 * r * tonemap_srgb_grad(f) / r.size


def keyframe_of(frame: int, period: int = 10):
    """Sec. 4 (implementation): every `period`-th frame is a keyframe with its own environment
    map; a frame in between linearly interpolates its two neighbouring keyframes.  Returns
    (k, alpha): env(frame) = (1 - alpha) env_k + alpha env_{k+1}."""
    return frame // period, (frame % period) / period


def keyframe_lerp(env_a, env_b, alpha: float):
    return (1.0 - alpha) * np.asarray(env_a, np.float64) + alpha * np.asarray(env_b, np.float64)


GBUFFER_KEYS = ("depth", "normal", "albedo", "rough", "metal")


def composite_gbuffer(scene: dict, obj: dict):
    """Object insertion (Sec. 4, "Object Insertion"): the object's G-buffer, rendered on its own,
    is merged into the scene's by depth comparison.  A pixel takes all five of the object's
    channels where the object's depth is strictly smaller (nearer) than the scene's; ties and
    object background (+inf) keep the scene.  Returns (merged channels, mask of object pixels)."""
    win = np.asarray(obj["depth"]) < np.asarray(scene["depth"])
    out = {}
    for k in GBUFFER_KEYS:
        a, b = np.asarray(scene[k]), np.asarray(obj[k])
        w = win[..., None] if a.ndim == win.ndim + 1 else win
        out[k] = np.where(w, b, a)
    return out, win


def depth_normals(depth, cams) -> np.ndarray:
    """World-space normals [V,H,W,3] from the depth buffer by finite differences (Sec. 3.1)."""
    dep = _d(depth)
    V, H, W = dep.shape
    cm = _d(cams)
    out = np.zeros((V, H, W, 3))
    lib().orc_depth_normals(V, H, W, _p(dep), _p(cm), _p(out))
    return out


def set_pathwise_step(h: float, mode: int = 0) -> None:
    """Step (default 1e-6) and form (0 central, +1 forward, -1 backward) of the oracle's
    differences for pathwise n / rho derivatives."""
    lib().orc_set_pathwise_step(float(h), int(mode))


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def max_threads() -> int:
    return lib().orc_max_threads()


def forward(wl, lut=None, flags=None, brute=False, pix_list=None):
    """Whole forward pass of a workload (ssgi_inputs.Workload): env mips, Hi-Z, direct shading,
    trace.  Returns a dict with every intermediate."""
    p = wl.params
    fl = p.flags if flags is None else flags
    if brute:
        fl |= FLAG_BRUTE_FORCE
    He, We = wl.env.shape[:2]
    if lut is None:
        lut = build_lut()
    mips = build_env_mips(wl.env)
    hiz = build_hiz(wl.depth, p.hiz_levels)
    cd, cs, c1 = shade_direct(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, mips, He, We, lut)
    tr = trace(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, mips, He, We, hiz, c1, cd, p.spp,
               p.max_steps, p.hiz_levels, p.thickness, p.max_distance, p.seed, fl, pix_list=pix_list)
    tr.update({"mips": mips, "hiz": hiz, "cd": cd, "cs": cs, "c1": c1, "lut": lut})
    return tr
