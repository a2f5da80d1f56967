"""Seeded synthetic inputs for the SSGI hot path (shared by the oracle tests and the CUDA path).

This module only *makes inputs*: analytic scenes ray-cast into an FP32 G-buffer, cameras,
log-normal environment maps and loss targets.  It holds none of the shading or tracing
arithmetic of the method; both the CPU oracle and the CUDA library consume what it returns.

The scenes stand in for the paper's garage/campus captures (Sec. 4, "Datasets"), which are not
available: an enclosed, floor-dominated view with a reflective ground, boxes and tilted mirror
quads, shaped like the workloads the paper renders (Sec. 3.3, Table 2).

Conventions (the same ones the library header documents):
  * world is right-handed, y up; a camera looks down its own -z axis;
  * camera record = 14 float32: cam_to_world 3x4 row-major [R | eye] (columns of R are the
    camera's right, up and back axes in world space), vertical FOV in radians, z_near;
  * pixel (x, y) centre is (x + 0.5, y + 0.5) with y pointing down; focal length in pixels
    f = (H / 2) / tan(fov_y / 2); principal point (W / 2, H / 2);
  * depth is linear depth (distance along the camera's forward axis); background = +inf.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

CAM_FLOATS = 14


# --------------------------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------------------------
def look_at(eye, target, fov_y_deg: float = 60.0, z_near: float = 0.01, up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """Camera record (14 float32) for a pinhole camera at `eye` looking at `target`."""
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up, np.float64))
    right /= np.linalg.norm(right)
    upv = np.cross(right, fwd)
    rot = np.stack([right, upv, -fwd], axis=1)  # columns: camera x, y, z in world
    rec = np.zeros(CAM_FLOATS, np.float64)
    rec[0:12] = np.concatenate([rot, eye[:, None]], axis=1).reshape(-1)
    rec[12] = math.radians(fov_y_deg)
    rec[13] = z_near
    return rec.astype(np.float32)


def pixel_rays(cam: np.ndarray, H: int, W: int) -> Tuple[np.ndarray, np.ndarray]:
    """World-space pixel-centre ray directions with unit forward component, and the eye."""
    cam = cam.astype(np.float64)
    m = cam[:12].reshape(3, 4)
    rot, eye = m[:, :3], m[:, 3]
    f = (H / 2.0) / math.tan(cam[12] / 2.0)
    xs = (np.arange(W) + 0.5 - W / 2.0) / f
    ys = -(np.arange(H) + 0.5 - H / 2.0) / f
    dc = np.stack(np.broadcast_arrays(xs[None, :], ys[:, None], -np.ones((H, W))), axis=-1)
    return dc @ rot.T, eye


# --------------------------------------------------------------------------------------------
# analytic scene
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Material:
    albedo: Tuple[float, float, float]
    rough: float
    metal: float


@dataclasses.dataclass
class Box:
    lo: np.ndarray
    hi: np.ndarray
    mat: Material


@dataclasses.dataclass
class Quad:
    centre: np.ndarray
    axis_u: np.ndarray  # unit, half extent hu
    axis_v: np.ndarray  # unit, half extent hv
    hu: float
    hv: float
    mat: Material


@dataclasses.dataclass
class Scene:
    ground: Optional[Material]
    ground_half: float
    boxes: List[Box]
    quads: List[Quad]


def _rand_material(rng: np.random.Generator) -> Material:
    a = rng.uniform(0.05, 0.95, size=3)
    r = rng.uniform(0.05, 1.0)
    m = 1.0 if rng.uniform() < 0.2 else 0.0
    return Material(tuple(float(x) for x in a), float(r), float(m))


def make_scene(seed: int, n_boxes: int, spread: float, n_mirrors: int = 0,
               ground_half: float = 40.0) -> Scene:
    """Ground plane y=0 + `n_boxes` axis-aligned boxes (sides U[0.3,1.5], centres x,z ~
    U[-spread, spread], resting on the ground) + `n_mirrors` 3x2 mirror quads tilted 15 degrees
    about x then given a random yaw (roughness 0.02, metallic 1, albedo 0.95)."""
    rng = np.random.default_rng(seed)
    ground = _rand_material(rng)
    boxes = []
    for _ in range(n_boxes):
        size = rng.uniform(0.3, 1.5, size=3)
        cx, cz = rng.uniform(-spread, spread, size=2)
        lo = np.array([cx - size[0] / 2, 0.0, cz - size[2] / 2])
        hi = np.array([cx + size[0] / 2, size[1], cz + size[2] / 2])
        boxes.append(Box(lo, hi, _rand_material(rng)))
    quads = []
    for _ in range(n_mirrors):
        cx, cz = rng.uniform(-spread, spread, size=2)
        yaw = rng.uniform(0.0, 2.0 * math.pi)
        tilt = math.radians(15.0)
        # local frame: u horizontal (width 3), v "up" (height 2) tilted about x, then yawed
        u0 = np.array([1.0, 0.0, 0.0])
        v0 = np.array([0.0, math.cos(tilt), -math.sin(tilt)])
        cy, sy = math.cos(yaw), math.sin(yaw)
        rot_y = np.array([[cy, 0.0, sy], [0.0, 1.0, 0.0], [-sy, 0.0, cy]])
        u, v = rot_y @ u0, rot_y @ v0
        centre = np.array([cx, 0.0, cz]) + v * 1.0 + np.array([0.0, 0.05, 0.0])
        quads.append(Quad(centre, u, v, 1.5, 1.0, Material((0.95, 0.95, 0.95), 0.02, 1.0)))
    return Scene(ground, ground_half, boxes, quads)


def _screen_rect(cam: np.ndarray, H: int, W: int, lo, hi):
    """Pixel slices covering the projection of the box [lo, hi] (the whole image if a corner
    lies behind the camera).  Only narrows the search; every covered pixel is still ray-cast."""
    c = cam.astype(np.float64)
    m = c[:12].reshape(3, 4)
    rot, eye = m[:, :3], m[:, 3]
    f = (H / 2.0) / math.tan(c[12] / 2.0)
    corners = np.array([[x, y, z] for x in (lo[0], hi[0]) for y in (lo[1], hi[1]) for z in (lo[2], hi[2])])
    q = (corners - eye) @ rot
    z = -q[:, 2]
    if np.any(z <= 1e-3):
        return slice(0, H), slice(0, W)
    sx = W / 2.0 + f * q[:, 0] / z
    sy = H / 2.0 - f * q[:, 1] / z
    x0, x1 = int(max(0, math.floor(sx.min()) - 1)), int(min(W, math.ceil(sx.max()) + 1))
    y0, y1 = int(max(0, math.floor(sy.min()) - 1)), int(min(H, math.ceil(sy.max()) + 1))
    if x0 >= x1 or y0 >= y1:
        return slice(0, 0), slice(0, 0)
    return slice(y0, y1), slice(x0, x1)


def raycast_gbuffer(scene: Scene, cam: np.ndarray, H: int, W: int) -> dict:
    """Ray-cast the analytic scene through the pixel centres of `cam` into an FP32 G-buffer.

    Returns depth [H,W] (linear, +inf for background), normal [H,W,3] (unit, facing the camera),
    albedo [H,W,3], rough [H,W], metal [H,W]."""
    d, eye = pixel_rays(cam, H, W)  # forward component of d is 1, so t == linear depth
    t_best = np.full((H, W), np.inf)
    nrm = np.zeros((H, W, 3))
    alb = np.zeros((H, W, 3))
    rough = np.zeros((H, W))
    metal = np.zeros((H, W))

    def commit(t, normal, mat):
        better = t < t_best
        t_best[better] = t[better]
        if normal.ndim == 1:
            nrm[better] = normal
        else:
            nrm[better] = normal[better]
        alb[better] = mat.albedo
        rough[better] = mat.rough
        metal[better] = mat.metal

    with np.errstate(divide="ignore", invalid="ignore"):
        if scene.ground is not None:
            t = -eye[1] / d[..., 1]
            p = eye + t[..., None] * d
            ok = (t > 1e-6) & (np.abs(p[..., 0]) <= scene.ground_half) & (np.abs(p[..., 2]) <= scene.ground_half)
            commit(np.where(ok, t, np.inf), np.array([0.0, 1.0, 0.0]), scene.ground)
        for b in scene.boxes:
            ys, xs = _screen_rect(cam, H, W, b.lo, b.hi)
            dd = d[ys, xs]
            t0 = (b.lo - eye) / dd
            t1 = (b.hi - eye) / dd
            tmin = np.minimum(t0, t1)
            tmax = np.maximum(t0, t1)
            t_in = tmin.max(axis=-1)
            t_out = tmax.min(axis=-1)
            ok = (t_in <= t_out) & (t_in > 1e-6)
            axis = tmin.argmax(axis=-1)
            sign = -np.sign(np.take_along_axis(dd, axis[..., None], axis=-1)[..., 0])
            n = np.zeros(dd.shape)
            np.put_along_axis(n, axis[..., None], sign[..., None], axis=-1)
            tb = t_best[ys, xs]
            better = np.where(ok, t_in, np.inf) < tb
            tb[better] = t_in[better]
            t_best[ys, xs] = tb
            sub = nrm[ys, xs]
            sub[better] = n[better]
            nrm[ys, xs] = sub
            sub = alb[ys, xs]
            sub[better] = b.mat.albedo
            alb[ys, xs] = sub
            sub = rough[ys, xs]
            sub[better] = b.mat.rough
            rough[ys, xs] = sub
            sub = metal[ys, xs]
            sub[better] = b.mat.metal
            metal[ys, xs] = sub
        for q in scene.quads:
            nq = np.cross(q.axis_u, q.axis_v)
            denom = d @ nq
            t = ((q.centre - eye) @ nq) / denom
            p = eye + t[..., None] * d - q.centre
            ok = (t > 1e-6) & (np.abs(p @ q.axis_u) <= q.hu) & (np.abs(p @ q.axis_v) <= q.hv)
            n = np.where((denom > 0)[..., None], -nq, nq)
            commit(np.where(ok, t, np.inf), n, q.mat)

    return {
        "depth": t_best.astype(np.float32),
        "normal": nrm.astype(np.float32),
        "albedo": alb.astype(np.float32),
        "rough": rough.astype(np.float32),
        "metal": metal.astype(np.float32),
    }


# --------------------------------------------------------------------------------------------
# environment maps and targets
# --------------------------------------------------------------------------------------------
def lognormal_env(seed: int, He: int, We: int, sigma: float = 1.0) -> np.ndarray:
    """Lat-long RGB environment map [He, We, 3] float32, i.i.d. exp(N(0, sigma^2)) per texel/channel."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.normal(0.0, sigma, size=(He, We, 3))).astype(np.float32)


def uniform_target(seed: int, V: int, H: int, W: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, 1.0, size=(V, H, W, 3)).astype(np.float32)


# --------------------------------------------------------------------------------------------
# workload presets
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class TraceParams:
    spp: int
    max_steps: int
    hiz_levels: int = 8
    thickness: float = 0.05
    max_distance: float = 100.0
    seed: int = 0
    flags: int = 0


@dataclasses.dataclass
class Workload:
    name: str
    depth: np.ndarray   # [V,H,W]
    normal: np.ndarray  # [V,H,W,3]
    albedo: np.ndarray  # [V,H,W,3]
    rough: np.ndarray   # [V,H,W]
    metal: np.ndarray   # [V,H,W]
    cams: np.ndarray    # [V,14]
    env: np.ndarray     # [He,We,3]
    params: TraceParams
    target: Optional[np.ndarray] = None

    @property
    def dims(self):
        return self.depth.shape


def _stack_views(scene: Scene, cams: List[np.ndarray], H: int, W: int) -> dict:
    bufs = [raycast_gbuffer(scene, c, H, W) for c in cams]
    return {k: np.stack([b[k] for b in bufs]) for k in bufs[0]}


def single_view(name, seed, H, W, n_boxes, spread, n_mirrors, env_hw, params,
                eye=(0.0, 1.6, 5.0), target=(0.0, 0.5, 0.0), with_target=False) -> Workload:
    scene = make_scene(seed, n_boxes, spread, n_mirrors)
    cam = look_at(eye, target)
    g = _stack_views(scene, [cam], H, W)
    env = lognormal_env(seed + 1000, *env_hw)
    tgt = uniform_target(seed + 2000, 1, H, W) if with_target else None
    return Workload(name, g["depth"], g["normal"], g["albedo"], g["rough"], g["metal"],
                    cam[None, :], env, dataclasses.replace(params, seed=seed), tgt)


def config1() -> Workload:
    """256x256, 60 deg FOV, ground + 3 boxes, env 64x128 log-normal, 4 spp, 32 steps."""
    return single_view("1view-256x256-4spp", 1, 256, 256, 3, 3.0, 0, (64, 128),
                       TraceParams(spp=4, max_steps=32))


def config2(with_target: bool = False) -> Workload:
    """1600x900, ground + 40 boxes + 2 tilted mirrors, env 256x512 log-normal, 16 spp, 64 steps."""
    return single_view("1view-1600x900-16spp", 2, 900, 1600, 40, 8.0, 2, (256, 512),
                       TraceParams(spp=16, max_steps=64), with_target=with_target)


def config3() -> Workload:
    """Config 2's scene plus a seeded U[0,1] target image for the L2 loss (forward + backward)."""
    w = config2(with_target=True)
    w.name = "1view-1600x900-16spp-fwd+bwd"
    return w


def config4() -> Workload:
    """8 views at 1245x825 on a ring of radius 6 (y=2, yaw k*45 deg) around one 60-box scene,
    shared env 512x1024, 32 spp."""
    seed = 4
    scene = make_scene(seed, 60, 8.0, 0)
    cams = []
    for k in range(8):
        yaw = math.radians(45.0 * k)
        eye = (6.0 * math.sin(yaw), 2.0, 6.0 * math.cos(yaw))
        cams.append(look_at(eye, (0.0, 0.0, 0.0)))
    g = _stack_views(scene, cams, 825, 1245)
    env = lognormal_env(seed + 1000, 512, 1024)
    tgt = uniform_target(seed + 2000, 8, 825, 1245)
    return Workload("8view-1245x825-32spp-fwd+bwd", g["depth"], g["normal"], g["albedo"], g["rough"],
                    g["metal"], np.stack(cams), env, TraceParams(spp=32, max_steps=64, seed=seed), tgt)


def small_case(seed: int = 7, H: int = 48, W: int = 64, spp: int = 4, n_boxes: int = 3,
               n_mirrors: int = 1, env_hw=(16, 32), max_steps: int = 32, with_target: bool = True) -> Workload:
    """A few-tile case the oracle finishes in well under a second (ragged in both axes)."""
    return single_view(f"small-{H}x{W}-{spp}spp", seed, H, W, n_boxes, 2.5, n_mirrors, env_hw,
                       TraceParams(spp=spp, max_steps=max_steps), with_target=with_target)
