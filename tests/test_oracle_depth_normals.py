"""Pins of the oracle's depth normals (Sec. 3.1: surface normals from the rendered depth buffer by
finite differences) against analytic geometry: a plane (exact, including pixels next to the
background, where the difference is one-sided), a sphere (second-order convergence of the
central differences), the rules for isolated and background pixels, and orientation."""
import math

import numpy as np

import oracle as O
import ssgi_inputs as si


def _rays(cam, H, W):
    """World directions through the pixel centres, forward component 1 (FP64)."""
    R = cam[:12].reshape(3, 4)[:, :3].astype(np.float64)
    eye = cam[:12].reshape(3, 4)[:, 3].astype(np.float64)
    f = (H / 2.0) / math.tan(float(cam[12]) / 2.0)
    x, y = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    dc = np.stack([(x - W / 2.0) / f, -(y - H / 2.0) / f, -np.ones_like(x)], -1)
    return dc @ R.T, eye


def _plane_depth(cam, H, W, n, c):
    d, eye = _rays(cam, H, W)
    den = d @ n
    with np.errstate(divide="ignore", invalid="ignore"):
        z = (c - n @ eye) / den
    z[~(z > 0)] = np.inf
    return z


def _sphere_depth(cam, H, W, C, r):
    d, eye = _rays(cam, H, W)
    oc = eye - C
    a = np.sum(d * d, -1)
    b = d @ oc
    c0 = oc @ oc - r * r
    disc = b * b - a * c0
    z = np.full((H, W), np.inf)
    hit = disc > 0
    z[hit] = (-b[hit] - np.sqrt(disc[hit])) / a[hit]
    z[~(z > 0)] = np.inf
    return z, d, eye


def test_plane_normals_are_exact_also_next_to_the_background():
    cam = si.look_at((0.3, 2.0, 4.0), (0.0, 0.0, 0.0))
    H, W = 40, 56
    n = np.array([0.2, 0.9, -0.3])
    n /= np.linalg.norm(n)
    z = _plane_depth(cam, H, W, n, -0.4)
    z[:, :9] = np.inf  # a background band: the pixels beside it take one-sided differences
    z[15:19, 30:33] = np.inf
    fg = np.isfinite(z)
    assert fg.sum() > 1000
    nn = O.depth_normals(z[None], cam[None])[0]
    facing = n if n @ (np.array([0.3, 2.0, 4.0])) > -0.4 else -n
    err = np.abs(nn[fg] - facing).max()
    assert err < 1e-6, err  # the camera record is FP32: its rotation is orthonormal to ~1e-7
    assert np.all(nn[~fg] == 0.0)


def test_sphere_normals_converge_at_second_order():
    C, r = np.array([0.0, 0.5, 0.0]), 1.0
    cam = si.look_at((0.0, 1.2, 4.0), (0.0, 0.5, 0.0))
    errs = []
    for H in (64, 128, 256):
        z, d, eye = _sphere_depth(cam, H, H, C, r)
        nn = O.depth_normals(z[None], cam[None])[0]
        X = eye + z[..., None] * d
        exact = (X - C) / r
        # interior pixels: every neighbour on the sphere, away from the silhouette
        fg = np.isfinite(z)
        inner = fg.copy()
        for dy, dx in ((0, 1), (0, -1), (1, 0), (-1, 0), (0, 2), (0, -2), (2, 0), (-2, 0)):
            inner &= np.roll(np.roll(fg, dy, 0), dx, 1)
        cosang = np.clip(np.sum(nn[inner] * exact[inner], -1), -1, 1)
        errs.append(float(np.median(np.arccos(cosang))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.0 < r1 < 5.5 and 3.0 < r2 < 5.5, errs


def test_isolated_pixels_face_the_camera_and_background_is_zero():
    cam = si.look_at((0.0, 1.0, 3.0), (0.0, 0.0, 0.0))
    H, W = 9, 11
    z = np.full((H, W), np.inf)
    z[4, 5] = 3.0        # isolated
    z[1, 2:5] = 2.5      # a row: no vertical neighbour
    nn = O.depth_normals(z[None], cam[None])[0]
    d, eye = _rays(cam, H, W)
    for (y, x) in ((4, 5), (1, 3)):
        v = -d[y, x] / np.linalg.norm(d[y, x])
        np.testing.assert_allclose(nn[y, x], v, atol=1e-6)
    assert np.all(nn[~np.isfinite(z)] == 0.0)


def test_normals_are_unit_and_face_the_camera(cfg1):
    nn = O.depth_normals(cfg1.depth, cfg1.cams)[0]
    fg = np.isfinite(cfg1.depth[0])
    np.testing.assert_allclose(np.linalg.norm(nn[fg], axis=-1), 1.0, atol=1e-6)
    d, eye = _rays(cfg1.cams[0], *cfg1.depth.shape[1:])
    assert np.all(np.sum(nn[fg] * (-d[fg]), -1) >= 0.0)
    # and on the flat interior of the floor and box faces they are the analytic normals
    assert np.mean(np.sum(nn[fg] * cfg1.normal[0][fg], -1) > 0.999) > 0.95
