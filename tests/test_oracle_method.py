"""Pins of the oracle's direct shading, trace, Monte-Carlo sum and adjoint (Sec. 3.2, Sec. 3.3).

These check the whole-image oracle against closed forms (white furnace, split-sum integral by
quadrature, mirror reflection geometry), invariants (no self-hits on a fronto-parallel plane,
zero albedo), a brute-force pixel walk, the O(1/sqrt(spp)) Monte-Carlo rate and central finite
differences -- never against the oracle itself.
"""
import math

import numpy as np
import pytest

import oracle as O
import ssgi_inputs as si
from test_oracle_primitives import _exact_split


def _wl_from_scene(scene, cam, H, W, env, params, name="custom"):
    g = si.raycast_gbuffer(scene, cam, H, W)
    return si.Workload(name, g["depth"][None], g["normal"][None], g["albedo"][None], g["rough"][None],
                       g["metal"][None], cam[None], env.astype(np.float32), params)


# --------------------------------------------------------------------------------------------
# direct shading
# --------------------------------------------------------------------------------------------
def test_white_furnace_diffuse(small, lut):
    """m = 0 under a uniform environment L: c_d = a L (prefiltered mips of a constant are that
    constant; the lookup weights sum to one)."""
    L = np.array([0.7, 1.3, 0.25])
    env = np.broadcast_to(L, (16, 32, 3)).copy()
    mips = O.build_env_mips(env)
    metal = np.zeros_like(small.metal)
    cd, cs, c1 = O.shade_direct(small.depth, small.normal, small.albedo, small.rough, metal, small.cams, mips, 16,
                                32, lut)
    fg = np.isfinite(small.depth)
    np.testing.assert_allclose(cd[fg], small.albedo[fg].astype(np.float64) * L, rtol=1e-13)
    np.testing.assert_allclose(c1[~fg], np.broadcast_to(L, c1[~fg].shape), rtol=1e-13)


def test_uniform_env_specular_is_split_sum_integral(small, lut):
    """Under a uniform environment L, c_s = L (F0 A + B) where A, B are the Appendix C integrals
    at (rho, n.v); compared with a sampling-free quadrature (table + bilinear error band)."""
    L = 0.9
    env = np.full((16, 32, 3), L)
    mips = O.build_env_mips(env)
    cd, cs, c1 = O.shade_direct(small.depth, small.normal, small.albedo, small.rough, small.metal, small.cams, mips,
                                16, 32, lut)
    H, W = small.depth.shape[1:]
    rng = np.random.default_rng(0)
    cam = small.cams[0].astype(np.float64)
    d, _ = si.pixel_rays(small.cams[0], H, W)
    checked = 0
    for _ in range(400):
        y, x = rng.integers(0, H), rng.integers(0, W)
        if not np.isfinite(small.depth[0, y, x]):
            continue
        v = -d[y, x] / np.linalg.norm(d[y, x])
        nv = float(small.normal[0, y, x].astype(np.float64) @ v)
        rho = float(small.rough[0, y, x])
        if nv < 0.15 or rho < 0.2:
            continue
        A, B = _exact_split(rho, min(nv, 1.0))
        m = float(small.metal[0, y, x])
        F0 = 0.04 * (1 - m) + small.albedo[0, y, x].astype(np.float64) * m
        np.testing.assert_allclose(cs[0, y, x], L * (F0 * A + B), rtol=0, atol=4e-3 * L)
        checked += 1
        if checked >= 6:
            break
    assert checked >= 3
    del cam


def _tilt_case(env, normal, rough=0.02, metal=0.0, albedo=(0.5, 0.5, 0.5)):
    """A 1x1 G-buffer seen from eye (0,1,1) looking at the origin (view direction 45 deg down)."""
    cam = si.look_at((0.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    depth = np.full((1, 1, 1), math.sqrt(2.0), np.float32)
    nrm = np.array(normal, np.float32).reshape(1, 1, 1, 3)
    alb = np.array(albedo, np.float32).reshape(1, 1, 1, 3)
    mips = O.build_env_mips(env)
    He, We = env.shape[:2]
    return O.shade_direct(depth, nrm, alb, np.full((1, 1, 1), rough), np.full((1, 1, 1), metal), cam[None], mips,
                          He, We, O.build_lut(8, 256))


def test_diffuse_looks_up_the_normal_and_specular_the_mirror_direction():
    """c_d queries L_E(n), c_s queries L_E(r) with r = 2 (v.n) n - v.  Floor normal (0,1,0) seen
    45 degrees from above: n is the zenith, r leaves at 45 degrees elevation towards -z."""
    He, We = 32, 64
    vs = (np.arange(He) + 0.5) / He
    us = (np.arange(We) + 0.5) / We
    zen = np.zeros((He, We, 3))
    zen[vs < 0.12] = 1.0  # a cap around the zenith
    cd, cs, _ = _tilt_case(zen, (0, 1, 0))
    assert cd[0, 0, 0, 0] > 0.2 and cs[0, 0, 0, 0] == 0.0
    # a cap around r = (0, 1/sqrt2, -1/sqrt2): v = 0.25, u = 0.5
    capr = np.zeros((He, We, 3))
    capr[np.ix_(np.abs(vs - 0.25) < 0.08, np.abs(us - 0.5) < 0.08)] = 1.0
    cd, cs, _ = _tilt_case(capr, (0, 1, 0), metal=1.0, albedo=(0.9, 0.9, 0.9))
    assert cd[0, 0, 0, 0] == 0.0 and cs[0, 0, 0, 0] > 0.5
    # the same metal under the zenith cap: nothing reaches the specular lookup
    cd, cs, _ = _tilt_case(zen, (0, 1, 0), metal=1.0, albedo=(0.9, 0.9, 0.9))
    assert cd[0, 0, 0, 0] == 0.0 and cs[0, 0, 0, 0] == 0.0


def test_zero_albedo_gives_zero_indirect(small, lut):
    """a = 0: the diffuse-indirect channel is exactly zero; with a = 0 and a black environment
    every channel (c_d, c_s, c1, c_s', final) is exactly zero."""
    w = small
    alb0 = np.zeros_like(w.albedo)
    mips = O.build_env_mips(w.env)
    He, We = w.env.shape[:2]
    hiz = O.build_hiz(w.depth, w.params.hiz_levels)
    cd, cs, c1 = O.shade_direct(w.depth, w.normal, alb0, w.rough, w.metal, w.cams, mips, He, We, lut)
    p = w.params
    tr = O.trace(w.depth, w.normal, alb0, w.rough, w.metal, w.cams, mips, He, We, hiz, c1, cd, p.spp, p.max_steps,
                 p.hiz_levels, p.thickness, p.max_distance, p.seed, O.FLAG_DIFFUSE_INDIRECT)
    assert np.all(tr["cid"] == 0.0)
    assert (tr["hit_idx"] >= 0).any()
    black = O.build_env_mips(np.zeros_like(w.env))
    metal0 = np.zeros_like(w.metal)
    cd, cs, c1 = O.shade_direct(w.depth, w.normal, alb0, w.rough, metal0, w.cams, black, He, We, lut)
    tr = O.trace(w.depth, w.normal, alb0, w.rough, metal0, w.cams, black, He, We, hiz, c1, cd, p.spp, p.max_steps,
                 p.hiz_levels, p.thickness, p.max_distance, p.seed, O.FLAG_DIFFUSE_INDIRECT)
    for a in (cd, cs, c1, tr["cs_mc"], tr["final"], tr["cid"]):
        assert np.all(a == 0.0)


# --------------------------------------------------------------------------------------------
# trace
# --------------------------------------------------------------------------------------------
def test_fronto_parallel_plane_has_no_self_hits(lut):
    """A plane facing the camera and filling the screen: every valid reflected ray moves towards
    the camera, so it stays in front of the depth buffer and never hits."""
    cam = si.look_at((0.0, 0.0, 0.0), (0.0, 0.0, -1.0))
    q = si.Quad(np.array([0.0, 0.0, -3.0]), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), 50.0, 50.0,
                si.Material((0.5, 0.6, 0.7), 0.6, 0.0))
    scene = si.Scene(None, 0.0, [], [q])
    env = si.lognormal_env(3, 16, 32)
    w = _wl_from_scene(scene, cam, 40, 56, env, si.TraceParams(spp=8, max_steps=200, hiz_levels=6, seed=9))
    assert np.all(w.depth == np.float32(3.0))
    r = O.forward(w, lut=lut)
    h = r["hit_idx"]
    assert np.all(h < 0)
    assert (h == O.MISS).mean() > 0.5


def _mirror_setup():
    wall = si.Box(np.array([-10.0, 0.0, -6.0]), np.array([10.0, 4.0, -5.0]), si.Material((0.3, 0.5, 0.7), 0.5, 0.0))
    scene = si.Scene(si.Material((1.0, 1.0, 1.0), 0.0, 1.0), 40.0, [wall], [])
    cam = si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0))
    return scene, cam


def test_mirror_floor_hits_the_closed_form_reflected_pixel(lut):
    """rho = 0 floor (h = n exactly) facing a wall: each floor pixel's reflected ray must hit the
    pixel holding the closed-form intersection of the mirrored ray with the wall's front face
    (within one pixel along the ray), and rays that clear the wall must miss."""
    scene, cam = _mirror_setup()
    H, W = 120, 160
    env = si.lognormal_env(5, 16, 32)
    w = _wl_from_scene(scene, cam, H, W, env, si.TraceParams(spp=2, max_steps=400, hiz_levels=6, seed=3))
    r = O.forward(w, lut=lut)
    hit = r["hit_idx"][0]
    d, eye = si.pixel_rays(cam, H, W)
    f = (H / 2.0) / math.tan(cam[12] / 2.0)
    rot = cam[:12].reshape(3, 4)[:, :3].astype(np.float64)
    n_hit = n_exact = n_miss = 0
    for y in range(H):
        for x in range(W):
            if not (np.isfinite(w.depth[0, y, x]) and w.normal[0, y, x, 1] > 0.5):
                continue  # floor pixels only
            assert hit[y, x, 0] == hit[y, x, 1]  # a delta lobe: both samples identical
            p = eye + float(w.depth[0, y, x]) * d[y, x]
            v = -d[y, x] / np.linalg.norm(d[y, x])
            om = 2 * v[1] * np.array([0, 1.0, 0]) - v
            if om[2] >= -1e-9:
                continue
            t = (-5.0 - p[2]) / om[2]
            X = p + t * om
            Xc = rot.T @ (X - eye)
            z = -Xc[2]
            sx, sy = W / 2 + f * Xc[0] / z, H / 2 - f * Xc[1] / z
            inside = (abs(X[0]) < 9.5) and (X[1] < 3.8) and (X[1] > 0.05)
            on_screen = (1 <= sx < W - 1) and (1 <= sy < H - 1)
            if inside and on_screen:
                qx, qy = int(math.floor(sx)), int(math.floor(sy))
                if abs(w.depth[0, qy, qx] - z) > 0.02:
                    continue  # the wall point is hidden in the depth buffer
                q = hit[y, x, 0]
                assert q >= 0, (y, x)
                hx, hy = q % W, q // W
                assert max(abs(hx - qx), abs(hy - qy)) <= 1, ((y, x), (hx, hy), (qx, qy))
                n_hit += 1
                n_exact += (hx == qx and hy == qy)
            elif X[1] > 4.3 or not (0 <= sx < W and 0 <= sy < H):
                assert hit[y, x, 0] == O.MISS, (y, x)
                n_miss += 1
    assert n_hit > 300 and n_miss > 100
    assert n_exact / n_hit > 0.8


@pytest.mark.parametrize("name", ["cfg1", "small"])
def test_hiz_traversal_equals_brute_force_pixel_walk(name, request, lut):
    """Conservative Hi-Z skipping never changes the first hit: identical hit indices to the
    pixel-by-pixel walk (one level, no step budget) on every ray that did not run out of steps."""
    w = request.getfixturevalue(name)
    r = O.forward(w, lut=lut)
    b = O.forward(w, lut=lut, brute=True)
    h, hb = r["hit_idx"], b["hit_idx"]
    exhausted = (h == O.MISS) & (r["iters"] >= w.params.max_steps)
    assert exhausted.mean() < 0.05
    assert np.array_equal(h[~exhausted], hb[~exhausted])
    assert (h >= 0).sum() > 1000 if name == "cfg1" else (h >= 0).sum() > 50


@pytest.mark.parametrize("K", [4, 12, 32])
def test_one_more_step_counts_the_rays_the_budget_stopped(small, lut, K):
    """The march with budget K is the first K iterations of the march with budget K + 1, so the
    total iterations grow by exactly one for each ray the budget stopped (a ray that, with no
    budget to speak of, takes more than K iterations) and by nothing for any other ray, whether
    it hit, left the screen or ended its segment.  The benchmark counts budget-stopped rays this
    way from the kernel's own iteration totals."""
    import dataclasses
    runs = [O.forward(dataclasses.replace(small, params=dataclasses.replace(small.params, max_steps=k)), lut=lut)
            for k in (K, K + 1, 100000)]
    stopped = runs[2]["iters"] > K
    assert stopped.sum() > 0
    assert int(runs[1]["iters"].sum()) - int(runs[0]["iters"].sum()) == int(stopped.sum())
    d = runs[1]["iters"].astype(np.int64) - runs[0]["iters"]
    assert np.array_equal(d, stopped.astype(np.int64))
    # a stopped ray is reported as a miss; every other ray's result is its unbounded result
    assert np.all(runs[0]["hit_idx"][stopped] == O.MISS)
    assert np.array_equal(runs[0]["hit_idx"][~stopped], runs[2]["hit_idx"][~stopped])


def test_hiz_levels_do_not_change_hits(small, lut):
    import dataclasses
    ref = None
    for L in (1, 2, 4, 7):
        w = dataclasses.replace(small, params=dataclasses.replace(small.params, hiz_levels=L, max_steps=100000))
        h = O.forward(w, lut=lut)["hit_idx"]
        if ref is None:
            ref = h
        assert np.array_equal(h, ref), L


def test_monte_carlo_error_falls_as_inverse_sqrt_spp(lut):
    """RMS error of c_s' against an independent 2048-spp estimate: log-log slope -1/2."""
    import dataclasses
    base = si.small_case(seed=11, H=32, W=40, spp=1)
    mips = O.build_env_mips(base.env)
    He, We = base.env.shape[:2]
    hiz = O.build_hiz(base.depth, base.params.hiz_levels)
    cd, cs, c1 = O.shade_direct(base.depth, base.normal, base.albedo, base.rough, base.metal, base.cams, mips, He,
                                We, lut)
    p = base.params

    def est(spp, seed):
        return O.trace(base.depth, base.normal, base.albedo, base.rough, base.metal, base.cams, mips, He, We, hiz,
                       c1, cd, spp, p.max_steps, p.hiz_levels, p.thickness, p.max_distance, seed, 0)["cs_mc"]

    ref = est(2048, 999)
    fg = np.isfinite(base.depth)
    spps = [1, 4, 16, 64, 256]
    errs = []
    for spp in spps:
        e2 = np.mean([np.mean((est(spp, s)[fg] - ref[fg]) ** 2) for s in (1, 2, 3)])
        errs.append(math.sqrt(e2))
    slope = np.polyfit(np.log(spps), np.log(errs), 1)[0]
    assert -0.55 <= slope <= -0.45, (slope, errs)
    del dataclasses


def test_all_miss_furnace_matches_split_sum_integral(small, lut):
    """With every ray forced to miss (step budget 0) under a uniform environment L, the Monte-
    Carlo specular c_s' converges to L (F0 A + B), the same integral the table holds (Appendix C)."""
    w = small
    L = 1.7
    env = np.full((16, 32, 3), L)
    mips = O.build_env_mips(env)
    cd, cs, c1 = O.shade_direct(w.depth, w.normal, w.albedo, w.rough, w.metal, w.cams, mips, 16, 32, lut)
    H, W = w.depth.shape[1:]
    d, _ = si.pixel_rays(w.cams[0], H, W)
    rng = np.random.default_rng(4)
    picks = []
    for _ in range(2000):
        y, x = rng.integers(0, H), rng.integers(0, W)
        if not np.isfinite(w.depth[0, y, x]):
            continue
        v = -d[y, x] / np.linalg.norm(d[y, x])
        nv = float(w.normal[0, y, x].astype(np.float64) @ v)
        if nv > 0.25 and w.rough[0, y, x] > 0.15 and (y * W + x) not in [q for q, _, _ in picks]:
            picks.append((y * W + x, nv, float(w.rough[0, y, x])))
        if len(picks) == 6:
            break
    pl = [q for q, _, _ in picks]
    hiz = O.build_hiz(w.depth, 4)
    tr = O.trace(w.depth, w.normal, w.albedo, w.rough, w.metal, w.cams, mips, 16, 32, hiz, c1, cd, 8192, 0, 4, 0.05,
                 100.0, 17, 0, pix_list=pl)
    assert np.all(tr["hit_idx"] != O.INVALID - 10)
    assert not (tr["hit_idx"] >= 0).any()
    for k, (q, nv, rho) in enumerate(picks):
        y, x = divmod(q, W)
        A, B = _exact_split(rho, nv)
        m = float(w.metal[0, y, x])
        F0 = 0.04 * (1 - m) + w.albedo[0, y, x].astype(np.float64) * m
        np.testing.assert_allclose(tr["cs_mc"][k], L * (F0 * A + B), rtol=0.03, atol=2e-3)
        # and the split-sum c_s of the direct pass agrees within the table's error
        np.testing.assert_allclose(cs[0, y, x], L * (F0 * A + B), rtol=0.0, atol=6e-3 * L)


# --------------------------------------------------------------------------------------------
# adjoint (replay mode)
# --------------------------------------------------------------------------------------------
def _loss(final, target):
    return float(np.mean((final - target) ** 2))


def _replay(w, lut, flags, nb, rb, ne, ae, re_, me, ee, hit):
    He, We = w.env.shape[:2]
    return O.replay_final(w.depth, w.cams, He, We, lut, w.params.spp, w.params.seed, flags, nb, rb, ne, ae, re_, me,
                          ee, hit)


def test_replay_at_the_base_point_is_the_forward_pass(small, lut):
    for flags in (0, O.FLAG_DIFFUSE_INDIRECT):
        r = O.forward(small, lut=lut, flags=flags)
        f = _replay(small, lut, flags, small.normal, small.rough, small.normal, small.albedo, small.rough, small.metal,
                    small.env, r["hit_idx"])
        np.testing.assert_allclose(f, r["final"], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("flags", [0, 1])
def test_adjoint_matches_central_finite_differences(small, lut, flags):
    """Analytic adjoint vs central differences of the replay forward, FP64, h = 1e-6 max(1,|x|),
    on 256 random parameters over albedo, roughness, metallic, normal and environment texels.
    Normals pointing at a pole of the lat-long map (the floor's (0,1,0)) are skipped: the
    lookup L_E(n) jumps in azimuth there, so the forward is not differentiable at that point."""
    w = small
    r = O.forward(w, lut=lut, flags=flags)
    target = w.target.astype(np.float64)
    N = r["final"].size
    g_final = 2.0 * (r["final"] - target) / N
    He, We = w.env.shape[:2]
    grads = O.backward(w.depth, w.normal, w.albedo, w.rough, w.metal, w.cams, r["mips"], He, We, lut, r["c1"],
                       r["hit_idx"], g_final, w.params.spp, w.params.seed, flags)
    base = {"albedo": w.albedo.astype(np.float64), "rough": w.rough.astype(np.float64),
            "metal": w.metal.astype(np.float64), "normal": w.normal.astype(np.float64),
            "env": w.env.astype(np.float64)}
    rng = np.random.default_rng(100 + flags)
    fg = np.argwhere(np.isfinite(w.depth))
    kinds = ["albedo", "rough", "metal", "normal", "env"]
    errs = []
    n_checked = 0
    while n_checked < 256:
        kind = kinds[n_checked % 5]
        if kind == "env":
            idx = (rng.integers(0, He), rng.integers(0, We), rng.integers(0, 3))
        else:
            v, y, x = fg[rng.integers(0, len(fg))]
            if kind == "normal" and abs(w.normal[v, y, x, 1]) > 0.999:
                continue
            idx = (v, y, x) if kind in ("rough", "metal") else (v, y, x, rng.integers(0, 3))
        x0 = base[kind][idx]
        h = 1e-6 * max(1.0, abs(x0))
        vals = []
        for sgn in (+1, -1):
            p = {k: a.copy() for k, a in base.items()}
            p[kind][idx] = x0 + sgn * h
            f = _replay(w, lut, flags, base["normal"], base["rough"], p["normal"], p["albedo"], p["rough"], p["metal"],
                        p["env"], r["hit_idx"])
            vals.append(_loss(f, target))
        fd = (vals[0] - vals[1]) / (2 * h)
        g = grads[kind][idx]
        scale = max(abs(fd), abs(g), 1e-7)
        errs.append(abs(fd - g) / scale)
        n_checked += 1
    errs = np.array(errs)
    assert np.max(errs) < 1e-2, (np.argmax(errs), np.max(errs))


# --------------------------------------------------------------------------------------------
# adjoint (pathwise mode: directions re-drawn from n and rho, hits frozen)
# --------------------------------------------------------------------------------------------
def test_pathwise_replay_at_the_base_point_is_the_forward_pass(small, lut):
    for flags in (0, O.FLAG_DIFFUSE_INDIRECT):
        r = O.forward(small, lut=lut, flags=flags)
        f = _replay(small, lut, flags | O.FLAG_PATHWISE, small.normal, small.rough, small.normal, small.albedo,
                    small.rough, small.metal, small.env, r["hit_idx"])
        np.testing.assert_allclose(f, r["final"], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("flags", [0, 1])
def test_pathwise_adjoint_matches_central_finite_differences(small, lut, flags):
    """The pathwise adjoint (flag 4) vs central differences of the pathwise replay forward over the
    whole image: 256 random parameters over albedo, roughness, metallic, normal, env texels."""
    w = small
    fl = flags | O.FLAG_PATHWISE
    r = O.forward(w, lut=lut, flags=flags)
    target = w.target.astype(np.float64)
    g_final = 2.0 * (r["final"] - target) / r["final"].size
    He, We = w.env.shape[:2]
    grads = O.backward(w.depth, w.normal, w.albedo, w.rough, w.metal, w.cams, r["mips"], He, We, lut, r["c1"],
                       r["hit_idx"], g_final, w.params.spp, w.params.seed, fl)
    base = {"albedo": w.albedo.astype(np.float64), "rough": w.rough.astype(np.float64),
            "metal": w.metal.astype(np.float64), "normal": w.normal.astype(np.float64),
            "env": w.env.astype(np.float64)}
    rng = np.random.default_rng(300 + flags)
    fg = np.argwhere(np.isfinite(w.depth))
    kinds = ["albedo", "rough", "metal", "normal", "env"]
    errs = []
    while len(errs) < 256:
        kind = kinds[len(errs) % 5]
        if kind == "env":
            idx = (rng.integers(0, He), rng.integers(0, We), rng.integers(0, 3))
        else:
            v, y, x = fg[rng.integers(0, len(fg))]
            if kind == "normal" and abs(w.normal[v, y, x, 1]) > 0.999:
                continue
            idx = (v, y, x) if kind in ("rough", "metal") else (v, y, x, rng.integers(0, 3))
        x0 = base[kind][idx]
        h = 1e-6 * max(1.0, abs(x0))
        vals = []
        for sgn in (+1, -1):
            p = {k: a.copy() for k, a in base.items()}
            p[kind][idx] = x0 + sgn * h
            f = _replay(w, lut, fl, base["normal"], base["rough"], p["normal"], p["albedo"], p["rough"], p["metal"],
                        p["env"], r["hit_idx"])
            vals.append(_loss(f, target))
        fd = (vals[0] - vals[1]) / (2 * h)
        g = grads[kind][idx]
        errs.append(abs(fd - g) / max(abs(fd), abs(g), 1e-7))
    errs = np.array(errs)
    assert np.max(errs) < 1e-2, (np.argmax(errs), np.max(errs))


@pytest.mark.parametrize("flags", [0, O.FLAG_PATHWISE])
def test_furnace_gradient_is_the_derivative_of_the_split_sum_integral(flags):
    """Unbiasedness of both adjoints.  One pixel under a uniform environment L with every ray a
    miss: E[c_s'] = L (F0 A(rho, mu) + B(rho, mu)) (Appendix C), so the expected roughness
    gradient is L d/drho (F0 A + B) and the expected normal gradient along the tangent towards v
    is L d/dmu (F0 A + B) (t.v); A, B come from a sampling-free quadrature.  8 seeds x 4096
    samples; the mean must lie within 4 standard errors of the quadrature derivative."""
    L = 1.3
    cam = si.look_at((0.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    v = np.array([0.0, 1.0, 1.0]) / math.sqrt(2.0)
    n = np.array([0.9, 0.45, -0.2])
    n /= np.linalg.norm(n)
    mu = float(n @ v)
    rho, m = 0.45, 0.3
    a = np.array([0.6, 0.3, 0.8])
    g = np.array([0.3, 0.5, 0.2])
    t1 = v - mu * n
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    gr, gt1, gt2 = [], [], []
    for seed in range(8):
        params = si.TraceParams(spp=4096, max_steps=0, hiz_levels=1, seed=1000 + seed, flags=0)
        wl = si.Workload("furnace", np.full((1, 1, 1), math.sqrt(2.0), np.float32),
                         n.astype(np.float32).reshape(1, 1, 1, 3), a.astype(np.float32).reshape(1, 1, 1, 3),
                         np.full((1, 1, 1), rho, np.float32), np.full((1, 1, 1), m, np.float32), cam[None],
                         np.full((8, 16, 3), L, np.float32), params)
        r = O.forward(wl, lut=O.build_lut(16, 256))
        assert not (r["hit_idx"] >= 0).any()
        gd = O.backward(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], 8, 16,
                        O.build_lut(16, 256), r["c1"], r["hit_idx"], g.reshape(1, 1, 1, 3), 4096, params.seed, flags)
        gn = gd["normal"][0, 0, 0]
        gr.append(gd["rough"][0, 0, 0])
        gt1.append(gn @ t1)
        gt2.append(gn @ t2)
    F0 = 0.04 * (1 - m) + a * m
    def S(r_, mu_):
        A, B = _exact_split(r_, mu_)
        return float(g @ (F0 * A + B)) * L
    hr, hm = 2e-3, 2e-3
    dS_dr = (S(rho + hr, mu) - S(rho - hr, mu)) / (2 * hr)
    dS_dmu = (S(rho, mu + hm) - S(rho, mu - hm)) / (2 * hm)
    for vals, expect in ((gr, dS_dr), (gt1, dS_dmu * float(t1 @ v)), (gt2, 0.0)):
        vals = np.array(vals)
        se = vals.std(ddof=1) / math.sqrt(len(vals))
        assert abs(vals.mean() - expect) < 4 * se + 2e-3 * abs(expect) + 1e-5, (vals.mean(), expect, se)
