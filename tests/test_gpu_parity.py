"""GPU (libssgi.so through the C ABI) vs the FP64 oracle, element by element on the same seeded
inputs.  Sizes span several tiles with ragged tails; config 2 runs at full size (1600x900,
16 spp) in the bench's launch configuration and is checked on a pixel sample, and the bench's
whole step (config 3: forward, loss gradient, backward) is checked at full size on every pixel."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle as O
import ssgi_inputs as si
from parity import (GRAD_RTOL, affected_pixels, assert_direct_parity, assert_forward_parity, direct_kinks,
                    gpu_forward, gradient_report, orc_forward)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2504_01358_gb300 as S
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return S


@pytest.fixture(scope="module")
def olut():
    return O.build_lut()


# --------------------------------------------------------------------------------------------
# precomputation
# --------------------------------------------------------------------------------------------
def test_brdf_lut_matches_oracle(S, olut):
    lut = S.ssgi_build_brdf_lut().cpu().numpy()
    assert lut.shape == olut.shape
    np.testing.assert_allclose(lut, olut, rtol=0, atol=2e-5)


@pytest.mark.parametrize("hw", [(64, 128), (256, 512), (1, 4), (8, 8)])
def test_env_mips_match_oracle(S, hw):
    env = si.lognormal_env(11, *hw)
    mips = S.ssgi_build_env_mips(torch.from_numpy(env).cuda()).mips.cpu().numpy()
    ref = O.build_env_mips(env)
    np.testing.assert_allclose(mips, ref, rtol=2e-6, atol=0)


@pytest.mark.parametrize("shape,levels", [((1, 256, 256), 8), ((3, 37, 53), 6), ((2, 900, 1600), 8), ((1, 1, 1), 8),
                                          ((1, 70, 33), 16)])
def test_hiz_is_bitwise_equal(S, shape, levels):
    rng = np.random.default_rng(sum(shape) + levels)
    depth = rng.uniform(0.5, 50.0, size=shape).astype(np.float32)
    depth[..., : shape[1] // 3, : shape[2] // 2] = np.inf
    hiz = S.ssgi_build_hiz(torch.from_numpy(depth).cuda(), levels).cpu().numpy()
    ref = O.build_hiz(depth, levels).astype(np.float32).reshape(-1)
    assert hiz.size >= ref.size
    assert np.array_equal(hiz[: ref.size], ref)


# --------------------------------------------------------------------------------------------
# forward
# --------------------------------------------------------------------------------------------
def test_shade_direct_matches_oracle(S, small, cfg1, olut):
    for wl in (small, cfg1):
        g = gpu_forward(wl)
        r = orc_forward(wl, lut=olut)
        assert_direct_parity(g, r, wl, wl.name)


@pytest.mark.parametrize("flags", [0, 1])
def test_trace_matches_oracle_small(S, small, olut, flags):
    g = gpu_forward(small, flags=flags)
    r = orc_forward(small, lut=olut, flags=flags)
    assert_forward_parity(g, r, f"small flags={flags}", wl=small, flags=flags)


def test_trace_matches_oracle_config1(S, cfg1, olut):
    g = gpu_forward(cfg1)
    r = orc_forward(cfg1, lut=olut)
    assert_forward_parity(g, r, "config1", wl=cfg1)
    assert (g["hit_idx"] >= 0).sum() > 10000


def test_trace_matches_oracle_multiview_ragged(S, olut):
    scene = si.make_scene(21, 12, 4.0, 2)
    cams = [si.look_at((5 * np.sin(a), 1.8, 5 * np.cos(a)), (0, 0.4, 0)) for a in (0.0, 2.1, 4.2)]
    bufs = [si.raycast_gbuffer(scene, c, 75, 131) for c in cams]
    st = lambda k: np.stack([b[k] for b in bufs])  # noqa: E731
    wl = si.Workload("3view-75x131", st("depth"), st("normal"), st("albedo"), st("rough"), st("metal"),
                     np.stack(cams), si.lognormal_env(22, 32, 64), si.TraceParams(spp=8, max_steps=48, seed=77))
    g = gpu_forward(wl)
    r = orc_forward(wl, lut=olut)
    assert_forward_parity(g, r, "3 views", wl=wl)


def test_brute_force_mode_matches_oracle(S, small, olut):
    g = gpu_forward(small, brute=True)
    r = orc_forward(small, lut=olut, brute=True)
    assert_forward_parity(g, r, "brute force", wl=small)


def test_config2_full_size_sampled(S, olut):
    """1600x900, 16 spp, 40 boxes + 2 mirrors, 64 steps -- the benchmark's launch -- against the
    oracle on 30k sampled pixels (480k rays)."""
    wl = si.config2()
    g = gpu_forward(wl)
    rng = np.random.default_rng(0)
    V, H, W = wl.depth.shape
    pl = np.sort(rng.choice(V * H * W, size=30000, replace=False))
    r = O.forward(wl, lut=olut, pix_list=pl)
    sub = {k: g[k].reshape((V * H * W,) + g[k].shape[3:])[pl] for k in ("hit_idx", "final", "cs_mc", "c_id")}
    assert_forward_parity(sub, r, "config2 sample", wl=wl, pix=pl)
    # the Hi-Z pyramid and direct pass at full size
    assert np.array_equal(g["hiz"][: r["hiz"].size], r["hiz"].astype(np.float32).reshape(-1))
    assert_direct_parity(g, r, wl, "config2", keys=("c1",))
    assert (sub["hit_idx"] >= 0).mean() > 0.05


# --------------------------------------------------------------------------------------------
# special cases
# --------------------------------------------------------------------------------------------
def test_zero_albedo_and_black_env_are_exactly_zero(S, small, olut):
    wl = dataclasses.replace(small, albedo=np.zeros_like(small.albedo))
    g = gpu_forward(wl, flags=1)
    assert np.all(g["c_id"] == 0.0) and (g["hit_idx"] >= 0).any()
    wl = dataclasses.replace(wl, env=np.zeros_like(small.env), metal=np.zeros_like(small.metal))
    g = gpu_forward(wl, flags=1)
    for k in ("cd", "cs", "c1", "cs_mc", "final", "c_id"):
        assert np.all(g[k] == 0.0), k


def test_fronto_parallel_plane_no_hits_on_gpu(S):
    cam = si.look_at((0.0, 0.0, 0.0), (0.0, 0.0, -1.0))
    q = si.Quad(np.array([0.0, 0.0, -3.0]), np.array([1.0, 0, 0]), np.array([0, 1.0, 0]), 50.0, 50.0,
                si.Material((0.5, 0.6, 0.7), 0.6, 0.0))
    gb = si.raycast_gbuffer(si.Scene(None, 0.0, [], [q]), cam, 64, 96)
    wl = si.Workload("fronto", gb["depth"][None], gb["normal"][None], gb["albedo"][None], gb["rough"][None],
                     gb["metal"][None], cam[None], si.lognormal_env(3, 16, 32), si.TraceParams(spp=8, max_steps=200))
    g = gpu_forward(wl)
    assert np.all(g["hit_idx"] < 0)


@pytest.mark.parametrize("case", ["1x1", "all_background", "spp1", "steps0", "levels1", "odd"])
def test_edge_cases_match_oracle(S, olut, case):
    base = si.small_case(seed=5, H=37, W=53, spp=4)
    p = base.params
    if case == "1x1":
        wl = dataclasses.replace(base, depth=base.depth[:, 30:31, 20:21].copy(), normal=base.normal[:, 30:31, 20:21].copy(),
                                 albedo=base.albedo[:, 30:31, 20:21].copy(), rough=base.rough[:, 30:31, 20:21].copy(),
                                 metal=base.metal[:, 30:31, 20:21].copy())
    elif case == "all_background":
        wl = dataclasses.replace(base, depth=np.full_like(base.depth, np.inf))
    elif case == "spp1":
        wl = dataclasses.replace(base, params=dataclasses.replace(p, spp=1))
    elif case == "steps0":
        wl = dataclasses.replace(base, params=dataclasses.replace(p, max_steps=0))
    elif case == "levels1":
        wl = dataclasses.replace(base, params=dataclasses.replace(p, hiz_levels=1))
    else:
        wl = dataclasses.replace(base, params=dataclasses.replace(p, spp=7, hiz_levels=3, max_steps=5))
    g = gpu_forward(wl)
    r = orc_forward(wl, lut=olut)
    assert_forward_parity(g, r, case, wl=wl)
    assert_direct_parity(g, r, wl, case, keys=("c1",))


def test_invalid_arguments_are_rejected(S):
    d = torch.zeros((1, 8, 8), device="cuda")
    with pytest.raises(S._native.SSGIError):
        S.ssgi_build_hiz(d, 99)
    with pytest.raises(ValueError):
        S.ssgi_build_env_mips(torch.zeros((3, 8, 3), device="cuda"))
    with pytest.raises(ValueError):
        S.ssgi_build_hiz(d.cpu(), 4)


# --------------------------------------------------------------------------------------------
# backward
# --------------------------------------------------------------------------------------------
def _backward_pair(S, wl, olut, flags, forward_out=None):
    g = gpu_forward(wl, flags=flags)
    r = orc_forward(wl, lut=olut, flags=flags)
    target = wl.target.astype(np.float64)
    g_final = (2.0 * (r["final"] - target) / r["final"].size).astype(np.float32)
    gb, env, cams, em, lut_t, c1, hit_idx, p = g["_dev"]
    grads = S.ssgi_backward(torch.from_numpy(g_final).cuda(), gb, cams, c1, em, lut_t, hit_idx, p)
    torch.cuda.synchronize()
    ggpu = {k: v.cpu().numpy() for k, v in grads.items()}
    He, We = wl.env.shape[:2]
    gorc = O.backward(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], He, We, olut, r["c1"],
                      r["hit_idx"], g_final, wl.params.spp, wl.params.seed, flags)
    aff = affected_pixels(g["hit_idx"], r["hit_idx"])
    if forward_out is not None:
        forward_out.update(gpu=g, orc=r)
    return ggpu, gorc, aff


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("name", ["small", "cfg1"])
def test_backward_matches_oracle_adjoint(S, olut, request, name, flags):
    wl = request.getfixturevalue(name)
    if wl.target is None:
        wl = dataclasses.replace(wl, target=si.uniform_target(99, *wl.depth.shape))
    _assert_backward_parity(*_backward_pair(S, wl, olut, flags), label=f"{name} flags={flags}",
                            kinks=direct_kinks(wl))


def _assert_backward_parity(ggpu, gorc, aff, excuse=None, excused_max=0, label="", kinks=None):
    """Per-pixel gradients within GRAD_RTOL of their scale outside `aff`; with `excuse`, a pixel
    over the bound must be one of the excused pixels (at most `excused_max` of them).  Elements of
    at least a tenth of their buffer's scale are also checked relative to themselves (GRAD_RTOL),
    outside `aff`, the excused pixels and `kinks` (direct-shading lookups whose bilinear cells
    differ between the two sides, where the one-sided derivatives legitimately differ)."""
    ok = ~aff
    skip = aff.copy()
    for m in (excuse, kinks):
        if m is not None:
            skip |= m
    gradient_report(ggpu, gorc, ~skip, label, check=True)
    for k in ("albedo", "rough", "metal", "normal"):
        scale = np.abs(gorc[k][ok]).max()
        err = np.abs(ggpu[k] - gorc[k]) / scale
        if err.ndim == ok.ndim + 1:
            err = err.max(axis=-1)
        over = ok & (err > GRAD_RTOL)
        if excuse is not None:
            assert not (over & ~excuse).any(), (k, float(err[over & ~excuse].max()))
            assert int(over.sum()) <= excused_max, (k, int(over.sum()))
        else:
            assert not over.any(), (k, float(err[ok].max()))
    a, b = ggpu["env"], gorc["env"]
    rel = np.linalg.norm(a - b) / np.linalg.norm(b)
    assert rel <= GRAD_RTOL, ("env", rel)


@pytest.mark.parametrize("flags", [0, 1])
def test_config3_full_size_backward(S, olut, flags):
    """The benchmark's step at full size (1600x900, 16 spp, 64 steps, 8 levels: forward, L2 loss
    gradient, ssgi_backward with its workspace, as bench.py launches them) against the oracle's
    forward and adjoint on every pixel and every texel of the map; pixels whose samples hit
    differently on the two sides, and the pixels those samples reach, are left out (a small
    share, asserted)."""
    wl = si.config3()
    assert wl.target is not None
    fw = {}
    ggpu, gorc, aff = _backward_pair(S, wl, olut, flags, forward_out=fw)
    # the forward at full size on every pixel: hits, images (the same bounds as every forward test)
    _, _, replayed = assert_forward_parity(fw["gpu"], fw["orc"], f"config3 flags={flags}", wl=wl, flags=flags)
    # a mismatching sample leaves out at most three pixels (its receiver and the two pixels hit),
    # so the forward bound (>= 99.9 % of samples equal) allows up to 3 x 16 x 0.1 % of the
    # pixels; about 0.1 % are left out at this size
    assert aff.mean() < 0.01, float(aff.mean())
    # A pixel's gradient may exceed the bound only where it is not defined to FP32 precision:
    # where its forward value was shown to be a rounding effect by the replay at the GPU's own
    # lookup coordinates (a steep lookup: its albedo, normal and roughness gradients are linear
    # in the same radiance), or where a direct-shading lookup of the GPU falls in another cell of
    # its bilinear filter than the oracle's (the one-sided derivatives differ there).  Such
    # pixels over the bound must be few.
    excuse = replayed | direct_kinks(wl)
    _assert_backward_parity(ggpu, gorc, aff, excuse=excuse, excused_max=int(1e-5 * aff.size) + 1,
                            label=f"config3 flags={flags}")


def test_config4_eight_views_full_size_step():
    """Config 4 (8 views of 1245x825 around one scene, 32 spp, 512x1024 map: the fused step's
    workload) through the per-stage path, every pixel of every view and every texel against the
    oracle's forward and adjoint, under the same rules as config 3.  The fused step equals this
    path bit for bit in final and hit indices (test_gpu_fused)."""
    import paper_2504_01358_gb300 as S
    wl = si.config4()
    olut = O.build_lut()
    fw = {}
    ggpu, gorc, aff = _backward_pair(S, wl, olut, 0, forward_out=fw)
    _, _, replayed = assert_forward_parity(fw["gpu"], fw["orc"], "config4", wl=wl, flags=0)
    assert aff.mean() < 0.01, float(aff.mean())
    excuse = replayed | direct_kinks(wl)
    _assert_backward_parity(ggpu, gorc, aff, excuse=excuse, excused_max=int(1e-5 * aff.size) + 1,
                            label="config4")


@pytest.mark.parametrize("flags", [0, 1])
@pytest.mark.parametrize("name", ["small", "cfg1"])
def test_pathwise_backward_matches_oracle_adjoint(S, olut, request, name, flags):
    """SSGI_PATHWISE: directions re-drawn from (n, rho) at frozen uniforms, hits frozen.  Albedo,
    metallic and texel gradients as in replay mode (same bound).  Normal and roughness gradients
    against the oracle's FP64 central differences of the per-sample summand, 1e-3 of the scale on
    every element where the summand is differentiable; a point where it is not (a sample on a
    bilinear kink of the map, a texel centre, or on the edge of validity) shows up as a change
    of the oracle's difference with its step (1e-6 vs 1e-7) or as forward and backward
    differences that disagree, and is left out (<= 0.1 % of the elements)."""
    wl = request.getfixturevalue(name)
    if wl.target is None:
        wl = dataclasses.replace(wl, target=si.uniform_target(99, *wl.depth.shape))
    fl = flags | O.FLAG_PATHWISE
    ggpu, gorc, aff = _backward_pair(S, wl, olut, fl)
    ok = ~aff
    for k in ("albedo", "metal"):
        a, b = ggpu[k][ok], gorc[k][ok]
        assert np.abs(a - b).max() / np.abs(b).max() <= GRAD_RTOL, k
    a, b = ggpu["env"], gorc["env"]
    assert np.linalg.norm(a - b) / np.linalg.norm(b) <= GRAD_RTOL, "env"
    # the oracle's derivative at a second step and as one-sided differences: where they disagree
    # the summand is not differentiable (a kink within the step of the base point)
    r = orc_forward(wl, lut=olut, flags=flags)
    g_final = (2.0 * (r["final"] - wl.target.astype(np.float64)) / r["final"].size).astype(np.float32)
    He, We = wl.env.shape[:2]
    alt = {}
    try:
        for key, h, mode in (("c7", 1e-7, 0), ("f7", 1e-7, 1), ("b7", 1e-7, -1)):
            O.set_pathwise_step(h, mode)
            alt[key] = O.backward(wl.depth, wl.normal, wl.albedo, wl.rough, wl.metal, wl.cams, r["mips"], He, We,
                                  olut, r["c1"], r["hit_idx"], g_final, wl.params.spp, wl.params.seed, fl)
    finally:
        O.set_pathwise_step(1e-6, 0)
    for k in ("rough", "normal"):
        scale = np.abs(gorc[k][ok]).max()
        kink = ((np.abs(gorc[k] - alt["c7"][k]) > 1e-4 * scale) |
                (np.abs(alt["f7"][k] - alt["b7"][k]) > 1e-4 * scale))
        if kink.ndim == ok.ndim + 1:  # per pixel
            kink = kink.any(axis=-1)
        sel = ok & ~kink
        assert float(np.mean(kink[ok])) <= 1e-3, (k, "non-differentiable share", float(np.mean(kink[ok])))
        err = np.abs(ggpu[k][sel] - gorc[k][sel]) / scale
        assert err.max() <= GRAD_RTOL, (k, float(err.max()))


def test_pathwise_differs_from_replay_only_in_normal_and_roughness(S, small, olut):
    wl = dataclasses.replace(small, target=si.uniform_target(98, *small.depth.shape))
    g0, _, _ = _backward_pair(S, wl, olut, 0)
    g4, _, _ = _backward_pair(S, wl, olut, O.FLAG_PATHWISE)
    for k in ("albedo", "metal", "env"):
        np.testing.assert_allclose(g4[k], g0[k], rtol=0, atol=1e-6 * np.abs(g0[k]).max())
    for k in ("rough", "normal"):
        assert np.abs(g4[k] - g0[k]).max() > 1e-3 * np.abs(g0[k]).max(), k


def test_autograd_function_matches_backward_call(S, small, olut):
    wl = small
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    lut = S.ssgi_build_brdf_lut()
    leaves = {k: getattr(g, k).clone().requires_grad_(True) for k in ("normal", "albedo", "rough", "metal")}
    env_l = env.clone().requires_grad_(True)
    final = S.ssgi_render(g.depth, leaves["normal"], leaves["albedo"], leaves["rough"], leaves["metal"], env_l, cams,
                          p, lut)
    loss = ((final - tgt) ** 2).mean()
    loss.backward()
    # same through the explicit calls
    em = S.ssgi_build_env_mips(env)
    hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels)
    c_d, _, c1 = S.ssgi_shade_direct(g, cams, em, lut)
    tr = S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p, want_hits=True)
    gf, _ = S.ssgi_l2_loss(tr["final"], tgt)
    gr = S.ssgi_backward(gf, g, cams, c1, em, lut, tr["hit_idx"], p)
    torch.cuda.synchronize()
    for k in ("normal", "albedo", "rough", "metal"):
        a, b = leaves[k].grad.cpu().numpy(), gr[k].cpu().numpy()
        assert np.abs(a - b).max() <= 1e-5 * max(np.abs(b).max(), 1e-12), k
    a, b = env_l.grad.cpu().numpy(), gr["env"].cpu().numpy()
    assert np.abs(a - b).max() <= 1e-5 * np.abs(b).max()


# --------------------------------------------------------------------------------------------
# the interface's maximum sizes
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("case", ["32views", "16384wide", "1024spp", "16levels"])
def test_maximum_sizes_match_oracle(S, olut, case):
    """The limits include/ssgi.h states, each at its maximum: SSGI_MAX_VIEWS (32) views of one
    scene; a frame 16384 pixels wide (the width limit; 3 rows, so the pyramid's top levels are
    ragged 1-row strips); 1024 samples per pixel (the spp limit); 16 pyramid levels (the level
    limit, above the frame's own height) -- forward against the oracle on every pixel, backward
    on the 32-view case."""
    scene = si.make_scene(61, 8, 3.0, 1)
    if case == "32views":
        cams = [si.look_at((4.5 * np.sin(a), 1.4 + 0.3 * np.cos(3 * a), 4.5 * np.cos(a)), (0, 0.3, 0))
                for a in np.linspace(0.0, 2 * np.pi, 32, endpoint=False)]
        H, W, params = 12, 20, si.TraceParams(spp=4, max_steps=32, seed=61)
    elif case == "16384wide":
        cams = [si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0), fov_y_deg=2.0)]
        H, W, params = 3, 16384, si.TraceParams(spp=2, max_steps=64, seed=62)
    elif case == "1024spp":
        cams = [si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0))]
        H, W, params = 6, 7, si.TraceParams(spp=1024, max_steps=32, seed=63)
    else:
        cams = [si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0))]
        H, W, params = 33, 47, si.TraceParams(spp=4, max_steps=48, hiz_levels=16, seed=64)
    bufs = [si.raycast_gbuffer(scene, c, H, W) for c in cams]
    st = lambda k: np.stack([b[k] for b in bufs])  # noqa: E731
    wl = si.Workload(f"max-{case}", st("depth"), st("normal"), st("albedo"), st("rough"), st("metal"),
                     np.stack(cams), si.lognormal_env(65, 16, 32), params,
                     si.uniform_target(66, len(cams), H, W))
    g = gpu_forward(wl)
    r = orc_forward(wl, lut=olut)
    assert_forward_parity(g, r, f"maximum {case}", wl=wl)
    assert_direct_parity(g, r, wl, f"maximum {case}", keys=("c1",))
    assert np.isfinite(wl.depth).any()
    if case == "32views":
        _assert_backward_parity(*_backward_pair(S, wl, olut, 0), label="maximum 32views",
                                kinks=direct_kinks(wl))
