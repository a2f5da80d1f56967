"""Depth normals on the GPU (ssgi_depth_normals) against the FP64 oracle: small, 256x256 and
1600x900 frames, ragged multi-view frames with background holes, all-background and 1x1 frames.
The bound, 2e-5 per component, is FP32 rounding of the well-conditioned differences, the cross
product and the rotation (a few units of 1.2e-7 each), with margin."""
import numpy as np
import pytest
import torch

import oracle as O
import ssgi_inputs as si

pytestmark = pytest.mark.gpu
TOL = 2e-5


@pytest.fixture(scope="module")
def S():
    import paper_2504_01358_gb300 as S
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return S


def _compare(S, depth, cams):
    got = S.ssgi_depth_normals(torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda(), cams).cpu().numpy()
    ref = O.depth_normals(depth, cams)
    err = np.abs(got - ref).max() if got.size else 0.0
    assert err <= TOL, err
    bg = ~np.isfinite(depth)
    assert np.all(got[bg] == 0.0)
    return got


@pytest.mark.parametrize("name", ["small", "cfg1"])
def test_depth_normals_match_oracle(S, request, name):
    wl = request.getfixturevalue(name)
    _compare(S, wl.depth, wl.cams)


def test_depth_normals_full_size_frame(S):
    wl = si.config2()
    got = _compare(S, wl.depth, wl.cams)
    fg = np.isfinite(wl.depth)
    assert np.mean(np.sum(got[fg] * wl.normal[fg], -1) > 0.999) > 0.95


def test_depth_normals_ragged_views_with_holes(S):
    scene = si.make_scene(12, 6, 3.0, 1)
    cams = np.stack([si.look_at((4 * np.sin(a), 1.5, 4 * np.cos(a)), (0, 0.4, 0)) for a in (0.2, 2.2, 4.1)])
    depth = np.stack([si.raycast_gbuffer(scene, c, 37, 53)["depth"] for c in cams])
    rng = np.random.default_rng(3)
    depth[rng.random(depth.shape) < 0.05] = np.inf  # isolated holes: one-sided differences around them
    _compare(S, depth, cams)


def test_depth_normals_degenerate_frames(S):
    cam = si.look_at((0.0, 1.0, 3.0), (0.0, 0.0, 0.0))[None]
    _compare(S, np.full((1, 5, 7), np.inf, np.float32), cam)
    _compare(S, np.full((1, 1, 1), 2.0, np.float32), cam)


@pytest.mark.parametrize("case", ["256", "ragged3", "1600x900", "1x1", "levels1", "levels16"])
def test_fused_pyramid_and_normals_equal_the_separate_passes(S, case):
    """ssgi_build_hiz_normals (the depth normals computed while the pyramid's tiles are read)
    against ssgi_build_hiz and ssgi_depth_normals on the same depth: bit for bit, on ragged
    multi-view frames with background holes and at 1600x900; and the normals against the
    oracle to the same bound."""
    levels = 8
    if case == "256":
        wl = si.config1()
        depth, cams = wl.depth, wl.cams
    elif case == "1600x900":
        wl = si.config2()
        depth, cams = wl.depth, wl.cams
    else:
        scene = si.make_scene(41, 9, 3.0, 1)
        cams = np.stack([si.look_at((4 * np.sin(a), 1.5, 4 * np.cos(a)), (0, 0.3, 0)) for a in (0.4, 2.5, 4.4)])
        H, W = (1, 1) if case == "1x1" else (45, 77)
        depth = np.stack([si.raycast_gbuffer(scene, c, H, W)["depth"] for c in cams])
        levels = {"levels1": 1, "levels16": 16}.get(case, 6)
    d = torch.from_numpy(np.ascontiguousarray(depth, np.float32)).cuda()
    hz_f, n_f = S.ssgi_build_hiz_normals(d, cams, levels)
    n_s = S.ssgi_depth_normals(d, cams)
    assert torch.equal(n_f, n_s)
    if levels > 1:
        hz_s = S.ssgi_build_hiz(d, levels)
        assert torch.equal(hz_f, hz_s)
    ref = O.depth_normals(depth, cams)
    assert np.abs(n_f.cpu().numpy() - ref).max() <= TOL
