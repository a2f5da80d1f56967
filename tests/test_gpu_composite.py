"""Object insertion on the GPU (ssgi_composite_gbuffer) against the oracle, bit for bit, in place
and into separate planes; and end to end: inserting an object and rendering gives exactly the
frame of the union scene."""
import numpy as np
import pytest
import torch

import oracle as O
import ssgi_inputs as si

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2504_01358_gb300 as S
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return S


def _renders(V=2, H=45, W=67):
    scene = si.make_scene(21, 5, 3.0, 0)  # no mirrors: no quad can tie with the object in depth
    box = si.Box(np.array([-0.6, 0.4, -0.3]), np.array([0.5, 1.3, 0.6]), si.Material((0.9, 0.2, 0.1), 0.3, 1.0))
    obj = si.Scene(None, 40.0, [box], [])
    union = si.Scene(scene.ground, scene.ground_half, scene.boxes + [box], scene.quads)
    cams = np.stack([si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0)), si.look_at((3.0, 2.5, 3.0), (0.0, 0.7, 0.0))])[:V]
    st = lambda sc: {k: np.stack([si.raycast_gbuffer(sc, c, H, W)[k] for c in cams]) for k in O.GBUFFER_KEYS}  # noqa
    return st(scene), st(obj), st(union), cams


def _dev(S, gb):
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()  # noqa: E731
    return S.GBuffer(*(t(gb[k]) for k in O.GBUFFER_KEYS))


@pytest.mark.parametrize("in_place", [True, False])
def test_composite_matches_oracle_bit_for_bit(S, in_place):
    sc, ob, _, _ = _renders()
    ref, win = O.composite_gbuffer(sc, ob)
    gs, go = _dev(S, sc), _dev(S, ob)
    out = None if in_place else S.GBuffer(*(torch.full_like(getattr(gs, k), -7.0) for k in O.GBUFFER_KEYS))
    res, mask = S.ssgi_composite_gbuffer(gs, go, out=out, mask=True)
    torch.cuda.synchronize()
    assert np.array_equal(mask.cpu().numpy().astype(bool), win)
    for k in O.GBUFFER_KEYS:
        assert np.array_equal(getattr(res, k).cpu().numpy(), ref[k].astype(np.float32)), k
    if not in_place:  # the scene's planes are untouched
        assert np.array_equal(gs.depth.cpu().numpy(), sc["depth"].astype(np.float32))


def test_object_background_leaves_the_scene_untouched(S):
    sc, ob, _, _ = _renders(V=1)
    gs = _dev(S, sc)
    ob["depth"] = np.full_like(ob["depth"], np.inf)
    _, mask = S.ssgi_composite_gbuffer(gs, _dev(S, ob), mask=True)
    torch.cuda.synchronize()
    assert not mask.any()
    for k in O.GBUFFER_KEYS:
        assert np.array_equal(getattr(gs, k).cpu().numpy(), sc[k].astype(np.float32)), k


def test_inserted_object_renders_like_the_union_scene(S):
    """Composite then mips -> Hi-Z -> shade -> trace equals the same passes on the union's
    G-buffer bit for bit (final and hit indices): the object receives light and, through c1 and
    the hit indices, lights the scene (Sec. 4)."""
    sc, ob, un, cams = _renders()
    env = torch.from_numpy(si.lognormal_env(4, 32, 64)).cuda()
    p = S.TraceParams(spp=8, max_steps=48, seed=3)
    lut = S.ssgi_build_brdf_lut()

    def render(g):
        em = S.ssgi_build_env_mips(env)
        hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels)
        c_d, _, c1 = S.ssgi_shade_direct(g, cams, em, lut)
        return S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p, want_hits=True)

    gs = _dev(S, sc)
    S.ssgi_composite_gbuffer(gs, _dev(S, ob))
    a, b = render(gs), render(_dev(S, un))
    torch.cuda.synchronize()
    assert torch.equal(a["final"], b["final"]) and torch.equal(a["hit_idx"], b["hit_idx"])
    assert (a["hit_idx"] >= 0).any()
