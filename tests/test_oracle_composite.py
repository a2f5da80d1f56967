"""Pins of the oracle's object-insertion composite (Sec. 4 "Object Insertion": the object's
G-buffer merged into the scene's by depth comparison): the composite of two separately
ray-cast G-buffers equals the ray cast of the union scene, channel for channel, and the special
cases (object behind, object background, ties, the scene with itself)."""
import numpy as np

import oracle as O
import ssgi_inputs as si


def _gb(scene, cam, H, W):
    return si.raycast_gbuffer(scene, cam, H, W)


def test_composite_of_two_renders_is_the_render_of_the_union():
    scene = si.make_scene(21, 5, 3.0, 0)
    # the inserted object: a floating box (no contact with the floor, so no depth ties)
    obj_box = si.Box(np.array([-0.6, 0.4, -0.3]), np.array([0.5, 1.3, 0.6]), si.Material((0.9, 0.2, 0.1), 0.3, 1.0))
    obj = si.Scene(None, 40.0, [obj_box], [])
    union = si.Scene(scene.ground, scene.ground_half, scene.boxes + [obj_box], scene.quads)
    for cam in (si.look_at((0.0, 1.6, 5.0), (0.0, 0.5, 0.0)), si.look_at((3.0, 2.5, 3.0), (0.0, 0.7, 0.0))):
        a, b, u = _gb(scene, cam, 61, 83), _gb(obj, cam, 61, 83), _gb(union, cam, 61, 83)
        merged, win = O.composite_gbuffer(a, b)
        assert 0.02 < win.mean() < 0.6
        for k in O.GBUFFER_KEYS:
            assert np.array_equal(merged[k], u[k]), k


def test_special_cases():
    rng = np.random.default_rng(5)
    H, W = 7, 9
    sc = {"depth": rng.uniform(1, 5, (1, H, W)).astype(np.float32), "normal": rng.normal(size=(1, H, W, 3)),
          "albedo": rng.random((1, H, W, 3)), "rough": rng.random((1, H, W)), "metal": rng.random((1, H, W))}
    far = {k: (v + 1.0 if k != "depth" else v + 10.0) for k, v in sc.items()}
    out, win = O.composite_gbuffer(sc, far)              # object behind everything: unchanged
    assert not win.any() and all(np.array_equal(out[k], sc[k]) for k in O.GBUFFER_KEYS)
    bg = dict(far, depth=np.full_like(sc["depth"], np.inf))
    out, win = O.composite_gbuffer(sc, bg)               # object background: unchanged
    assert not win.any()
    out, win = O.composite_gbuffer(sc, sc)               # ties keep the scene
    assert not win.any()
    near = dict(far, depth=sc["depth"] - 0.5)
    out, win = O.composite_gbuffer(sc, near)             # object in front everywhere: the object
    assert win.all() and all(np.array_equal(out[k], near[k]) for k in O.GBUFFER_KEYS)
    sky = dict(sc, depth=np.full_like(sc["depth"], np.inf))
    out, win = O.composite_gbuffer(sky, near)            # scene background: the object wins
    assert win.all()
