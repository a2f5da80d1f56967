"""Pins of the oracle's output transform (tone mapping + gamma to sRGB after the composite,
Sec. 3.3) and keyframe lighting (Sec. 4 implementation details): the sRGB transfer function
against its inverse (IEC 61966-2-1), continuity at its breakpoint and known grey levels; the
loss gradient against central differences; keyframe selection and blending."""
import numpy as np

import oracle as O


def _eotf(y):
    y = np.asarray(y, np.float64)
    return np.where(y <= 0.04045, y / 12.92, np.power((y + 0.055) / 1.055, 2.4))


def test_transfer_function_inverts_and_is_continuous():
    x = np.linspace(0.0, 1.0, 10001)
    np.testing.assert_allclose(_eotf(O.srgb_oetf(x)), x, rtol=0, atol=1e-12)
    b = 0.0031308
    assert abs(12.92 * b - (1.055 * b ** (1 / 2.4) - 0.055)) < 1e-7
    assert O.srgb_oetf(0.0) == 0.0 and abs(O.srgb_oetf(1.0) - 1.0) < 1e-12
    # the 18 % and 50 % linear greys (ratios of the published function, not retyped constants)
    assert 0.46 < O.srgb_oetf(0.18) < 0.462 and 0.735 < O.srgb_oetf(0.5) < 0.736


def test_tonemap_clamps_and_is_monotone():
    x = np.array([-3.0, -1e-9, 0.0, 0.002, 0.01, 0.3, 0.999, 1.0, 1.5, 40.0])
    y = O.tonemap_srgb(x)
    assert y[0] == 0.0 and y[1] == 0.0 and abs(y[-1] - 1.0) < 1e-12 and y[-1] == y[-2] == y[-3]
    assert np.all(np.diff(y) >= 0)


def test_srgb_loss_gradient_matches_central_differences():
    rng = np.random.default_rng(6)
    f = rng.uniform(-0.2, 1.3, size=(4, 5, 3))
    f[0, 0, 0] = 0.001  # the linear segment
    t = rng.uniform(0, 1, size=f.shape)
    _, g = O.l2_loss_srgb(f, t)
    for idx in [(0, 0, 0), (1, 2, 1), (3, 4, 2), (2, 1, 0)]:
        if not (0.0 < f[idx] < 1.0):
            assert g[idx] == 0.0
            continue
        h = 1e-7
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = (O.l2_loss_srgb(fp, t)[0] - O.l2_loss_srgb(fm, t)[0]) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(abs(fd), 1e-9), (idx, fd, g[idx])


def test_keyframes():
    assert O.keyframe_of(0) == (0, 0.0) and O.keyframe_of(7) == (0, 0.7) and O.keyframe_of(10) == (1, 0.0)
    assert O.keyframe_of(29, 10) == (2, 0.9)
    a, b = np.zeros((2, 4, 3)), np.ones((2, 4, 3))
    np.testing.assert_array_equal(O.keyframe_lerp(a, b, 0.0), a)
    np.testing.assert_array_equal(O.keyframe_lerp(a, b, 1.0), b)
    np.testing.assert_allclose(O.keyframe_lerp(a, b, 0.3), 0.3)
