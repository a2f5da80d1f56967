"""The output transform (tone mapping + gamma to sRGB, Sec. 3.3) and keyframe lighting (Sec. 4)
on the GPU against the oracle.  Bounds: a few FP32 ulps on the transfer function (powf) and the
blend; the loss gradient relative to its largest element."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import paper_2504_01358_gb300 as S
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return S


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def test_tonemap_matches_oracle(S):
    rng = np.random.default_rng(8)
    x = np.concatenate([rng.uniform(-0.5, 1.5, 200000), rng.lognormal(0, 2, 50000), [0.0, 1.0, 0.0031308, -0.0, 3e-5]])
    x = x.astype(np.float32)
    got = S.ssgi_tonemap_srgb(_t(x)).cpu().numpy()
    ref = O.tonemap_srgb(x)
    assert np.abs(got - ref).max() <= 4e-7
    y = _t(x)
    S.ssgi_tonemap_srgb(y, out=y)  # in place
    assert torch.equal(y.cpu(), torch.from_numpy(got))


@pytest.mark.parametrize("n", [1, 257, 3 * 97 * 61, 3 * 1600 * 900])
def test_srgb_loss_and_gradient_match_oracle(S, n):
    rng = np.random.default_rng(n)
    f = rng.uniform(-0.2, 1.4, n).astype(np.float32)
    t = rng.uniform(0, 1, n).astype(np.float32)
    g, loss = S.ssgi_l2_loss_srgb(_t(f), _t(t))
    lo, go = O.l2_loss_srgb(f, t)
    assert abs(float(loss.item()) - lo) <= 1e-5 * lo
    g = g.cpu().numpy()
    assert np.abs(g - go).max() <= 1e-5 * np.abs(go).max()
    assert np.all(g[(f < 0) | (f > 1)] == 0.0)


def test_keyframe_blend_and_adjoint(S):
    rng = np.random.default_rng(9)
    a, b = rng.lognormal(0, 1, (32, 64, 3)), rng.lognormal(0, 1, (32, 64, 3))
    for frame in (0, 3, 10, 17):
        k, alpha = S.ssgi_keyframe_of(frame)
        out = S.ssgi_env_keyframe_lerp(_t(a), _t(b), alpha).cpu().numpy()
        ref = O.keyframe_lerp(a.astype(np.float32), b.astype(np.float32), alpha)
        assert np.abs(out - ref).max() <= 3e-7 * np.abs(ref).max()
    g = rng.normal(size=(32, 64, 3))
    ga, gb = _t(np.ones_like(g)), _t(np.zeros_like(g))
    S.ssgi_env_keyframe_lerp_backward(_t(g), 0.25, ga, gb, accumulate=True)
    np.testing.assert_allclose(ga.cpu().numpy(), 1.0 + 0.75 * g, rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(gb.cpu().numpy(), 0.25 * g, rtol=1e-6, atol=1e-6)
    S.ssgi_env_keyframe_lerp_backward(_t(g), 0.25, ga, gb, accumulate=False)
    np.testing.assert_allclose(ga.cpu().numpy(), 0.75 * g, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("flags", [0, 1])
def test_trace_srgb_epilogue_equals_the_separate_transform(S, flags):
    """SSGI_SRGB_FINAL: the trace writes the display image itself (the output transform as its
    epilogue), bit for bit the separate ssgi_tonemap_srgb of its linear final, on foreground and
    background pixels; the linear parts and the hits are unchanged, and the oracle's transform of
    the oracle's final agrees to the transfer function's bound."""
    import ssgi_inputs as si
    from parity import gpu_forward
    wl = si.small_case()
    base = gpu_forward(wl, flags=flags)
    enc = gpu_forward(wl, flags=flags | S._native.SRGB_FINAL)
    assert np.array_equal(enc["hit_idx"], base["hit_idx"])
    assert np.array_equal(enc["cs_mc"], base["cs_mc"])
    sep = S.ssgi_tonemap_srgb(_t(base["final"])).cpu().numpy()
    assert np.array_equal(enc["final"], sep)
    r = O.forward(wl, lut=O.build_lut(), flags=flags)
    assert np.abs(enc["final"] - O.tonemap_srgb(r["final"])).max() <= 1e-4
    # not a flag of the fused step (its loss reads the linear image)
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    p.flags |= S._native.SRGB_FINAL
    with pytest.raises(S._native.SSGIError):
        S.ssgi_step_fused(g, cams, env, S.ssgi_build_brdf_lut(), tgt, p)
