"""The fused step (ssgi_step_fused: all stages of a multi-view inverse-rendering step
in one launch) against the per-stage calls and the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import ssgi_inputs as si
from parity import GRAD_RTOL, assert_forward_parity

pytestmark = pytest.mark.gpu


def _per_stage(S, wl, lut):
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    em = S.ssgi_build_env_mips(env)
    hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels) if p.hiz_levels > 1 else None
    c_d, _, c1 = S.ssgi_shade_direct(g, cams, em, lut)
    tr = S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p, want_hits=True)
    lossf = S.ssgi_l2_loss_srgb if p.flags & 8 else S.ssgi_l2_loss
    gf, loss = lossf(tr["final"], tgt)
    gr = S.ssgi_backward(gf, g, cams, c1, em, lut, tr["hit_idx"], p)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in gr.items()}
    out.update(final=tr["final"].cpu().numpy(), hit_idx=tr["hit_idx"].cpu().numpy(), loss=float(loss.item()))
    return out


def _fused(S, wl, lut, reps=1):
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    out = None
    for _ in range(reps):
        out = S.ssgi_step_fused(g, cams, env, lut, tgt, p, out=out)
    torch.cuda.synchronize()
    assert not S.ssgi_step_fused_check(out["_workspace"])
    res = {k: v.cpu().numpy() for k, v in out.items() if k != "_workspace"}
    res["loss"] = float(res["loss"][0])
    return res


def _compare(a, b):
    assert np.array_equal(a["final"], b["final"])
    assert np.array_equal(a["hit_idx"], b["hit_idx"])
    assert abs(a["loss"] - b["loss"]) <= 1e-5 * abs(b["loss"])
    for k in ("albedo", "rough", "metal", "normal", "env"):
        scale = max(float(np.abs(b[k]).max()), 1e-30)
        assert float(np.abs(a[k] - b[k]).max()) / scale <= 1e-4, k


@pytest.mark.parametrize("flags", [0, 1, 4, 5, 8, 9])
def test_fused_step_equals_the_per_stage_path(flags):
    import paper_2504_01358_gb300 as S
    scene = si.make_scene(31, 10, 4.0, 1)
    cams = [si.look_at((5 * np.sin(a), 1.7, 5 * np.cos(a)), (0, 0.3, 0)) for a in (0.3, 1.9, 3.5, 5.1)]
    bufs = [si.raycast_gbuffer(scene, c, 61, 97) for c in cams]
    st = lambda k: np.stack([b[k] for b in bufs])  # noqa: E731
    wl = si.Workload("4view-61x97", st("depth"), st("normal"), st("albedo"), st("rough"), st("metal"),
                     np.stack(cams), si.lognormal_env(33, 32, 64),
                     si.TraceParams(spp=8, max_steps=48, seed=5, flags=flags), si.uniform_target(34, 4, 61, 97))
    lut = S.ssgi_build_brdf_lut()
    ref = _per_stage(S, wl, lut)
    got = _fused(S, wl, lut, reps=2)  # a second launch reuses the workspace
    _compare(got, ref)


def test_config4_eight_views_fused_against_per_stage_and_oracle():
    """Config 4: 8 views at 1245x825 on a ring around a 60-box scene, shared 512x1024 env,
    32 spp, 8 levels, fused forward+backward in one launch with stored hit indices."""
    import paper_2504_01358_gb300 as S
    wl = si.config4()
    lut = S.ssgi_build_brdf_lut()
    ref = _per_stage(S, wl, lut)
    got = _fused(S, wl, lut)
    _compare(got, ref)
    # forward parity with the oracle on sampled pixels of all views
    V, H, W = wl.depth.shape
    rng = np.random.default_rng(4)
    pl = np.sort(rng.choice(V * H * W, size=6000, replace=False))
    r = O.forward(wl, lut=O.build_lut(), pix_list=pl)
    sub = {"hit_idx": got["hit_idx"].reshape(V * H * W, -1)[pl], "final": got["final"].reshape(-1, 3)[pl]}
    assert_forward_parity(sub, r, "config4 sample", wl=wl, pix=pl)
    assert (sub["hit_idx"] >= 0).mean() > 0.02


def test_fused_phase_wait_gives_up_and_the_next_step_is_clean():
    """The phase boundary's bounded wait: with the wait limit at 0 polls a block whose previous
    phase has not finished gives up at once, marks the error word, and every later block returns
    (no hang, no fault); ssgi_step_fused_check reports it.  With the default limit restored the
    next launch on the same workspace runs to the end and equals the per-stage path."""
    import paper_2504_01358_gb300 as S
    wl = si.small_case()
    lut = S.ssgi_build_brdf_lut()
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    try:
        S.ssgi_step_fused_set_wait_limit(0)
        out = S.ssgi_step_fused(g, cams, env, lut, tgt, p)
        torch.cuda.synchronize()
        assert S.ssgi_step_fused_check(out["_workspace"])
    finally:
        S.ssgi_step_fused_set_wait_limit(-1)
    out = S.ssgi_step_fused(g, cams, env, lut, tgt, p, out=out, workspace=out["_workspace"])
    torch.cuda.synchronize()
    assert not S.ssgi_step_fused_check(out["_workspace"])
    got = {k: v.cpu().numpy() for k, v in out.items() if k != "_workspace"}
    got["loss"] = float(got["loss"][0])
    _compare(got, _per_stage(S, wl, lut))


def _up256(n):
    return (n + 255) & ~255


@pytest.mark.parametrize("H,W,levels,he,we", [(61, 97, 8, 32, 64), (77, 133, 9, 64, 128), (33, 200, 3, 8, 16),
                                              (150, 40, 16, 128, 256), (16, 16, 2, 2, 4)])
def test_fused_pyramids_equal_the_stand_alone_builders(H, W, levels, he, we):
    """The Hi-Z pyramid and the environment mip chain the fused step builds in its workspace
    (its own tiling: 16 x 16 tiles through level 4, the levels above by the block that finishes
    a pyramid's last item) equal ssgi_build_hiz and ssgi_build_env_mips bit for bit: minima and
    2 x 2 means of the same four values in the same order, however the work is cut.  The
    workspace holds a 512-byte control block, then the mip chain, then the pyramid (each start
    256-byte aligned)."""
    import paper_2504_01358_gb300 as S
    scene = si.make_scene(41, 6, 4.0, 1)
    cams = [si.look_at((5 * np.sin(a), 1.5, 5 * np.cos(a)), (0, 0.3, 0)) for a in (0.4, 2.6, 4.4)]
    bufs = [si.raycast_gbuffer(scene, c, H, W) for c in cams]
    st = lambda k: np.stack([b[k] for b in bufs])  # noqa: E731
    wl = si.Workload(f"3view-{H}x{W}", st("depth"), st("normal"), st("albedo"), st("rough"), st("metal"),
                     np.stack(cams), si.lognormal_env(43, he, we),
                     si.TraceParams(spp=4, max_steps=24, seed=7, hiz_levels=levels), si.uniform_target(44, 3, H, W))
    lut = S.ssgi_build_brdf_lut()
    g, env, cams_d, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    out = S.ssgi_step_fused(g, cams_d, env, lut, tgt, p)
    torch.cuda.synchronize()
    assert not S.ssgi_step_fused_check(out["_workspace"])
    ws = out["_workspace"]
    n_mips = S.ssgi_env_mip_floats(he, we)
    n_hiz = S.ssgi_hiz_floats((3, H, W), levels)
    o_mips = 512
    o_hiz = o_mips + _up256(4 * n_mips)
    mips_f = ws[o_mips:o_mips + 4 * n_mips].view(torch.float32).cpu().numpy()
    mips_s = S.ssgi_build_env_mips(env).mips.cpu().numpy()
    assert np.array_equal(mips_f.view(np.uint32), mips_s.view(np.uint32))
    if levels > 1:
        hiz_f = ws[o_hiz:o_hiz + 4 * n_hiz].view(torch.float32).cpu().numpy()
        hiz_s = S.ssgi_build_hiz(g.depth, levels).cpu().numpy()[:n_hiz]
        assert np.array_equal(hiz_f.view(np.uint32), hiz_s.view(np.uint32))
