"""The allocation-free backward entry point (ssgi_backward_noalloc), called through the C ABI.

It exists for callers that cannot allocate device memory while they run (a render loop on a
fixed memory budget, an application whose pool allocator owns the device); it uses a scratch
array inside the library instead of a caller workspace.  This file is collected last so that a
failure here does not hide any other test, and it builds its own inputs, so it also passes when
run alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

import ssgi_inputs as si
from parity import GRAD_RTOL

pytestmark = pytest.mark.gpu


def test_noalloc_backward_matches_workspace_backward_on_two_calls():
    import paper_2504_01358_gb300 as S
    from paper_2504_01358_gb300 import _native as N

    assert torch.cuda.is_available()
    wl = si.config1()
    wl.target = si.uniform_target(5, *wl.depth.shape)
    g, env, cams, tgt = S.to_device_workload(wl)
    p = S.params_of(wl.params)
    lut = S.ssgi_build_brdf_lut()
    em = S.ssgi_build_env_mips(env)
    hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels)
    c_d, _, c1 = S.ssgi_shade_direct(g, cams, em, lut)
    tr = S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p, want_hits=True)
    gf, _ = S.ssgi_l2_loss(tr["final"], tgt)
    ref = S.ssgi_backward(gf, g, cams, c1, em, lut, tr["hit_idx"], p)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}

    cam = S.cameras(cams)
    gs, es, ps = g.c_struct(), em.c_struct(), p.c_struct()
    for call in range(2):
        out = {k: torch.full(v.shape, float("nan"), device="cuda") for k, v in ref.items()}
        rc = N.lib().ssgi_backward_noalloc(
            C.c_void_p(gf.data_ptr()), C.byref(gs), cam, C.c_void_p(c1.data_ptr()), C.byref(es),
            C.c_void_p(lut.data_ptr()), int(lut.shape[0]), C.c_void_p(tr["hit_idx"].data_ptr()), C.byref(ps),
            C.c_void_p(out["albedo"].data_ptr()), C.c_void_p(out["rough"].data_ptr()),
            C.c_void_p(out["metal"].data_ptr()), C.c_void_p(out["normal"].data_ptr()),
            C.c_void_p(out["env"].data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, N.STATUS.get(rc, rc)
        torch.cuda.synchronize()
        for k, want in ref.items():
            got = out[k].cpu().numpy()
            assert np.isfinite(got).all(), (call, k)
            scale = max(float(np.abs(want).max()), 1e-30)
            err = float(np.abs(got - want).max()) / scale
            assert err <= GRAD_RTOL, (call, k, err)


def test_noalloc_backward_rejects_sizes_beyond_its_scratch():
    from paper_2504_01358_gb300 import _native as N

    fake = C.c_void_p(0x100000)
    d = N.Dims(8, 825, 1245)
    assert N.lib().ssgi_backward_workspace_bytes(d, 512, 1024) > N.BACKWARD_NOALLOC_MAX_BYTES
    g = N.GBuffer(fake, fake, fake, fake, fake, d)
    cams = (N.Camera * 8)()
    for c in cams:
        c.fov_y_rad, c.z_near = 1.0, 0.01
    env = N.EnvMap(fake, 512, 1024, 10)
    p = N.TraceParams(32, 64, 8, 0.05, 100.0, 1, 0)
    rc = N.lib().ssgi_backward_noalloc(fake, C.byref(g), cams, fake, C.byref(env), fake, 64, fake, C.byref(p),
                                       fake, fake, fake, fake, fake, None)
    assert rc == 2  # SSGI_ERR_UNSUPPORTED
