"""CPU checks of the C ABI: libssgi.so builds, loads without a GPU, exports every function
include/ssgi.h declares, and its host-side size queries and argument validation behave.
No call here reaches a CUDA API (validation fails before any launch)."""
import ctypes as C
import os
import re

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def N():
    from paper_2504_01358_gb300 import _native
    _native.lib()
    return _native


def _declared():
    src = open(os.path.join(ROOT, "include", "ssgi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ssgi_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(N):
    names = _declared()
    assert len(names) >= 12
    lib = C.CDLL(N.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(N.EXPORTED), set(names) - set(N.EXPORTED)


def test_status_strings_and_version(N):
    L = N.lib()
    assert L.ssgi_status_string(0) == b"ok"
    assert L.ssgi_status_string(1) == b"invalid argument"
    assert b"sm_103a" in L.ssgi_version()


def test_size_queries_match_the_oracle_layout(N):
    L = N.lib()
    for h, w in [(64, 128), (256, 512), (1, 2), (8, 8)]:
        assert L.ssgi_env_levels(h, w) == O.env_levels(h, w)
        assert L.ssgi_env_mip_floats(h, w) == O.build_env_mips(__import__("numpy").zeros((h, w, 3))).size
    assert L.ssgi_env_levels(3, 8) == -1 and L.ssgi_env_levels(8, 4) == -1
    for (V, H, W), lev in [((1, 900, 1600), 8), ((3, 37, 53), 6), ((1, 1, 1), 1)]:
        assert L.ssgi_hiz_floats(N.Dims(V, H, W), lev) == V * O.hiz_floats_per_view(H, W, lev)
    ws = L.ssgi_backward_workspace_bytes(N.Dims(1, 900, 1600), 256, 512)
    assert ws >= 4 * (3 * 900 * 1600 + O.build_env_mips(__import__("numpy").zeros((256, 512, 3))).size)
    assert L.ssgi_backward_workspace_bytes(N.Dims(0, 9, 9), 256, 512) == 0


def test_invalid_arguments_fail_before_any_launch(N):
    L = N.lib()
    fake = C.c_void_p(0x100000)
    assert L.ssgi_build_hiz(None, N.Dims(1, 8, 8), 4, fake, None) == 1
    assert L.ssgi_build_hiz(fake, N.Dims(1, 8, 8), 0, fake, None) == 1
    assert L.ssgi_build_hiz(fake, N.Dims(0, 8, 8), 4, fake, None) == 1
    assert L.ssgi_build_env_mips(fake, 6, 8, fake, None) == 1
    assert L.ssgi_build_brdf_lut(1, 64, fake, None) == 1
    g = N.GBuffer(fake, fake, fake, fake, fake, N.Dims(1, 8, 8))
    cam = (N.Camera * 1)()
    cam[0].fov_y_rad, cam[0].z_near = 1.0, 0.01
    env = N.EnvMap(fake, 8, 16, 4)
    p = N.TraceParams(4, 32, 8, 0.05, 100.0, 1, 0)
    bad_p = N.TraceParams(0, 32, 8, 0.05, 100.0, 1, 0)
    assert L.ssgi_trace_indirect(C.byref(g), cam, fake, fake, fake, C.byref(env), C.byref(bad_p), None, None, fake,
                                 None, None, None) == 1
    bad_env = N.EnvMap(fake, 8, 16, 3)
    assert L.ssgi_shade_direct(C.byref(g), cam, C.byref(bad_env), fake, 64, fake, None, fake, None) == 1
    bad_cam = (N.Camera * 1)()
    assert L.ssgi_shade_direct(C.byref(g), bad_cam, C.byref(env), fake, 64, fake, None, fake, None) == 1
    # workspace too small
    assert L.ssgi_backward(fake, C.byref(g), cam, fake, C.byref(env), fake, 64, fake, C.byref(p), fake, fake, fake,
                           fake, fake, fake, 16, None) == 1
    assert L.ssgi_l2_loss(fake, fake, 0, fake, None, None) == 1


def test_serving_host_side_checks(N):
    L = N.lib()
    d = N.Dims(1, 90, 160)
    full = L.ssgi_serve_request_bytes(d, 16, 32, 8, 0)
    resident = L.ssgi_serve_request_bytes(d, 16, 32, 8, 1)
    px = 90 * 160
    assert resident >= px * 36 and full >= resident + px * 36 + 4 * O.hiz_floats_per_view(90, 160, 8)
    assert L.ssgi_serve_request_bytes(d, 3, 8, 8, 0) == 0
    cfg = N.ServeConfig(16, 4, 8, 0, 0)  # budget below the minimum
    h = C.c_void_p()
    assert L.ssgi_serve_create(C.byref(cfg), C.byref(h)) == 1
    cfg = N.ServeConfig(1 << 30, 0, 8, 0, 0)  # no slots
    assert L.ssgi_serve_create(C.byref(cfg), C.byref(h)) == 1
    assert L.ssgi_serve_submit(None, None, None) == 1
    assert L.ssgi_serve_poll(None, 1, None) == 1
    assert L.ssgi_serve_destroy(None, 0) == 1


def test_fused_phase_names_match_the_header():
    from paper_2504_01358_gb300 import ssgi
    src = open(os.path.join(ROOT, "include", "ssgi.h")).read()
    m = re.search(r"#define\s+SSGI_FUSED_PHASES\s+(\d+)", src)
    assert m and int(m.group(1)) == len(ssgi.FUSED_PHASES)


def test_bandwidth_probe_rejects_bad_arguments(N):
    L = N.lib()
    fake, sink = C.c_void_p(0x100000), C.c_void_p(0x200000)
    assert L.ssgi_read_bandwidth_probe(None, 64, 1, sink, None) == 1
    assert L.ssgi_read_bandwidth_probe(C.c_void_p(0x100008), 64, 1, sink, None) == 1  # not 16-byte aligned
    assert L.ssgi_read_bandwidth_probe(fake, 60, 1, sink, None) == 1                  # not a multiple of 16
    assert L.ssgi_read_bandwidth_probe(fake, 0, 1, sink, None) == 1
    assert L.ssgi_read_bandwidth_probe(fake, 64, 0, sink, None) == 1
    assert L.ssgi_read_bandwidth_probe(fake, 64, 1, None, None) == 1


def test_depth_normals_rejects_bad_arguments(N):
    L = N.lib()
    fake = C.c_void_p(0x100000)
    cams = (N.Camera * 1)()
    assert L.ssgi_depth_normals(None, N.Dims(1, 8, 8), cams, fake, None) == 1
    assert L.ssgi_depth_normals(fake, N.Dims(1, 8, 8), cams, None, None) == 1
    assert L.ssgi_depth_normals(fake, N.Dims(0, 8, 8), cams, fake, None) == 1
    assert L.ssgi_depth_normals(fake, N.Dims(1, 8, 8), None, fake, None) == 1


def test_composite_rejects_bad_arguments(N):
    L = N.lib()
    f = [C.c_void_p(0x100000 + 0x1000 * i) for i in range(10)]
    sc = N.GBuffer(f[0], f[1], f[2], f[3], f[4], N.Dims(1, 8, 8))
    ob = N.GBuffer(f[5], f[6], f[7], f[8], f[9], N.Dims(1, 8, 8))
    bad = N.GBuffer(f[5], f[6], f[7], f[8], f[9], N.Dims(1, 8, 9))
    o = [C.c_void_p(0x900000 + 0x1000 * i) for i in range(5)]
    assert L.ssgi_composite_gbuffer(C.byref(sc), C.byref(bad), *o, None, None) == 1        # dims differ
    assert L.ssgi_composite_gbuffer(None, C.byref(ob), *o, None, None) == 1
    assert L.ssgi_composite_gbuffer(C.byref(sc), C.byref(ob), None, *o[1:], None, None) == 1
    mixed = [f[0], o[1], o[2], o[3], o[4]]                                                   # partly in place
    assert L.ssgi_composite_gbuffer(C.byref(sc), C.byref(ob), *mixed, None, None) == 1


def test_keyframe_of_matches_the_oracle_and_rejects_bad_arguments(N):
    L = N.lib()
    k, a = C.c_int64(), C.c_float()
    for frame in (0, 1, 9, 10, 11, 27, 99, 100, 12345):
        for period in (1, 3, 10):
            assert L.ssgi_keyframe_of(frame, period, C.byref(k), C.byref(a)) == 0
            ko, ao = O.keyframe_of(frame, period)
            assert k.value == ko and abs(a.value - ao) <= 1e-7
    assert L.ssgi_keyframe_of(-1, 10, C.byref(k), C.byref(a)) == 1
    assert L.ssgi_keyframe_of(5, 0, C.byref(k), C.byref(a)) == 1
    fake = C.c_void_p(0x100000)
    assert L.ssgi_tonemap_srgb(fake, None, 16, None) == 1
    assert L.ssgi_tonemap_srgb(fake, fake, 0, None) == 1
    assert L.ssgi_l2_loss_srgb(fake, fake, 0, fake, None, None) == 1
    assert L.ssgi_env_keyframe_lerp(fake, fake, C.c_float(1.5), 4, 8, fake, None) == 1
    assert L.ssgi_env_keyframe_lerp_backward(fake, C.c_float(0.5), 4, 8, fake, fake, 1, None) == 1  # g_a == g_b
