"""The FP32 model of the kernels' direction and coordinate arithmetic (tests/fp32_emu.py), pinned
on the CPU against exact arithmetic, the FP64 library functions and the oracle's own lookup and
sampler: its one-rounding operations round exactly once, its sine / cosine / arctangent stay
within a few FP32 ulps of the true functions, and the coordinates and directions it forms are
the oracle's (in FP64) up to FP32 rounding."""
import math
from fractions import Fraction

import numpy as np

import fp32_emu as E
import oracle as O

F32 = np.float32


def test_round_f32_matches_numpy_and_breaks_ties_to_even():
    rng = np.random.default_rng(0)
    for x in rng.standard_normal(2000) * 10.0 ** rng.integers(-30, 30, 2000):
        assert E.round_f32(Fraction(float(x))) == float(F32(x))
    one = Fraction(1)
    ulp = Fraction(1, 2 ** 23)
    assert E.round_f32(one + ulp / 2) == 1.0                    # tie -> even (1.0)
    assert E.round_f32(one + ulp + ulp / 2) == float(1 + 2 * ulp)  # tie -> even (1 + 2 ulp)
    assert E.round_f32(Fraction(1, 2 ** 150)) == 0.0            # half the smallest subnormal -> 0 (even)
    assert E.round_f32(Fraction(3, 2 ** 151)) == 2.0 ** -149


def test_fma_rounds_once():
    rng = np.random.default_rng(1)
    a = rng.standard_normal(3000).astype(F32)
    b = rng.standard_normal(3000).astype(F32)
    c = (-(a.astype(np.float64) * b) * (1 + rng.standard_normal(3000) * 1e-6)).astype(F32)  # cancellation
    got = E.fma(a, b, c)
    for x, y, z, g in zip(a, b, c, got):
        want = E.round_f32(Fraction(float(x)) * Fraction(float(y)) + Fraction(float(z)))
        assert float(g) == want
    # a sum that lands exactly on an FP32 midpoint in FP64 but not exactly: the rational sum decides
    x, y = 1.0 + 2.0 ** -12, 1.0 + 2.0 ** -12          # x y = 1 + 2^-11 + 2^-24 exactly
    z = -(2.0 ** -11) + 2.0 ** -30
    assert float(E.fma(x, y, z)) == E.round_f32(Fraction(x) * Fraction(y) + Fraction(z))


def _ulps(got, want):
    return abs(got - want) / float(np.spacing(F32(max(abs(want), 2.0 ** -126))))


def test_sincospi_within_two_ulps_on_the_uniform_grid():
    rng = np.random.default_rng(2)
    xs = np.concatenate([rng.integers(0, 2 ** 24, 4000) * 2.0 ** -23,
                         np.arange(0, 2.0, 0.125), [2.0 - 2.0 ** -23, 2.0 ** -23]])
    worst = 0.0
    S, C = E.sincospi(xs.astype(F32))
    for x, s, c in zip(xs, S.astype(float), C.astype(float)):
        ts, tc = math.sin(math.pi * x), math.cos(math.pi * x)
        assert abs(s - ts) <= 2.5e-7 and abs(c - tc) <= 2.5e-7, x
        worst = max(worst, _ulps(s, ts) if abs(ts) > 1e-3 else 0.0, _ulps(c, tc) if abs(tc) > 1e-3 else 0.0)
    assert worst <= 2.0, worst
    # quarter turns are exact
    for x, (s0, c0) in ((0.0, (0.0, 1.0)), (0.5, (1.0, 0.0)), (1.0, (0.0, -1.0)), (1.5, (-1.0, 0.0))):
        s, c = E.sincospi(x)
        assert float(s) == s0 and float(c) == c0


def test_atan_octant_within_three_ulps():
    rng = np.random.default_rng(3)
    worst = 0.0
    den = rng.uniform(1e-3, 10.0, 5000).astype(F32)
    num = (den * rng.uniform(-1.0, 1.0, 5000)).astype(F32)
    got_all = E.atan_octant(num, den)
    for n_, d_, got in zip(num.astype(float), den.astype(float), got_all.astype(float)):
        want = math.atan2(n_, d_)
        worst = max(worst, _ulps(got, want) if abs(want) > 1e-6 else abs(got - want) / 1e-13)
        assert abs(got - want) <= 1.2e-7, (n_, d_)
    # the largest errors (~2.7 ulp) sit just above the reduction threshold tan(pi/8), where
    # pi/4 + atan(r) cancels to ~0.41
    assert worst <= 3.0, worst
    assert float(E.atan_octant(0.0, 0.0)) == 0.0
    assert float(E.atan_octant(-0.0, 0.0)) == 0.0 and np.signbit(E.atan_octant(-0.0, 0.0))
    assert float(E.atan_octant(0.0, -0.0)) == float(F32(math.pi)) == -float(E.atan_octant(-0.0, -0.0))
    assert float(E.atan_octant(1.0, 1.0)) == float(F32(math.pi / 4))


def test_texel_coordinates_follow_the_latitude_longitude_mapping():
    """x = (0.5 + atan2(d.x, -d.z) / 2pi) w - 0.5 and y = acos(d.y) / pi h - 0.5 (mod w in x), to
    FP32 rounding of the angles, in every octant and at the poles."""
    rng = np.random.default_rng(4)
    h, w = 256, 512
    dirs = list(rng.standard_normal((3000, 3)))
    dirs += [np.array(v, float) for v in ((0, 1, 0), (0, -1, 0), (1e-4, 1, 0), (0, -1, -1e-5), (1, 0, 0),
                                          (-1, 0, 0), (0, 0, 1), (0, 0, -1), (1, 0, 1), (-1, 0, -1),
                                          (0.0, 1.0, -0.0), (-0.0, -1.0, 0.0))]
    D32 = np.array(dirs, F32)
    X0, Y0, TX, TY = E.texel_coords(D32, h, w)
    for d, x0, y0, tx, ty in zip(D32, X0, Y0, TX.astype(float), TY.astype(float)):
        assert 0.0 <= tx < 1.0 and 0.0 <= ty < 1.0
        dd = d.astype(np.float64)
        u = 0.5 + math.atan2(dd[0], -dd[2]) / (2 * math.pi)
        vt = math.atan2(math.hypot(dd[0], dd[2]), dd[1]) / math.pi
        xe, ye = u * w - 0.5, vt * h - 0.5
        dx = (x0 + tx - xe) % w
        dx = min(dx, w - dx)
        q = math.hypot(dd[0], dd[2]) / np.linalg.norm(dd)
        if q == 0.0:  # on the axis itself: the longitude of atan2's signed zeros
            assert dx <= 2e-4, (d, x0 + tx, xe)
        elif q > 1e-6:
            assert dx <= 2e-4 + 4e-7 * w / q, (d, x0 + tx, xe)
        assert abs(y0 + ty - ye) <= 2e-4, (d, y0 + ty, ye)


def test_emulated_lookup_equals_the_oracle_lookup_away_from_steep_texels():
    """FP64 bilinear at the model's coordinates against the oracle's own mip-0 lookup: the same
    texels and weights up to the FP32 rounding of the coordinates."""
    rng = np.random.default_rng(5)
    He, We = 32, 64
    env = np.exp(rng.standard_normal((He, We, 3))).astype(F32)
    mips = O.build_env_mips(env)
    base = mips[: He * We * 3].reshape(He, We, 3)
    D32 = rng.standard_normal((500, 3)).astype(F32)
    X0, Y0, TX, TY = E.texel_coords(D32, He, We)
    for d32, x0, y0, tx, ty in zip(D32, X0, Y0, TX.astype(float), TY.astype(float)):
        c0, c1 = x0 % We, (x0 + 1) % We
        r0, r1 = min(max(y0, 0), He - 1), min(max(y0 + 1, 0), He - 1)
        got = ((1 - tx) * (1 - ty) * base[r0, c0] + tx * (1 - ty) * base[r0, c1] + (1 - tx) * ty * base[r1, c0]
               + tx * ty * base[r1, c1])
        want = O.env_lookup(mips, He, We, d32.astype(np.float64), 0.0)
        assert np.allclose(got, want, rtol=2e-5, atol=0.0), (d, got, want)


def test_emulated_sample_is_the_oracles_sample_in_fp32():
    """The model's half vector and reflected direction against the oracle's FP64 sampler at the
    same uniforms (the frame, the angles and the reflection are the oracle's)."""
    rng = np.random.default_rng(6)
    for _ in range(400):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        n32 = n.astype(F32)
        v = rng.standard_normal(3)
        v /= np.linalg.norm(v)
        v32 = v.astype(F32)
        rho = F32(rng.uniform(0.02, 1.0))
        xi0 = F32(float(rng.integers(0, 2 ** 24)) * 2.0 ** -24)
        xi1 = F32(float(rng.integers(0, 2 ** 24)) * 2.0 ** -24)
        nv = E.dot3(n32, v32)
        sm = E.make_sample(n32, v32, nv, rho, xi0, xi1)
        h = O.ggx_sample_h(n32.astype(np.float64), float(rho), float(xi0), float(xi1))
        assert np.allclose(sm["h"], h, atol=2e-6), (n32, rho, xi0, xi1)
        w = 2.0 * float(np.dot(v32.astype(np.float64), h)) * h - v32.astype(np.float64)
        assert np.allclose(sm["w"], w, atol=4e-6)


def test_view_vector_and_pixel_ray_match_the_camera_convention():
    import ssgi_inputs as si
    cam = si.look_at((0.3, 1.6, 5.0), (0.0, 0.5, 0.0))
    H, W = 90, 160
    c = E.Cam(cam, H, W)
    rays, eye = si.pixel_rays(cam, H, W)
    for (x, y) in ((0, 0), (W - 1, H - 1), (W // 2, H // 2), (17, 61)):
        d = E.pix_dir_world(c, x, y)
        assert np.allclose(d, rays[y, x], rtol=0, atol=2e-6)
        v = E.view_vector(d)
        assert np.allclose(v, -rays[y, x] / np.linalg.norm(rays[y, x]), atol=2e-7)
