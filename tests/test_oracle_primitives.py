"""Pins of the oracle's building blocks against what the paper and the mathematics fix.

Each test checks an oracle function against something other than itself: an independent
library implementation, a textbook identity, a quadrature, or a brute-force computation.
"""
import json
import math
import os
import subprocess
import sys

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O

pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")


# --------------------------------------------------------------------------------------------
# Philox4x32-10 (the counter-based RNG both sides implement from its published definition)
# --------------------------------------------------------------------------------------------
_TRITON_PROBE = r"""
import os, json, sys
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def k(c_ptr, out_ptr, seed, N: tl.constexpr):
    i = tl.arange(0, N)
    c0 = tl.load(c_ptr + i * 4 + 0).to(tl.uint32)
    c1 = tl.load(c_ptr + i * 4 + 1).to(tl.uint32)
    c2 = tl.load(c_ptr + i * 4 + 2).to(tl.uint32)
    c3 = tl.load(c_ptr + i * 4 + 3).to(tl.uint32)
    a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
    tl.store(out_ptr + i * 4 + 0, a)
    tl.store(out_ptr + i * 4 + 1, b)
    tl.store(out_ptr + i * 4 + 2, c)
    tl.store(out_ptr + i * 4 + 3, d)

cases = json.loads(sys.stdin.read())
res = []
for seed, ctrs in cases:
    c = torch.tensor(np.array(ctrs, dtype=np.uint32).view(np.int32).reshape(-1))
    out = torch.zeros(len(ctrs) * 4, dtype=torch.int32)
    k[(1,)](c, out, seed, N=len(ctrs))
    res.append((out.numpy().view(np.uint32)).reshape(-1, 4).tolist())
print(json.dumps(res))
"""


def _kat_vectors():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "philox4x32_10_kat.txt")
    out = []
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(t, 16) for t in line.split()]
                out.append((w[0:4], w[4:6], w[6:10]))
    return out


def test_philox_known_answer_vectors():
    """Philox4x32-10 against the generator's published known-answer vectors (no other
    implementation needed): all-zero, all-ones and the pi-digit counter/key."""
    kat = _kat_vectors()
    assert len(kat) == 3
    for ctr, key, want in kat:
        assert O.philox4x32_10(ctr, key).tolist() == want, (ctr, key)


def test_philox_matches_triton_reference_implementation():
    """Philox4x32-10 against triton's independent implementation (its CPU interpreter)."""
    pytest.importorskip("triton")
    rng = np.random.default_rng(123)
    cases = []
    for seed in [0, 1, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, int(rng.integers(0, 2**63))]:
        ctrs = rng.integers(0, 2**32, size=(8, 4), dtype=np.uint64).tolist()
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        cases.append((seed, ctrs))
    env = dict(os.environ, TRITON_INTERPRET="1")
    p = subprocess.run([sys.executable, "-c", _TRITON_PROBE], input=json.dumps(cases), capture_output=True,
                       text=True, env=env, timeout=600)
    if p.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + p.stderr[-300:])
    ref = json.loads(p.stdout.strip().splitlines()[-1])
    for (seed, ctrs), want in zip(cases, ref):
        key = [seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF]
        for ctr, w in zip(ctrs, want):
            got = O.philox4x32_10(ctr, key).tolist()
            assert got == w, (seed, ctr, got, w)


def test_uniforms_are_uniform_and_uncorrelated():
    """xi = (out >> 8) 2^-24 over a counter sweep: chi-square uniformity and no lag correlation."""
    n = 40000
    xs = np.array([O.philox4x32_10([i, 3, 0, 0], [7, 9]) for i in range(n)], dtype=np.uint64)
    xi = (xs >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    for k in range(4):
        hist, _ = np.histogram(xi[:, k], bins=50, range=(0, 1))
        assert stats.chisquare(hist).pvalue > 1e-4
    assert abs(np.corrcoef(xi[:, 0], xi[:, 1])[0, 1]) < 0.03
    assert abs(np.corrcoef(xi[:-1, 0], xi[1:, 0])[0, 1]) < 0.03


# --------------------------------------------------------------------------------------------
# Microfacet terms (Appendix B)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("rho", [0.05, 0.1, 0.3, 0.5, 0.8, 1.0])
def test_ggx_ndf_is_normalised(rho):
    """int D(h) (n.h) dw_h = 1 over the hemisphere (eq:ndf is a normalised microfacet density)."""
    f = lambda c: O.ggx_D(c, rho) * c * 2.0 * math.pi
    val, _ = integrate.quad(f, 0.0, 1.0, points=[1.0 - 1e-3, 1.0 - 1e-2, 1.0 - 0.1], limit=400, epsabs=1e-12)
    assert abs(val - 1.0) < 1e-7


def test_smith_G1_matches_lambda_form():
    """eq:geometry equals the Smith form 1 / (1 + Lambda), Lambda = (-1 + sqrt(1 + a^2 tan^2)) / 2
    (Walter et al. 2007 / Heitz 2014)."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        z = rng.uniform(0.01, 1.0)
        a = rng.uniform(0.0, 1.0)
        tan2 = (1 - z * z) / (z * z)
        lam = (-1.0 + math.sqrt(1.0 + a * a * tan2)) / 2.0
        assert O.ggx_G1(z, a) == pytest.approx(1.0 / (1.0 + lam), rel=1e-12)
    assert O.ggx_G1(0.3, 0.0) == pytest.approx(1.0, rel=1e-15)
    assert O.ggx_G1(1.0, 0.7) == pytest.approx(1.0, rel=1e-15)


@pytest.mark.parametrize("rho,theta_o", [(0.3, 0.2), (0.6, 0.9), (1.0, 1.3), (0.45, 0.0)])
def test_masking_normalisation(rho, theta_o):
    """Projected-area identity of a microsurface (Heitz 2014, eq. 1-2):
    int G1(o) <o.m>+ D(m) dm = cos(theta_o).  Pins D and G1 together."""
    so, co = math.sin(theta_o), math.cos(theta_o)

    def integrand(phi, tm):
        om = so * math.sin(tm) * math.cos(phi) + co * math.cos(tm)
        return max(om, 0.0) * O.ggx_D(math.cos(tm), rho) * math.sin(tm)

    val, _ = integrate.dblquad(integrand, 0.0, math.pi / 2, 0.0, 2 * math.pi, epsabs=1e-9, epsrel=1e-9)
    assert O.ggx_G1(co, rho) * val == pytest.approx(co, rel=2e-5, abs=1e-7)


def test_schlick_fresnel_tracks_exact_dielectric_fresnel():
    """Schlick with F0 = 0.04 approximates the exact unpolarised Fresnel reflectance of an
    IOR-1.5 dielectric (textbook Fresnel equations) to within 0.04 up to 85 degrees; the garbled
    (1 - (w.h)^5) reading would be off by ~0.9 at 60 degrees."""
    eta = 1.5
    for deg in np.linspace(0.0, 85.0, 35):
        ci = math.cos(math.radians(deg))
        st = math.sin(math.radians(deg)) / eta
        ct = math.sqrt(1 - st * st)
        rs = ((ci - eta * ct) / (ci + eta * ct)) ** 2
        rp = ((ct - eta * ci) / (ct + eta * ci)) ** 2
        exact = 0.5 * (rs + rp)
        assert abs(O.fresnel(0.04, ci) - exact) < 0.04, deg
    assert O.fresnel(0.3, 1.0) == pytest.approx(0.3, abs=1e-15)
    assert O.fresnel(0.3, 0.0) == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("rho", [0.1, 0.5, 0.9])
def test_ggx_sampling_follows_D_cos(rho):
    """Half vectors drawn by the oracle's sampler have density D(h)(n.h) around an arbitrary n:
    Kolmogorov-Smirnov on cos(theta_h) against the CDF of 2 pi D(c) c, uniform azimuth, unit h."""
    rng = np.random.default_rng(1)
    n = rng.normal(size=3)
    n /= np.linalg.norm(n)
    t = np.cross(n, [0.3, 0.5, 0.8])
    t /= np.linalg.norm(t)
    b = np.cross(n, t)
    cs, phis = [], []
    for _ in range(4000):
        h = O.ggx_sample_h(n, rho, rng.uniform(), rng.uniform())
        assert abs(np.linalg.norm(h) - 1.0) < 1e-12
        cs.append(h @ n)
        phis.append(math.atan2(h @ b, h @ t))
    cdf_cache = {}

    def cdf(c):
        key = round(float(c), 6)
        if key not in cdf_cache:
            cdf_cache[key] = integrate.quad(lambda x: 2 * math.pi * O.ggx_D(x, rho) * x, 0.0, key, limit=200)[0]
        return cdf_cache[key]

    res = stats.kstest(np.array(cs), np.vectorize(cdf))
    assert res.pvalue > 1e-3
    assert stats.kstest((np.array(phis) + math.pi) / (2 * math.pi), "uniform").pvalue > 1e-3


# --------------------------------------------------------------------------------------------
# Environment map (Sec. 3.2 SampleEnvMap): mip chain and lat-long lookup
# --------------------------------------------------------------------------------------------
def test_env_mips_are_box_means_of_the_base():
    rng = np.random.default_rng(2)
    He, We = 16, 64
    env = rng.uniform(0, 5, size=(He, We, 3))
    mips = O.build_env_mips(env)
    L = O.env_levels(He, We)
    assert L == 5
    off = 0
    for l in range(L):
        h, w = He >> l, We >> l
        lev = mips[off:off + h * w * 3].reshape(h, w, 3)
        s = 1 << l
        brute = env.reshape(h, s, w, s, 3).mean(axis=(1, 3))
        np.testing.assert_allclose(lev, brute, rtol=1e-13, atol=0)
        off += h * w * 3
    assert off == mips.size
    const = O.build_env_mips(np.full((He, We, 3), 0.625))
    assert np.all(const == 0.625)


def _texel_dir(u, v):
    phi = 2 * math.pi * (u - 0.5)
    return np.array([math.sin(phi) * math.sin(math.pi * v), math.cos(math.pi * v),
                     -math.cos(phi) * math.sin(math.pi * v)])


def test_env_lookup_hits_texel_centres_and_blends_levels():
    rng = np.random.default_rng(3)
    He, We = 8, 16
    env = rng.uniform(0, 1, size=(He, We, 3))
    mips = O.build_env_mips(env)
    for r in range(He):
        for c in range(We):
            d = _texel_dir((c + 0.5) / We, (r + 0.5) / He) * rng.uniform(0.5, 2.0)  # any length
            np.testing.assert_allclose(O.env_lookup(mips, He, We, d, 0.0), env[r, c], rtol=1e-9, atol=1e-12)
    # level 1 texel centres
    lev1 = env.reshape(He // 2, 2, We // 2, 2, 3).mean(axis=(1, 3))
    for r in range(He // 2):
        for c in range(We // 2):
            d = _texel_dir((c + 0.5) / (We // 2), (r + 0.5) / (He // 2))
            np.testing.assert_allclose(O.env_lookup(mips, He, We, d, 1.0), lev1[r, c], rtol=1e-9)
    # linear in lambda between integer levels
    d = rng.normal(size=3)
    a0 = O.env_lookup(mips, He, We, d, 1.0)
    a1 = O.env_lookup(mips, He, We, d, 2.0)
    np.testing.assert_allclose(O.env_lookup(mips, He, We, d, 1.3), 0.7 * a0 + 0.3 * a1, rtol=1e-12)
    # clamped beyond the last level
    np.testing.assert_allclose(O.env_lookup(mips, He, We, d, 99.0), O.env_lookup(mips, He, We, d, 3.0))


def test_env_lookup_is_continuous_across_the_seam_and_pole():
    rng = np.random.default_rng(4)
    He, We = 8, 16
    mips = O.build_env_mips(rng.uniform(0, 1, size=(He, We, 3)))
    eps = 1e-9
    a = O.env_lookup(mips, He, We, _texel_dir(eps, 0.4), 0.0)
    b = O.env_lookup(mips, He, We, _texel_dir(1 - eps, 0.4), 0.0)
    np.testing.assert_allclose(a, b, atol=1e-6)
    # at the zenith every azimuth returns the same value (top row is clamped)
    vals = [O.env_lookup(mips, He, We, _texel_dir(u, 1e-12), 0.0) for u in np.linspace(0.01, 0.99, 7)]
    top = mips[:We * 3].reshape(We, 3)
    for v in vals:
        assert np.all(v <= top.max(axis=0) + 1e-12) and np.all(v >= top.min(axis=0) - 1e-12)


# --------------------------------------------------------------------------------------------
# BRDF-integral table (Appendix C)
# --------------------------------------------------------------------------------------------
def _exact_split(rho, mu):
    """A, B of Appendix C by 2-D quadrature over the incident hemisphere (no sampling):
    A = int D G / (4 mu) (1 - (1 - v.h)^5) dw_i, B = int D G / (4 mu) (1 - v.h)^5 dw_i."""
    v = np.array([math.sqrt(1 - mu * mu), 0.0, mu])

    def parts(phi, th, which):
        l = np.array([math.sin(th) * math.cos(phi), math.sin(th) * math.sin(phi), math.cos(th)])
        h = l + v
        h /= np.linalg.norm(h)
        vh = float(v @ h)
        f = O.ggx_D(h[2], rho) * O.ggx_G1(l[2], rho) * O.ggx_G1(mu, rho) / (4 * mu)
        fc = (1 - vh) ** 5
        return f * ((1 - fc) if which == 0 else fc) * math.sin(th)

    A = 2 * integrate.dblquad(lambda p, t: parts(p, t, 0), 0, math.pi / 2, 0, math.pi, epsabs=1e-7)[0]
    B = 2 * integrate.dblquad(lambda p, t: parts(p, t, 1), 0, math.pi / 2, 0, math.pi, epsabs=1e-7)[0]
    return A, B


@pytest.mark.parametrize("i,j", [(40, 10), (40, 50), (63, 1), (25, 30), (63, 63), (16, 5), (8, 3), (2, 8)])
def test_lut_matches_quadrature_of_the_brdf_integral(lut, i, j):
    """Table entries against a sampling-free quadrature.  The Hammersley estimate converges
    slowly where the lobe is narrow and grazing (the n.l > 0 cut), so corners get a wider band."""
    N = lut.shape[0]
    rho, mu = (i + 0.5) / N, (j + 0.5) / N
    A, B = _exact_split(rho, mu)
    tol = 2e-3 if (rho > 0.2 and mu > 0.1) else 1.2e-2
    assert lut[i, j, 0] == pytest.approx(A, abs=tol)
    assert lut[i, j, 1] == pytest.approx(B, abs=tol)


def test_lut_small_roughness_limit_and_energy(lut):
    """rho -> 0: the lobe is a delta at h = n, G1 -> 1, so A = 1 - (1 - mu)^5, B = (1 - mu)^5
    (checked on the first row, rho = 0.5/N, away from grazing mu where G1(mu) < 1 still shows).
    Everywhere A + B (directional albedo with F = 1) stays <= 1."""
    N = lut.shape[0]
    mus = (np.arange(N) + 0.5) / N
    np.testing.assert_allclose(lut[0, 16:, 0], 1 - (1 - mus[16:]) ** 5, atol=1e-3)
    np.testing.assert_allclose(lut[0, 16:, 1], (1 - mus[16:]) ** 5, atol=1e-3)
    assert np.all(lut[..., 0] + lut[..., 1] <= 1.0 + 1e-3)
    assert np.all(lut >= 0)


def test_lut_bilinear_sampling_is_exact_at_texel_centres(lut):
    N = lut.shape[0]
    for i, j in [(0, 0), (5, 17), (N - 1, N - 1), (30, 2)]:
        np.testing.assert_allclose(O.lut_sample(lut, (i + 0.5) / N, (j + 0.5) / N), lut[i, j], rtol=1e-12)
    # clamped outside the texel-centre range
    np.testing.assert_allclose(O.lut_sample(lut, 0.0, 0.0), lut[0, 0], rtol=1e-12)
    np.testing.assert_allclose(O.lut_sample(lut, 1.0, 1.0), lut[N - 1, N - 1], rtol=1e-12)


# --------------------------------------------------------------------------------------------
# Hierarchical-Z pyramid
# --------------------------------------------------------------------------------------------
def test_hiz_is_brute_force_min_over_each_footprint():
    rng = np.random.default_rng(5)
    V, H, W, L = 2, 37, 53, 6
    depth = rng.uniform(1, 10, size=(V, H, W))
    depth[0, 3:9, 4:20] = np.inf
    hiz = O.build_hiz(depth, L)
    for v in range(V):
        levels = O.hiz_levels_split(hiz[v], H, W, L)
        for l, lev in enumerate(levels, start=1):
            s = 1 << l
            for i in range(lev.shape[0]):
                for j in range(lev.shape[1]):
                    assert lev[i, j] == depth[v, i * s:(i + 1) * s, j * s:(j + 1) * s].min()
