"""Helpers shared by the GPU parity tests: run a workload through libssgi.so (via the binding)
and through the FP64 oracle on the same seeded inputs, and compare.

Tolerances (written here, used by every parity test):
  * hit indices: bit-exact on >= 99.9 % of samples; every mismatching sample must be a
    near-tie in the oracle (decision margin < MARGIN_TOL), i.e. a rounding-order case.  The
    largest margin a rounding case can have is a positional one (the distance in pixels of an
    exit point to a pixel boundary) at the far end of a long ray: the FP32 direction error
    (DIR_EPS) displaces a point l pixels down the ray by about l x DIR_EPS x z0 / z pixels, so
    with l up to the screen diagonal (1836 px at 1600x900) and z0 / z up to 2 it reaches
    ~3.7e-3 px (measured: 2.06e-3 at the end of a 440-pixel ray, the largest of 5482 mismatches
    among the 263 M samples of the 8-view 1245x825 workload);
  * per-pixel RGB: |gpu - oracle|_inf <= RGB_RTOL * max(|oracle|_inf, RGB_FLOOR) on pixels
    whose samples all match;
  * a pixel above that bound must be explained by its own conditioning (checked when the test
    passes the workload; a hit sample carries the two sides' difference of the c1 it gathers,
    itself checked by the direct-shading tests): the FP32 direction of a missed sample differs from the oracle's by a few
    roundings (DIR_EPS per component), and where the latitude-longitude lookup is steep in the
    direction (near the map's poles, where the longitude atan2(x, -z) is ill-conditioned, or
    across a bright texel) that changes the sample's radiance by far more than a rounding; such a
    pixel may exceed RGB_RTOL_MAX by at most the sum over its missed samples of |weight| x the
    largest change of the lookup under a DIR_EPS move of the direction, and such pixels are at
    most OUTLIER_SHARE_MAX of the compared ones;
  * gradients: <= GRAD_RTOL relative (per element against the vector's scale, and as a norm).
"""
import math

import numpy as np

import oracle as O

HIT_MATCH_MIN = 0.999
MARGIN_TOL = 5e-3
RGB_RTOL = 1e-4
RGB_FRAC_MIN = 0.99999  # share of pixels within RGB_RTOL (all pixels below 1e5 pixels)
RGB_RTOL_MAX = 3e-4     # bound for the rest: FP32 direction error (~1e-7 rad) x env texel contrast
RGB_FLOOR = 1e-3
GRAD_RTOL = 1e-3
DIR_EPS = 1e-6          # FP32 error of a sampled direction's components: ~8 ulp of 1 (normalisation,
                        # the GGX sample's square roots and sine/cosine, the reflection)
OUTLIER_SHARE_MAX = 1e-3
ANGLE_EPS = 4.0 / 2 ** 24  # FP32 rounding of a lookup's longitude and latitude, in turns


def assert_rgb(err, label):
    """err: per-pixel relative errors.  <= RGB_RTOL on all but a 1e-5 share, <= RGB_RTOL_MAX on all."""
    if err.size == 0:
        return
    frac = (err <= RGB_RTOL).mean()
    assert frac >= RGB_FRAC_MIN or err.size < 1e5 and frac == 1.0, \
        f"{label}: {1 - frac:.2e} of pixels above {RGB_RTOL} (max {err.max():.3e})"
    assert err.max() <= RGB_RTOL_MAX, f"{label}: max rel err {err.max():.3e}"


def gpu_forward(wl, flags=None, brute=False, lut=None, want_cs=True):
    import torch
    import paper_2504_01358_gb300 as S
    p = S.params_of(wl.params)
    if flags is not None:
        p.flags = flags
    if brute:
        p.flags |= S._native.BRUTE_FORCE
    g, env, cams, _ = S.to_device_workload(wl)
    lut_t = S.ssgi_build_brdf_lut() if lut is None else lut
    em = S.ssgi_build_env_mips(env)
    hiz = S.ssgi_build_hiz(g.depth, p.hiz_levels) if p.hiz_levels > 1 else None
    c_d, c_s, c1 = S.ssgi_shade_direct(g, cams, em, lut_t, want_cs=want_cs)
    tr = S.ssgi_trace_indirect(g, cams, hiz, c1, c_d, em, p, want_hits=True, want_parts=True)
    torch.cuda.synchronize()
    out = {{"c_s_mc": "cs_mc"}.get(k, k): v.cpu().numpy() for k, v in tr.items() if v is not None}
    out.update({"cd": c_d.cpu().numpy(), "c1": c1.cpu().numpy(), "mips": em.mips.cpu().numpy(),
                "lut": lut_t.cpu().numpy()})
    if c_s is not None:
        out["cs"] = c_s.cpu().numpy()
    if hiz is not None:
        out["hiz"] = hiz.cpu().numpy()
    out["_dev"] = (g, env, cams, em, lut_t, c1, tr["hit_idx"], p)
    return out


def orc_forward(wl, flags=None, brute=False, lut=None):
    return O.forward(wl, lut=O.build_lut() if lut is None else lut, flags=flags, brute=brute)


def pixel_rel_err(a, b, floor=RGB_FLOOR):
    """per-pixel |a - b|_inf / max(|b|_inf, floor) over the last axis"""
    num = np.abs(a.astype(np.float64) - b).max(axis=-1)
    den = np.maximum(np.abs(b).max(axis=-1), floor)
    return num / den


def compare_hits(h_gpu, r_orc):
    h_orc = r_orc["hit_idx"]
    same = h_gpu == h_orc
    frac = same.mean()
    bad = ~same
    margins = r_orc["margin"][bad]
    return frac, bad, margins


def direction_bound(wl, view, y, x, hits, flags, eps=DIR_EPS, c1_diff=None):
    """Per-channel bound on |gpu - oracle| of pixel (x, y)'s Monte-Carlo sums from the
    conditioning of its missed samples' environment lookups (a background pixel: of its own
    lookup in the view direction) (Sec. 3.3 estimator; the lookup is
    the oracle's): each valid missed sample adds |weight| x the largest change of its lookup when
    one component of the direction moves by +-eps.  A hit gathers c1 at an index both sides agree
    on, and adds |weight| x the two sides' difference of that c1 (`c1_diff`, [V,H,W,3], when
    given).  The samples are redrawn with the oracle's own generator and GGX sampler."""
    V, H, W = wl.depth.shape
    He, We = wl.env.shape[:2]
    mips = _mips_of(wl)
    cam = wl.cams[view].astype(np.float64)
    R = cam[:12].reshape(3, 4)[:, :3]
    f = (H / 2.0) / math.tan(cam[12] / 2.0)
    d = R @ np.array([(x + 0.5 - W / 2.0) / f, -(y + 0.5 - H / 2.0) / f, -1.0])
    v = -d / np.linalg.norm(d)
    n = wl.normal[view, y, x].astype(np.float64)
    rho, m = float(wl.rough[view, y, x]), float(wl.metal[view, y, x])
    a = wl.albedo[view, y, x].astype(np.float64)
    nv = float(n @ v)
    F0 = 0.04 * (1.0 - m) + a * m
    seed, spp = wl.params.seed, wl.params.spp
    z = float(wl.depth[view, y, x])
    if not (np.isfinite(z) and z > 0):  # background: the map at mip 0 in the view direction
        return _lookup_dev(mips, He, We, -v, eps)
    key = np.array([seed & 0xffffffff, (seed >> 32) ^ view], np.uint32)
    out = np.zeros(3)
    for s in range(spp):
        if hits[s] < -1 or (hits[s] >= 0 and c1_diff is None):
            continue  # an invalid sample, background, or a hit without c1 to compare
        o = O.philox4x32_10(np.array([y * W + x, s, 0, 0], np.uint32), key)
        xi0, xi1 = float(int(o[0]) >> 8) / 16777216.0, float(int(o[1]) >> 8) / 16777216.0
        h = O.ggx_sample_h(n, rho, xi0, xi1)
        vh, nh = float(v @ h), float(n @ h)
        w = 2.0 * vh * h - v
        nw = float(n @ w)
        if not (nv > 0 and nw > 0 and vh > 0 and nh > 0):
            continue
        dev = c1_diff[view].reshape(-1, 3)[hits[s]] if hits[s] >= 0 else _lookup_dev(mips, He, We, w, eps)
        K = O.ggx_G1(nw, rho) * O.ggx_G1(nv, rho) * vh / (nv * nh)
        out += (F0 + (1.0 - F0) * (1.0 - vh) ** 5) * K * dev / spp
        if flags & O.FLAG_DIFFUSE_INDIRECT:
            pdf = O.ggx_D(nh, rho) * nh / (4.0 * vh)
            if pdf > 0 and np.isfinite(pdf):
                out += (1.0 - m) * a / math.pi * nw / pdf * dev / spp
    return out


def _lookup_dev(mips, He, We, d, eps):
    """Largest change of the mip-0 lookup (per channel) when one component of d moves by +-eps."""
    L = O.env_lookup(mips, He, We, d, 0.0)
    dev = np.zeros(3)
    for k in range(3):
        for sg in (1.0, -1.0):
            d2 = np.array(d, np.float64)
            d2[k] += sg * eps
            dev = np.maximum(dev, np.abs(O.env_lookup(mips, He, We, d2 / np.linalg.norm(d2), 0.0) - L))
    return dev


_MIPS = {}


def _mips_of(wl):
    k = id(wl.env)
    if k not in _MIPS:
        _MIPS.clear()
        _MIPS[k] = O.build_env_mips(wl.env)
    return _MIPS[k]


def assert_forward_parity(gpu, orc, label="", wl=None, pix=None, flags=0):
    """Hits and images of a forward pass against the oracle (module docstring).  With the
    workload `wl` (and `pix`, the linear pixel indices of a sampled comparison), a pixel over the
    RGB bounds passes if its conditioning explains it (direction_bound)."""
    frac, bad, margins = compare_hits(gpu["hit_idx"], orc)
    assert frac >= HIT_MATCH_MIN, f"{label}: hit-index match {frac:.6f}"
    assert np.all(margins < MARGIN_TOL), f"{label}: mismatch with decision margin {margins.max()}"
    pix_ok = ~bad.any(axis=-1)
    scale = np.maximum(np.abs(orc["final"]).max(axis=-1), RGB_FLOOR)
    bounds = {}
    c1_diff = np.abs(gpu["c1"].astype(np.float64) - orc["c1"]) if ("c1" in gpu and "c1" in orc) else None
    for key in [k for k in ("final", "cs_mc", "c_id") if k in gpu]:
        okey = {"c_id": "cid"}.get(key, key)
        # error of each channel in units of the pixel's output RGB
        err_all = np.abs(gpu[key].astype(np.float64) - orc[okey]).max(axis=-1) / scale
        err = err_all[pix_ok]
        if wl is None:
            assert_rgb(err, f"{label}: {key}")
            continue
        out = np.argwhere(pix_ok & (err_all > RGB_RTOL))
        assert len(out) <= OUTLIER_SHARE_MAX * max(int(pix_ok.sum()), 1), \
            f"{label}: {key}: {len(out)} of {int(pix_ok.sum())} pixels above {RGB_RTOL}"
        V, H, W = wl.depth.shape
        for idx in out:
            t = tuple(int(i) for i in idx)
            lin = int(pix[t[0]]) if pix is not None else (t[0] * H + t[1]) * W + t[2]
            if lin not in bounds:
                vv, rem = divmod(lin, H * W)
                bounds[lin] = direction_bound(wl, vv, rem // W, rem % W, gpu["hit_idx"][t], flags,
                                              c1_diff=c1_diff).max()
            allowed = RGB_RTOL_MAX + bounds[lin] / scale[t]
            assert err_all[t] <= allowed, \
                f"{label}: {key}: pixel {lin} rel err {err_all[t]:.3e} > {allowed:.3e} (conditioning bound)"
    return frac, int(bad.sum())


def forward_outliers(gpu, orc):
    """Pixels whose samples all hit alike but whose RGB differs by more than RGB_RTOL: the ones
    assert_forward_parity admits only through their conditioning (direction_bound).  Their own
    material gradients are linear in the same radiance, so they inherit its conditioning."""
    same = ~(gpu["hit_idx"] != orc["hit_idx"]).any(axis=-1)
    scale = np.maximum(np.abs(orc["final"]).max(axis=-1), RGB_FLOOR)
    out = np.zeros(same.shape, bool)
    for key in [k for k in ("final", "cs_mc", "c_id") if k in gpu]:
        okey = {"c_id": "cid"}.get(key, key)
        out |= np.abs(gpu[key].astype(np.float64) - orc[okey]).max(axis=-1) / scale > RGB_RTOL
    return out & same


def direct_kinks(wl, eps=DIR_EPS):
    """Foreground pixels whose direct-shading lookups (Sec. 3.2) lie within the FP32 rounding of
    a kink of their bilinear filters, where the adjoint is one-sided and the two sides may take
    different branches: the latitude-longitude lookups at r = 2 (v.n) n - v and at n, on levels
    floor(lambda) and floor(lambda) + 1, within eps x (texels per unit of direction) of a
    texel-centre line; lambda = log2(rho + 1) lambda_max within eps lambda_max of an integer;
    n.v within eps N of a texel centre of the N x N BRDF table."""
    V, H, W = wl.depth.shape
    He, We = wl.env.shape[:2]
    lmax = O.env_levels(He, We) - 1
    xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
    kink = np.zeros((V, H, W), bool)
    for view in range(V):
        cam = wl.cams[view].astype(np.float64)
        R = cam[:12].reshape(3, 4)[:, :3]
        f = (H / 2.0) / math.tan(cam[12] / 2.0)
        d = np.stack([(xs - W / 2.0) / f, -(ys - H / 2.0) / f, -np.ones_like(xs)], -1) @ R.T
        v = -d / np.linalg.norm(d, axis=-1, keepdims=True)
        n = wl.normal[view].astype(np.float64)
        nv = np.sum(n * v, -1)
        lam = np.log2(wl.rough[view].astype(np.float64) + 1.0) * lmax
        l0 = np.clip(np.floor(lam), 0, lmax).astype(np.int64)
        levels = (l0, np.minimum(l0 + 1, lmax))
        k = np.abs(lam - np.round(lam)) < eps * lmax
        # r is computed (an error of eps per component, i.e. eps / q in longitude and eps in
        # latitude); n is an input, exact on both sides, and only its angles are rounded
        # (ANGLE_EPS of a turn; at the exact pole both sides take the same longitude)
        for dv, de, da in ((2.0 * nv[..., None] * n - v, eps, 0.0), (n, 0.0, ANGLE_EPS)):
            q = np.hypot(dv[..., 0], dv[..., 2])
            u = 0.5 + np.arctan2(dv[..., 0], -dv[..., 2]) / (2.0 * math.pi)
            vt = np.arctan2(q, dv[..., 1]) / math.pi
            du = np.where(q > 0, de / (2.0 * math.pi * np.maximum(q, 1e-30)) + da, 0.0)
            dvt = de / math.pi + da
            for lv in levels:
                wl_, hl = (We >> lv).astype(np.float64), (He >> lv).astype(np.float64)
                tx, ty = u * wl_ - 0.5, vt * hl - 0.5
                k |= np.abs(tx - np.round(tx)) < du * wl_
                k |= np.abs(ty - np.round(ty)) < dvt * hl
        tm = np.clip(nv, 0.0, 1.0) * O.LUT_N - 0.5
        k |= np.abs(tm - np.round(tm)) < eps * O.LUT_N
        kink[view] = k
    return kink & np.isfinite(wl.depth) & (wl.depth > 0)


def affected_pixels(h_gpu, h_orc):
    """Pixels whose gradients may legitimately differ because some sample's hit differs:
    the receivers of mismatching samples and the pixels either side says they hit."""
    V = h_gpu.shape[0]
    bad = h_gpu != h_orc
    aff = bad.any(axis=-1)
    for hh in (h_gpu, h_orc):
        vv, yy, xx, ss = np.nonzero(bad & (hh >= 0))
        q = hh[vv, yy, xx, ss]
        W = h_gpu.shape[2]
        aff[vv, q // W, q % W] = True
    del V
    return aff
