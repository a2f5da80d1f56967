"""Helpers shared by the GPU parity tests: run a workload through libssgi.so (via the binding)
and through the FP64 oracle on the same seeded inputs, and compare.

Tolerances (written here, used by every parity test):
  * hit indices: bit-exact on >= 99.9 % of samples; every mismatching sample must be a
    near-tie in the oracle (decision margin < MARGIN_TOL), i.e. a rounding-order case.  The
    largest margin a rounding case can have is a positional one (the distance in pixels of an
    exit point to a pixel boundary) at the far end of a long ray: an FP32 direction error of
    ~1e-6 displaces a point l pixels down the ray by about l x 1e-6 x z0 / z pixels, so with l up
    to the screen diagonal (1836 px at 1600x900) and z0 / z up to 2 it reaches ~3.7e-3 px
    (measured: 2.06e-3 at the end of a 440-pixel ray, the largest of 5482 mismatches among the
    263 M samples of the 8-view 1245x825 workload);
  * per-pixel RGB, on pixels whose samples all hit alike: |gpu - oracle|_inf <= RGB_RTOL (1e-4)
    x max(|oracle|_inf, RGB_FLOOR).  A pixel over that bound passes only if replaying its sums
    in the oracle's FP64 arithmetic at the lookup coordinates the GPU itself used (Replay: the
    kernels' FP32 directions and texel coordinates, reproduced bit for bit by fp32_emu) agrees
    with the GPU to EMU_RTOL (1e-5): then the difference is the FP32 rounding of a direction
    or texel coordinate, amplified by a steep lookup, and nothing else.  The share within
    RGB_RTOL, the largest error and the number of replayed pixels are reported (ParityReport);
  * gradients: <= GRAD_RTOL relative per element against the vector's scale, and as a norm for
    the environment; per-element relative errors on elements above fractions of the scale are
    reported.
"""
import math

import numpy as np

import fp32_emu as E
import oracle as O

HIT_MATCH_MIN = 0.999
MARGIN_TOL = 5e-3
RGB_RTOL = 1e-4
EMU_RTOL = 1e-5
RGB_FLOOR = 1e-3
GRAD_RTOL = 1e-3
F32 = np.float32

# every forward comparison of a test run, for the report printed at the end of the session
REPORTS = []


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


# ---------------------------------------------------------------------------------------------
# replay of pixels in FP64 at the GPU's own lookup coordinates
# ---------------------------------------------------------------------------------------------
def _g1(z, rho):
    a2 = rho * rho
    return 2.0 * z / (z + np.sqrt(a2 + (1.0 - a2) * z * z))


class Replay:
    """The oracle's arithmetic (FP64; its mip chain, BRDF table and Philox generator) for chosen
    pixels, with every environment lookup taken at the texel coordinates the kernels compute in
    FP32 (fp32_emu) instead of the exact ones, and every sample's weight taken from the FP32
    dot products v.h, n.h, n.w and sampler denominator (bit for bit the kernels'; the trace's
    n.v, which shapes no direction, to within an ulp).  It follows the kernels' order
    of evaluation: direct shading (Sec. 3.2: c_d, c_s, c1), then per sample the GGX direction,
    the hit's c1 or the map at mip 0, the Monte-Carlo sums and the composite (Sec. 3.3)."""

    def __init__(self, wl, lut=None):
        self.wl = wl
        self.V, self.H, self.W = wl.depth.shape
        self.He, self.We = wl.env.shape[:2]
        self.levels = O.env_levels(self.He, self.We)
        flat = O.build_env_mips(wl.env)
        self.mips, off = [], 0
        for l in range(self.levels):
            h, w = self.He >> l, self.We >> l
            self.mips.append(flat[off: off + h * w * 3].reshape(h, w, 3))
            off += h * w * 3
        self.lut = O.build_lut() if lut is None else lut
        self.cams = [E.Cam(wl.cams[v], self.H, self.W) for v in range(self.V)]
        self._c1 = {}

    # -- geometry of pixels (linear indices over [V,H,W]) ---------------------------------------
    def _pixel_geometry(self, pix):
        HW = self.H * self.W
        view, rem = np.divmod(pix, HW)
        y, x = np.divmod(rem, self.W)
        d = np.zeros((len(pix), 3), F32)
        for vv in np.unique(view):
            sel = view == vv
            d[sel] = E.pix_dir_world(self.cams[vv], x[sel], y[sel])
        return view, rem, d

    def _bilinear(self, l, x0, y0, tx, ty):
        T = self.mips[l]
        h, w = T.shape[:2]
        c0 = np.mod(x0, w)
        c1 = np.mod(c0 + 1, w)
        r0, r1 = np.clip(y0, 0, h - 1), np.clip(y0 + 1, 0, h - 1)
        tx = tx.astype(np.float64)[:, None]
        ty = ty.astype(np.float64)[:, None]
        return ((1 - tx) * (1 - ty) * T[r0, c0] + tx * (1 - ty) * T[r0, c1] + (1 - tx) * ty * T[r1, c0]
                + tx * ty * T[r1, c1])

    def lookup0(self, d):
        """Mip-0 lookups in directions d [N,3] (FP32)."""
        if len(d) == 0:
            return np.zeros((0, 3))
        x0, y0, tx, ty = E.texel_coords(d, self.He, self.We)
        return self._bilinear(0, x0, y0, tx, ty)

    def lookup(self, d, lam):
        """SampleEnvMap(d, lambda) at FP32 lambda [N]: floor level and the next, blended."""
        lmax = F32(self.levels - 1)
        lam = np.minimum(np.maximum(lam, F32(0.0)), lmax).astype(F32)
        l0 = np.floor(lam).astype(np.int64)
        l1 = np.minimum(l0 + 1, self.levels - 1)
        t = (lam - l0.astype(F32)).astype(F32).astype(np.float64)
        ang = E.dir_angles(d)
        out = np.zeros((len(d), 3))
        for lvl in np.unique(np.concatenate([l0, l1])):
            wt = np.where(l0 == lvl, 1.0 - t, 0.0) + np.where((l1 == lvl) & (t > 0), t, 0.0)
            sel = wt > 0
            if not np.any(sel):
                continue
            h, w = self.He >> lvl, self.We >> lvl
            x0, y0, tx, ty = E.texel_coords(d[sel], h, w, angles=tuple(a[sel] for a in ang))
            out[sel] += wt[sel][:, None] * self._bilinear(lvl, x0, y0, tx, ty)
        return out

    def lam_of(self, rho):
        """lambda = log2(rho + 1) lambda_max as the kernels round it."""
        lp = np.log2(E.add(rho, F32(1.0)).astype(np.float64)).astype(F32)
        return E.mul(lp, F32(self.levels - 1))

    # -- direct shading -------------------------------------------------------------------------
    def direct(self, pix):
        """(c_d, c_s, c1) [N,3] of pixels `pix`."""
        wl = self.wl
        pix = np.asarray(pix, np.int64)
        n_ = len(pix)
        cd, cs, c1 = np.zeros((n_, 3)), np.zeros((n_, 3)), np.zeros((n_, 3))
        if n_ == 0:
            return cd, cs, c1
        view, rem, d = self._pixel_geometry(pix)
        z = wl.depth.reshape(-1)[pix]
        bg = ~(np.isfinite(z) & (z > 0))
        c1[bg] = self.lookup0(d[bg])
        fg = ~bg
        if np.any(fg):
            df = d[fg]
            pf = pix[fg]
            v = E.view_vector(df)
            n = wl.normal.reshape(-1, 3)[pf].astype(F32)
            nv = E.dot3(n, v)
            mu = np.minimum(np.maximum(nv, F32(1e-4)), F32(1.0)).astype(F32)
            r = E.reflect_about(n, nv, v)
            rho = wl.rough.reshape(-1)[pf].astype(F32)
            m = wl.metal.reshape(-1)[pf].astype(np.float64)[:, None]
            a = wl.albedo.reshape(-1, 3)[pf].astype(np.float64)
            lam = self.lam_of(rho)
            Er = self.lookup(r, lam)
            En = self.lookup(n, lam)
            AB = np.array([O.lut_sample(self.lut, float(rr), float(mm)) for rr, mm in zip(rho, mu)])
            F0 = 0.04 * (1.0 - m) + a * m
            cs[fg] = Er * (F0 * AB[:, :1] + AB[:, 1:])
            cd[fg] = (1.0 - m) * a * En
            c1[fg] = cd[fg] + cs[fg]
        return cd, cs, c1

    def c1_of(self, pix):
        pix = np.asarray(pix, np.int64)
        need = [int(p) for p in np.unique(pix) if int(p) not in self._c1]
        if need:
            _, _, c1 = self.direct(np.array(need, np.int64))
            for p, c in zip(need, c1):
                self._c1[p] = c
        return np.array([self._c1[int(p)] for p in pix]).reshape(-1, 3)

    # -- the Monte-Carlo sums -------------------------------------------------------------------
    def trace(self, pix, hits, flags):
        """(cs_mc, c_id, final) [N,3] of pixels `pix` whose samples hit `hits` [N, spp] (the
        indices both sides agree on)."""
        wl = self.wl
        pix = np.asarray(pix, np.int64)
        N = len(pix)
        hits = np.asarray(hits).reshape(N, -1)
        spp = hits.shape[1]
        cd, _, final = self.direct(pix)
        cs_mc, cid = np.zeros((N, 3)), np.zeros((N, 3))
        view, rem, d = self._pixel_geometry(pix)
        z = wl.depth.reshape(-1)[pix]
        fg = np.nonzero(np.isfinite(z) & (z > 0))[0]
        if len(fg) == 0:
            return cs_mc, cid, final
        # every sample of every foreground pixel, pixel-major
        P = pix[fg]
        v = E.view_vector(d[fg])
        n = wl.normal.reshape(-1, 3)[P].astype(F32)
        nv = E.dot3(n, v)
        rho = wl.rough.reshape(-1)[P].astype(F32)
        seed = wl.params.seed
        xi = np.zeros((len(fg), spp, 2), np.uint32)
        for j, i in enumerate(fg):
            key = np.array([seed & 0xFFFFFFFF, ((seed >> 32) ^ int(view[i])) & 0xFFFFFFFF], np.uint32)
            for s in range(spp):
                xi[j, s] = O.philox4x32_10(np.array([rem[i], s, 0, 0], np.uint32), key)[:2]
        u = ((xi >> 8).astype(np.float64) * 2.0 ** -24).astype(F32).reshape(-1, 2)
        rep = lambda a: np.repeat(a, spp, axis=0)  # noqa: E731
        sm = E.make_sample(rep(n), rep(v), rep(nv), rep(rho), u[:, 0], u[:, 1])
        hs = hits[fg].reshape(-1)
        # the trace forms n.v in the compiler's own order (it shapes no direction), so the model's
        # n.v may differ from it by an ulp: the GPU's verdict on validity (its hit codes) decides,
        # and the model must agree with it wherever n.v and n.w are not within rounding of 0
        valid = hs != O.INVALID
        clear = (np.abs(sm["nw"]) > 1e-5) & (np.abs(rep(nv)) > 1e-5)
        bad = np.nonzero((sm["valid"] != valid) & clear)[0]
        assert len(bad) == 0, ("sample validity differs from the hits at pixel", int(P[bad[0] // spp]))
        L = np.zeros((len(hs), 3))
        hit = valid & (hs >= 0)
        miss = valid & ~hit
        HW = self.H * self.W
        if np.any(hit):
            L[hit] = self.c1_of(rep(view[fg])[hit] * HW + hs[hit])
        L[miss] = self.lookup0(sm["w"][miss])
        nv64, r64 = rep(nv).astype(np.float64), rep(rho).astype(np.float64)
        vh, nh, nw, ds = (sm[k].astype(np.float64) for k in ("vh", "nh", "nw", "ds"))
        m = rep(wl.metal.reshape(-1)[P].astype(np.float64))[:, None]
        a = rep(wl.albedo.reshape(-1, 3)[P].astype(np.float64))
        F0 = 0.04 * (1.0 - m) + a * m
        with np.errstate(divide="ignore", invalid="ignore"):
            K = _g1(nw, r64) * _g1(nv64, r64) * vh / (nv64 * nh)
            Fr = F0 + (1.0 - F0) * ((1.0 - vh) ** 5)[:, None]
            term = np.where(valid[:, None], Fr * L * K[:, None], 0.0)
            cs_mc[fg] = term.reshape(len(fg), spp, 3).sum(axis=1) / spp
            if flags & O.FLAG_DIFFUSE_INDIRECT:
                pdf = ds * ds / (math.pi * r64 * r64) * nh / (4.0 * vh)
                use = valid & (pdf > 0) & np.isfinite(pdf)
                wd = np.where(use, (1.0 - m[:, 0]) * nw / pdf / math.pi, 0.0)
                cid[fg] = (a * L * wd[:, None]).reshape(len(fg), spp, 3).sum(axis=1) / spp
        final[fg] = cd[fg] + cs_mc[fg] + (cid[fg] if flags & O.FLAG_DIFFUSE_INDIRECT else 0.0)
        return cs_mc, cid, final


_REPLAYS = {}


def replay_of(wl):
    k = id(wl)
    if k not in _REPLAYS:
        _REPLAYS.clear()
        _REPLAYS[k] = Replay(wl)
    return _REPLAYS[k]


# ---------------------------------------------------------------------------------------------
# the assertions
# ---------------------------------------------------------------------------------------------
class ParityReport:
    """The spec check of one comparison: pixels compared, share within RGB_RTOL of the
    oracle, the largest error, and the pixels over it that the replay proves rounding-only."""

    def __init__(self, label, channel, compared, within, max_err, replayed, replay_max):
        self.label, self.channel = label, channel
        self.compared, self.within, self.max_err = compared, within, max_err
        self.replayed, self.replay_max = replayed, replay_max

    def line(self):
        share = self.within / max(self.compared, 1)
        return (f"{self.label} [{self.channel}]: {self.within}/{self.compared} pixels ({share:.6f}) within "
                f"{RGB_RTOL:g} of the FP64 oracle, max rel err {self.max_err:.3e}; {self.replayed} over it, all "
                f"within {EMU_RTOL:g} of the FP64 replay at the GPU's lookup coordinates (max {self.replay_max:.2e})")


def check_pixels(gpu_img, orc_img, label, channel, pix_ok=None, replay_fn=None, scale=None):
    """Per-pixel check of one image [..., 3] against the oracle (module docstring).  replay_fn(idx)
    gives the replayed values [len(idx), 3] of pixels at flat indices idx of the image; returns
    the mask of replayed pixels."""
    g = gpu_img.reshape(-1, 3).astype(np.float64)
    o = orc_img.reshape(-1, 3)
    sc = np.maximum(np.abs(o).max(axis=-1), RGB_FLOOR) if scale is None else scale.reshape(-1)
    err = np.abs(g - o).max(axis=-1) / sc
    ok = np.ones(len(err), bool) if pix_ok is None else pix_ok.reshape(-1)
    out = np.nonzero(ok & (err > RGB_RTOL))[0]
    rmax = 0.0
    if len(out):
        assert replay_fn is not None, f"{label}: {channel}: {len(out)} pixels above {RGB_RTOL} (max {err[ok].max():.3e})"
        rep = replay_fn(out)
        rerr = np.abs(g[out] - rep).max(axis=-1) / sc[out]
        rmax = float(rerr.max())
        worst = int(np.argmax(rerr))
        assert rmax <= EMU_RTOL, (f"{label}: {channel}: pixel {int(out[worst])} rel err {err[out[worst]]:.3e} vs the "
                                  f"oracle and {rmax:.3e} vs its replay at the GPU's coordinates")
    rep = ParityReport(label, channel, int(ok.sum()), int((ok & (err <= RGB_RTOL)).sum()),
                       float(err[ok].max()) if ok.any() else 0.0, len(out), rmax)
    REPORTS.append(rep)
    print(rep.line())
    mask = np.zeros(len(err), bool)
    mask[out] = True
    return mask.reshape(gpu_img.shape[:-1])


def assert_direct_parity(gpu, orc, wl, label, keys=("cd", "cs", "c1")):
    """c_d, c_s and c1 of every pixel (Sec. 3.2) against the oracle, outliers through the replay."""
    rp = replay_of(wl)
    masks = []
    for key in keys:
        if key not in gpu:
            continue
        idx = {"cd": 0, "cs": 1, "c1": 2}[key]
        masks.append(check_pixels(gpu[key], orc[key], label, key,
                                  replay_fn=lambda out, i=idx: rp.direct(out)[i]))
    return np.any(masks, axis=0)


def assert_forward_parity(gpu, orc, label="", wl=None, pix=None, flags=0):
    """Hits and images of a forward pass against the oracle (module docstring).  With the
    workload `wl` (and `pix`, the linear pixel indices of a sampled comparison), a pixel over
    RGB_RTOL passes only if the replay at the GPU's coordinates reproduces the GPU's value.
    Returns (hit match, mismatching samples, mask of replayed pixels)."""
    frac, bad, margins = compare_hits(gpu["hit_idx"], orc)
    assert frac >= HIT_MATCH_MIN, f"{label}: hit-index match {frac:.6f}"
    assert np.all(margins < MARGIN_TOL), f"{label}: mismatch with decision margin {margins.max()}"
    pix_ok = ~bad.any(axis=-1)
    scale = np.maximum(np.abs(orc["final"]).max(axis=-1), RGB_FLOOR)
    rp = replay_of(wl) if wl is not None else None
    flat_pix = None if pix is None else np.asarray(pix, np.int64)
    hits = gpu["hit_idx"].reshape(pix_ok.size, -1)
    cache = {}

    def replay(out, part):
        keyset = tuple(out.tolist())
        if keyset not in cache:
            lin = out if flat_pix is None else flat_pix[out]
            cache[keyset] = rp.trace(lin, hits[out], flags)
        return cache[keyset][part]

    masks = []
    for key, part in (("final", 2), ("cs_mc", 0), ("c_id", 1)):
        if key not in gpu:
            continue
        okey = {"c_id": "cid"}.get(key, key)
        fn = None if rp is None else (lambda out, k=part: replay(out, k))
        masks.append(check_pixels(gpu[key], orc[okey], label, key, pix_ok=pix_ok, replay_fn=fn, scale=scale))
    return frac, int(bad.sum()), np.any(masks, axis=0)


# ---------------------------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------------------------
def direct_kinks(wl):
    """Foreground pixels where a direct-shading lookup (Sec. 3.2) of the GPU and of the oracle
    falls in different cells of its bilinear filter, so that the one-sided derivatives the two
    adjoints take differ there (the values agree: the filter is continuous): the latitude-
    longitude lookups at r = 2 (v.n) n - v and at n on levels floor(lambda) and floor(lambda)+1,
    the level pair itself, and the cell of the BRDF table in n.v.  The GPU's cells are those of
    its own FP32 coordinates (fp32_emu), the oracle's those of the exact FP64 ones."""
    V, H, W = wl.depth.shape
    He, We = wl.env.shape[:2]
    levels = O.env_levels(He, We)
    lmax = levels - 1
    kink = np.zeros((V, H, W), bool)
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    for view in range(V):
        fgm = np.isfinite(wl.depth[view]) & (wl.depth[view] > 0)
        y, x = ys[fgm], xs[fgm]
        c = E.Cam(wl.cams[view], H, W)
        d32 = E.pix_dir_world(c, x, y)
        v32 = E.view_vector(d32)
        n32 = wl.normal[view][fgm].astype(F32)
        nv32 = E.dot3(n32, v32)
        r32 = E.reflect_about(n32, nv32, v32)
        rho = wl.rough[view][fgm].astype(F32)
        lp = np.log2(E.add(rho, F32(1.0)).astype(np.float64)).astype(F32)
        lam32 = np.clip(E.mul(lp, F32(lmax)), 0, lmax)
        # FP64 side
        cam = wl.cams[view].astype(np.float64)
        R = cam[:12].reshape(3, 4)[:, :3]
        f = (H / 2.0) / math.tan(cam[12] / 2.0)
        d64 = np.stack([(x + 0.5 - W / 2.0) / f, -(y + 0.5 - H / 2.0) / f, -np.ones(len(x))], -1) @ R.T
        v64 = -d64 / np.linalg.norm(d64, axis=-1, keepdims=True)
        n64 = n32.astype(np.float64)
        nv64 = np.sum(n64 * v64, -1)
        r64 = 2.0 * nv64[:, None] * n64 - v64
        lam64 = np.clip(np.log2(rho.astype(np.float64) + 1.0) * lmax, 0, lmax)
        l0_32, l0_64 = np.floor(lam32).astype(int), np.floor(lam64).astype(int)
        k = l0_32 != l0_64
        for dir32, dir64 in ((r32, r64), (n32, n64)):
            ang = E.dir_angles(dir32)
            u = 0.5 + np.arctan2(dir64[:, 0], -dir64[:, 2]) / (2.0 * math.pi)
            vt = np.arctan2(np.hypot(dir64[:, 0], dir64[:, 2]), dir64[:, 1]) / math.pi
            for lv in np.unique(np.concatenate([l0_32, np.minimum(l0_32 + 1, lmax)])):
                sel = (l0_32 == lv) | (np.minimum(l0_32 + 1, lmax) == lv)
                h, w = He >> lv, We >> lv
                x0, y0, _, _ = E.texel_coords(dir32[sel], h, w, angles=tuple(a[sel] for a in ang))
                xe, ye = np.floor(u[sel] * w - 0.5).astype(int), np.floor(vt[sel] * h - 0.5).astype(int)
                k[sel] |= (np.mod(x0, w) != np.mod(xe, w)) | (y0 != ye)
        mu32 = np.clip(nv32, 1e-4, 1.0).astype(np.float64)
        mu64 = np.clip(nv64, 1e-4, 1.0)
        N = O.LUT_N
        k |= np.floor(mu32 * N - 0.5) != np.floor(mu64 * N - 0.5)
        kk = np.zeros((H, W), bool)
        kk[fgm] = k
        kink[view] = kk
    return kink


ELEM_FLOOR = 0.1  # per-element relative check on gradient elements at least this share of the scale


def gradient_report(ggpu, gorc, ok, label="", check=False):
    """Per-element relative errors of each gradient on elements whose size is at least a
    fraction (1e-1, 1e-2) of the buffer's scale, over the pixels `ok`; printed, and returned as
    a dict.  With check=True every element of at least ELEM_FLOOR of the scale must be within
    GRAD_RTOL of the oracle's, relative to itself."""
    out = {}
    for k in ("albedo", "rough", "metal", "normal", "env"):
        a, b = ggpu[k], gorc[k]
        if k != "env":
            sel = np.broadcast_to(ok[..., None], a.shape) if a.ndim == ok.ndim + 1 else ok
            a, b = a[sel], b[sel]
        scale = float(np.abs(b).max()) if b.size else 0.0
        rec = {}
        for fl in (1e-1, 1e-2):
            big = np.abs(b) >= fl * scale
            rec[f"{fl:g}"] = float((np.abs(a - b)[big] / np.abs(b[big])).max()) if big.any() else 0.0
        out[k] = rec
        print(f"{label} gradient {k}: per-element rel err on elements >= 0.1 / 0.01 of the scale: "
              f"{rec['0.1']:.2e} / {rec['0.01']:.2e}")
        if check:
            assert rec[f"{ELEM_FLOOR:g}"] <= GRAD_RTOL, (label, k, rec)
    return out


def affected_pixels(h_gpu, h_orc):
    """Pixels whose gradients may legitimately differ because some sample's hit differs:
    the receivers of mismatching samples and the pixels either side says they hit."""
    bad = h_gpu != h_orc
    aff = bad.any(axis=-1)
    for hh in (h_gpu, h_orc):
        vv, yy, xx, ss = np.nonzero(bad & (hh >= 0))
        q = hh[vv, yy, xx, ss]
        W = h_gpu.shape[2]
        aff[vv, q // W, q % W] = True
    return aff
