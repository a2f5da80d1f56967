"""Helpers shared by the GPU parity tests: run a workload through libssgi.so (via the binding)
and through the FP64 oracle on the same seeded inputs, and compare.

Tolerances (written here, used by every parity test):
  * hit indices: bit-exact on >= 99.9 % of samples; every mismatching sample must be a
    near-tie in the oracle (decision margin < MARGIN_TOL), i.e. a rounding-order case;
  * per-pixel RGB: |gpu - oracle|_inf <= RGB_RTOL * max(|oracle|_inf, RGB_FLOOR) on pixels
    whose samples all match;
  * gradients: <= GRAD_RTOL relative (per element against the vector's scale, and as a norm).
"""
import numpy as np

import oracle as O

HIT_MATCH_MIN = 0.999
MARGIN_TOL = 2e-3
RGB_RTOL = 1e-4
RGB_FRAC_MIN = 0.99999  # share of pixels within RGB_RTOL (all pixels below 1e5 pixels)
RGB_RTOL_MAX = 3e-4     # bound for the rest: FP32 direction error (~1e-7 rad) x env texel contrast
RGB_FLOOR = 1e-3
GRAD_RTOL = 1e-3


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


def assert_forward_parity(gpu, orc, label=""):
    frac, bad, margins = compare_hits(gpu["hit_idx"], orc)
    assert frac >= HIT_MATCH_MIN, f"{label}: hit-index match {frac:.6f}"
    assert np.all(margins < MARGIN_TOL), f"{label}: mismatch with decision margin {margins.max()}"
    pix_ok = ~bad.any(axis=-1)
    scale = np.maximum(np.abs(orc["final"]).max(axis=-1), RGB_FLOOR)
    for key in [k for k in ("final", "cs_mc", "c_id") if k in gpu]:
        okey = {"c_id": "cid"}.get(key, key)
        # error of each channel in units of the pixel's output RGB
        err = (np.abs(gpu[key].astype(np.float64) - orc[okey]).max(axis=-1) / scale)[pix_ok]
        assert_rgb(err, f"{label}: {key}")
    return frac, int(bad.sum())


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
