"""The parity tests' replay (tests/parity.py: Replay, the oracle's FP64 arithmetic at the lookup
coordinates and sample weights the kernels form in FP32) pinned on the CPU against the oracle
itself: on every pixel of a few-tile case it reproduces the oracle's direct shading and
Monte-Carlo sums up to the FP32 rounding of directions and coordinates, and a pixel it replays
differs from the oracle by no more than the conditioning of its lookups explains."""
import numpy as np
import pytest

import oracle as O
import ssgi_inputs as si
from parity import Replay, pixel_rel_err


@pytest.mark.parametrize("flags", [0, O.FLAG_DIFFUSE_INDIRECT])
def test_replay_reproduces_the_oracle(flags, small, lut):
    wl = small
    r = O.forward(wl, lut=lut, flags=flags)
    rp = Replay(wl, lut=lut)
    V, H, W = wl.depth.shape
    pix = np.arange(V * H * W)
    cd, cs, c1 = rp.direct(pix)
    errs = {}
    for name, got, want in (("cd", cd, r["cd"]), ("cs", cs, r["cs"]), ("c1", c1, r["c1"])):
        errs[name] = pixel_rel_err(got.reshape(want.shape), want).ravel()
    cs_mc, cid, final = rp.trace(pix, r["hit_idx"].reshape(V * H * W, -1), flags)
    for name, got, want in (("cs_mc", cs_mc, r["cs_mc"]), ("final", final, r["final"])):
        errs[name] = pixel_rel_err(got.reshape(want.shape), want).ravel()
    if flags:
        errs["cid"] = pixel_rel_err(cid.reshape(r["cid"].shape), r["cid"]).ravel()
    for name, e in errs.items():
        assert np.median(e) < 1e-6, (name, float(np.median(e)))
        assert np.mean(e <= 1e-4) >= 0.999, (name, float(np.mean(e <= 1e-4)), float(e.max()))
        assert e.max() < 1e-2, (name, float(e.max()))
