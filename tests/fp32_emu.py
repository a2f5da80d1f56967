"""Bit-exact host model of the FP32 arithmetic by which the CUDA kernels form directions and
environment-map coordinates: the pixel ray, the view vector, the mirror direction, the GGX
half vector and reflected direction of a sample, and the octant-reduced angles and texel
coordinates of a latitude-longitude lookup.

Test infrastructure.  It is NOT the oracle (the oracle computes in FP64 and shares nothing with
the kernels); it models the kernels' rounding so that a parity test can replay a pixel's
Monte-Carlo sum in the oracle's FP64 arithmetic at exactly the lookup coordinates the GPU used,
and so tell an ill-conditioned lookup (a direction that FP32 rounding moves across a steep
texel edge or near the map's pole) from a wrong result.  The kernels write every step of that
arithmetic with explicitly rounded operations (one IEEE rounding per add, multiply, divide,
square root or fused multiply-add, never re-fused by the compiler), and their sine, cosine and
arctangent are polynomials of their own; this module performs the same steps in the same order
on numpy float32 arrays: numpy's float32 add, multiply, divide and square root (IEEE, round to
nearest even) and a fused multiply-add that rounds the exact value once.  Every function takes
and returns arrays (or numpy scalars) and works elementwise.
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

F32 = np.float32


def f32(x):
    return np.asarray(x, dtype=F32)


# ---------------------------------------------------------------------------------------------
# one-rounding operations
# ---------------------------------------------------------------------------------------------
def round_f32(x: Fraction) -> float:
    """x rounded to the nearest FP32 value, ties to even (subnormals included)."""
    if x == 0:
        return 0.0
    sg = -1.0 if x < 0 else 1.0
    a = -x if x < 0 else x
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    elif Fraction(2) ** (e + 1) <= a:
        e += 1
    q = max(e - 23, -149)  # quantum of the result's binade
    m = a / (Fraction(2) ** q)
    n = m.numerator // m.denominator
    rem = m - n
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sg * float(Fraction(n) * Fraction(2) ** q)


def lit(s: str) -> np.float32:
    """An FP32 literal as a C compiler reads it: the decimal string rounded once to FP32."""
    return F32(round_f32(Fraction(s)))


_ERR = dict(divide="ignore", invalid="ignore", over="ignore", under="ignore")


def add(a, b):
    with np.errstate(**_ERR):
        return f32(a) + f32(b)


def sub(a, b):
    with np.errstate(**_ERR):
        return f32(a) - f32(b)


def mul(a, b):
    with np.errstate(**_ERR):
        return f32(a) * f32(b)


def div(a, b):
    with np.errstate(**_ERR):
        return f32(a) / f32(b)


def sqrt(a):
    with np.errstate(**_ERR):
        return np.sqrt(f32(a))


def fma(a, b, c):
    """a * b + c rounded once.  The product of two FP32 values is exact in FP64; the FP64 sum is
    one more rounding, which changes the FP32 result only where it lands exactly on an FP32
    midpoint (or in the subnormal range): those elements are recomputed in exact arithmetic."""
    a, b, c = np.broadcast_arrays(f32(a), f32(b), f32(c))
    with np.errstate(**_ERR):
        s = a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)
        r = s.astype(F32)
        r64 = r.astype(np.float64)
        lo = np.nextafter(r, F32(-np.inf)).astype(np.float64)
        hi = np.nextafter(r, F32(np.inf)).astype(np.float64)
        bad = np.isfinite(s) & (s != r64) & ((s == (r64 + lo) / 2) | (s == (r64 + hi) / 2) |
                                             (np.abs(r64) < 2.0 ** -126))
    if np.any(bad):
        r = np.array(r, copy=True)
        for i in zip(*np.nonzero(bad)) if r.ndim else [()]:
            r[i] = round_f32(Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i])))
    return r


def dot3(a, b):
    """x y z order, as the kernels' dot3."""
    return fma(a[..., 2], b[..., 2], fma(a[..., 1], b[..., 1], mul(a[..., 0], b[..., 0])))


def vec(x, y, z):
    return np.stack([f32(x), f32(y), f32(z)], axis=-1)


# constants as the kernels spell them
K_INV_2PI = lit("0.15915494309189533577")
K_INV_PI = lit("0.31830988618379067154")
TAN_PI_8 = lit("0.41421356237309505")
PI_4 = lit("0.78539816339744831")
_SIN = [lit(c) for c in ("8.2145886611128190e-02", "-5.9926452932079207e-01", "2.5501640398773455e+00",
                         "-5.1677127800499703e+00", "3.1415926535897932e+00")]
_COS = [lit(c) for c in ("-2.5806891390014061e-02", "2.3533063035889320e-01", "-1.3352627688545895e+00",
                         "4.0587121264167682e+00", "-4.9348022005446793e+00")]
_ATAN = [F32(round_f32(Fraction(n, d))) for n, d in ((-1, 15), (1, 13), (-1, 11), (1, 9), (-1, 7), (1, 5),
                                                       (-1, 3))]


# ---------------------------------------------------------------------------------------------
# sine / cosine of pi x and the octant arctangent (the kernels' own polynomials)
# ---------------------------------------------------------------------------------------------
def sincospi(x):
    x = f32(x)
    k = np.rint(mul(2.0, x))
    f = fma(k, F32(-0.5), x)
    f2 = mul(f, f)
    ps = fma(f2, _SIN[0], _SIN[1])
    for c in _SIN[2:]:
        ps = fma(ps, f2, c)
    ps = mul(ps, f)
    pc = fma(f2, _COS[0], _COS[1])
    for c in _COS[2:]:
        pc = fma(pc, f2, c)
    pc = fma(pc, f2, F32(1.0))
    q = k.astype(np.int64) & 3
    s = np.select([q == 0, q == 1, q == 2], [ps, pc, -ps], -pc).astype(F32)
    c = np.select([q == 0, q == 1, q == 2], [pc, -ps, -pc], ps).astype(F32)
    return s, c


PI = lit("3.14159265358979323846")


def atan_octant(num, den):
    """atan(num / den) for |num| <= den; at den = 0 the signed zeros decide as in atan2 (+-0 for
    den = +0, +-pi for den = -0)."""
    num, den = np.broadcast_arrays(f32(num), f32(den))
    an = np.abs(num)
    big = an > mul(TAN_PI_8, den)
    r = div(np.where(big, sub(an, den), an), np.where(big, add(an, den), den))
    r2 = mul(r, r)
    p = fma(r2, _ATAN[0], _ATAN[1])
    for c in _ATAN[2:]:
        p = fma(p, r2, c)
    at = fma(mul(r, r2), p, r)
    a = np.where(big, add(PI_4, at), at).astype(F32)
    a = np.where(num < 0, -a, a).astype(F32)
    zero = np.copysign(np.where(np.signbit(den), PI, F32(0.0)), num).astype(F32)
    return np.where(den == 0, zero, a).astype(F32)


# ---------------------------------------------------------------------------------------------
# camera, view vector, mirror direction
# ---------------------------------------------------------------------------------------------
class Cam:
    """A camera record as the library holds it (FP32 rotation, focal length and principal point)."""

    def __init__(self, rec, H: int, W: int):
        rec = np.asarray(rec, np.float32)
        self.R = rec[:12].reshape(3, 4)[:, :3].reshape(-1).astype(F32)
        self.f = F32((H / 2.0) / math.tan(float(rec[12]) / 2.0))
        self.cx, self.cy = F32(W / 2.0), F32(H / 2.0)


def pix_dir_world(c: Cam, x, y):
    """Ray through pixel centres (x, y) (integer arrays), forward component 1 in camera space."""
    x = np.asarray(x).astype(F32)
    y = np.asarray(y).astype(F32)
    dx = div((x + F32(0.5)) - c.cx, c.f)          # the numerators are exact half-integers
    dy = -div((y + F32(0.5)) - c.cy, c.f)
    R = c.R
    return vec(fma(R[0], dx, fma(R[1], dy, -R[2])), fma(R[3], dx, fma(R[4], dy, -R[5])),
               fma(R[6], dx, fma(R[7], dy, -R[8])))


def view_vector(d):
    s = div(F32(-1.0), sqrt(dot3(d, d)))
    return vec(mul(d[..., 0], s), mul(d[..., 1], s), mul(d[..., 2], s))


def reflect_about(n, nv, v):
    t = mul(F32(2.0), nv)  # exact
    return vec(fma(n[..., 0], t, -v[..., 0]), fma(n[..., 1], t, -v[..., 1]), fma(n[..., 2], t, -v[..., 2]))


# ---------------------------------------------------------------------------------------------
# one sample: GGX half vector (Duff et al. frame), reflected direction, validity
# ---------------------------------------------------------------------------------------------
def ggx_sample_h(n, rho, xi0, xi1):
    """(h, n.h, den) of the kernels' sampler."""
    rho, xi0, xi1 = f32(rho), f32(xi0), f32(xi1)
    a2 = mul(rho, rho)
    om = F32(1.0) - xi0  # exact on the 2^-24 grid
    den = fma(a2, xi0, om)
    ct = sqrt(div(om, den))
    st = sqrt(div(mul(a2, xi0), den))
    sp, cp = sincospi(mul(F32(2.0), xi1))
    nx, ny, nz = n[..., 0], n[..., 1], n[..., 2]
    sgn = np.where(nz >= 0, F32(1.0), F32(-1.0)).astype(F32)
    aa = div(F32(-1.0), add(sgn, nz))
    bb = mul(mul(nx, ny), aa)
    t1 = vec(fma(mul(sgn * nx, nx), aa, F32(1.0)), sgn * bb, -sgn * nx)
    t2 = vec(bb, fma(mul(ny, ny), aa, sgn), -ny)
    c1, c2 = mul(st, cp), mul(st, sp)
    h = vec(*[fma(n[..., i], ct, fma(t2[..., i], c2, mul(t1[..., i], c1))) for i in range(3)])
    return h, ct, den


def make_sample(n, v, nv, rho, xi0, xi1):
    h, nh, den = ggx_sample_h(n, rho, xi0, xi1)
    vh = dot3(v, h)
    w = reflect_about(h, vh, v)
    nw = fma(mul(F32(2.0), vh), nh, -f32(nv))
    valid = (f32(nv) > 0) & (nw > 0) & (vh > 0) & (nh > 0)
    return {"h": h, "w": w, "vh": vh, "nh": nh, "nw": nw, "ds": den, "valid": valid}


# ---------------------------------------------------------------------------------------------
# latitude-longitude coordinates
# ---------------------------------------------------------------------------------------------
def dir_angles(d):
    X, Y = -d[..., 2], d[..., 0]
    aX, aY = np.abs(X), np.abs(Y)
    xa, xb, xc = aY <= X, Y > aX, -X >= aY
    num = np.select([xa, xb, xc], [Y, -X, -Y], X).astype(F32)
    den = np.select([xa, xb, xc], [X, Y, -X], -Y).astype(F32)
    bx = np.select([xa, xb, xc], [0.5, 0.75, 1.0], 0.25).astype(F32)
    ax = atan_octant(num, den)
    q = sqrt(fma(d[..., 2], d[..., 2], mul(d[..., 0], d[..., 0])))
    dyv = d[..., 1]
    ya, yb = dyv >= q, -dyv >= q
    ny = np.where(ya | yb, q, dyv).astype(F32)
    dy = np.select([ya, yb], [dyv, -dyv], q).astype(F32)
    sg = np.where(ya, F32(1.0), F32(-1.0)).astype(F32)
    by = np.select([ya, yb], [0.0, 1.0], 0.5).astype(F32)
    ay = sg * atan_octant(ny, dy)
    return ax, bx, ay, by


def split_coord(base, ang, n: int, k):
    b = fma(base, F32(n), F32(-0.5))  # exact: n is a power of two
    f0 = np.floor(fma(ang, k, b))
    t = fma(ang, k, sub(b, f0))
    lo, hi = t < 0, t >= 1
    t = np.where(lo, add(t, F32(1.0)), np.where(hi, sub(t, F32(1.0)), t)).astype(F32)
    f0 = f0 - lo + hi
    return f0.astype(np.int64), t


def texel_coords(d, h: int, w: int, angles=None):
    """(x0, y0, tx, ty) of the lookup in direction d on an h x w level: the texel column / row
    below the sample point (before wrapping and clamping) and the bilinear fractions."""
    ax, bx, ay, by = dir_angles(d) if angles is None else angles
    x0, tx = split_coord(bx, ax, w, mul(F32(w), K_INV_2PI))
    y0, ty = split_coord(by, ay, h, mul(F32(h), K_INV_PI))
    return x0, y0, tx, ty
