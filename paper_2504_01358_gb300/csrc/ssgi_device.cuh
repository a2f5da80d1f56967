// ssgi_device.cuh -- device-side math shared by the SSGI kernels (FP32, sm_103a).
//
// Microfacet terms (Appendix B), the lat-long environment lookup with its mip blend
// (Sec. 3.2, SampleEnvMap), the BRDF-table lookup (Appendix C), GGX sampling (Sec. 3.3) and
// the Philox4x32-10 generator (Salmon et al., SC'11).  Everything here follows the data
// formats of include/ssgi.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssgi_internal.h"

namespace ssgi {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInv2Pi = 0.15915494309189533577f;
constexpr float kInvPi = 0.31830988618379067154f;

// ------------------------------------------------------------------------------------------
// float3 helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul3(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
// The same in x y z order with one rounding per step, never re-fused by the compiler: for the
// dot products that shape a sampled direction or a lookup coordinate (n.v, v.h, |d|^2), whose
// bits a host model reproduces.  (Everywhere else the compiler's own fusion measured faster.)
__device__ __forceinline__ float dot3_rn(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 ld3(const float* __restrict__ p) { return f3(__ldg(p), __ldg(p + 1), __ldg(p + 2)); }
__device__ __forceinline__ void st3(float* p, float3 v) { p[0] = v.x; p[1] = v.y; p[2] = v.z; }
__device__ __forceinline__ float comp(float3 v, int c) { return c == 0 ? v.x : (c == 1 ? v.y : v.z); }

// ------------------------------------------------------------------------------------------
// Camera
// ------------------------------------------------------------------------------------------
// Camera-space direction through the centre of pixel (x, y); forward component is 1.
__device__ __forceinline__ float3 pix_dir_cam(const DevCam& c, int x, int y) {
  return f3(((float)x + 0.5f - c.cx) / c.f, -((float)y + 0.5f - c.cy) / c.f, -1.0f);
}
__device__ __forceinline__ float3 cam_to_world(const DevCam& c, float3 d) {
  return f3(fmaf(c.R[0], d.x, fmaf(c.R[1], d.y, c.R[2] * d.z)), fmaf(c.R[3], d.x, fmaf(c.R[4], d.y, c.R[5] * d.z)),
            fmaf(c.R[6], d.x, fmaf(c.R[7], d.y, c.R[8] * d.z)));
}
// World-space direction through the centre of pixel (x, y) (camera-space forward component 1;
// the -1 z term is exact, so each component takes two roundings).
__device__ __forceinline__ float3 pix_dir_world(const DevCam& c, int x, int y) {
  // the numerators are exact (half-integers); one rounding in each quotient
  const float dx = __fdiv_rn((float)x + 0.5f - c.cx, c.f), dy = -__fdiv_rn((float)y + 0.5f - c.cy, c.f);
  return f3(fmaf(c.R[0], dx, fmaf(c.R[1], dy, -c.R[2])), fmaf(c.R[3], dx, fmaf(c.R[4], dy, -c.R[5])),
            fmaf(c.R[6], dx, fmaf(c.R[7], dy, -c.R[8])));
}
// Unit vector from the surface point of a pixel to the camera: -d / |d| for the pixel's ray d.
__device__ __forceinline__ float3 view_vector(float3 d) {
  const float s = __fdiv_rn(-1.0f, __fsqrt_rn(dot3_rn(d, d)));
  return f3(__fmul_rn(d.x, s), __fmul_rn(d.y, s), __fmul_rn(d.z, s));
}
// Mirror direction r = 2 (v.n) n - v.
__device__ __forceinline__ float3 reflect_about(float3 n, float nv, float3 v) {
  const float t = 2.0f * nv;  // exact
  return f3(__fmaf_rn(n.x, t, -v.x), __fmaf_rn(n.y, t, -v.y), __fmaf_rn(n.z, t, -v.z));
}
__device__ __forceinline__ float3 world_to_cam(const DevCam& c, float3 d) {
  return f3(c.R[0] * d.x + c.R[3] * d.y + c.R[6] * d.z, c.R[1] * d.x + c.R[4] * d.y + c.R[7] * d.z,
            c.R[2] * d.x + c.R[5] * d.y + c.R[8] * d.z);
}
__device__ __forceinline__ bool is_background(float z) { return !(isfinite(z) && z > 0.0f); }

// ------------------------------------------------------------------------------------------
// sin(pi x), cos(pi x) and atan(num / den) in FP32 with explicitly rounded steps, so that the
// sampled directions and the environment-map coordinates are the same bits wherever this
// arithmetic is replayed.  sin/cos: exact reduction to the nearest quarter turn k/2 (2x and
// x - k/2 are exact), then the Taylor series of sin(pi f) and cos(pi f) on |f| <= 1/4 through
// f^9 and f^10 (truncation below 2e-9).  atan: for |t| > tan(pi/8) the identity
// atan(t) = pi/4 + atan((t - 1)/(t + 1)) brings the argument to |r| <= tan(pi/8), where the
// alternating series through r^15 is within 2e-8.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ void sincospi_rn(float x, float* s, float* c) {
  const float k = rintf(2.0f * x);
  const float f = __fmaf_rn(k, -0.5f, x);
  const float f2 = __fmul_rn(f, f);
  float ps = __fmaf_rn(f2, 8.2145886611128190e-02f, -5.9926452932079207e-01f);  // pi^9/9!, -pi^7/7!
  ps = __fmaf_rn(ps, f2, 2.5501640398773455e+00f);                               // pi^5/5!
  ps = __fmaf_rn(ps, f2, -5.1677127800499703e+00f);                              // -pi^3/3!
  ps = __fmaf_rn(ps, f2, 3.1415926535897932e+00f);                               // pi
  ps = __fmul_rn(ps, f);
  float pc = __fmaf_rn(f2, -2.5806891390014061e-02f, 2.3533063035889320e-01f);  // -pi^10/10!, pi^8/8!
  pc = __fmaf_rn(pc, f2, -1.3352627688545895e+00f);                               // -pi^6/6!
  pc = __fmaf_rn(pc, f2, 4.0587121264167682e+00f);                                // pi^4/4!
  pc = __fmaf_rn(pc, f2, -4.9348022005446793e+00f);                               // -pi^2/2!
  pc = __fmaf_rn(pc, f2, 1.0f);
  const int q = ((int)k) & 3;
  *s = q == 0 ? ps : (q == 1 ? pc : (q == 2 ? -ps : -pc));
  *c = q == 0 ? pc : (q == 1 ? -ps : (q == 2 ? -pc : ps));
}

// atan(num / den) for |num| <= den (an octant-reduced angle, in [-pi/4, pi/4]).  With den = 0
// (and so num = 0: a direction along the map's axis) the signed zeros decide as in atan2:
// +-0 for den = +0, +-pi for den = -0.
__device__ __forceinline__ float atan_octant_rn(float num, float den) {
  if (den == 0.0f) return copysignf(signbit(den) ? kPi : 0.0f, num);
  const float an = fabsf(num);
  const bool big = an > __fmul_rn(0.41421356237309505f, den);
  // one division: the reduced argument's numerator and denominator are selected first
  const float r = __fdiv_rn(big ? __fsub_rn(an, den) : an, big ? __fadd_rn(an, den) : den);
  const float r2 = __fmul_rn(r, r);
  float p = __fmaf_rn(r2, -1.0f / 15.0f, 1.0f / 13.0f);
  p = __fmaf_rn(p, r2, -1.0f / 11.0f);
  p = __fmaf_rn(p, r2, 1.0f / 9.0f);
  p = __fmaf_rn(p, r2, -1.0f / 7.0f);
  p = __fmaf_rn(p, r2, 1.0f / 5.0f);
  p = __fmaf_rn(p, r2, -1.0f / 3.0f);
  const float at = __fmaf_rn(__fmul_rn(r, r2), p, r);
  const float a = big ? __fadd_rn(0.78539816339744831f, at) : at;
  return num < 0.0f ? -a : a;
}

// ------------------------------------------------------------------------------------------
// Philox4x32-10: ten rounds of the 4x32 S-box, multipliers 0xD2511F53 / 0xCD9E8D57 and key
// increments 0x9E3779B9 / 0xBB67AE85 (Salmon, Moraes, Dror, Shaw 2011).
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// (xi0, xi1) of sample s at pixel `pix` of view `view`.
__device__ __forceinline__ float2 sample_uniforms(uint64_t seed, int view, uint32_t pix, uint32_t s) {
  const uint2 key = make_uint2((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ (uint32_t)view);
  const uint4 o = philox4x32_10(make_uint4(pix, s, 0u, 0u), key);
  return make_float2((float)(o.x >> 8) * (1.0f / 16777216.0f), (float)(o.y >> 8) * (1.0f / 16777216.0f));
}

// ------------------------------------------------------------------------------------------
// Microfacet terms (Appendix B); alpha = rho as printed.
// ------------------------------------------------------------------------------------------
// D at a half vector drawn by ggx_sample_h with denominator ds: there
// 1 + (n.h)^2 (rho^2 - 1) = rho^2 / ds exactly, so D = ds^2 / (pi rho^2), free of the
// cancellation that 1 + (n.h)^2 (rho^2 - 1) suffers for n.h -> 1 at low roughness (n.h
// rounded to FP32 near 1 has lost most of the information that sin(theta_h) keeps).
__device__ __forceinline__ float ggx_D_sampled(float ds, float rho) { return ds * ds / (kPi * (rho * rho)); }
__device__ __forceinline__ float ggx_G1(float z, float rho) {
  const float a2 = rho * rho;
  return 2.0f * z / (z + sqrtf(a2 + (1.0f - a2) * z * z));
}
__device__ __forceinline__ float pow5(float c) {
  const float c2 = c * c;
  return c2 * c2 * c;
}
__device__ __forceinline__ float f0_of(float a, float m) { return 0.04f * (1.0f - m) + a * m; }

// GGX half vector around n (Walter et al. 2007 inversion; frame of Duff et al. 2017).
// cos^2 = (1 - xi0) / den and sin^2 = rho^2 xi0 / den with den = 1 + (rho^2 - 1) xi0: the
// same values as sqrt(1 - cos^2) without its cancellation for near-mirror lobes.  *ct
// receives cos(theta_h) = n.h and *den_out den.
// den is formed as (1 - xi0) + rho^2 xi0: the same number without the cancellation of the
// first form as xi0 -> 1 (1 - xi0 is exact on the uniforms' 2^-24 grid), so that
// cos^2 + sin^2 stays 1 to a few ulp and h stays a unit vector; with the first form a
// low-roughness sample's h could be ~1e-5 too long, turning its reflection by as much.
__device__ __forceinline__ float3 ggx_sample_h(float3 n, float rho, float xi0, float xi1, float* ct_out = nullptr,
                                               float* den_out = nullptr) {
  const float a2 = __fmul_rn(rho, rho);
  const float om = 1.0f - xi0;  // exact on the 2^-24 grid
  const float den = __fmaf_rn(a2, xi0, om);
  const float ct = __fsqrt_rn(__fdiv_rn(om, den));
  const float st = __fsqrt_rn(__fdiv_rn(__fmul_rn(a2, xi0), den));
  if (ct_out) *ct_out = ct;
  if (den_out) *den_out = den;
  float sp, cp;
  sincospi_rn(2.0f * xi1, &sp, &cp);
  const float sgn = n.z >= 0.0f ? 1.0f : -1.0f;
  const float aa = __fdiv_rn(-1.0f, __fadd_rn(sgn, n.z));
  const float bb = __fmul_rn(__fmul_rn(n.x, n.y), aa);
  const float3 t1 = f3(__fmaf_rn(__fmul_rn(sgn * n.x, n.x), aa, 1.0f), sgn * bb, -sgn * n.x);
  const float3 t2 = f3(bb, __fmaf_rn(__fmul_rn(n.y, n.y), aa, sgn), -n.y);
  const float c1 = __fmul_rn(st, cp), c2 = __fmul_rn(st, sp);
  return f3(__fmaf_rn(n.x, ct, __fmaf_rn(t2.x, c2, __fmul_rn(t1.x, c1))),
            __fmaf_rn(n.y, ct, __fmaf_rn(t2.y, c2, __fmul_rn(t1.y, c1))),
            __fmaf_rn(n.z, ct, __fmaf_rn(t2.z, c2, __fmul_rn(t1.z, c1))));
}

// Derivatives of ggx_sample_h's half vector at fixed uniforms with respect to n.x, n.y, n.z
// (dh[0..2]; the components taken independently, as the formula is written) and rho (dh[3]).
// With q = sqrt(xi0 / den): sin = rho q, d sin / d rho = q (1 - xi0) / den, and
// d cos / d rho = -cos rho xi0 / den; the frame's derivatives follow from aa' = aa^2 (n.z).
__device__ __forceinline__ void ggx_sample_h_jac(float3 n, float rho, float xi0, float xi1, float3 dh[4]) {
  const float a2 = rho * rho;
  const float den = fmaf(a2, xi0, 1.0f - xi0);
  const float ct = sqrtf((1.0f - xi0) / den);
  const float q = sqrtf(xi0 / den);
  const float st = rho * q;
  float sp, cp;
  sincospi_rn(2.0f * xi1, &sp, &cp);
  const float sgn = n.z >= 0.0f ? 1.0f : -1.0f;
  const float aa = -1.0f / (sgn + n.z);
  const float aa2 = aa * aa;
  const float bb = n.x * n.y * aa;
  const float3 t1 = f3(1.0f + sgn * n.x * n.x * aa, sgn * bb, -sgn * n.x);
  const float3 t2 = f3(bb, sgn + n.y * n.y * aa, -n.y);
  const float c1 = st * cp, c2 = st * sp;
  dh[0] = f3(2.0f * sgn * n.x * aa, sgn * n.y * aa, -sgn) * c1 + f3(n.y * aa, 0.0f, 0.0f) * c2 + f3(ct, 0.0f, 0.0f);
  dh[1] = f3(0.0f, sgn * n.x * aa, 0.0f) * c1 + f3(n.x * aa, 2.0f * n.y * aa, -1.0f) * c2 + f3(0.0f, ct, 0.0f);
  dh[2] = f3(sgn * n.x * n.x * aa2, sgn * n.x * n.y * aa2, 0.0f) * c1 + f3(n.x * n.y * aa2, n.y * n.y * aa2, 0.0f) * c2 +
          f3(0.0f, 0.0f, ct);
  dh[3] = (t1 * cp + t2 * sp) * (q * (1.0f - xi0) / den) + n * (-ct * rho * xi0 / den);
}

struct Sample {
  float3 h, w;
  float vh, nh, nw;
  float ds;  // the sampler's denominator (1 - xi0) + rho^2 xi0 (ggx_D_sampled)
  bool valid;
};

// n.h is the sampled cosine and n.w = 2 (v.h)(n.h) - n.v (identities of w = 2 (v.h) h - v),
// both better conditioned in FP32 than dot products with the rounded vectors.
__device__ __forceinline__ Sample make_sample(float3 n, float3 v, float nv, float rho, float2 xi) {
  Sample s;
  s.h = ggx_sample_h(n, rho, xi.x, xi.y, &s.nh, &s.ds);
  s.vh = dot3_rn(v, s.h);
  s.w = reflect_about(s.h, s.vh, v);
  s.nw = fmaf(2.0f * s.vh, s.nh, -nv);
  s.valid = (nv > 0.0f) && (s.nw > 0.0f) && (s.vh > 0.0f) && (s.nh > 0.0f);
  return s;
}

// ------------------------------------------------------------------------------------------
// Environment lookup
// ------------------------------------------------------------------------------------------
struct Taps {
  int idx[4];  // float offsets of the four texels
  float tx, ty;
};

// Octant-reduced angles of a direction: the texel coordinates x = u w - 0.5 and y = v h - 0.5
// of the lat-long mapping are written as base + ang * scale with |ang| <= pi/4 and an exact
// base, so the bilinear fractions keep full FP32 precision (a full-range atan2 near +-pi would
// cost ~4e-5 texel at w = 512).  The mapping is u = 0.5 + atan2(x, -z) / (2 pi) and
// v = atan2(sqrt(x^2 + z^2), y) / pi.
struct DirAngles {
  float ax, bx;  // x = bx + ax * w / (2 pi)
  float ay, by;  // y = by + ay * h / pi  (by in units of h: 0, 1/2 or 1)
};

__device__ __forceinline__ DirAngles dir_angles(float3 d) {
  DirAngles r;
  // azimuth: pick the octant-reduced (numerator, denominator) pair with selects, one arctangent
  const float X = -d.z, Y = d.x;
  const float aX = fabsf(X), aY = fabsf(Y);
  const bool xa = aY <= X, xb = Y > aX, xc = -X >= aY;
  const float num = xa ? Y : (xb ? -X : (xc ? -Y : X));
  const float den = xa ? X : (xb ? Y : (xc ? -X : -Y));
  r.bx = xa ? 0.5f : (xb ? 0.75f : (xc ? 1.0f : 0.25f));
  r.ax = atan_octant_rn(num, den);
  // polar angle from +y, likewise
  const float q = __fsqrt_rn(__fmaf_rn(d.z, d.z, __fmul_rn(d.x, d.x)));
  const bool ya = d.y >= q, yb = -d.y >= q;
  const float ny = ya ? q : (yb ? q : d.y);
  const float dy = ya ? d.y : (yb ? -d.y : q);
  const float sg = (ya ? 1.0f : -1.0f);
  r.by = ya ? 0.0f : (yb ? 1.0f : 0.5f);
  r.ay = sg * atan_octant_rn(ny, dy);
  return r;
}

// integer part and fraction of base * n - 0.5 + ang * k
__device__ __forceinline__ void split_coord(float base, float ang, int n, float k, int& i0, float& t) {
  const float b = __fmaf_rn(base, (float)n, -0.5f);  // exact: n is a power of two
  float f0 = floorf(__fmaf_rn(ang, k, b));
  t = __fmaf_rn(ang, k, __fsub_rn(b, f0));
  if (t < 0.0f) {
    t = __fadd_rn(t, 1.0f);
    f0 -= 1.0f;
  } else if (t >= 1.0f) {
    t = __fsub_rn(t, 1.0f);
    f0 += 1.0f;
  }
  i0 = (int)f0;
}

// kMask: wrap the column with a mask (the map's widths are powers of two, and a two's-complement
// mask wraps negative columns too) instead of a remainder and two tests: the same taps, measured
// 9 % faster in direct shading and 2.5 % in the adjoint, but 0.6 % slower in the trace, whose
// miss lookup keeps the remainder.
template <bool kMask = true>
__device__ __forceinline__ Taps env_taps(const EnvInfo& e, int l, const DirAngles& a) {
  Taps t;
  const int h = e.h[l], w = e.w[l];
  int x0, y0;
  split_coord(a.bx, a.ax, w, __fmul_rn((float)w, kInv2Pi), x0, t.tx);
  split_coord(a.by, a.ay, h, __fmul_rn((float)h, kInvPi), y0, t.ty);
  int c0, c1;
  if (kMask) {
    c0 = x0 & (w - 1);
    c1 = (x0 + 1) & (w - 1);
  } else {
    c0 = x0 % w;
    if (c0 < 0) c0 += w;
    c1 = c0 + 1;
    if (c1 >= w) c1 -= w;
  }
  const int r0 = min(max(y0, 0), h - 1), r1 = min(max(y0 + 1, 0), h - 1);
  const int base = e.off[l];
  t.idx[0] = base + (r0 * w + c0) * 3;
  t.idx[1] = base + (r0 * w + c1) * 3;
  t.idx[2] = base + (r1 * w + c0) * 3;
  t.idx[3] = base + (r1 * w + c1) * 3;
  return t;
}

__device__ __forceinline__ float3 bilinear(const float* __restrict__ mips, const Taps& t) {
  const float3 a = ld3(mips + t.idx[0]), b = ld3(mips + t.idx[1]);
  const float3 c = ld3(mips + t.idx[2]), d = ld3(mips + t.idx[3]);
  const float w00 = (1.0f - t.tx) * (1.0f - t.ty), w01 = t.tx * (1.0f - t.ty);
  const float w10 = (1.0f - t.tx) * t.ty, w11 = t.tx * t.ty;
  return a * w00 + b * w01 + c * w10 + d * w11;
}

// SampleEnvMap(d, lambda): bilinear at floor(lambda) and the next level, blended linearly.
__device__ __forceinline__ float3 env_lookup(const float* __restrict__ mips, const EnvInfo& e, float3 d, float lam) {
  const float lmax = (float)(e.levels - 1);
  lam = fminf(fmaxf(lam, 0.0f), lmax);
  const int l0 = (int)floorf(lam);
  const int l1 = min(l0 + 1, e.levels - 1);
  const float t = lam - (float)l0;
  const DirAngles ang = dir_angles(d);
  const float3 a = bilinear(mips, env_taps(e, l0, ang));
  if (t == 0.0f) return a;
  const float3 b = bilinear(mips, env_taps(e, l1, ang));
  return a * (1.0f - t) + b * t;
}

__device__ __forceinline__ float3 env_lookup0(const float* __restrict__ mips, const EnvInfo& e, float3 d) {
  return bilinear(mips, env_taps(e, 0, dir_angles(d)));
}
// The trace's miss lookup (see env_taps).
__device__ __forceinline__ float3 env_lookup0_trace(const float* __restrict__ mips, const EnvInfo& e, float3 d) {
  return bilinear(mips, env_taps<false>(e, 0, dir_angles(d)));
}

// ------------------------------------------------------------------------------------------
// BRDF table lookup: bilinear at texel centres, clamped.  Also returns d/drho, d/dmu of A, B
// (zero where the coordinate is clamped).
// ------------------------------------------------------------------------------------------
struct LutVal {
  float A, B, dA_drho, dB_drho, dA_dmu, dB_dmu;
};

__device__ __forceinline__ LutVal lut_sample(const float* __restrict__ lut, int N, float rho, float mu) {
  LutVal r;
  float x = mu * (float)N - 0.5f, y = rho * (float)N - 0.5f;
  const bool xin = (x > 0.0f && x < (float)(N - 1)), yin = (y > 0.0f && y < (float)(N - 1));
  x = fminf(fmaxf(x, 0.0f), (float)(N - 1));
  y = fminf(fmaxf(y, 0.0f), (float)(N - 1));
  const int x0 = min((int)floorf(x), N - 2), y0 = min((int)floorf(y), N - 2);
  const float tx = x - (float)x0, ty = y - (float)y0;
  const float2 v00 = __ldg(reinterpret_cast<const float2*>(lut) + (y0 * N + x0));
  const float2 v01 = __ldg(reinterpret_cast<const float2*>(lut) + (y0 * N + x0 + 1));
  const float2 v10 = __ldg(reinterpret_cast<const float2*>(lut) + ((y0 + 1) * N + x0));
  const float2 v11 = __ldg(reinterpret_cast<const float2*>(lut) + ((y0 + 1) * N + x0 + 1));
  r.A = (1 - ty) * ((1 - tx) * v00.x + tx * v01.x) + ty * ((1 - tx) * v10.x + tx * v11.x);
  r.B = (1 - ty) * ((1 - tx) * v00.y + tx * v01.y) + ty * ((1 - tx) * v10.y + tx * v11.y);
  const float fN = (float)N;
  r.dA_dmu = xin ? fN * ((1 - ty) * (v01.x - v00.x) + ty * (v11.x - v10.x)) : 0.0f;
  r.dB_dmu = xin ? fN * ((1 - ty) * (v01.y - v00.y) + ty * (v11.y - v10.y)) : 0.0f;
  r.dA_drho = yin ? fN * ((1 - tx) * (v10.x - v00.x) + tx * (v11.x - v01.x)) : 0.0f;
  r.dB_drho = yin ? fN * ((1 - tx) * (v10.y - v00.y) + tx * (v11.y - v01.y)) : 0.0f;
  return r;
}

}  // namespace ssgi
