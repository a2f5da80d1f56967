// ssgi_ops.cuh -- the per-item device code of every SSGI stage, shared by the stand-alone
// kernels (one launch per stage) and the fused persistent step (all stages in one launch).
//
// FrameArgs describes one frame's buffers; each stage reads the fields it needs.
#pragma once

#include <limits.h>

#include "ssgi_device.cuh"

namespace ssgi {

struct FrameArgs {
  Views vs;
  EnvInfo e;
  HizInfo hz;
  const float* __restrict__ depth;
  const float* __restrict__ normal;
  const float* __restrict__ albedo;
  const float* __restrict__ rough;
  const float* __restrict__ metal;
  const float* __restrict__ mips;  // packed mip chain (built before the stages that read it)
  const float* __restrict__ lut;
  const float* __restrict__ hiz;
  const float* __restrict__ target;
  int lut_n;
  float* c_d;
  float* c_s;
  float* c1;
  float* c_s_mc;
  float* c_id;
  float* final_out;
  int32_t* hit_idx;
  unsigned long long* step_count;
  float* g_final;
  float* g_albedo;
  float* g_rough;
  float* g_metal;
  float* g_normal;
  float4* g_c1;    // backward workspace [V,H,W] RGB + pad: one 16-byte atomic per scatter
  float4* g_mips;  // backward workspace, one RGB + pad per texel, levels packed like the mips
  int spp, max_steps, levels;
  float thickness, max_distance;
  uint64_t seed;
  uint32_t flags;
};

// ==========================================================================================
// Precomputation (Appendix C table, Sec. 3.2 mips, Sec. 3.3 pyramid)
// ==========================================================================================
// The pyramid builders read the level below through ld.global.cg (L2, coherent): in the fused
// step that level was written earlier in the same launch, possibly by another SM.
__device__ __forceinline__ float env_avg4(float a, float b, float d, float e) { return 0.25f * (((a + b) + d) + e); }

__device__ __forceinline__ void env_down_item(const float* src, int hs, int ws, float* dst, int t) {
  const int wd = ws >> 1;
  const int c = t % 3, j = (t / 3) % wd, i = t / (3 * wd);
  const float a = __ldcg(src + ((2 * i) * ws + 2 * j) * 3 + c), b = __ldcg(src + ((2 * i) * ws + 2 * j + 1) * 3 + c);
  const float d = __ldcg(src + ((2 * i + 1) * ws + 2 * j) * 3 + c), e = __ldcg(src + ((2 * i + 1) * ws + 2 * j + 1) * 3 + c);
  dst[t] = env_avg4(a, b, d, e);
}

constexpr int kHizTile = 32;  // level-0 pixels per block side; covers levels 1..5

// A kT x kT tile in shared memory (a padded row: no bank conflicts on the 2 x 2 reads).
template <int kT>
using TileBufT = float[kT][kT + 1];
typedef TileBufT<kHizTile> TileBuf;

// Pyramid levels a kT x kT tile covers (levels 1..log2 kT).
template <int kT>
__host__ __device__ constexpr int tile_levels() {
  return kT == 1 ? 0 : 1 + tile_levels<kT / 2>();
}

// Block-level: reduces the kT x kT level-0 tile in s (filled by the caller, +inf outside the
// image; the caller synchronised after filling it) through levels 1..log2 kT of the pyramid
// and writes them; every thread of the block calls it for the same tile (it synchronises the
// block); the block has at least 128 threads.
template <int kT>
__device__ __forceinline__ void hiz_tile_reduce(int H, int W, const HizInfo& hz, float* __restrict__ hiz, int view,
                                                int tile_x, int tile_y, TileBufT<kT>& s) {
  const int bx = tile_x * kT, by = tile_y * kT;
  float* out = hiz + (size_t)view * hz.per_view;
  int n = kT;
  const int top = min(hz.levels - 1, tile_levels<kT>());
  // a level has at most (kT / 2)^2 outputs: with >= 128 threads each thread owns at most kPer
  constexpr int kPer = ((kT / 2) * (kT / 2) + 127) / 128;
  for (int l = 1; l <= top; ++l) {
    n >>= 1;
    float m[kPer];
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int k = threadIdx.x + j * blockDim.x;
      m[j] = INFINITY;
      if (k < n * n) {
        const int ty = k / n, tx = k % n;
        m[j] = fminf(fminf(s[2 * ty][2 * tx], s[2 * ty][2 * tx + 1]), fminf(s[2 * ty + 1][2 * tx], s[2 * ty + 1][2 * tx + 1]));
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int k = threadIdx.x + j * blockDim.x;
      if (k < n * n) {
        const int ty = k / n, tx = k % n;
        s[ty][tx] = m[j];
        const int gy = (by >> l) + ty, gx = (bx >> l) + tx;
        if (gy < hz.h[l] && gx < hz.w[l]) out[hz.off[l] + gy * hz.w[l] + gx] = m[j];
      }
    }
    __syncthreads();
  }
  (void)H;
  (void)W;
}

// Block-level: loads the tile of depth and reduces it (hiz_tile_reduce).
template <int kT>
__device__ __forceinline__ void hiz_tile_block(const float* __restrict__ depth, int H, int W, const HizInfo& hz,
                                               float* __restrict__ hiz, int view, int tile_x, int tile_y,
                                               TileBufT<kT>& s) {
  const int bx = tile_x * kT, by = tile_y * kT;
  const float* d0 = depth + (size_t)view * H * W;
  for (int k = threadIdx.x; k < kT * kT; k += blockDim.x) {
    const int ty = k / kT, tx = k % kT;
    const int y = by + ty, x = bx + tx;
    s[ty][tx] = (y < H && x < W) ? __ldg(d0 + (size_t)y * W + x) : INFINITY;
  }
  __syncthreads();
  hiz_tile_reduce<kT>(H, W, hz, hiz, view, tile_x, tile_y, s);
}

__device__ __forceinline__ void hiz_level_item(const HizInfo& hz, int l, float* __restrict__ hiz, int t) {
  const int w = hz.w[l], h = hz.h[l];
  const int view = t / (w * h), rem = t % (w * h);
  const int i = rem / w, j = rem % w;
  const float* src = hiz + (size_t)view * hz.per_view + hz.off[l - 1];
  const int ws = hz.w[l - 1], hs = hz.h[l - 1];
  float m = __ldcg(src + (2 * i) * ws + 2 * j);
  if (2 * j + 1 < ws) m = fminf(m, __ldcg(src + (2 * i) * ws + 2 * j + 1));
  if (2 * i + 1 < hs) {
    m = fminf(m, __ldcg(src + (2 * i + 1) * ws + 2 * j));
    if (2 * j + 1 < ws) m = fminf(m, __ldcg(src + (2 * i + 1) * ws + 2 * j + 1));
  }
  hiz[(size_t)view * hz.per_view + hz.off[l] + rem] = m;
}

// Block-level: a kT x kT texel tile of the base environment level (tiles are exact: the sizes
// are powers of two) copied into level 0 of the chain and reduced through level log2 kT in
// shared memory, one channel at a time, with env_down_item's arithmetic.
template <int kT>
__device__ __forceinline__ void env_tile_block(const float* __restrict__ env0, const EnvInfo& e, float* mips,
                                               int tile_x, int tile_y, TileBufT<kT>& s) {
  const int w0 = e.w[0];
  const int th = min(kT, e.h[0]), tw = min(kT, w0);
  const int by = tile_y * th, bx = tile_x * tw;
  for (int k = threadIdx.x; k < th * tw * 3; k += blockDim.x) {
    const size_t o = ((size_t)(by + k / (tw * 3)) * w0 + bx) * 3 + k % (tw * 3);
    mips[e.off[0] + o] = __ldg(env0 + o);
  }
  const int top = min(e.levels - 1, tile_levels<kT>());
  constexpr int kPer = ((kT / 2) * (kT / 2) + 127) / 128;
  for (int c = 0; c < 3; ++c) {
    __syncthreads();
    for (int k = threadIdx.x; k < th * tw; k += blockDim.x)
      s[k / tw][k % tw] = __ldg(env0 + ((size_t)(by + k / tw) * w0 + bx + k % tw) * 3 + c);
    __syncthreads();
    int nh = th, nw = tw;
    for (int l = 1; l <= top; ++l) {
      nh >>= 1;
      nw >>= 1;
      float m[kPer];
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int k = threadIdx.x + j * blockDim.x;
        m[j] = 0.0f;
        if (k < nh * nw) {
          const int i = k / nw, q = k % nw;
          m[j] = env_avg4(s[2 * i][2 * q], s[2 * i][2 * q + 1], s[2 * i + 1][2 * q], s[2 * i + 1][2 * q + 1]);
        }
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        const int k = threadIdx.x + j * blockDim.x;
        if (k < nh * nw) {
          const int i = k / nw, q = k % nw;
          s[i][q] = m[j];
          mips[e.off[l] + ((size_t)((by >> l) + i) * e.w[l] + (bx >> l) + q) * 3 + c] = m[j];
        }
      }
      __syncthreads();
    }
  }
}

// Block-level: environment levels `from`.. from level from - 1 (which is complete).
__device__ __forceinline__ void env_upper_block(const EnvInfo& e, float* mips, int from = 6) {
  for (int l = from; l < e.levels; ++l) {
    for (int t = threadIdx.x; t < e.h[l] * e.w[l] * 3; t += blockDim.x)
      env_down_item(mips + e.off[l - 1], e.h[l - 1], e.w[l - 1], mips + e.off[l], t);
    __threadfence();
    __syncthreads();
  }
}

// Block-level: Hi-Z levels `from`.. of one view from its level from - 1 (which is complete).
__device__ __forceinline__ void hiz_upper_block(const HizInfo& hz, int view, float* hiz, int from = 6) {
  for (int l = from; l < hz.levels; ++l) {
    const int n = hz.w[l] * hz.h[l];
    for (int t = threadIdx.x; t < n; t += blockDim.x) hiz_level_item(hz, l, hiz, view * n + t);
    __threadfence();
    __syncthreads();
  }
}

// ==========================================================================================
// Direct shading (Sec. 3.2)
// ==========================================================================================
// Direct shading of pixel p (flat index over [V,H,W]).
__device__ __forceinline__ void shade_pixel(const FrameArgs& A, long long p) {
  const Views& vs = A.vs;
  const EnvInfo& e = A.e;
  const long long HW = (long long)vs.H * vs.W;
  const int view = (int)(p / HW);
  const int rem = (int)(p - (long long)view * HW);
  const int y = rem / vs.W, x = rem - (rem / vs.W) * vs.W;
  const DevCam& cam = vs.cam[view];
  const float3 d = pix_dir_world(cam, x, y);
  const float z = __ldg(A.depth + p);
  float3 od = f3(0.f, 0.f, 0.f), os = f3(0.f, 0.f, 0.f), o1;
  if (is_background(z)) {
    o1 = env_lookup0(A.mips, e, d);
  } else {
    const float3 v = view_vector(d);
    const float3 n = ld3(A.normal + 3 * p);
    const float nv = dot3_rn(n, v);
    const float mu = fminf(fmaxf(nv, 1e-4f), 1.0f);
    const float3 r = reflect_about(n, nv, v);
    const float rho = __ldg(A.rough + p), m = __ldg(A.metal + p);
    const float lam = log2f(rho + 1.0f) * (float)(e.levels - 1);
    const LutVal ab = lut_sample(A.lut, A.lut_n, rho, mu);
    const float3 Er = env_lookup(A.mips, e, r, lam);
    const float3 En = env_lookup(A.mips, e, n, lam);
    const float3 a = ld3(A.albedo + 3 * p);
    const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
    os = mul3(Er, F0 * ab.A + f3(ab.B, ab.B, ab.B));
    od = mul3(a * (1.0f - m), En);
    o1 = od + os;
  }
  st3(A.c_d + 3 * p, od);
  if (A.c_s) st3(A.c_s + 3 * p, os);
  st3(A.c1 + 3 * p, o1);
}


// ==========================================================================================
// Output transform: tone mapping + gamma to sRGB after the composite (Sec. 3.3): clamp to
// [0, 1], then the sRGB transfer function (IEC 61966-2-1).
// ==========================================================================================
// x^(1/2.4) through CUDA's fast __powf: its error grows with |y log2 x|, here at most 3.5, and
// the transfer function's tests bound the encoded value's error by 4e-7 on [0, 1]; it costs the
// trace's epilogue less than half of what powf does.
__device__ __forceinline__ float tonemap_srgb(float x) {
  x = fminf(fmaxf(x, 0.0f), 1.0f);
  return x <= 0.0031308f ? 12.92f * x : fmaf(1.055f, __powf(x, 1.0f / 2.4f), -0.055f);
}

// The display encoding of one RGB value, out of line: the trace's epilogue calls it once per
// pixel, and inlined its transfer function measured 2.5 % slower in the trace's march.
static __device__ __noinline__ float3 tonemap3_srgb(float3 v) {
  return f3(tonemap_srgb(v.x), tonemap_srgb(v.y), tonemap_srgb(v.z));
}

// d tonemap_srgb / dx: 0 outside [0, 1].
__device__ __forceinline__ float tonemap_srgb_slope(float x) {
  if (!(x >= 0.0f && x <= 1.0f)) return 0.0f;
  return x <= 0.0031308f ? 12.92f : (1.055f / 2.4f) * powf(x, 1.0f / 2.4f - 1.0f);
}

// ==========================================================================================
// Trace (Sec. 3.3, Appendix D)
// ==========================================================================================
// Per-level base pointer and row width of the pyramid of one view, level 0 being the depth
// buffer itself, so that the march reads every level through the same code (shared memory,
// filled by the block for the view it traces).
struct __align__(16) LevelEntry {  // one 16-byte shared-memory load per march iteration
  const float* base;
  int w, pad;
};
struct LevelTable {
  LevelEntry lv[SSGI_MAX_HIZ_LEVELS];
};

// Block-level part: threads 0..SSGI_MAX_HIZ_LEVELS-1 fill the table; the caller synchronises.
__device__ __forceinline__ void fill_levels(const FrameArgs& A, int view, LevelTable& t) {
  const int l = threadIdx.x;
  if (l < SSGI_MAX_HIZ_LEVELS) {
    const long long HW = (long long)A.vs.H * A.vs.W;
    t.lv[l].base = l == 0 ? A.depth + view * HW
                          : (A.hiz && l < A.hz.levels ? A.hiz + (long long)view * A.hz.per_view + A.hz.off[l] : nullptr);
    t.lv[l].w = l == 0 ? A.vs.W : A.hz.w[l];
    t.lv[l].pad = 0;
  }
}

// One ray's march state.  The segment constants give the exit parameter of a cell edge bx as
// s_x = bx * iDx + ox (iDx = 0, ox = +inf when the segment has no x extent).  Depth is handled
// as k = 1/z, which is linear in the screen parameter, and the tests are written on k:
//   z_hi < hz          <=>  k_min * hz > 1
//   z_lo <= hz + thick <=>  k_max * (hz + thick) >= 1
// (k > 0 on the clipped segment), so an iteration has no division; ka caches k at the cell
// entry.
struct Ray {
  float P0x, P0y, Dx, Dy, iDx, iDy, ox, oy, k0, dk, ka;
  int ix, iy, L, sgx, sgy;
};

// Exit parameters of the level-L cell holding (ix, iy).
__device__ __forceinline__ void exits(const Ray& r, float& sx, float& sy) {
  sx = fmaf((float)(((r.ix >> r.L) + r.sgx) << r.L), r.iDx, r.ox);
  sy = fmaf((float)(((r.iy >> r.L) + r.sgy) << r.L), r.iDy, r.oy);
}

// Enter the pixel across the exit side of the level-L cell (ties go to x), on the row (column)
// of the exit point clamped to the cell.
// Written with selects instead of a branch on the exit side: lanes of a warp that leave their
// cells through different sides do not diverge here.
__device__ __forceinline__ void step_out(Ray& r, float sx, float sy) {
  const int lo_x = (r.ix >> r.L) << r.L, lo_y = (r.iy >> r.L) << r.L;
  const int S1 = (1 << r.L) - 1;
  const bool xe = sx <= sy;
  // the coordinate along the side that is not crossed, at the exit point, clamped to the cell
  const int f = __float2int_rd(xe ? fmaf(sx, r.Dy, r.P0y) : fmaf(sy, r.Dx, r.P0x));
  const int lo_o = xe ? lo_y : lo_x;
  const int along = min(max(f, lo_o), lo_o + S1);
  // the crossed coordinate: the first pixel beyond the cell
  const int lo_m = xe ? lo_x : lo_y;
  const int across = (xe ? r.sgx : r.sgy) ? lo_m + S1 + 1 : lo_m - 1;
  r.ix = xe ? across : along;
  r.iy = xe ? along : across;
}

// March from pixel (x, y) at linear depth z0 (k0 = 1/z0) along camera-space direction w.
// Returns the hit pixel's index within the view, or SSGI_HIT_MISS; `it` gets the iterations.
__device__ __forceinline__ int march(const FrameArgs& A, const DevCam& c, const LevelTable& lt, int levels,
                                     int max_steps, int x, int y,
                                     float z0, float k0, float3 w, int& it) {
  const int H = A.vs.H, W = A.vs.W;
  it = 0;
  const float3 o = pix_dir_cam(c, x, y) * z0;
  const float wz = -w.z;
  float t_end = A.max_distance;
  if (wz < 0.0f) t_end = fminf(t_end, (c.znear - z0) / wz);
  if (!(t_end > 0.0f)) return SSGI_HIT_MISS;
  const float3 X1 = o + w * t_end;
  const float z1 = -X1.z;
  Ray r;
  r.P0x = (float)x + 0.5f;
  r.P0y = (float)y + 0.5f;
  r.Dx = (c.cx + c.f * X1.x / z1) - r.P0x;
  r.Dy = (c.cy - c.f * X1.y / z1) - r.P0y;
  r.iDx = r.Dx != 0.0f ? 1.0f / r.Dx : 0.0f;
  r.iDy = r.Dy != 0.0f ? 1.0f / r.Dy : 0.0f;
  r.ox = r.Dx != 0.0f ? -r.P0x * r.iDx : INFINITY;
  r.oy = r.Dy != 0.0f ? -r.P0y * r.iDy : INFINITY;
  r.sgx = r.Dx > 0.0f ? 1 : 0;
  r.sgy = r.Dy > 0.0f ? 1 : 0;
  r.k0 = k0;
  r.dk = 1.0f / z1 - k0;
  r.ix = x;
  r.iy = y;
  r.L = 0;
  float sx, sy;
  exits(r, sx, sy);  // leave the origin pixel untested
  const float s0 = fminf(sx, sy);
  if (!(s0 < 1.0f)) return SSGI_HIT_MISS;
  step_out(r, sx, sy);
  r.ka = fmaf(s0, r.dk, r.k0);
  const float thick = A.thickness;
  // off screen is checked where the position changes: after leaving a cell, not after refining
  if ((unsigned)r.ix >= (unsigned)W || (unsigned)r.iy >= (unsigned)H) return SSGI_HIT_MISS;

  // The loop is exits() and step_out() written out on the cell's corner and exit edges, which
  // gives the same integers and floats with fewer integer operations (the march is bound by
  // the ALU pipe): with cs = 2^L and ix >= 0, (ix >> L) << L = ix & -cs, the exit edge
  // ((ix >> L) + sgx) << L = lo_x + sgx cs, the pixel across it is that edge + sgx - 1, and
  // the cell's pyramid index (iy >> L) w + (ix >> L) = (lo_y w + lo_x) >> L exactly (a sum of
  // multiples of cs; lo_y w < 2^28 by the size limits).
  for (;;) {
    if (it >= max_steps) return SSGI_HIT_MISS;
    ++it;
    const int cs = 1 << r.L;
    const int lo_x = r.ix & -cs, lo_y = r.iy & -cs;
    const int bx = lo_x + r.sgx * cs, by = lo_y + r.sgy * cs;
    const float sx = fmaf((float)bx, r.iDx, r.ox);
    const float sy = fmaf((float)by, r.iDy, r.oy);
    const float se = fminf(sx, sy);
    const float kb = fmaf(fminf(se, 1.0f), r.dk, r.k0);
    const float kmin = fminf(r.ka, kb), kmax = fmaxf(r.ka, kb);
    // one load for every level (level 0 is the depth buffer itself)
    const LevelEntry le = lt.lv[r.L];
    const float hzv = __ldg(le.base + ((lo_y * le.w + lo_x) >> r.L));
    const bool skip = kmin * hzv > 1.0f;
    if (!skip) {
      if (r.L > 0) {  // something in this cell may be hit: refine
        --r.L;
        continue;
      }
      if (kmax * (hzv + thick) >= 1.0f) return r.iy * W + r.ix;
    }
    // leave the cell: skipped at any level, or passed behind a level-0 pixel (one code path for
    // both, so a warp whose lanes do either runs it once)
    if (!(se < 1.0f)) return SSGI_HIT_MISS;  // the cell holds the end of the segment
    const bool xe = sx <= sy;
    const int f = __float2int_rd(xe ? fmaf(sx, r.Dy, r.P0y) : fmaf(sy, r.Dx, r.P0x));
    const int lo_o = xe ? lo_y : lo_x;
    const int along = min(max(f, lo_o), lo_o + cs - 1);
    const int across = xe ? bx + r.sgx - 1 : by + r.sgy - 1;
    r.ix = xe ? across : along;
    r.iy = xe ? along : across;
    r.ka = kb;
    r.L = min(r.L + (int)skip, levels - 1);  // up a level after a skip, up to the top
    if ((unsigned)r.ix >= (unsigned)W || (unsigned)r.iy >= (unsigned)H) return SSGI_HIT_MISS;
  }
}

// Trace all samples of pixel (x, y) of `view`: GGX sampling, march, gather, Monte-Carlo sum
// and composite (one thread per pixel).  kSrgb: the output transform as the epilogue (its own
// instantiation: with it off the kernel carries no trace of it, which measured 6 % faster than
// a run-time test; with it on the trace takes ~1 % longer than the linear trace plus the
// separate 13-17 us pass, so the epilogue is for callers that want one launch, not for speed).
template <bool kCid, bool kSrgb = false>
__device__ __forceinline__ float3 trace_pixel(const FrameArgs& A, int x, int y, int view, const LevelTable& lt) {
  const int W = A.vs.W, H = A.vs.H;
  const long long HW = (long long)H * W;
  const int rem = y * W + x;
  const long long p = (long long)view * HW + rem;
  const int spp = A.spp;
  const float z0 = __ldg(A.depth + p);
  if (is_background(z0)) {
    const float3 v1 = ld3(A.c1 + 3 * p);
    st3(A.final_out + 3 * p, kSrgb ? tonemap3_srgb(v1) : v1);
    if (A.c_s_mc) st3(A.c_s_mc + 3 * p, f3(0.f, 0.f, 0.f));
    if (A.c_id) st3(A.c_id + 3 * p, f3(0.f, 0.f, 0.f));
    if (A.hit_idx)
      for (int s = 0; s < spp; ++s) A.hit_idx[p * spp + s] = SSGI_HIT_BACKGROUND;
    return v1;
  }
  const DevCam& cam = A.vs.cam[view];
  const bool brute = (A.flags & SSGI_BRUTE_FORCE) != 0;
  const int levels = brute ? 1 : A.levels;
  const int max_steps = brute ? INT_MAX : A.max_steps;

  const float3 d = pix_dir_world(cam, x, y);
  const float3 v = view_vector(d);
  const float3 n = ld3(A.normal + 3 * p);
  const float nv = dot3(n, v);  // weights and validity only (no direction): the compiler's own form
  const float rho = __ldg(A.rough + p), m = __ldg(A.metal + p);
  const float3 a = ld3(A.albedo + 3 * p);
  const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
  const float g1v = ggx_G1(nv, rho);
  const float k0 = 1.0f / z0;
  float3 acc = f3(0.f, 0.f, 0.f), accd = f3(0.f, 0.f, 0.f);
  unsigned long long steps = 0;

  for (int s = 0; s < spp; ++s) {
    const float2 xi = sample_uniforms(A.seed, view, (uint32_t)rem, (uint32_t)s);
    const Sample sm = make_sample(n, v, nv, rho, xi);
    int q = SSGI_HIT_INVALID;
    if (sm.valid) {
      int it;
      q = march(A, cam, lt, levels, max_steps, x, y, z0, k0, world_to_cam(cam, sm.w), it);
      steps += (unsigned long long)it;
      const float3 Li = q >= 0 ? ld3(A.c1 + 3 * (view * HW + q)) : env_lookup0_trace(A.mips, A.e, sm.w);
      const float K = ggx_G1(sm.nw, rho) * g1v * sm.vh / (nv * sm.nh);
      const float fc = pow5(1.0f - sm.vh);
      const float3 F = F0 + (f3(1.f, 1.f, 1.f) - F0) * fc;
      acc = acc + mul3(F, Li) * K;
      if (kCid) {
        const float pdf = ggx_D_sampled(sm.ds, rho) * sm.nh / (4.0f * sm.vh);
        if (pdf > 0.0f && isfinite(pdf)) accd = accd + mul3(a, Li) * ((1.0f - m) * kInvPi * sm.nw / pdf);
      }
    }
    if (A.hit_idx) A.hit_idx[p * spp + s] = q;
  }
  const float fs = (float)spp;
  const float3 csm = f3(acc.x / fs, acc.y / fs, acc.z / fs);
  const float3 cid = f3(accd.x / fs, accd.y / fs, accd.z / fs);
  float3 fin = ld3(A.c_d + 3 * p) + csm;
  if (kCid) fin = fin + cid;
  // the output transform as an epilogue: the display image leaves the kernel already encoded
  st3(A.final_out + 3 * p, kSrgb ? tonemap3_srgb(fin) : fin);
  if (A.c_s_mc) st3(A.c_s_mc + 3 * p, csm);
  if (A.c_id) st3(A.c_id + 3 * p, cid);
  if (A.step_count && steps) atomicAdd(A.step_count, steps);
  return fin;
}

// ==========================================================================================
// Backward (replay adjoint) and L2 loss
// ==========================================================================================
// Adds v to the RGB of *p (w unused), summing first over the lanes of the warp that add to the
// same address; one 16-byte vector atomic per distinct address.
__device__ __forceinline__ void atomic_add4(float4* p, float3 v) {
  const unsigned act = __activemask();
  const unsigned grp = __match_any_sync(act, (unsigned long long)p);
  const int lane = threadIdx.x & 31;
  if (grp == 0xffffffffu) {
    // the whole warp adds to one texel (coarse mip levels): butterfly sum, one atomic per channel
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
      v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
      v.z += __shfl_xor_sync(0xffffffffu, v.z, o);
    }
    if (lane == 0) atomicAdd(p, make_float4(v.x, v.y, v.z, 0.0f));
    return;
  }
  // lanes sharing an address form a list in lane order; pointer jumping doubles the span of
  // each lane's suffix sum per step, so the group's first lane holds the total after at most
  // five steps whatever the grouping
  int nxt = __ffs(grp & ((0xffffffffu << lane) << 1)) - 1;
  while (__any_sync(act, nxt >= 0)) {
    const int src = nxt >= 0 ? nxt : lane;
    const float tx = __shfl_sync(act, v.x, src), ty = __shfl_sync(act, v.y, src), tz = __shfl_sync(act, v.z, src);
    const int nn = __shfl_sync(act, nxt, src);
    if (nxt >= 0) {
      v = v + f3(tx, ty, tz);
      nxt = nn;
    }
  }
  if (lane == __ffs(grp) - 1) atomicAdd(p, make_float4(v.x, v.y, v.z, 0.0f));
}

// d ln G1(z; rho) / dz, / drho.  The adjoint's own quotients use the approximate division
// (__fdividef, 2 ulp): the gradients are compared at 1e-3, and it measured 3.4 % faster.
// Anything that shapes a direction, a hit or the forward's radiance keeps IEEE division.
__device__ __forceinline__ void dlnG1(float z, float rho, float& dz, float& dr) {
  const float a2 = rho * rho;
  const float s = sqrtf(a2 + (1.0f - a2) * z * z);
  const float izs = __fdividef(1.0f, z + s), is = __fdividef(1.0f, s);
  dz = __fdividef(1.0f, z) - (1.0f + (1.0f - a2) * z * is) * izs;
  dr = -(rho * (1.0f - z * z) * is) * izs;
}

// d ln D(c; rho) / dc, / drho with c = n.h, at a half vector drawn by ggx_sample_h with
// denominator ds (1 + c^2 (rho^2 - 1) = rho^2 / ds there, see ggx_D_sampled):
//   dc = -4 c (rho^2 - 1) / (1 + c^2 (rho^2 - 1)),  dr = 2 / rho - 4 rho c^2 / (1 + c^2 (rho^2 - 1)).
__device__ __forceinline__ void dlnD(float c, float ds, float rho, float& dc, float& dr) {
  const float q = __fdividef(ds, rho * rho);  // 1 / (1 + c^2 (rho^2 - 1))
  dc = 4.0f * c * (1.0f - rho * rho) * q;
  dr = __fdividef(2.0f, rho) - 4.0f * rho * c * c * q;
}

// Scatter g (per channel) with weight `scale` through the bilinear taps into gm, and return
// the derivatives of the bilinear value contracted with g along x and y (texel units).
// Plain 16-byte atomic add of v to the RGB of *p.
__device__ __forceinline__ void atomic_add4_plain(float4* p, float3 v) {
  atomicAdd(p, make_float4(v.x, v.y, v.z, 0.0f));
}

// aggregate: sum over the warp's lanes that share a texel first (atomic_add4).  Worth it where
// many lanes land on one texel (the coarse levels of the direct adjoint); where they rarely do
// (mip 0 under scattered directions) the matching costs more than it saves.
__device__ __forceinline__ void bilin_adj(const float* __restrict__ mips, const Taps& t, float3 g, float scale,
                                          float4* gm, float& gx, float& gy, bool aggregate = true) {
  const float3 a = ld3(mips + t.idx[0]), b = ld3(mips + t.idx[1]);
  const float3 c = ld3(mips + t.idx[2]), d = ld3(mips + t.idx[3]);
  gx = dot3(g, (b - a) * (1.0f - t.ty) + (d - c) * t.ty);
  gy = dot3(g, (c - a) * (1.0f - t.tx) + (d - b) * t.tx);
  if (scale != 0.0f) {
    const float w00 = (1.0f - t.tx) * (1.0f - t.ty), w01 = t.tx * (1.0f - t.ty);
    const float w10 = (1.0f - t.tx) * t.ty, w11 = t.tx * t.ty;
    // tap offsets count floats of the packed RGB chain (3 per texel); gm holds one float4 per texel
    if (aggregate) {
      atomic_add4(gm + t.idx[0] / 3, g * (scale * w00));
      atomic_add4(gm + t.idx[1] / 3, g * (scale * w01));
      atomic_add4(gm + t.idx[2] / 3, g * (scale * w10));
      atomic_add4(gm + t.idx[3] / 3, g * (scale * w11));
    } else {
      atomic_add4_plain(gm + t.idx[0] / 3, g * (scale * w00));
      atomic_add4_plain(gm + t.idx[1] / 3, g * (scale * w01));
      atomic_add4_plain(gm + t.idx[2] / 3, g * (scale * w10));
      atomic_add4_plain(gm + t.idx[3] / 3, g * (scale * w11));
    }
  }
}

// Adjoint of SampleEnvMap(d, lambda): texel gradients into gm (all levels), returns d/dd and
// d/dlambda (zero where lambda is clamped).
__device__ __forceinline__ float3 env_lookup_adj(const float* __restrict__ mips, const EnvInfo& e, float3 d,
                                                 float lam, float3 g, float4* gm, float& glam, bool aggregate = true) {
  const float lmax = (float)(e.levels - 1);
  const bool inside = lam > 0.0f && lam < lmax;
  lam = fminf(fmaxf(lam, 0.0f), lmax);
  const int l0 = (int)floorf(lam);
  const int l1 = min(l0 + 1, e.levels - 1);
  const float t = lam - (float)l0;
  const DirAngles ang = dir_angles(d);
  const Taps t0 = env_taps(e, l0, ang), t1 = env_taps(e, l1, ang);
  float gx0, gy0, gx1 = 0.0f, gy1 = 0.0f;
  bilin_adj(mips, t0, g, 1.0f - t, gm, gx0, gy0, aggregate);
  if (t != 0.0f) bilin_adj(mips, t1, g, t, gm, gx1, gy1, aggregate);
  const float gu = (1.0f - t) * gx0 * (float)e.w[l0] + t * gx1 * (float)e.w[l1];
  const float gv = (1.0f - t) * gy0 * (float)e.h[l0] + t * gy1 * (float)e.h[l1];
  glam = 0.0f;
  if (inside && l1 != l0) glam = dot3(g, bilinear(mips, t1) - bilinear(mips, t0));
  const float q2 = d.x * d.x + d.z * d.z;
  if (!(q2 > 0.0f)) return f3(0.f, 0.f, 0.f);
  const float q = sqrtf(q2);
  const float r2 = q2 + d.y * d.y;
  const float iq2 = __fdividef(kInv2Pi, q2), iqr = __fdividef(kInvPi, q * r2);
  const float dux = -d.z * iq2, duz = d.x * iq2;
  const float dvx = d.y * d.x * iqr, dvz = d.y * d.z * iqr, dvy = __fdividef(-q * kInvPi, r2);
  return f3(gu * dux + gv * dvx, gv * dvy, gu * duz + gv * dvz);
}

// Adjoint of one receiver pixel's Monte-Carlo sum.  kPathwise = false: replay (direction and
// pdf frozen; d/d{n, rho} of f_s (n.w) / p_frozen).  kPathwise = true: the direction is a
// function of (n, rho) at frozen uniforms (ggx_sample_h_jac), the weight is the cancelled
// F G1 G1 (v.h) / ((n.v)(n.h)) and a miss's radiance follows the direction through the map.
// kOwn: the calling thread traced this pixel itself (the fused step's trace item), so its hit
// indices are read with ordinary loads (not the read-only path) and dL/dfinal comes in g_own.
template <bool kPathwise, bool kOwn = false>
__device__ __forceinline__ void bwd_mc_pixel(const FrameArgs& A, long long p, float3 g_own = float3{}) {
  const long long HW = (long long)A.vs.H * A.vs.W;
  const int view = (int)(p / HW);
  const int rem = (int)(p - view * HW);
  const int y = rem / A.vs.W, x = rem - y * A.vs.W;
  float3 ga = f3(0.f, 0.f, 0.f), gn = f3(0.f, 0.f, 0.f);
  float gr = 0.0f, gm = 0.0f;
  const float z = __ldg(A.depth + p);
  if (!is_background(z)) {
    const DevCam& cam = A.vs.cam[view];
    const float3 d = pix_dir_world(cam, x, y);
    const float3 v = view_vector(d);
    const float3 n = ld3(A.normal + 3 * p);
    const float nv = dot3(n, v);  // weights and validity only (no direction): the compiler's own form
    const float rho = __ldg(A.rough + p), m = __ldg(A.metal + p);
    const float3 a = ld3(A.albedo + 3 * p);
    const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
    const float3 gC = (kOwn ? g_own : ld3(A.g_final + 3 * p)) * (1.0f / (float)A.spp);
    const float g1v = ggx_G1(nv, rho);
    float dgv_z, dgv_r;
    dlnG1(nv, rho, dgv_z, dgv_r);
    const bool want_cid = (A.flags & SSGI_DIFFUSE_INDIRECT) != 0;
    for (int s = 0; s < A.spp; ++s) {
      const float2 xi = sample_uniforms(A.seed, view, (uint32_t)rem, (uint32_t)s);
      const Sample sm = make_sample(n, v, nv, rho, xi);
      const int q = kOwn ? A.hit_idx[p * A.spp + s] : __ldg(A.hit_idx + p * A.spp + s);
      // the forward's verdict on validity decides (n.v and n.w here may round differently)
      if (!sm.valid || q == SSGI_HIT_INVALID) continue;
      if (q >= HW) continue;  // not an index this G-buffer's trace can produce
      float3 Li;
      Taps tm;
      if (q >= 0) {
        Li = ld3(A.c1 + 3 * (view * HW + q));
      } else {
        tm = env_taps(A.e, 0, dir_angles(sm.w));
        Li = bilinear(A.mips, tm);
      }
      const float K = __fdividef(ggx_G1(sm.nw, rho) * g1v * sm.vh, nv * sm.nh);
      const float fc = pow5(1.0f - sm.vh);
      const float3 F = F0 + (f3(1.f, 1.f, 1.f) - F0) * fc;
      float3 gL = mul3(gC, F) * K;
      const float3 gF = mul3(gC, Li) * K;
      ga = ga + gF * (m * (1.0f - fc));
      gm += dot3(gF, a - f3(0.04f, 0.04f, 0.04f)) * (1.0f - fc);
      const float gKK = dot3(gC, mul3(F, Li)) * K;
      float dgw_z, dgw_r;
      dlnG1(sm.nw, rho, dgw_z, dgw_r);
      float dd_c = 0.0f, dd_r = 0.0f;
      if (rho > 0.0f) dlnD(sm.nh, sm.ds, rho, dd_c, dd_r);
      if (!kPathwise) {
        float dlnK_r = dgw_r + dgv_r;
        float3 dlnK_n = sm.w * dgw_z + v * (dgv_z - 1.0f / nv);
        if (rho > 0.0f) {
          dlnK_r += dd_r;
          dlnK_n = dlnK_n + sm.h * dd_c;
        }
        gr += gKK * dlnK_r;
        gn = gn + dlnK_n * gKK;
      }
      float gcid = 0.0f;  // d loss / d ln(n.w / pdf) of the diffuse-indirect summand
      if (want_cid) {
        const float pdf = ggx_D_sampled(sm.ds, rho) * sm.nh / (4.0f * sm.vh);
        if (pdf > 0.0f && isfinite(pdf)) {
          const float kk = kInvPi / pdf;
          ga = ga + mul3(gC, Li) * ((1.0f - m) * kk * sm.nw);
          gm -= dot3(gC, mul3(a, Li)) * kk * sm.nw;
          if (!kPathwise) gn = gn + sm.w * (dot3(gC, mul3(a, Li)) * (1.0f - m) * kk);
          gL = gL + mul3(gC, a) * ((1.0f - m) * kk * sm.nw);
          gcid = dot3(gC, mul3(a, Li)) * (1.0f - m) * kk * sm.nw;
        }
      }
      float3 gdir = f3(0.f, 0.f, 0.f);  // d loss / d w through a miss's lookup
      if (q >= 0) {
        // receivers' hits land on scattered pixels and misses on scattered mip-0 texels: no
        // warp aggregation in this kernel (see bilin_adj)
        atomic_add4_plain(A.g_c1 + (view * HW + q), gL);
      } else if (kPathwise) {
        float glam;
        gdir = env_lookup_adj(A.mips, A.e, sm.w, 0.0f, gL, A.g_mips, glam, false);
      } else {
        float gx, gy;
        bilin_adj(A.mips, tm, gL, 1.0f, A.g_mips, gx, gy, false);
      }
      if (kPathwise) {
        // total derivative through h(n, rho), w = 2 (v.h) h - v and the dot products
        float3 dh[4];
        ggx_sample_h_jac(n, rho, xi.x, xi.y, dh);
        const float om = 1.0f - sm.vh, om2 = om * om;
        const float gFdvh = -5.0f * om2 * om2 * dot3(mul3(gC, Li), f3(1.f, 1.f, 1.f) - F0) * K;
        float gth[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float dvh = dot3(v, dh[k]);
          const float3 dw = sm.h * (2.0f * dvh) + dh[k] * (2.0f * sm.vh);
          const float en_h = k == 0 ? sm.h.x : (k == 1 ? sm.h.y : (k == 2 ? sm.h.z : 0.0f));
          const float en_w = k == 0 ? sm.w.x : (k == 1 ? sm.w.y : (k == 2 ? sm.w.z : 0.0f));
          const float dnv = k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : 0.0f));
          const float dnh = dot3(n, dh[k]) + en_h;
          const float dnw = dot3(n, dw) + en_w;
          const float dr = k == 3 ? 1.0f : 0.0f;
          const float dlnK = dgw_z * dnw + dgv_z * dnv + (dgw_r + dgv_r) * dr + dvh / sm.vh - dnv / nv - dnh / sm.nh;
          float g = gKK * dlnK + gFdvh * dvh + dot3(gdir, dw);
          if (gcid != 0.0f) g += gcid * (dnw / sm.nw + dvh / sm.vh - dd_c * dnh - dd_r * dr - dnh / sm.nh);
          gth[k] = g;
        }
        gn = gn + f3(gth[0], gth[1], gth[2]);
        gr += gth[3];
      }
    }
  }
  st3(A.g_albedo + 3 * p, ga);
  st3(A.g_normal + 3 * p, gn);
  A.g_rough[p] = gr;
  A.g_metal[p] = gm;
}

__device__ __forceinline__ void bwd_direct_pixel(const FrameArgs& A, long long p) {
  const long long HW = (long long)A.vs.H * A.vs.W;
  const int view = (int)(p / HW);
  const int rem = (int)(p - view * HW);
  const int y = rem / A.vs.W, x = rem - y * A.vs.W;
  const DevCam& cam = A.vs.cam[view];
  const float3 d = pix_dir_world(cam, x, y);
  const float4 gq = __ldcg(A.g_c1 + p);  // written by atomics earlier: read through L2
  const float3 gc1 = f3(gq.x, gq.y, gq.z);
  const float3 gcd = ld3(A.g_final + 3 * p) + gc1;
  const float3 gcs = gc1;
  const float z = __ldg(A.depth + p);
  if (is_background(z)) {
    float gx, gy;
    bilin_adj(A.mips, env_taps(A.e, 0, dir_angles(d)), gcd, 1.0f, A.g_mips, gx, gy);
    return;
  }
  const float3 v = view_vector(d);
  const float3 n = ld3(A.normal + 3 * p);
  const float nv = dot3_rn(n, v);
  const float mu = fminf(fmaxf(nv, 1e-4f), 1.0f);
  const float3 r = reflect_about(n, nv, v);
  const float rho = __ldg(A.rough + p), m = __ldg(A.metal + p);
  const float lmax = (float)(A.e.levels - 1);
  const float lam = log2f(rho + 1.0f) * lmax;
  const LutVal ab = lut_sample(A.lut, A.lut_n, rho, mu);
  const float3 Er = env_lookup(A.mips, A.e, r, lam);
  const float3 En = env_lookup(A.mips, A.e, n, lam);
  const float3 a = ld3(A.albedo + 3 * p);
  const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
  const float3 ga = mul3(gcd, En) * (1.0f - m) + mul3(gcs, Er) * (ab.A * m);
  const float gm = -dot3(gcd, mul3(a, En)) + dot3(gcs, mul3(Er, a - f3(0.04f, 0.04f, 0.04f))) * ab.A;
  const float3 gEn = mul3(gcd, a) * (1.0f - m);
  const float3 gEr = mul3(gcs, F0 * ab.A + f3(ab.B, ab.B, ab.B));
  const float gA = dot3(gcs, mul3(Er, F0));
  const float gB = dot3(gcs, Er);
  float gl1, gl2;
  const float3 gdn = env_lookup_adj(A.mips, A.e, n, lam, gEn, A.g_mips, gl1);
  const float3 gdr = env_lookup_adj(A.mips, A.e, r, lam, gEr, A.g_mips, gl2);
  float gnv = 0.0f;
  if (nv > 1e-4f && nv < 1.0f) gnv = gA * ab.dA_dmu + gB * ab.dB_dmu;
  // r = 2 (n.v) n - v
  const float3 gn = gdn + v * (2.0f * dot3(gdr, n)) + gdr * (2.0f * nv) + v * gnv;
  const float gr = gA * ab.dA_drho + gB * ab.dB_drho + __fdividef((gl1 + gl2) * lmax, (rho + 1.0f) * 0.69314718055994531f);
  float* pa = A.g_albedo + 3 * p;
  float* pn = A.g_normal + 3 * p;
  st3(pa, ld3(pa) + ga);
  st3(pn, ld3(pn) + gn);
  A.g_rough[p] += gr;
  A.g_metal[p] += gm;
}

__device__ __forceinline__ void bwd_env_item(const EnvInfo& e, const float4* __restrict__ g_mips,
                                             float* __restrict__ g_env, int t) {
  const int w0 = e.w[0];
  const int c = t % 3, j = (t / 3) % w0, i = t / (3 * w0);
  const float* gm = reinterpret_cast<const float*>(g_mips);
  float acc = 0.0f, scale = 1.0f;
  for (int l = 0; l < e.levels; ++l) {
    // texel (i >> l, j >> l) of level l; e.off counts floats of the packed RGB chain
    acc += scale * __ldcg(gm + 4 * (e.off[l] / 3 + (i >> l) * e.w[l] + (j >> l)) + c);
    scale *= 0.25f;
  }
  g_env[t] = acc;
}

// Block-level: adds the block's sum of acc (one value per thread) times scale to *out.
__device__ __forceinline__ void block_sum_add(float acc, float* out, float scale) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
    atomicAdd(out, s * scale);
  }
  __syncthreads();
}

// The L2 loss term of one pixel's final colour (already in registers); returns |r|^2 and
// stores g = dL/dfinal (also returned in g).
__device__ __forceinline__ float l2_pixel(const FrameArgs& A, long long p, float3 fin, float inv, float3& g) {
  const float3 t = ld3(A.target + 3 * p);
  const float rx = fin.x - t.x, ry = fin.y - t.y, rz = fin.z - t.z;
  g = f3(2.0f * rx * inv, 2.0f * ry * inv, 2.0f * rz * inv);
  st3(A.g_final + 3 * p, g);
  return rx * rx + ry * ry + rz * rz;
}

// One element of the L2 loss: writes g and returns r^2 (kSrgb: against T(f), T = tonemap_srgb).
template <bool kSrgb>
__device__ __forceinline__ float l2_elem(float f, float t, float inv, float& g) {
  if (kSrgb) {
    const float r = tonemap_srgb(f) - t;
    g = 2.0f * r * tonemap_srgb_slope(f) * inv;
    return r * r;
  }
  const float r = f - t;
  g = 2.0f * r * inv;
  return r * r;
}

// Block-level (blockDim <= 256) L2 loss over n floats with 16-byte accesses (f, t and g
// 16-byte aligned when vec4 is set), the ragged tail element by element: g = d/df of the mean,
// loss += the mean.
template <bool kSrgb>
__device__ __forceinline__ void l2_block_vec(const float* __restrict__ f, const float* __restrict__ t, long long n,
                                             float* __restrict__ g, float* __restrict__ loss, bool vec4) {
  const float inv = 1.0f / (float)n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n4 = vec4 ? n / 4 : 0;
  float acc = 0.0f;
  for (long long i = t0; i < n4; i += stride) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(f) + i), b = __ldg(reinterpret_cast<const float4*>(t) + i);
    float4 o;
    acc += l2_elem<kSrgb>(a.x, b.x, inv, o.x);
    acc += l2_elem<kSrgb>(a.y, b.y, inv, o.y);
    acc += l2_elem<kSrgb>(a.z, b.z, inv, o.z);
    acc += l2_elem<kSrgb>(a.w, b.w, inv, o.w);
    reinterpret_cast<float4*>(g)[i] = o;
  }
  for (long long i = 4 * n4 + t0; i < n; i += stride) acc += l2_elem<kSrgb>(__ldg(f + i), __ldg(t + i), inv, g[i]);
  if (!loss) return;  // block-uniform
  block_sum_add(acc, loss, inv);
}

// The sRGB loss term of one pixel's final colour in registers; returns |r|^2 and stores (and
// returns in g) dL/dfinal.
__device__ __forceinline__ float l2_srgb_pixel(const FrameArgs& A, long long p, float3 fin, float inv, float3& g) {
  const float3 t = ld3(A.target + 3 * p);
  const float rx = tonemap_srgb(fin.x) - t.x, ry = tonemap_srgb(fin.y) - t.y, rz = tonemap_srgb(fin.z) - t.z;
  g = f3(2.0f * rx * tonemap_srgb_slope(fin.x) * inv, 2.0f * ry * tonemap_srgb_slope(fin.y) * inv,
         2.0f * rz * tonemap_srgb_slope(fin.z) * inv);
  st3(A.g_final + 3 * p, g);
  return rx * rx + ry * ry + rz * rz;
}

}  // namespace ssgi
