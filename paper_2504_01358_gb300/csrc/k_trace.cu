// k_trace.cu -- Monte-Carlo screen-space ray tracing for one-bounce indirect light
// (Sec. 3.3, Appendix D) with a conservative hierarchical-Z traversal, plus the Monte-Carlo
// sum and the composite final = c_d + c_s'.
//
// March definition: the ray o + t w is clipped to z >= z_near and t <= max_distance and
// projected to the screen segment P(s) = P0 + s D, s in [0, 1], along which 1/z is linear in
// s.  The state is a level-0 pixel (ix, iy) entered at parameter s and a level L.  Each
// iteration takes the level-L cell holding (ix, iy) and the ray's depth interval over
// [s, min(s_exit, 1)]:
//   entirely in front of the cell's minimum depth            -> skip the cell, go up a level;
//   otherwise, above level 0                                 -> go down a level;
//   at level 0, reaching no deeper than depth + thickness    -> hit (ix, iy);
//   at level 0 otherwise (passes behind)                     -> step to the next pixel.
// Leaving a cell through its x side (ties go to x) enters the pixel across that side, on
// the row of the exit point clamped to the cell's rows; symmetrically for y.  The origin
// pixel is left before the first iteration and is never a hit.  Off screen, past the end of
// the segment, or max_steps iterations without a hit is a miss.  The skip test is
// conservative, so the first hit is the one a pixel-by-pixel walk finds.
#include <limits.h>

#include "ssgi_device.cuh"

namespace ssgi {

struct TraceArgs {
  Views vs;
  EnvInfo e;
  HizInfo hz;
  const float* __restrict__ depth;
  const float* __restrict__ normal;
  const float* __restrict__ albedo;
  const float* __restrict__ rough;
  const float* __restrict__ metal;
  const float* __restrict__ hiz;
  const float* __restrict__ c1;
  const float* __restrict__ c_d;
  const float* __restrict__ mips;
  float* __restrict__ c_s_mc;
  float* __restrict__ c_id;
  float* __restrict__ final_out;
  int32_t* __restrict__ hit_idx;
  unsigned long long* step_count;
  int spp, max_steps, levels;
  float thickness, max_distance;
  uint64_t seed;
  uint32_t flags;
};

constexpr int kTileW = 8;   // a warp covers an 8 x 4 pixel tile
constexpr int kTileH = 16;  // a 128-thread block covers 8 x 16 pixels

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
__device__ __forceinline__ void step_out(Ray& r, float sx, float sy) {
  const int lo_x = (r.ix >> r.L) << r.L, lo_y = (r.iy >> r.L) << r.L;
  const int S1 = (1 << r.L) - 1;
  if (sx <= sy) {
    const int fy = __float2int_rd(fmaf(sx, r.Dy, r.P0y));
    r.iy = min(max(fy, lo_y), lo_y + S1);
    r.ix = r.sgx ? lo_x + S1 + 1 : lo_x - 1;
  } else {
    const int fx = __float2int_rd(fmaf(sy, r.Dx, r.P0x));
    r.ix = min(max(fx, lo_x), lo_x + S1);
    r.iy = r.sgy ? lo_y + S1 + 1 : lo_y - 1;
  }
}

// March from pixel (x, y) at linear depth z0 (k0 = 1/z0) along camera-space direction w.
// Returns the hit pixel's index within the view, or SSGI_HIT_MISS; `it` gets the iterations.
__device__ __forceinline__ int march(const TraceArgs& A, const DevCam& c, const float* __restrict__ dep,
                                     const float* __restrict__ hz_v, const int* __restrict__ s_hoff,
                                     const int* __restrict__ s_hw, int levels, int max_steps, int x, int y,
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

  for (;;) {
    if ((unsigned)r.ix >= (unsigned)W || (unsigned)r.iy >= (unsigned)H || it >= max_steps) return SSGI_HIT_MISS;
    ++it;
    exits(r, sx, sy);
    const float se = fminf(sx, sy);
    const float kb = fmaf(fminf(se, 1.0f), r.dk, r.k0);
    const float kmin = fminf(r.ka, kb), kmax = fmaxf(r.ka, kb);
    const float hzv = (r.L == 0) ? __ldg(dep + r.iy * W + r.ix)
                                 : __ldg(hz_v + s_hoff[r.L] + (r.iy >> r.L) * s_hw[r.L] + (r.ix >> r.L));
    if (kmin * hzv > 1.0f) {
      if (!(se < 1.0f)) return SSGI_HIT_MISS;  // the cell holds the end of the segment
      step_out(r, sx, sy);
      r.ka = kb;
      if (r.L + 1 < levels) ++r.L;
    } else if (r.L > 0) {
      --r.L;
    } else if (kmax * (hzv + thick) >= 1.0f) {
      return r.iy * W + r.ix;
    } else {
      if (!(se < 1.0f)) return SSGI_HIT_MISS;
      step_out(r, sx, sy);
      r.ka = kb;
    }
  }
}

// One thread per pixel, looping over its samples; a warp covers an 8 x 4 tile so that its
// rays start close together and touch the same pyramid cells.
template <bool kCid>
__global__ void __launch_bounds__(kTileW * kTileH, 8) k_trace(TraceArgs A) {
  __shared__ int s_hoff[SSGI_MAX_HIZ_LEVELS], s_hw[SSGI_MAX_HIZ_LEVELS];
  if (threadIdx.x < SSGI_MAX_HIZ_LEVELS) {
    s_hoff[threadIdx.x] = A.hz.off[threadIdx.x];
    s_hw[threadIdx.x] = A.hz.w[threadIdx.x];
  }
  __syncthreads();
  const int W = A.vs.W, H = A.vs.H;
  const int x = blockIdx.x * kTileW + (threadIdx.x % kTileW);
  const int y = blockIdx.y * kTileH + (threadIdx.x / kTileW);
  const int view = blockIdx.z;
  if (x >= W || y >= H) return;
  const long long HW = (long long)H * W;
  const int rem = y * W + x;
  const long long p = (long long)view * HW + rem;
  const int spp = A.spp;
  const float z0 = __ldg(A.depth + p);
  if (is_background(z0)) {
    const float3 v1 = ld3(A.c1 + 3 * p);
    st3(A.final_out + 3 * p, v1);
    if (A.c_s_mc) st3(A.c_s_mc + 3 * p, f3(0.f, 0.f, 0.f));
    if (A.c_id) st3(A.c_id + 3 * p, f3(0.f, 0.f, 0.f));
    if (A.hit_idx)
      for (int s = 0; s < spp; ++s) A.hit_idx[p * spp + s] = SSGI_HIT_BACKGROUND;
    return;
  }
  const DevCam& cam = A.vs.cam[view];
  const bool brute = (A.flags & SSGI_BRUTE_FORCE) != 0;
  const int levels = brute ? 1 : A.levels;
  const int max_steps = brute ? INT_MAX : A.max_steps;
  const float* dep = A.depth + view * HW;
  const float* hz_v = A.hiz ? A.hiz + (long long)view * A.hz.per_view : nullptr;

  const float3 d = pix_dir_world(cam, x, y);
  const float3 v = d * (-1.0f / sqrtf(dot3(d, d)));
  const float3 n = ld3(A.normal + 3 * p);
  const float nv = dot3(n, v);
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
      q = march(A, cam, dep, hz_v, s_hoff, s_hw, levels, max_steps, x, y, z0, k0, world_to_cam(cam, sm.w), it);
      steps += (unsigned long long)it;
      const float3 Li = q >= 0 ? ld3(A.c1 + 3 * (view * HW + q)) : env_lookup0(A.mips, A.e, sm.w);
      const float K = ggx_G1(sm.nw, rho) * g1v * sm.vh / (nv * sm.nh);
      const float fc = pow5(1.0f - sm.vh);
      const float3 F = F0 + (f3(1.f, 1.f, 1.f) - F0) * fc;
      acc = acc + mul3(F, Li) * K;
      if (kCid) {
        const float pdf = ggx_D(sm.nh, rho) * sm.nh / (4.0f * sm.vh);
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
  st3(A.final_out + 3 * p, fin);
  if (A.c_s_mc) st3(A.c_s_mc + 3 * p, csm);
  if (A.c_id) st3(A.c_id + 3 * p, cid);
  if (A.step_count && steps) atomicAdd(A.step_count, steps);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" ssgi_status ssgi_trace_indirect(const ssgi_gbuffer* g, const ssgi_camera* cams, const float* hiz,
                                           const float* c1, const float* c_d, const ssgi_envmap* env,
                                           const ssgi_trace_params* p, float* c_s_mc, float* c_id, float* final_out,
                                           int32_t* hit_idx, uint64_t* step_count, ssgi_stream_t stream) {
  if (gbuffer_ok(g) != SSGI_OK || trace_params_ok(p) != SSGI_OK || !c1 || !c_d || !final_out)
    return SSGI_ERR_INVALID_ARG;
  const bool brute = (p->flags & SSGI_BRUTE_FORCE) != 0;
  if (!brute && p->hiz_levels > 1 && !hiz) return SSGI_ERR_INVALID_ARG;
  TraceArgs A;
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  make_hiz_info(g->d, p->hiz_levels, &A.hz);
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.hiz = hiz;
  A.c1 = c1;
  A.c_d = c_d;
  A.mips = env->mips;
  A.c_s_mc = c_s_mc;
  A.c_id = c_id;
  A.final_out = final_out;
  A.hit_idx = hit_idx;
  A.step_count = reinterpret_cast<unsigned long long*>(step_count);
  A.spp = p->spp;
  A.max_steps = p->max_steps;
  A.levels = p->hiz_levels;
  A.thickness = p->thickness;
  A.max_distance = p->max_distance;
  A.seed = p->seed;
  A.flags = p->flags;
  dim3 grid(ceil_div(g->d.width, kTileW), ceil_div(g->d.height, kTileH), g->d.views);
  if (p->flags & SSGI_DIFFUSE_INDIRECT)
    k_trace<true><<<grid, kTileW * kTileH, 0, (cudaStream_t)stream>>>(A);
  else
    k_trace<false><<<grid, kTileW * kTileH, 0, (cudaStream_t)stream>>>(A);
  return launch_status();
}
