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
#include "ssgi_ops.cuh"

namespace ssgi {

constexpr int kTileW = 16;  // a warp covers a 16 x 2 pixel tile
constexpr int kTileH = 8;   // a 128-thread block covers 16 x 8 pixels

// One thread per pixel, looping over its samples; a warp covers a 16 x 2 tile so that its
// rays start close together and touch the same pyramid cells (measured 0.7 % faster than 8 x 4
// and 1.8 % faster than 4 x 8 tiles).  Seven blocks per SM leave 72
// registers a thread, enough for the march and the pixel's shading inputs without spills
// (measured faster than eight blocks at 64 registers and six at 80).
template <bool kCid, bool kSrgb>
__global__ void __launch_bounds__(kTileW * kTileH, 7) k_trace(FrameArgs A) {
  __shared__ LevelTable s_lv;
  fill_levels(A, blockIdx.z, s_lv);
  __syncthreads();
  const int x = blockIdx.x * kTileW + (threadIdx.x % kTileW);
  const int y = blockIdx.y * kTileH + (threadIdx.x / kTileW);
  if (x >= A.vs.W || y >= A.vs.H) return;
  trace_pixel<kCid, kSrgb>(A, x, y, blockIdx.z, s_lv);
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
  FrameArgs A = {};
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  make_hiz_info(g->d, p->hiz_levels, &A.hz);
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.hiz = hiz;
  A.c1 = const_cast<float*>(c1);
  A.c_d = const_cast<float*>(c_d);
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
  const bool cid = (p->flags & SSGI_DIFFUSE_INDIRECT) != 0, srgb = (p->flags & SSGI_SRGB_FINAL) != 0;
  auto kern = cid ? (srgb ? k_trace<true, true> : k_trace<true, false>) : (srgb ? k_trace<false, true> : k_trace<false, false>);
  kern<<<grid, kTileW * kTileH, 0, (cudaStream_t)stream>>>(A);
  return launch_status();
}
