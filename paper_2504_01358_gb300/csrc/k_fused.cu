// k_fused.cu -- one inverse-rendering step (all views of a frame: environment mips, Hi-Z,
// direct shading, trace with stored hits, L2 loss, backward) in a single persistent launch.
//
// The launch is cooperative, so every block is resident at once and the blocks may wait for
// each other: the stages run as grid-stride phases separated by a grid barrier.  The barrier
// is bounded: a block that waits longer than kBarrierSpinLimit sleeps marks the error word and
// every block leaves; nothing spins forever.  The per-item code is the same as the stand-alone
// kernels' (ssgi_ops.cuh), so the results match the per-stage path.
#include <algorithm>
#include <cstring>

#include "ssgi_ops.cuh"

namespace ssgi {

constexpr int kFusedThreads = 128;                // one 8 x 16 trace tile per block iteration
constexpr long long kBarrierSpinLimit = 1ll << 26;  // x ~100 ns sleeps: several seconds

struct FusedArgs {
  FrameArgs f;
  const float* env;  // base level of the environment (input)
  float* mips;       // workspace: the mip chain
  float* hiz;        // workspace: the pyramid
  float* g_env;      // output
  float* loss;       // output (one float)
  unsigned* bar;     // workspace: [0] arrivals, [1] generation, [2] error
  long long n_gc1;   // floats of g_c1
  int n_gmips;       // floats of g_mips
};

// Grid barrier for a cooperative launch; returns false if any block gave up waiting.
__device__ __forceinline__ bool grid_sync(unsigned* bar) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile unsigned* verr = bar + 2;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(const_cast<unsigned*>(vgen), 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (++spins > kBarrierSpinLimit) {
          atomicExch(const_cast<unsigned*>(verr), 1u);
          ok = 0;
          break;
        }
        __nanosleep(100);
      }
    }
    __threadfence();
    s_ok = ok && *verr == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

template <bool kCid>
__global__ void __launch_bounds__(kFusedThreads, 8) k_step_fused(const __grid_constant__ FusedArgs F) {
  const FrameArgs& A = F.f;
  __shared__ int s_hoff[SSGI_MAX_HIZ_LEVELS], s_hw[SSGI_MAX_HIZ_LEVELS];
  if (threadIdx.x < SSGI_MAX_HIZ_LEVELS) {
    s_hoff[threadIdx.x] = A.hz.off[threadIdx.x];
    s_hw[threadIdx.x] = A.hz.w[threadIdx.x];
  }
  const int V = A.vs.V, H = A.vs.H, W = A.vs.W;
  const long long npx = (long long)V * H * W;
  const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long gsz = (long long)gridDim.x * blockDim.x;
  const EnvInfo& e = A.e;

  // P0: clear the backward workspace and the loss; copy the base level into the mip chain
  for (long long i = gtid; i < F.n_gc1; i += gsz) A.g_c1[i] = 0.0f;
  for (long long i = gtid; i < F.n_gmips; i += gsz) A.g_mips[i] = 0.0f;
  for (long long i = gtid; i < (long long)e.h[0] * e.w[0] * 3; i += gsz) F.mips[i] = __ldg(F.env + i);
  if (gtid == 0) *F.loss = 0.0f;
  if (!grid_sync(F.bar)) return;

  // P1: environment mips, one level per phase
  for (int l = 1; l < e.levels; ++l) {
    const int n = e.h[l] * e.w[l] * 3;
    for (long long t = gtid; t < n; t += gsz) env_down_item(F.mips + e.off[l - 1], e.h[l - 1], e.w[l - 1], F.mips + e.off[l], (int)t);
    if (!grid_sync(F.bar)) return;
  }

  // P2: Hi-Z, 32x32 tiles through level 5 (block-level), then the remaining levels
  if (A.levels > 1) {
    const int tx = (W + kHizTile - 1) / kHizTile, ty = (H + kHizTile - 1) / kHizTile;
    for (int t = blockIdx.x; t < tx * ty * V; t += gridDim.x) {
      const int v = t / (tx * ty), r = t - v * tx * ty;
      hiz_tile_block(A.depth, H, W, A.hz, F.hiz, v, r % tx, r / tx);
    }
    if (!grid_sync(F.bar)) return;
    for (int l = 6; l < A.levels; ++l) {
      const long long n = (long long)V * A.hz.w[l] * A.hz.h[l];
      for (long long t = gtid; t < n; t += gsz) hiz_level_item(A.hz, l, F.hiz, (int)t);
      if (!grid_sync(F.bar)) return;
    }
  }

  // P3: direct shading
  for (long long p = gtid; p < npx; p += gsz) shade_pixel(A, p);
  if (!grid_sync(F.bar)) return;

  // P4: trace, one 8 x 16 tile per block iteration
  {
    const int tx = (W + 7) / 8, ty = (H + 15) / 16;
    for (int t = blockIdx.x; t < tx * ty * V; t += gridDim.x) {
      const int v = t / (tx * ty), r = t - v * tx * ty;
      const int x = (r % tx) * 8 + (threadIdx.x % 8), y = (r / tx) * 16 + (threadIdx.x / 8);
      if (x < W && y < H) trace_pixel<kCid>(A, x, y, v, s_hoff, s_hw);
    }
  }
  if (!grid_sync(F.bar)) return;

  // P5: L2 loss and its gradient
  l2_block(A.final_out, A.target, npx * 3, A.g_final, F.loss, (long long)blockIdx.x * blockDim.x, gsz);
  if (!grid_sync(F.bar)) return;

  // P6: Monte-Carlo adjoint (scatters into g_c1 and g_mips)
  for (long long p = gtid; p < npx; p += gsz) bwd_mc_pixel(A, p);
  if (!grid_sync(F.bar)) return;

  // P7: direct-shading adjoint
  for (long long p = gtid; p < npx; p += gsz) bwd_direct_pixel(A, p);
  if (!grid_sync(F.bar)) return;

  // P8: mip-chain adjoint to the base texels
  for (long long t = gtid; t < (long long)e.h[0] * e.w[0] * 3; t += gsz) bwd_env_item(e, A.g_mips, F.g_env, (int)t);
}

struct FusedLayout {
  size_t bar, mips, hiz, cd, c1, gfinal, gc1, gmips, bytes;
};

inline size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

inline FusedLayout fused_layout(ssgi_dims d, int env_h, int env_w, int levels) {
  FusedLayout L;
  const size_t px = (size_t)d.views * d.height * d.width;
  size_t o = 0;
  L.bar = o; o += 256;
  L.mips = o; o += up256(ssgi_env_mip_floats(env_h, env_w) * 4);
  L.hiz = o; o += up256(std::max<size_t>(ssgi_hiz_floats(d, levels), 1) * 4);
  L.cd = o; o += up256(px * 12);
  L.c1 = o; o += up256(px * 12);
  L.gfinal = o; o += up256(px * 12);
  L.gc1 = o; o += up256(px * 12);
  L.gmips = o; o += up256(ssgi_env_mip_floats(env_h, env_w) * 4);
  L.bytes = o;
  return L;
}

}  // namespace ssgi

using namespace ssgi;

extern "C" {

size_t ssgi_step_fused_workspace_bytes(ssgi_dims d, int32_t env_h, int32_t env_w, int32_t hiz_levels) {
  if (!dims_ok(d) || ssgi_env_levels(env_h, env_w) < 1 || hiz_levels < 1 || hiz_levels > SSGI_MAX_HIZ_LEVELS) return 0;
  return fused_layout(d, env_h, env_w, hiz_levels).bytes;
}

ssgi_status ssgi_step_fused(const ssgi_gbuffer* g, const ssgi_camera* cams, const float* env, int32_t env_h,
                            int32_t env_w, const float* lut, int32_t lut_n, const float* target,
                            const ssgi_trace_params* p, float* final_out, int32_t* hit_idx, float* loss,
                            float* g_albedo, float* g_rough, float* g_metal, float* g_normal, float* g_env,
                            void* workspace, size_t ws_bytes, ssgi_stream_t stream) {
  if (gbuffer_ok(g) != SSGI_OK || trace_params_ok(p) != SSGI_OK || !env || !lut || lut_n < 2 || !target ||
      !final_out || !hit_idx || !loss || !g_albedo || !g_rough || !g_metal || !g_normal || !g_env || !workspace)
    return SSGI_ERR_INVALID_ARG;
  if (p->flags & SSGI_BRUTE_FORCE) return SSGI_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 255) != 0) return SSGI_ERR_INVALID_ARG;
  const size_t need = ssgi_step_fused_workspace_bytes(g->d, env_h, env_w, p->hiz_levels);
  if (need == 0 || ws_bytes < need) return SSGI_ERR_INVALID_ARG;
  FusedArgs F;
  memset(&F, 0, sizeof(F));
  FrameArgs& A = F.f;
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env_dims(env_h, env_w, &A.e) != SSGI_OK)
    return SSGI_ERR_INVALID_ARG;
  make_hiz_info(g->d, p->hiz_levels, &A.hz);
  const FusedLayout L = fused_layout(g->d, env_h, env_w, p->hiz_levels);
  char* ws = (char*)workspace;
  const long long npx = (long long)g->d.views * g->d.height * g->d.width;
  F.env = env;
  F.mips = (float*)(ws + L.mips);
  F.hiz = (float*)(ws + L.hiz);
  F.g_env = g_env;
  F.loss = loss;
  F.bar = (unsigned*)(ws + L.bar);
  F.n_gc1 = npx * 3;
  F.n_gmips = (int)ssgi_env_mip_floats(env_h, env_w);
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.mips = F.mips;
  A.lut = lut;
  A.lut_n = lut_n;
  A.hiz = p->hiz_levels > 1 ? F.hiz : nullptr;
  A.target = target;
  A.c_d = (float*)(ws + L.cd);
  A.c1 = (float*)(ws + L.c1);
  A.final_out = final_out;
  A.hit_idx = hit_idx;
  A.g_final = (float*)(ws + L.gfinal);
  A.g_albedo = g_albedo;
  A.g_rough = g_rough;
  A.g_metal = g_metal;
  A.g_normal = g_normal;
  A.g_c1 = (float*)(ws + L.gc1);
  A.g_mips = (float*)(ws + L.gmips);
  A.spp = p->spp;
  A.max_steps = p->max_steps;
  A.levels = p->hiz_levels;
  A.thickness = p->thickness;
  A.max_distance = p->max_distance;
  A.seed = p->seed;
  A.flags = p->flags;

  int dev = 0, sms = 0, coop = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess)
    return SSGI_ERR_CUDA;
  if (!coop) return SSGI_ERR_UNSUPPORTED;
  const bool cid = (p->flags & SSGI_DIFFUSE_INDIRECT) != 0;
  const void* fn = cid ? (const void*)k_step_fused<true> : (const void*)k_step_fused<false>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFusedThreads, 0) != cudaSuccess || per_sm < 1)
    return SSGI_ERR_CUDA;
  const int blocks = per_sm * sms;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws + L.bar, 0, 256, s) != cudaSuccess) return SSGI_ERR_CUDA;
  void* args[] = {(void*)&F};
  if (cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kFusedThreads), args, 0, s) != cudaSuccess) {
    cudaGetLastError();
    return SSGI_ERR_CUDA;
  }
  return SSGI_OK;
}

ssgi_status ssgi_step_fused_check(const void* workspace, int32_t* failed) {
  if (!workspace || !failed) return SSGI_ERR_INVALID_ARG;
  unsigned w[3];
  if (cudaMemcpy(w, workspace, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return SSGI_ERR_CUDA;
  *failed = w[2] != 0;
  return SSGI_OK;
}

}  // extern "C"
