// k_fused.cu -- one inverse-rendering step (all views of a frame: environment mips, Hi-Z,
// direct shading, trace with stored hits, L2 loss, backward) in a single persistent launch.
//
// The launch is cooperative, so every block is resident at once and the blocks may wait for
// each other.  The step has five grid barriers, one per true all-to-all dependency:
//   pyramids | shading | trace + loss | Monte-Carlo adjoint | direct adjoint | mip-chain adjoint
// (shading reads any mip level; the trace reads any pixel's c1; the direct adjoint of a pixel
// needs every receiver's scatter into its g_c1; the mip-chain adjoint needs every texel's
// gradient).  Inside the pyramid phase the top levels are built by whichever block finishes
// the last tile of a view (a counter, no waiting).  Work inside a phase is handed out from
// counters, block by block.  The barrier is bounded: a block that waits longer than
// kBarrierSpinLimit sleeps marks the error word and every block leaves; nothing spins forever.
// The per-item code is the stand-alone kernels' (ssgi_ops.cuh), so the results match the
// per-stage path bit for bit (gradients up to the order of atomic additions).
#include <algorithm>
#include <atomic>
#include <cstring>

#include "ssgi_ops.cuh"

namespace ssgi {

constexpr int kFusedThreads = 128;                // one 8 x 16 trace tile per block iteration
constexpr long long kBarrierSpinLimit = 1ll << 26;  // x ~100 ns sleeps: several seconds (default)
constexpr int kFusedBarBytes = 512;               // control block at the start of the workspace
constexpr int kFusedStampOffset = 256;            // bytes into it: 64-bit phase timestamps

// Control words (32-bit) of the control block.
enum : int {
  kArrive = 0,     // grid barrier: arrivals
  kGen = 1,        // grid barrier: generation
  kErr = 2,        // a block gave up waiting
  kPyrNext = 3,    // next pyramid tile
  kTraceNext = 4,  // next trace tile
  kMcNext = 5,     // next Monte-Carlo adjoint chunk
  kDirNext = 6,    // next direct adjoint chunk
  kEnvDone = 7,    // environment tiles finished
  kHizDone = 8,    // Hi-Z tiles finished, one word per view
};
static_assert((kHizDone + SSGI_MAX_VIEWS) * 4 <= kFusedStampOffset, "control words overlap the stamps");
static_assert(kFusedStampOffset + 8 * (SSGI_FUSED_PHASES + 1) <= kFusedBarBytes, "stamps overflow");

struct FusedArgs {
  FrameArgs f;
  const float* env;  // base level of the environment (input)
  float* mips;       // workspace: the mip chain
  float* hiz;        // workspace: the pyramid
  float* g_env;      // output
  float* loss;       // output (one float)
  unsigned* ctl;     // workspace: control block
  long long n_gc1;   // float4s of g_c1
  int n_gmips;       // float4s of g_mips
  long long wait_limit;  // polls a block makes at a grid barrier before it gives up
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Block 0 records when it leaves barrier `k` (slot 0 = its start): the phase durations.
__device__ __forceinline__ void stamp(unsigned* ctl, int k) {
  if (blockIdx.x == 0 && threadIdx.x == 0)
    reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctl) + kFusedStampOffset)[k] = global_ns();
}

// Block-level dynamic work loop: the block takes chunk after chunk from `counter` (zero at the
// start of the launch) until all `n` are taken; body(c) runs on every thread of the block.
template <class Body>
__device__ __forceinline__ void for_each_chunk(unsigned* counter, int n, Body body) {
  __shared__ int s_c;
  for (;;) {
    if (threadIdx.x == 0) s_c = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int c = s_c;
    __syncthreads();
    if (c >= n) break;
    body(c);
  }
}

// Block-level: counts this block's finished piece of work on `counter`; true for the block that
// finishes the last of `total` (its later loads see every other block's stores).
__device__ __forceinline__ bool last_arrival(unsigned* counter, unsigned total) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1u) == total - 1u;
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

// Grid barrier for a cooperative launch; returns false if any block gave up waiting (after
// `limit` polls of ~100 ns each).
__device__ __forceinline__ bool grid_sync(unsigned* ctl, long long limit) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = ctl + kGen;
    volatile unsigned* verr = ctl + kErr;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(ctl + kArrive, 1u) + 1u;
    int ok = 1;
    if (arrived == gridDim.x) {
      atomicExch(ctl + kArrive, 0u);
      __threadfence();
      atomicAdd(const_cast<unsigned*>(vgen), 1u);
    } else {
      long long spins = 0;
      while (*vgen == gen) {
        if (*verr) {
          ok = 0;
          break;
        }
        if (++spins > limit) {
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

// Sizes every phase needs, computed once per block into shared memory and read back inside
// each phase: a read after a grid barrier (which synchronises the block) cannot be merged with
// one before it, so no value stays in a register through the trace and adjoint loops.
struct PhaseConsts {
  long long HW, npx, gsz;
  int V, H, W, nchunks;
};

// Seven resident blocks per SM (72 registers a thread): fewer spills in the trace phase than at
// eight blocks and 64 registers, which measured slower (as did six at 80).
template <bool kCid, bool kPathwise>
__global__ void __launch_bounds__(kFusedThreads, 7) k_step_fused(const __grid_constant__ FusedArgs F) {
  const FrameArgs& A = F.f;
  const EnvInfo& e = A.e;
  __shared__ LevelTable s_lv;
  __shared__ TileBuf s_tile;
  __shared__ PhaseConsts s_k;
  if (threadIdx.x == 0) {
    s_k.V = A.vs.V;
    s_k.H = A.vs.H;
    s_k.W = A.vs.W;
    s_k.HW = (long long)A.vs.H * A.vs.W;
    s_k.npx = s_k.V * s_k.HW;
    s_k.gsz = (long long)gridDim.x * kFusedThreads;
    s_k.nchunks = (int)((s_k.npx + kFusedThreads - 1) / kFusedThreads);
  }
  __syncthreads();
  stamp(F.ctl, 0);

  // P0: clear the backward accumulators and the loss; Hi-Z and environment pyramids, 32 x 32
  // tiles through level 5, levels 6.. by the block that finishes a pyramid's last tile.
  {
    const long long gtid = (long long)blockIdx.x * kFusedThreads + threadIdx.x, gsz = s_k.gsz;
    const int V = s_k.V, H = s_k.H, W = s_k.W;
    for (long long i = gtid; i < F.n_gc1; i += gsz) A.g_c1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long i = gtid; i < F.n_gmips; i += gsz) A.g_mips[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gtid == 0) *F.loss = 0.0f;
    const int hx = (W + kHizTile - 1) / kHizTile, hy = (H + kHizTile - 1) / kHizTile;
    const int n_hz = A.levels > 1 ? hx * hy * V : 0;
    const int ex = e.w[0] / min(kHizTile, e.w[0]), ey = e.h[0] / min(kHizTile, e.h[0]);
    for_each_chunk(F.ctl + kPyrNext, n_hz + ex * ey, [&](int t) {
      if (t < n_hz) {
        const int v = t / (hx * hy), r = t - v * hx * hy;
        hiz_tile_block(A.depth, H, W, A.hz, F.hiz, v, r % hx, r / hx, s_tile);
        if (A.levels > 6 && last_arrival(F.ctl + kHizDone + v, hx * hy)) hiz_upper_block(A.hz, v, F.hiz);
      } else {
        const int r = t - n_hz;
        env_tile_block(F.env, e, F.mips, r % ex, r / ex, s_tile);
        if (e.levels > 6 && last_arrival(F.ctl + kEnvDone, ex * ey)) env_upper_block(e, F.mips);
      }
    });
  }
  if (!grid_sync(F.ctl, F.wait_limit)) return;
  stamp(F.ctl, 1);

  // P1: direct shading
  {
    const long long npx = s_k.npx, gsz = s_k.gsz;
    for (long long p = (long long)blockIdx.x * kFusedThreads + threadIdx.x; p < npx; p += gsz) shade_pixel(A, p);
  }
  if (!grid_sync(F.ctl, F.wait_limit)) return;
  stamp(F.ctl, 2);

  // P2: trace, one 8 x 16 tile per block iteration, and the L2 loss of each finished pixel.
  // The per-tile cost varies by an order of magnitude (sky vs. rays that run out of steps),
  // so blocks take the next tile from a counter instead of a fixed stride.
  {
    float acc = 0.0f;
    const int tx = (s_k.W + 7) / 8, ty = (s_k.H + 15) / 16;
    for_each_chunk(F.ctl + kTraceNext, tx * ty * s_k.V, [&](int t) {
      const int v = t / (tx * ty), r = t - v * tx * ty;
      const int x = (r % tx) * 8 + (threadIdx.x % 8), y = (r / tx) * 16 + (threadIdx.x / 8);
      fill_levels(A, v, s_lv);  // the previous tile's reads ended at for_each_chunk's barriers
      __syncthreads();
      if (x < s_k.W && y < s_k.H) {
        const float3 fin = trace_pixel<kCid>(A, x, y, v, s_lv);
        const long long p = v * s_k.HW + (long long)y * s_k.W + x;
        const float inv = 1.0f / (float)(s_k.npx * 3);
        acc += (A.flags & SSGI_SRGB_LOSS) ? l2_srgb_pixel(A, p, fin, inv) : l2_pixel(A, p, fin, inv);
      }
    });
    block_sum_add(acc, F.loss, 1.0f / (float)(s_k.npx * 3));
  }
  if (!grid_sync(F.ctl, F.wait_limit)) return;
  stamp(F.ctl, 3);

  // P3: Monte-Carlo adjoint (scatters into g_c1 and g_mips)
  for_each_chunk(F.ctl + kMcNext, s_k.nchunks, [&](int c) {
    const long long p = (long long)c * kFusedThreads + threadIdx.x;
    if (p < s_k.npx) bwd_mc_pixel<kPathwise>(A, p);
  });
  if (!grid_sync(F.ctl, F.wait_limit)) return;
  stamp(F.ctl, 4);

  // P4: direct-shading adjoint
  for_each_chunk(F.ctl + kDirNext, s_k.nchunks, [&](int c) {
    const long long p = (long long)c * kFusedThreads + threadIdx.x;
    if (p < s_k.npx) bwd_direct_pixel(A, p);
  });
  if (!grid_sync(F.ctl, F.wait_limit)) return;
  stamp(F.ctl, 5);

  // P5: mip-chain adjoint to the base texels
  {
    const long long gsz = s_k.gsz, n = (long long)e.h[0] * e.w[0] * 3;
    for (long long t = (long long)blockIdx.x * kFusedThreads + threadIdx.x; t < n; t += gsz)
      bwd_env_item(e, A.g_mips, F.g_env, (int)t);
  }
  stamp(F.ctl, 6);
}

struct FusedLayout {
  size_t bar, mips, hiz, cd, c1, gfinal, gc1, gmips, bytes;
};

inline size_t up256(size_t n) { return (n + 255) & ~(size_t)255; }

inline FusedLayout fused_layout(ssgi_dims d, int env_h, int env_w, int levels) {
  FusedLayout L;
  const size_t px = (size_t)d.views * d.height * d.width;
  size_t o = 0;
  L.bar = o; o += kFusedBarBytes;
  L.mips = o; o += up256(ssgi_env_mip_floats(env_h, env_w) * 4);
  L.hiz = o; o += up256(std::max<size_t>(ssgi_hiz_floats(d, levels), 1) * 4);
  L.cd = o; o += up256(px * 12);
  L.c1 = o; o += up256(px * 12);
  L.gfinal = o; o += up256(px * 12);
  L.gc1 = o; o += up256(px * 16);
  L.gmips = o; o += up256(ssgi_env_mip_floats(env_h, env_w) / 3 * 16);
  L.bytes = o;
  return L;
}

// Polls a block makes at a grid barrier before it gives up; negative = kBarrierSpinLimit.
std::atomic<long long> g_wait_limit{-1};

}  // namespace ssgi

using namespace ssgi;

extern "C" {

ssgi_status ssgi_step_fused_set_wait_limit(int64_t polls) {
  g_wait_limit.store(polls < 0 ? -1 : (long long)polls);
  return SSGI_OK;
}

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
  if (p->flags & (SSGI_BRUTE_FORCE | SSGI_SRGB_FINAL)) return SSGI_ERR_INVALID_ARG;
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
  F.ctl = (unsigned*)(ws + L.bar);
  F.n_gc1 = npx;
  F.n_gmips = (int)(ssgi_env_mip_floats(env_h, env_w) / 3);
  const long long lim = g_wait_limit.load();
  F.wait_limit = lim < 0 ? kBarrierSpinLimit : lim;
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
  A.g_c1 = (float4*)(ws + L.gc1);
  A.g_mips = (float4*)(ws + L.gmips);
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
  const bool cid = (p->flags & SSGI_DIFFUSE_INDIRECT) != 0, pw = (p->flags & SSGI_PATHWISE) != 0;
  const void* fn = cid ? (pw ? (const void*)k_step_fused<true, true> : (const void*)k_step_fused<true, false>)
                       : (pw ? (const void*)k_step_fused<false, true> : (const void*)k_step_fused<false, false>);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kFusedThreads, 0) != cudaSuccess || per_sm < 1)
    return SSGI_ERR_CUDA;
  const int blocks = per_sm * sms;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws + L.bar, 0, kFusedBarBytes, s) != cudaSuccess) return SSGI_ERR_CUDA;
  void* args[] = {(void*)&F};
  if (cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(kFusedThreads), args, 0, s) != cudaSuccess) {
    cudaGetLastError();
    return SSGI_ERR_CUDA;
  }
  return SSGI_OK;
}

ssgi_status ssgi_step_fused_check(const void* workspace, int32_t* failed) {
  if (!workspace || !failed) return SSGI_ERR_INVALID_ARG;
  unsigned w[kErr + 1];
  if (cudaMemcpy(w, workspace, sizeof(w), cudaMemcpyDeviceToHost) != cudaSuccess) return SSGI_ERR_CUDA;
  *failed = w[kErr] != 0;
  return SSGI_OK;
}

ssgi_status ssgi_step_fused_phase_ns(const void* workspace, uint64_t* ns) {
  if (!workspace || !ns) return SSGI_ERR_INVALID_ARG;
  unsigned long long t[SSGI_FUSED_PHASES + 1];
  if (cudaMemcpy(t, (const char*)workspace + kFusedStampOffset, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SSGI_ERR_CUDA;
  for (int k = 0; k < SSGI_FUSED_PHASES; ++k) ns[k] = t[k + 1] >= t[k] ? t[k + 1] - t[k] : 0;
  return SSGI_OK;
}

}  // extern "C"
