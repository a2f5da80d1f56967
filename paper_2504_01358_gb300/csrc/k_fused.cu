// k_fused.cu -- one inverse-rendering step (all views of a frame: environment mips, Hi-Z,
// direct shading, trace with stored hits, L2 loss, backward) in a single launch.
//
// One block per work item, in phase order:
//   clears | pyramids | shading | trace + loss + Monte-Carlo adjoint | direct adjoint | mip-chain adjoint
// (shading reads any mip level; the trace reads any pixel's c1; the direct adjoint of a pixel
// needs every receiver's scatter into its g_c1; the mip-chain adjoint needs every texel's
// gradient).  The Monte-Carlo adjoint of a pixel needs only that pixel's hits and dL/dfinal
// (the loss is a sum over pixels), so the block that traces a tile goes on to its adjoint: the
// scatter of one tile overlaps the march of the others, and no phase boundary separates them.
// A block takes a ticket from a counter when it starts; the ticket names its phase and item, so
// tickets go out in phase order.  Before working, a block of phase k waits until every item of
// phase k - 1 has finished (a completion count per phase; the trace phase counts warps, each of
// which leaves as soon as it is done).  That wait always ends: every item of phase k - 1 took
// its ticket earlier, so its block is already resident and running (no cooperative launch and
// no residency limit is needed), and it waits only for phase k - 2, which finished before.
// The wait is still bounded: a block that polls longer than the limit marks the error word and
// returns, and every later block sees the mark and returns; nothing spins forever.  Inside the
// pyramid phase the top levels are built by whichever block finishes the last item of a pyramid
// (a counter, no waiting).
//
// Why not persistent blocks: the trace's tiles vary in cost by an order of magnitude, and
// resident blocks that loop over tiles from a counter measured 12-21 % slower than the same
// tiles as a grid of blocks (one per tile) that the hardware schedules; with one block per item
// the trace phase keeps the grid's schedule.
//
// The per-item code is the stand-alone kernels' (ssgi_ops.cuh), so the results match the
// per-stage path bit for bit (gradients up to the order of atomic additions).  Data another
// block wrote earlier in the launch is read through L2 (ld.global.cg) where some block may have
// cached those lines before they were written; c1, the mip chain and the pyramid are read
// through the read-only path only in phases after the one that writes them, which reads none of
// them.
#include <algorithm>
#include <atomic>
#include <cstring>

#include "ssgi_ops.cuh"

namespace ssgi {

constexpr int kFusedThreads = 128;                  // one 16 x 8 trace tile per block
constexpr long long kBarrierSpinLimit = 1ll << 26;  // x ~100 ns sleeps: several seconds (default)
constexpr int kFusedBarBytes = 512;                 // control block at the start of the workspace
constexpr int kFusedStampOffset = 256;              // bytes into it: 64-bit phase timestamps
constexpr int kPhases = SSGI_FUSED_PHASES + 1;      // the clears, then the reported phases
constexpr int kClearPerBlock = kFusedThreads * 32;  // float4s a clearing block zeroes
// Pyramid tiles: 16 x 16 (levels 1..4), an item covering 2 x 2 of them (the stand-alone
// builder's 32 x 32 footprint); the levels above 4 are built by the block that finishes a
// pyramid's last item.  The tile buffer (1 KB) shares shared memory with the trace's level table,
// so seven blocks need at most 16 KB of shared memory and the rest of the SM's 256 KB stays L1
// for the march: with a 32 x 32 tile (4 KB) the carve-out became 64 KB and the trace phase ran
// 7 % slower (the stand-alone trace forced to that carve-out slows the same).
constexpr int kFusedTile = 16;
constexpr int kFusedTileLevels = tile_levels<kFusedTile>();
constexpr int kFusedRegion = 2 * kFusedTile;
// 128-pixel chunks per item in the per-pixel phases (the trace: one tile per item); coarser
// items measured slower
constexpr int kShadeChunks = 1;  // shading, direct adjoint, mip-chain adjoint

constexpr int kTracePhase = 3;  // trace + loss + Monte-Carlo adjoint

// Control words (32-bit) of the control block.
enum : int {
  kTicket = 0,                  // next ticket
  kErr = 1,                     // a block gave up waiting
  kEnvDone = 2,                 // environment tiles finished
  kDone = 3,                    // kDone + k: finished items of phase k
  kHizDone = kDone + kPhases,   // Hi-Z tiles finished, one word per view
};
// the loss's FP64 accumulator (the trace's ~10^5 tiles each add a partial sum: in FP32 their
// rounding would reach 1e-5 of the loss)
constexpr int kLossAccOffset = 248;
static_assert((kHizDone + SSGI_MAX_VIEWS) * 4 <= kLossAccOffset, "control words overlap the loss accumulator");
static_assert(kLossAccOffset + 8 <= kFusedStampOffset, "the loss accumulator overlaps the stamps");
// per phase: the start of its first item and the end of its last
static_assert(kFusedStampOffset + 16 * kPhases <= kFusedBarBytes, "stamps overflow");

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
  long long wait_limit;        // polls a block makes before it gives up
  int items[kPhases];          // work items of each phase
  int first[kPhases + 1];      // ticket of each phase's first item (prefix sums of items)
  int hx, hy, ex, ey, n_hz;    // pyramid items: Hi-Z regions per view, environment tiles, Hi-Z items in all views
  int tx, ty;                  // trace tiles (16 x 8) per view
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long* stamps(unsigned* ctl) {
  return reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctl) + kFusedStampOffset);
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

// Thread 0: waits until phase ph - 1 has finished all its items.  false if a block gave up
// (this one after `limit` polls of ~100 ns, or another one before).
__device__ __forceinline__ bool wait_for_phase(const FusedArgs& F, int ph) {
  volatile unsigned* err = F.ctl + kErr;
  if (ph > 0) {
    volatile unsigned* done = F.ctl + kDone + ph - 1;
    // the trace phase counts its warps (each leaves as soon as it is done), the others their items
    const unsigned need = (unsigned)F.items[ph - 1] * (ph - 1 == kTracePhase ? kFusedThreads / 32 : 1);
    long long spins = 0;
    while (*done < need) {
      if (*err) return false;
      if (++spins > F.wait_limit) {
        atomicExch(const_cast<unsigned*>(err), 1u);
        return false;
      }
      __nanosleep(100);
    }
    __threadfence();  // the finished phase's stores are visible to this block's loads
  }
  return *err == 0;
}

// Block-level: this block's item of phase ph is done; the block that completes the phase
// stamps its end (no contended atomics on the stamps).
__device__ __forceinline__ void finish_item(const FusedArgs& F, int ph) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();  // the item's stores before its count
    if (atomicAdd(F.ctl + kDone + ph, 1u) == (unsigned)F.items[ph] - 1u) stamps(F.ctl)[2 * ph + 1] = global_ns();
  }
}

// One item per block.  Seven resident blocks per SM (72 registers a thread): fewer spills in the
// trace than at eight blocks and 64 registers, which measured slower (as did six at 80).
template <bool kCid, bool kPathwise>
__global__ void __launch_bounds__(kFusedThreads, 7) k_step_fused(const __grid_constant__ FusedArgs F) {
  const FrameArgs& A = F.f;
  __shared__ union {
    LevelTable lv;                  // trace items
    TileBufT<kFusedTile> tile;      // pyramid items
  } s_u;
  __shared__ int s_phase, s_item, s_ok;
  if (threadIdx.x == 0) {
    const int t = (int)atomicAdd(F.ctl + kTicket, 1u);
    int ph = 0;
    while (ph + 1 < kPhases && t >= F.first[ph + 1]) ++ph;
    s_phase = ph;
    s_item = t - F.first[ph];
    s_ok = t < F.first[kPhases] && wait_for_phase(F, ph);
    if (s_ok && s_item == 0) stamps(F.ctl)[2 * ph] = global_ns();  // the phase's first item
  }
  __syncthreads();
  if (!s_ok) return;
  const int ph = s_phase, item = s_item;
  const long long HW = (long long)A.vs.H * A.vs.W, npx = A.vs.V * HW;

  if (ph == 0) {
    // the backward's accumulators and the loss
    const long long base = (long long)item * kClearPerBlock + threadIdx.x;
    for (int k = 0; k < kClearPerBlock / kFusedThreads; ++k) {
      const long long i = base + (long long)k * kFusedThreads;
      if (i < F.n_gc1) A.g_c1[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      else if (i - F.n_gc1 < F.n_gmips) A.g_mips[i - F.n_gc1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (item == 0 && threadIdx.x == 0) *F.loss = 0.0f;  // written again by the adjoint's first item
  } else if (ph == 1) {
    // Hi-Z and environment pyramids: 16 x 16 tiles through level 4, levels 5.. by the block
    // that finishes a pyramid's last item
    const EnvInfo& e = A.e;
    if (item < F.n_hz) {
      const int v = item / (F.hx * F.hy), r = item - v * F.hx * F.hy;
      for (int sub = 0; sub < 4; ++sub) {
        const int tx = 2 * (r % F.hx) + (sub & 1), ty = 2 * (r / F.hx) + (sub >> 1);
        if (tx * kFusedTile < A.vs.W && ty * kFusedTile < A.vs.H)  // block-uniform
          hiz_tile_block<kFusedTile>(A.depth, A.vs.H, A.vs.W, A.hz, F.hiz, v, tx, ty, s_u.tile);
      }
      if (A.levels > kFusedTileLevels + 1 && last_arrival(F.ctl + kHizDone + v, F.hx * F.hy))
        hiz_upper_block(A.hz, v, F.hiz, kFusedTileLevels + 1);
    } else {
      const int r = item - F.n_hz;
      env_tile_block<kFusedTile>(F.env, e, F.mips, r % F.ex, r / F.ex, s_u.tile);
      if (e.levels > kFusedTileLevels + 1 && last_arrival(F.ctl + kEnvDone, F.ex * F.ey))
        env_upper_block(e, F.mips, kFusedTileLevels + 1);
    }
  } else if (ph == 2) {
    for (int c = item * kShadeChunks; c < (item + 1) * kShadeChunks; ++c) {
      const long long p = (long long)c * kFusedThreads + threadIdx.x;
      if (p < npx) shade_pixel(A, p);
    }
  } else if (ph == kTracePhase) {
    // trace one 16 x 8 tile (16 x 2 per warp, as k_trace), the L2 loss of its pixels and their
    // Monte-Carlo adjoint (each thread's own pixel: its hits and dL/dfinal are this thread's)
    const int v = item / (F.tx * F.ty), r = item - v * F.tx * F.ty;
    const int x = (r % F.tx) * 16 + (threadIdx.x % 16), y = (r / F.tx) * 8 + (threadIdx.x / 16);
    fill_levels(A, v, s_u.lv);
    __syncthreads();
    float acc = 0.0f;
    const float inv = 1.0f / (float)(npx * 3);
    if (x < A.vs.W && y < A.vs.H) {
      const float3 fin = trace_pixel<kCid>(A, x, y, v, s_u.lv);
      const long long p = v * HW + (long long)y * A.vs.W + x;
      float3 gfin;
      acc = (A.flags & SSGI_SRGB_LOSS) ? l2_srgb_pixel(A, p, fin, inv, gfin) : l2_pixel(A, p, fin, inv, gfin);
      bwd_mc_pixel<kPathwise, true>(A, p, gfin);
    }
    // the warp's partial sum into the FP64 accumulator (zeroed with the control block); then the
    // warp counts itself done and leaves: its registers are not held until the block's slowest
    // warp finishes (the warps of a tile differ in march length; measured 1 % faster at config 4)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __threadfence();  // this lane's stores before the warp's count
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(reinterpret_cast<double*>(reinterpret_cast<char*>(F.ctl) + kLossAccOffset), (double)acc);
      __threadfence();
      const unsigned warps = (unsigned)F.items[kTracePhase] * (kFusedThreads / 32);
      if (atomicAdd(F.ctl + kDone + kTracePhase, 1u) == warps - 1u) stamps(F.ctl)[2 * kTracePhase + 1] = global_ns();
    }
    return;
  } else if (ph == 4) {
    // direct adjoint; its first item also writes the loss, which every trace tile has added to
    // by now
    if (item == 0 && threadIdx.x == 0)
      *F.loss = (float)(*reinterpret_cast<volatile double*>(reinterpret_cast<char*>(F.ctl) + kLossAccOffset) / (3.0 * (double)npx));
    for (int c = item * kShadeChunks; c < (item + 1) * kShadeChunks; ++c) {
      const long long p = (long long)c * kFusedThreads + threadIdx.x;
      if (p < npx) bwd_direct_pixel(A, p);
    }
  } else {
    // mip-chain adjoint to the base texels
    for (int c = item * kShadeChunks; c < (item + 1) * kShadeChunks; ++c) {
      const int t = c * kFusedThreads + threadIdx.x;
      if (t < A.e.h[0] * A.e.w[0] * 3) bwd_env_item(A.e, A.g_mips, F.g_env, t);
    }
  }
  finish_item(F, ph);
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

  const long long nch = (npx + kFusedThreads - 1) / kFusedThreads;
  const int H = g->d.height, W = g->d.width, V = g->d.views;
  F.hx = (W + kFusedRegion - 1) / kFusedRegion;
  F.hy = (H + kFusedRegion - 1) / kFusedRegion;
  F.n_hz = p->hiz_levels > 1 ? F.hx * F.hy * V : 0;
  F.ex = env_w / std::min(kFusedTile, env_w);
  F.ey = env_h / std::min(kFusedTile, env_h);
  F.tx = (W + 15) / 16;
  F.ty = (H + 7) / 8;
  const long long clear = (F.n_gc1 + F.n_gmips + kClearPerBlock - 1) / kClearPerBlock;
  const long long nenv = ((long long)env_h * env_w * 3 + kFusedThreads - 1) / kFusedThreads;
  const long long items[kPhases] = {clear, (long long)F.n_hz + F.ex * F.ey, (nch + kShadeChunks - 1) / kShadeChunks,
                                    (long long)F.tx * F.ty * V, (nch + kShadeChunks - 1) / kShadeChunks,
                                    (nenv + kShadeChunks - 1) / kShadeChunks};
  long long total = 0;
  for (int k = 0; k < kPhases; ++k) {
    F.first[k] = (int)total;
    F.items[k] = (int)items[k];
    total += items[k];
  }
  if (total >= (1ll << 31)) return SSGI_ERR_UNSUPPORTED;
  F.first[kPhases] = (int)total;
  const bool cid = (p->flags & SSGI_DIFFUSE_INDIRECT) != 0, pw = (p->flags & SSGI_PATHWISE) != 0;
  auto fn = cid ? (pw ? k_step_fused<true, true> : k_step_fused<true, false>)
                : (pw ? k_step_fused<false, true> : k_step_fused<false, false>);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(ws + L.bar, 0, kFusedBarBytes, s) != cudaSuccess) return SSGI_ERR_CUDA;
  fn<<<(unsigned)total, kFusedThreads, 0, s>>>(F);
  return launch_status();
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
  unsigned long long t[2 * kPhases];
  if (cudaMemcpy(t, (const char*)workspace + kFusedStampOffset, sizeof(t), cudaMemcpyDeviceToHost) != cudaSuccess)
    return SSGI_ERR_CUDA;
  // phase k (after the clears): from its first block's start to its last block's end; the
  // pyramids' span starts with the clears
  for (int k = 0; k < SSGI_FUSED_PHASES; ++k) {
    const unsigned long long start = t[2 * (k == 0 ? 0 : k + 1)], end = t[2 * (k + 1) + 1];
    ns[k] = end >= start ? end - start : 0;
  }
  return SSGI_OK;
}

}  // extern "C"
