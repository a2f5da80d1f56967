// k_backward.cu -- adjoint of the SSGI forward pass for inverse rendering, and the L2 loss.
//
// The march is not differentiable (Sec. 5 of the paper): the stored hit indices, the
// sampled directions and the sampling pdf are frozen ("replay" function).  Per sample the
// replayed contribution is  f_s(w; theta) (n.w) / p_frozen * L(theta)
//   = D(n.h) G1(n.w) G1(n.v) / (4 (n.v) p_frozen) * F(a, m) * L,
// whose value at the forward point equals G (v.h)/((n.v)(n.h)) F L (D cancels).  Kernels:
//   k_bwd_mc      per receiver pixel: d/d{a, m, rho, n} of the Monte-Carlo sum (replay or, with
//                 SSGI_PATHWISE, through the re-drawn directions); scatters
//                 d/dc1 to the hit pixels and d/dL_E to level-0 environment texels (atomics);
//   k_bwd_direct  per pixel: adjoint of c_d = (1-m) a L_E(n, lambda) and
//                 c_s = L_E(r, lambda) (F0 A + B) with d/dc_d = g_final + g_c1, d/dc_s = g_c1;
//   k_bwd_env     per base texel: adjoint of the 2x2 box mip chain (each level-l ancestor
//                 contributes its gradient / 4^l).
#include "ssgi_ops.cuh"

namespace ssgi {

// Three blocks per SM leave 80 registers a thread (32 bytes of spills instead of 120 at 64
// registers and four blocks): measured 6 % faster; at two blocks (118 registers, no spills) the
// lost occupancy costs more than the spills saved.
template <bool kPathwise>
__global__ void __launch_bounds__(256, 3) k_bwd_mc(FrameArgs A) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)A.vs.V * A.vs.H * A.vs.W) return;
  bwd_mc_pixel<kPathwise>(A, p);
}

// Monte-Carlo adjoint in the mode the flags select (replay or pathwise).
inline void launch_bwd_mc(const FrameArgs& A, int blocks, cudaStream_t s) {
  if (A.flags & SSGI_PATHWISE)
    k_bwd_mc<true><<<blocks, 256, 0, s>>>(A);
  else
    k_bwd_mc<false><<<blocks, 256, 0, s>>>(A);
}

__global__ void __launch_bounds__(256, 4) k_bwd_direct(FrameArgs A) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)A.vs.V * A.vs.H * A.vs.W) return;
  bwd_direct_pixel(A, p);
}

__global__ void k_bwd_env(EnvInfo e, const float4* __restrict__ g_mips, float* __restrict__ g_env) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= e.h[0] * e.w[0] * 3) return;
  bwd_env_item(e, g_mips, g_env, t);
}

__global__ void __launch_bounds__(256) k_l2(const float* __restrict__ f, const float* __restrict__ t, long long n,
                                            float* __restrict__ g, float* __restrict__ loss, bool vec4) {
  l2_block_vec<false>(f, t, n, g, loss, vec4);
}

// The three adjoint launches of one frame on `s`, with `workspace` (need bytes, 16-byte
// aligned) cleared first.  Both backward entry points end here after validating their
// arguments, so the two cannot drift apart.
ssgi_status run_backward(const float* g_final, const ssgi_gbuffer* g, const float* c1, const float* lut,
                         int32_t lut_n, const int32_t* hit_idx, const ssgi_trace_params* p, float* g_albedo,
                         float* g_rough, float* g_metal, float* g_normal, float* g_env, FrameArgs& A,
                         void* workspace, size_t need, cudaStream_t s) {
  const long long npx = (long long)g->d.views * g->d.height * g->d.width;
  const size_t c1_bytes = ((size_t)npx * sizeof(float4) + 255) & ~(size_t)255;
  A.g_c1 = (float4*)workspace;
  A.g_mips = (float4*)((char*)workspace + c1_bytes);
  if (cudaMemsetAsync(workspace, 0, need, s) != cudaSuccess) return SSGI_ERR_CUDA;
  A.g_final = const_cast<float*>(g_final);
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.c1 = const_cast<float*>(c1);
  A.lut = lut;
  A.hit_idx = const_cast<int32_t*>(hit_idx);
  A.g_albedo = g_albedo;
  A.g_rough = g_rough;
  A.g_metal = g_metal;
  A.g_normal = g_normal;
  A.lut_n = lut_n;
  A.spp = p->spp;
  A.seed = p->seed;
  A.flags = p->flags;
  const int blocks = ceil_div(npx, 256);
  launch_bwd_mc(A, blocks, s);
  ssgi_status st = launch_status();
  if (st != SSGI_OK) return st;
  k_bwd_direct<<<blocks, 256, 0, s>>>(A);
  st = launch_status();
  if (st != SSGI_OK) return st;
  const int nt = A.e.h[0] * A.e.w[0] * 3;
  k_bwd_env<<<ceil_div(nt, 256), 256, 0, s>>>(A.e, A.g_mips, g_env);
  return launch_status();
}

// Argument checks shared by both entry points; fills A's views and environment and *need.
ssgi_status check_backward(const float* g_final, const ssgi_gbuffer* g, const ssgi_camera* cams, const float* c1,
                           const ssgi_envmap* env, const float* lut, int32_t lut_n, const int32_t* hit_idx,
                           const ssgi_trace_params* p, const float* g_albedo, const float* g_rough,
                           const float* g_metal, const float* g_normal, const float* g_env, FrameArgs& A,
                           size_t* need) {
  if (!g_final || gbuffer_ok(g) != SSGI_OK || trace_params_ok(p) != SSGI_OK || !c1 || !lut || lut_n < 2 ||
      !hit_idx || !g_albedo || !g_rough || !g_metal || !g_normal || !g_env)
    return SSGI_ERR_INVALID_ARG;
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  A.mips = env->mips;
  *need = ssgi_backward_workspace_bytes(g->d, env->h, env->w);
  return *need == 0 ? SSGI_ERR_INVALID_ARG : SSGI_OK;
}

}  // namespace ssgi

using namespace ssgi;

extern "C" {

ssgi_status ssgi_l2_loss(const float* final_in, const float* target, int64_t n, float* g_final, float* loss_out,
                         ssgi_stream_t stream) {
  if (!final_in || !target || !g_final || n < 1) return SSGI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (loss_out && cudaMemsetAsync(loss_out, 0, sizeof(float), s) != cudaSuccess) return SSGI_ERR_CUDA;
  const int blocks = (int)((n + 255) / 256 < 152 * 8 ? (n + 255) / 256 : 152 * 8);
  const bool vec4 = (((uintptr_t)final_in | (uintptr_t)target | (uintptr_t)g_final) & 15) == 0;
  k_l2<<<blocks, 256, 0, s>>>(final_in, target, n, g_final, loss_out, vec4);
  return launch_status();
}

ssgi_status ssgi_backward(const float* g_final, const ssgi_gbuffer* g, const ssgi_camera* cams, const float* c1,
                          const ssgi_envmap* env, const float* lut, int32_t lut_n, const int32_t* hit_idx,
                          const ssgi_trace_params* p, float* g_albedo, float* g_rough, float* g_metal,
                          float* g_normal, float* g_env, void* workspace, size_t ws_bytes, ssgi_stream_t stream) {
  FrameArgs A = {};
  size_t need = 0;
  const ssgi_status chk = check_backward(g_final, g, cams, c1, env, lut, lut_n, hit_idx, p, g_albedo, g_rough,
                                         g_metal, g_normal, g_env, A, &need);
  if (chk != SSGI_OK) return chk;
  if (!workspace || ((uintptr_t)workspace & 15) != 0 || ws_bytes < need) return SSGI_ERR_INVALID_ARG;
  return run_backward(g_final, g, c1, lut, lut_n, hit_idx, p, g_albedo, g_rough, g_metal, g_normal, g_env, A,
                      workspace, need, (cudaStream_t)stream);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free backward: the workspace is a fixed array in the library's device image, so
// callers that must not allocate device memory can still run the adjoint.  Device code could
// name the array directly; host code needs its device address, which every call looks up
// with the caller's device current (a cheap table lookup once the module is loaded, and never
// stale: a cached address would outlive a cudaDeviceReset or a change of context).
// ------------------------------------------------------------------------------------------
namespace ssgi {
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[SSGI_BACKWARD_NOALLOC_MAX_BYTES];

// Device address of the scratch array in the current device's context.
ssgi_status noalloc_scratch(void** out) {
  void* ptr = nullptr;
  if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SSGI_ERR_CUDA;
  *out = ptr;
  return SSGI_OK;
}
}  // namespace
}  // namespace ssgi

extern "C" ssgi_status ssgi_backward_noalloc(const float* g_final, const ssgi_gbuffer* g, const ssgi_camera* cams,
                                             const float* c1, const ssgi_envmap* env, const float* lut,
                                             int32_t lut_n, const int32_t* hit_idx, const ssgi_trace_params* p,
                                             float* g_albedo, float* g_rough, float* g_metal, float* g_normal,
                                             float* g_env, ssgi_stream_t stream) {
  FrameArgs A = {};
  size_t need = 0;
  const ssgi_status chk = check_backward(g_final, g, cams, c1, env, lut, lut_n, hit_idx, p, g_albedo, g_rough,
                                         g_metal, g_normal, g_env, A, &need);
  if (chk != SSGI_OK) return chk;
  if (need > (size_t)SSGI_BACKWARD_NOALLOC_MAX_BYTES) return SSGI_ERR_UNSUPPORTED;
  void* workspace = nullptr;
  const ssgi_status ss = noalloc_scratch(&workspace);
  if (ss != SSGI_OK) return ss;
  return run_backward(g_final, g, c1, lut, lut_n, hit_idx, p, g_albedo, g_rough, g_metal, g_normal, g_env, A,
                      workspace, need, (cudaStream_t)stream);
}
