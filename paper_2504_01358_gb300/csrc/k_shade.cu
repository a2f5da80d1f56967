// k_shade.cu -- direct split-sum shading of the G-buffer (Sec. 3.2 "Shading").
//
//   v = unit vector to the camera, r = 2 (v.n) n - v, lambda = log2(rho + 1) lambda_max,
//   c_s = L_E(r, lambda) (F0 A + B), c_d = (1 - m) a L_E(n, lambda), c1 = c_d + c_s,
// with (A, B) the BRDF table at (rho, clamp(n.v, 1e-4, 1)) and F0 = lerp(0.04, a, m).
// One thread per pixel, consecutive threads on consecutive pixels (coalesced plane reads).
#include "ssgi_ops.cuh"

namespace ssgi {

__global__ void __launch_bounds__(256) k_shade_direct(FrameArgs A) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)A.vs.V * A.vs.H * A.vs.W) return;
  shade_pixel(A, p);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" ssgi_status ssgi_shade_direct(const ssgi_gbuffer* g, const ssgi_camera* cams, const ssgi_envmap* env,
                                         const float* lut, int32_t lut_n, float* c_d, float* c_s, float* c1,
                                         ssgi_stream_t stream) {
  if (gbuffer_ok(g) != SSGI_OK || !lut || lut_n < 2 || !c_d || !c1) return SSGI_ERR_INVALID_ARG;
  FrameArgs A = {};
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.mips = env->mips;
  A.lut = lut;
  A.lut_n = lut_n;
  A.c_d = c_d;
  A.c_s = c_s;
  A.c1 = c1;
  const long long n = (long long)g->d.views * g->d.height * g->d.width;
  k_shade_direct<<<ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(A);
  return launch_status();
}
