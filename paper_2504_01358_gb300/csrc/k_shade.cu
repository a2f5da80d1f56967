// k_shade.cu -- direct split-sum shading of the G-buffer (Sec. 3.2 "Shading").
//
//   v = unit vector to the camera, r = 2 (v.n) n - v, lambda = log2(rho + 1) lambda_max,
//   c_s = L_E(r, lambda) (F0 A + B), c_d = (1 - m) a L_E(n, lambda), c1 = c_d + c_s,
// with (A, B) the BRDF table at (rho, clamp(n.v, 1e-4, 1)) and F0 = lerp(0.04, a, m).
// One thread per pixel, consecutive threads on consecutive pixels (coalesced plane reads).
#include "ssgi_device.cuh"

namespace ssgi {

__global__ void __launch_bounds__(256) k_shade_direct(Views vs, const float* __restrict__ depth,
                                                      const float* __restrict__ normal,
                                                      const float* __restrict__ albedo,
                                                      const float* __restrict__ rough,
                                                      const float* __restrict__ metal,
                                                      const float* __restrict__ mips, EnvInfo e,
                                                      const float* __restrict__ lut, int lut_n,
                                                      float* __restrict__ c_d, float* __restrict__ c_s,
                                                      float* __restrict__ c1) {
  const long long HW = (long long)vs.H * vs.W;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW * vs.V) return;
  const int view = (int)(p / HW);
  const int rem = (int)(p - (long long)view * HW);
  const int y = rem / vs.W, x = rem - (rem / vs.W) * vs.W;
  const DevCam& cam = vs.cam[view];
  const float3 d = pix_dir_world(cam, x, y);
  const float z = __ldg(depth + p);
  float3 od = f3(0.f, 0.f, 0.f), os = f3(0.f, 0.f, 0.f), o1;
  if (is_background(z)) {
    o1 = env_lookup0(mips, e, d);
  } else {
    const float3 v = d * (-1.0f / sqrtf(dot3(d, d)));
    const float3 n = ld3(normal + 3 * p);
    const float nv = dot3(n, v);
    const float mu = fminf(fmaxf(nv, 1e-4f), 1.0f);
    const float3 r = n * (2.0f * nv) - v;
    const float rho = __ldg(rough + p), m = __ldg(metal + p);
    const float lam = log2f(rho + 1.0f) * (float)(e.levels - 1);
    const LutVal ab = lut_sample(lut, lut_n, rho, mu);
    const float3 Er = env_lookup(mips, e, r, lam);
    const float3 En = env_lookup(mips, e, n, lam);
    const float3 a = ld3(albedo + 3 * p);
    const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
    os = mul3(Er, F0 * ab.A + f3(ab.B, ab.B, ab.B));
    od = mul3(a * (1.0f - m), En);
    o1 = od + os;
  }
  st3(c_d + 3 * p, od);
  if (c_s) st3(c_s + 3 * p, os);
  st3(c1 + 3 * p, o1);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" ssgi_status ssgi_shade_direct(const ssgi_gbuffer* g, const ssgi_camera* cams, const ssgi_envmap* env,
                                         const float* lut, int32_t lut_n, float* c_d, float* c_s, float* c1,
                                         ssgi_stream_t stream) {
  if (gbuffer_ok(g) != SSGI_OK || !lut || lut_n < 2 || !c_d || !c1) return SSGI_ERR_INVALID_ARG;
  Views vs;
  EnvInfo e;
  if (make_views(cams, g->d, &vs) != SSGI_OK || make_env(env, &e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  const long long n = (long long)g->d.views * g->d.height * g->d.width;
  k_shade_direct<<<ceil_div(n, 256), 256, 0, (cudaStream_t)stream>>>(vs, g->depth, g->normal, g->albedo, g->rough,
                                                                     g->metal, env->mips, e, lut, lut_n, c_d, c_s, c1);
  return launch_status();
}
