// k_backward.cu -- adjoint of the SSGI forward pass for inverse rendering, and the L2 loss.
//
// The march is not differentiable (Sec. 5 of the paper): the stored hit indices, the
// sampled directions and the sampling pdf are frozen ("replay" function).  Per sample the
// replayed contribution is  f_s(w; theta) (n.w) / p_frozen * L(theta)
//   = D(n.h) G1(n.w) G1(n.v) / (4 (n.v) p_frozen) * F(a, m) * L,
// whose value at the forward point equals G (v.h)/((n.v)(n.h)) F L (D cancels).  Kernels:
//   k_bwd_mc      per receiver pixel: d/d{a, m, rho, n} of the Monte-Carlo sum; scatters
//                 d/dc1 to the hit pixels and d/dL_E to level-0 environment texels (atomics);
//   k_bwd_direct  per pixel: adjoint of c_d = (1-m) a L_E(n, lambda) and
//                 c_s = L_E(r, lambda) (F0 A + B) with d/dc_d = g_final + g_c1, d/dc_s = g_c1;
//   k_bwd_env     per base texel: adjoint of the 2x2 box mip chain (each level-l ancestor
//                 contributes its gradient / 4^l).
#include <mutex>

#include "ssgi_device.cuh"

namespace ssgi {

struct BwdArgs {
  Views vs;
  EnvInfo e;
  const float* __restrict__ g_final;
  const float* __restrict__ depth;
  const float* __restrict__ normal;
  const float* __restrict__ albedo;
  const float* __restrict__ rough;
  const float* __restrict__ metal;
  const float* __restrict__ c1;
  const float* __restrict__ mips;
  const float* __restrict__ lut;
  const int32_t* __restrict__ hit_idx;
  float* __restrict__ g_albedo;
  float* __restrict__ g_rough;
  float* __restrict__ g_metal;
  float* __restrict__ g_normal;
  float* __restrict__ g_c1;    // workspace [V,H,W,3]
  float* __restrict__ g_mips;  // workspace, packed like the mips
  int lut_n, spp;
  uint64_t seed;
  uint32_t flags;
};

// Warp-aggregated float3 atomic add: lanes of the calling (possibly partial) warp that
// target the same address are summed by shuffles and one lane issues the atomics.  Many
// pixels hit the same texels (a floor's normal always looks up the same polar texels, coarse
// mips have a handful of texels), and plain atomics on one address serialise in L2.
__device__ __forceinline__ void atomic_add3(float* p, float3 v) {
  const unsigned act = __activemask();
  const unsigned grp = __match_any_sync(act, (unsigned long long)p);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(grp) - 1;
  unsigned rest = grp & ~(1u << leader);
  float3 s = v;
  while (rest) {
    const int src = __ffs(rest) - 1;
    rest &= rest - 1;
    const float tx = __shfl_sync(grp, v.x, src), ty = __shfl_sync(grp, v.y, src), tz = __shfl_sync(grp, v.z, src);
    if (lane == leader) s = s + f3(tx, ty, tz);
  }
  if (lane == leader) {
    atomicAdd(p + 0, s.x);
    atomicAdd(p + 1, s.y);
    atomicAdd(p + 2, s.z);
  }
}

// d ln G1(z; rho) / dz, / drho
__device__ __forceinline__ void dlnG1(float z, float rho, float& dz, float& dr) {
  const float a2 = rho * rho;
  const float s = sqrtf(a2 + (1.0f - a2) * z * z);
  dz = 1.0f / z - (1.0f + (1.0f - a2) * z / s) / (z + s);
  dr = -(rho * (1.0f - z * z) / s) / (z + s);
}

// d ln D(c; rho) / dc, / drho with c = n.h
__device__ __forceinline__ void dlnD(float c, float rho, float& dc, float& dr) {
  const float a2 = rho * rho;
  const float den = c * c * (a2 - 1.0f) + 1.0f;
  dc = -4.0f * c * (a2 - 1.0f) / den;
  dr = 2.0f / rho - 4.0f * rho * c * c / den;
}

// Scatter g (per channel) with weight `scale` through the bilinear taps into gm, and return
// the derivatives of the bilinear value contracted with g along x and y (texel units).
__device__ __forceinline__ void bilin_adj(const float* __restrict__ mips, const Taps& t, float3 g, float scale,
                                          float* gm, float& gx, float& gy) {
  const float3 a = ld3(mips + t.idx[0]), b = ld3(mips + t.idx[1]);
  const float3 c = ld3(mips + t.idx[2]), d = ld3(mips + t.idx[3]);
  gx = dot3(g, (b - a) * (1.0f - t.ty) + (d - c) * t.ty);
  gy = dot3(g, (c - a) * (1.0f - t.tx) + (d - b) * t.tx);
  if (scale != 0.0f) {
    const float w00 = (1.0f - t.tx) * (1.0f - t.ty), w01 = t.tx * (1.0f - t.ty);
    const float w10 = (1.0f - t.tx) * t.ty, w11 = t.tx * t.ty;
    atomic_add3(gm + t.idx[0], g * (scale * w00));
    atomic_add3(gm + t.idx[1], g * (scale * w01));
    atomic_add3(gm + t.idx[2], g * (scale * w10));
    atomic_add3(gm + t.idx[3], g * (scale * w11));
  }
}

// Adjoint of SampleEnvMap(d, lambda): texel gradients into gm (all levels), returns d/dd and
// d/dlambda (zero where lambda is clamped).
__device__ __forceinline__ float3 env_lookup_adj(const float* __restrict__ mips, const EnvInfo& e, float3 d,
                                                 float lam, float3 g, float* gm, float& glam) {
  const float lmax = (float)(e.levels - 1);
  const bool inside = lam > 0.0f && lam < lmax;
  lam = fminf(fmaxf(lam, 0.0f), lmax);
  const int l0 = (int)floorf(lam);
  const int l1 = min(l0 + 1, e.levels - 1);
  const float t = lam - (float)l0;
  const DirAngles ang = dir_angles(d);
  const Taps t0 = env_taps(e, l0, ang), t1 = env_taps(e, l1, ang);
  float gx0, gy0, gx1 = 0.0f, gy1 = 0.0f;
  bilin_adj(mips, t0, g, 1.0f - t, gm, gx0, gy0);
  if (t != 0.0f) bilin_adj(mips, t1, g, t, gm, gx1, gy1);
  const float gu = (1.0f - t) * gx0 * (float)e.w[l0] + t * gx1 * (float)e.w[l1];
  const float gv = (1.0f - t) * gy0 * (float)e.h[l0] + t * gy1 * (float)e.h[l1];
  glam = 0.0f;
  if (inside && l1 != l0) glam = dot3(g, bilinear(mips, t1) - bilinear(mips, t0));
  const float q2 = d.x * d.x + d.z * d.z;
  if (!(q2 > 0.0f)) return f3(0.f, 0.f, 0.f);
  const float q = sqrtf(q2);
  const float r2 = q2 + d.y * d.y;
  const float dux = -d.z * kInv2Pi / q2, duz = d.x * kInv2Pi / q2;
  const float dvx = d.y * d.x * kInvPi / (q * r2), dvz = d.y * d.z * kInvPi / (q * r2), dvy = -q * kInvPi / r2;
  return f3(gu * dux + gv * dvx, gv * dvy, gu * duz + gv * dvz);
}

// ------------------------------------------------------------------------------------------
// K4a: Monte-Carlo adjoint, one thread per receiver pixel.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 4) k_bwd_mc(BwdArgs A) {
  const long long HW = (long long)A.vs.H * A.vs.W;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW * A.vs.V) return;
  const int view = (int)(p / HW);
  const int rem = (int)(p - view * HW);
  const int y = rem / A.vs.W, x = rem - y * A.vs.W;
  float3 ga = f3(0.f, 0.f, 0.f), gn = f3(0.f, 0.f, 0.f);
  float gr = 0.0f, gm = 0.0f;
  const float z = __ldg(A.depth + p);
  if (!is_background(z)) {
    const DevCam& cam = A.vs.cam[view];
    const float3 d = pix_dir_world(cam, x, y);
    const float3 v = d * (-1.0f / sqrtf(dot3(d, d)));
    const float3 n = ld3(A.normal + 3 * p);
    const float nv = dot3(n, v);
    const float rho = __ldg(A.rough + p), m = __ldg(A.metal + p);
    const float3 a = ld3(A.albedo + 3 * p);
    const float3 F0 = f3(f0_of(a.x, m), f0_of(a.y, m), f0_of(a.z, m));
    const float3 gC = ld3(A.g_final + 3 * p) * (1.0f / (float)A.spp);
    const float g1v = ggx_G1(nv, rho);
    float dgv_z, dgv_r;
    dlnG1(nv, rho, dgv_z, dgv_r);
    const bool want_cid = (A.flags & SSGI_DIFFUSE_INDIRECT) != 0;
    for (int s = 0; s < A.spp; ++s) {
      const float2 xi = sample_uniforms(A.seed, view, (uint32_t)rem, (uint32_t)s);
      const Sample sm = make_sample(n, v, nv, rho, xi);
      if (!sm.valid) continue;
      const int q = __ldg(A.hit_idx + p * A.spp + s);
      if (q >= HW) continue;  // not an index this G-buffer's trace can produce
      float3 Li;
      Taps tm;
      if (q >= 0) {
        Li = ld3(A.c1 + 3 * (view * HW + q));
      } else {
        tm = env_taps(A.e, 0, dir_angles(sm.w));
        Li = bilinear(A.mips, tm);
      }
      const float K = ggx_G1(sm.nw, rho) * g1v * sm.vh / (nv * sm.nh);
      const float fc = pow5(1.0f - sm.vh);
      const float3 F = F0 + (f3(1.f, 1.f, 1.f) - F0) * fc;
      float3 gL = mul3(gC, F) * K;
      const float3 gF = mul3(gC, Li) * K;
      ga = ga + gF * (m * (1.0f - fc));
      gm += dot3(gF, a - f3(0.04f, 0.04f, 0.04f)) * (1.0f - fc);
      const float gKK = dot3(gC, mul3(F, Li)) * K;
      float dgw_z, dgw_r;
      dlnG1(sm.nw, rho, dgw_z, dgw_r);
      float dlnK_r = dgw_r + dgv_r;
      float3 dlnK_n = sm.w * dgw_z + v * (dgv_z - 1.0f / nv);
      if (rho > 0.0f) {
        float dd_c, dd_r;
        dlnD(sm.nh, rho, dd_c, dd_r);
        dlnK_r += dd_r;
        dlnK_n = dlnK_n + sm.h * dd_c;
      }
      gr += gKK * dlnK_r;
      gn = gn + dlnK_n * gKK;
      if (want_cid) {
        const float pdf = ggx_D(sm.nh, rho) * sm.nh / (4.0f * sm.vh);
        if (pdf > 0.0f && isfinite(pdf)) {
          const float kk = kInvPi / pdf;
          ga = ga + mul3(gC, Li) * ((1.0f - m) * kk * sm.nw);
          gm -= dot3(gC, mul3(a, Li)) * kk * sm.nw;
          gn = gn + sm.w * (dot3(gC, mul3(a, Li)) * (1.0f - m) * kk);
          gL = gL + mul3(gC, a) * ((1.0f - m) * kk * sm.nw);
        }
      }
      if (q >= 0) {
        atomic_add3(A.g_c1 + 3 * (view * HW + q), gL);
      } else {
        float gx, gy;
        bilin_adj(A.mips, tm, gL, 1.0f, A.g_mips, gx, gy);
      }
    }
  }
  st3(A.g_albedo + 3 * p, ga);
  st3(A.g_normal + 3 * p, gn);
  A.g_rough[p] = gr;
  A.g_metal[p] = gm;
}

// ------------------------------------------------------------------------------------------
// K4b: direct-shading adjoint, one thread per pixel; adds to K4a's outputs.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bwd_direct(BwdArgs A) {
  const long long HW = (long long)A.vs.H * A.vs.W;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= HW * A.vs.V) return;
  const int view = (int)(p / HW);
  const int rem = (int)(p - view * HW);
  const int y = rem / A.vs.W, x = rem - y * A.vs.W;
  const DevCam& cam = A.vs.cam[view];
  const float3 d = pix_dir_world(cam, x, y);
  const float3 gc1 = ld3(A.g_c1 + 3 * p);
  const float3 gcd = ld3(A.g_final + 3 * p) + gc1;
  const float3 gcs = gc1;
  const float z = __ldg(A.depth + p);
  if (is_background(z)) {
    float gx, gy;
    bilin_adj(A.mips, env_taps(A.e, 0, dir_angles(d)), gcd, 1.0f, A.g_mips, gx, gy);
    return;
  }
  const float3 v = d * (-1.0f / sqrtf(dot3(d, d)));
  const float3 n = ld3(A.normal + 3 * p);
  const float nv = dot3(n, v);
  const float mu = fminf(fmaxf(nv, 1e-4f), 1.0f);
  const float3 r = n * (2.0f * nv) - v;
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
  const float gr = gA * ab.dA_drho + gB * ab.dB_drho + (gl1 + gl2) * lmax / ((rho + 1.0f) * 0.69314718055994531f);
  float* pa = A.g_albedo + 3 * p;
  float* pn = A.g_normal + 3 * p;
  st3(pa, ld3(pa) + ga);
  st3(pn, ld3(pn) + gn);
  A.g_rough[p] += gr;
  A.g_metal[p] += gm;
}

// ------------------------------------------------------------------------------------------
// K4c: mip-chain adjoint; base texel (i, j) collects g_mips[l][i >> l][j >> l] / 4^l.
// ------------------------------------------------------------------------------------------
__global__ void k_bwd_env(EnvInfo e, const float* __restrict__ g_mips, float* __restrict__ g_env) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int w0 = e.w[0];
  if (t >= e.h[0] * w0 * 3) return;
  const int c = t % 3, j = (t / 3) % w0, i = t / (3 * w0);
  float acc = 0.0f, scale = 1.0f;
  for (int l = 0; l < e.levels; ++l) {
    acc += scale * __ldg(g_mips + e.off[l] + ((i >> l) * e.w[l] + (j >> l)) * 3 + c);
    scale *= 0.25f;
  }
  g_env[t] = acc;
}

// ------------------------------------------------------------------------------------------
// L2 loss
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_l2(const float* __restrict__ f, const float* __restrict__ t, long long n,
                                            float* __restrict__ g, float* __restrict__ loss) {
  const float inv = 1.0f / (float)n;
  float acc = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float r = __ldg(f + i) - __ldg(t + i);
    g[i] = 2.0f * r * inv;
    acc += r * r;
  }
  if (!loss) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ float part[8];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.0f;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
    atomicAdd(loss, s * inv);
  }
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
  k_l2<<<blocks, 256, 0, s>>>(final_in, target, n, g_final, loss_out);
  return launch_status();
}

ssgi_status ssgi_backward(const float* g_final, const ssgi_gbuffer* g, const ssgi_camera* cams, const float* c1,
                          const ssgi_envmap* env, const float* lut, int32_t lut_n, const int32_t* hit_idx,
                          const ssgi_trace_params* p, float* g_albedo, float* g_rough, float* g_metal,
                          float* g_normal, float* g_env, void* workspace, size_t ws_bytes, ssgi_stream_t stream) {
  if (!g_final || gbuffer_ok(g) != SSGI_OK || trace_params_ok(p) != SSGI_OK || !c1 || !lut || lut_n < 2 ||
      !hit_idx || !g_albedo || !g_rough || !g_metal || !g_normal || !g_env || !workspace)
    return SSGI_ERR_INVALID_ARG;
  if (((uintptr_t)workspace & 15) != 0) return SSGI_ERR_INVALID_ARG;
  BwdArgs A;
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  const size_t need = ssgi_backward_workspace_bytes(g->d, env->h, env->w);
  if (need == 0 || ws_bytes < need) return SSGI_ERR_INVALID_ARG;
  const long long npx = (long long)g->d.views * g->d.height * g->d.width;
  const size_t c1_bytes = ((size_t)npx * 3 * sizeof(float) + 255) & ~(size_t)255;
  A.g_c1 = (float*)workspace;
  A.g_mips = (float*)((char*)workspace + c1_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, need, s) != cudaSuccess) return SSGI_ERR_CUDA;
  A.g_final = g_final;
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.c1 = c1;
  A.mips = env->mips;
  A.lut = lut;
  A.hit_idx = hit_idx;
  A.g_albedo = g_albedo;
  A.g_rough = g_rough;
  A.g_metal = g_metal;
  A.g_normal = g_normal;
  A.lut_n = lut_n;
  A.spp = p->spp;
  A.seed = p->seed;
  A.flags = p->flags;
  const int blocks = ceil_div(npx, 256);
  k_bwd_mc<<<blocks, 256, 0, s>>>(A);
  ssgi_status st = launch_status();
  if (st != SSGI_OK) return st;
  k_bwd_direct<<<blocks, 256, 0, s>>>(A);
  st = launch_status();
  if (st != SSGI_OK) return st;
  const int nt = env->h * env->w * 3;
  k_bwd_env<<<ceil_div(nt, 256), 256, 0, s>>>(A.e, A.g_mips, g_env);
  return launch_status();
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Allocation-free backward: the workspace is a fixed array in the library's device image, so
// callers that must not allocate device memory can still run the adjoint.  Device code could
// name the array directly; host code needs its device address, looked up once per device.
// ------------------------------------------------------------------------------------------
namespace ssgi {
namespace {
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[SSGI_BACKWARD_NOALLOC_MAX_BYTES];
std::mutex g_noalloc_mutex;
void* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (first call per device looks it
// up with that device current).
ssgi_status noalloc_scratch(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SSGI_ERR_CUDA;
  if (dev < 0 || dev >= kNoAllocMaxDevices) return SSGI_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return SSGI_ERR_CUDA;
    g_noalloc_addr[dev] = ptr;
  }
  *out = g_noalloc_addr[dev];
  return SSGI_OK;
}
}  // namespace
}  // namespace ssgi

extern "C" ssgi_status ssgi_backward_noalloc(const float* g_final, const ssgi_gbuffer* g, const ssgi_camera* cams,
                                             const float* c1, const ssgi_envmap* env, const float* lut,
                                             int32_t lut_n, const int32_t* hit_idx, const ssgi_trace_params* p,
                                             float* g_albedo, float* g_rough, float* g_metal, float* g_normal,
                                             float* g_env, ssgi_stream_t stream) {
  if (!g_final || gbuffer_ok(g) != SSGI_OK || trace_params_ok(p) != SSGI_OK || !c1 || !lut || lut_n < 2 ||
      !hit_idx || !g_albedo || !g_rough || !g_metal || !g_normal || !g_env)
    return SSGI_ERR_INVALID_ARG;
  BwdArgs A;
  if (make_views(cams, g->d, &A.vs) != SSGI_OK || make_env(env, &A.e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  const size_t need = ssgi_backward_workspace_bytes(g->d, env->h, env->w);
  if (need == 0) return SSGI_ERR_INVALID_ARG;
  if (need > (size_t)SSGI_BACKWARD_NOALLOC_MAX_BYTES) return SSGI_ERR_UNSUPPORTED;
  void* workspace = nullptr;
  const ssgi_status ss = noalloc_scratch(&workspace);
  if (ss != SSGI_OK) return ss;
  const long long npx = (long long)g->d.views * g->d.height * g->d.width;
  const size_t c1_bytes = ((size_t)npx * 3 * sizeof(float) + 255) & ~(size_t)255;
  A.g_c1 = (float*)workspace;
  A.g_mips = (float*)((char*)workspace + c1_bytes);
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(workspace, 0, need, s) != cudaSuccess) return SSGI_ERR_CUDA;
  A.g_final = g_final;
  A.depth = g->depth;
  A.normal = g->normal;
  A.albedo = g->albedo;
  A.rough = g->rough;
  A.metal = g->metal;
  A.c1 = c1;
  A.mips = env->mips;
  A.lut = lut;
  A.hit_idx = hit_idx;
  A.g_albedo = g_albedo;
  A.g_rough = g_rough;
  A.g_metal = g_metal;
  A.g_normal = g_normal;
  A.lut_n = lut_n;
  A.spp = p->spp;
  A.seed = p->seed;
  A.flags = p->flags;
  const int blocks = ceil_div(npx, 256);
  k_bwd_mc<<<blocks, 256, 0, s>>>(A);
  ssgi_status st = launch_status();
  if (st != SSGI_OK) return st;
  k_bwd_direct<<<blocks, 256, 0, s>>>(A);
  st = launch_status();
  if (st != SSGI_OK) return st;
  const int nt = env->h * env->w * 3;
  k_bwd_env<<<ceil_div(nt, 256), 256, 0, s>>>(A.e, A.g_mips, g_env);
  return launch_status();
}
