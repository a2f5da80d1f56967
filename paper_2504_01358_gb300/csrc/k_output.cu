// k_output.cu -- the output transform and keyframe lighting.
//
//   ssgi_tonemap_srgb           tone mapping + gamma to sRGB after the composite (Sec. 3.3):
//                               clamp to [0, 1], then the sRGB transfer function (IEC 61966-2-1)
//   ssgi_l2_loss_srgb           L2 loss of the sRGB image against an sRGB target and its gradient
//                               with respect to the linear image, in one pass
//   ssgi_env_keyframe_lerp      keyframe lighting (Sec. 4 implementation details): every 10th
//   (+ _backward)               frame has its own environment map, frames in between blend their
//                               two neighbouring keyframes linearly; the adjoint splits the map's
//                               gradient between them
//   ssgi_keyframe_of            which keyframes and weight a frame uses (host)
#include "ssgi_ops.cuh"

namespace ssgi {

// 16-byte accesses where both arrays are 16-byte aligned (x may equal y), the tail per element.
__global__ void __launch_bounds__(256) k_tonemap_srgb(const float* x, float* y, long long n, bool vec4) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long n4 = vec4 ? n / 4 : 0;
  for (long long i = t0; i < n4; i += stride) {
    const float4 v = reinterpret_cast<const float4*>(x)[i];
    reinterpret_cast<float4*>(y)[i] = make_float4(tonemap_srgb(v.x), tonemap_srgb(v.y), tonemap_srgb(v.z), tonemap_srgb(v.w));
  }
  for (long long i = 4 * n4 + t0; i < n; i += stride) y[i] = tonemap_srgb(x[i]);
}

__global__ void __launch_bounds__(256) k_l2_srgb(const float* __restrict__ f, const float* __restrict__ t, long long n,
                                                 float* __restrict__ g, float* __restrict__ loss, bool vec4) {
  l2_block_vec<true>(f, t, n, g, loss, vec4);
}

inline bool aligned16(const void* a, const void* b, const void* c = nullptr) {
  return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c) & 15) == 0;
}

__global__ void __launch_bounds__(256) k_env_lerp(const float* __restrict__ a, const float* __restrict__ b, float alpha,
                                                  float* __restrict__ out, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (1.0f - alpha) * __ldg(a + i) + alpha * __ldg(b + i);
}

__global__ void __launch_bounds__(256) k_env_lerp_bwd(const float* __restrict__ g, float alpha, float* __restrict__ ga,
                                                      float* __restrict__ gb, long long n, int accumulate) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float v = __ldg(g + i);
    const float wa = (1.0f - alpha) * v, wb = alpha * v;
    ga[i] = accumulate ? ga[i] + wa : wa;
    gb[i] = accumulate ? gb[i] + wb : wb;
  }
}

inline int grid_for(long long n) {
  const long long b = (n + 255) / 256;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" {

ssgi_status ssgi_tonemap_srgb(const float* linear, float* srgb, int64_t n, ssgi_stream_t stream) {
  if (!linear || !srgb || n < 1) return SSGI_ERR_INVALID_ARG;
  k_tonemap_srgb<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(linear, srgb, n, aligned16(linear, srgb));
  return launch_status();
}

ssgi_status ssgi_l2_loss_srgb(const float* final_in, const float* target, int64_t n, float* g_final, float* loss_out,
                              ssgi_stream_t stream) {
  if (!final_in || !target || !g_final || n < 1) return SSGI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (loss_out && cudaMemsetAsync(loss_out, 0, sizeof(float), s) != cudaSuccess) return SSGI_ERR_CUDA;
  k_l2_srgb<<<grid_for(n), 256, 0, s>>>(final_in, target, n, g_final, loss_out, aligned16(final_in, target, g_final));
  return launch_status();
}

ssgi_status ssgi_env_keyframe_lerp(const float* env_a, const float* env_b, float alpha, int32_t env_h, int32_t env_w,
                                   float* env_out, ssgi_stream_t stream) {
  if (!env_a || !env_b || !env_out || env_h < 1 || env_w < 1 || !(alpha >= 0.0f && alpha <= 1.0f))
    return SSGI_ERR_INVALID_ARG;
  const long long n = (long long)env_h * env_w * 3;
  k_env_lerp<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(env_a, env_b, alpha, env_out, n);
  return launch_status();
}

ssgi_status ssgi_env_keyframe_lerp_backward(const float* g_env, float alpha, int32_t env_h, int32_t env_w, float* g_a,
                                            float* g_b, int32_t accumulate, ssgi_stream_t stream) {
  if (!g_env || !g_a || !g_b || g_a == g_b || env_h < 1 || env_w < 1 || !(alpha >= 0.0f && alpha <= 1.0f))
    return SSGI_ERR_INVALID_ARG;
  const long long n = (long long)env_h * env_w * 3;
  k_env_lerp_bwd<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(g_env, alpha, g_a, g_b, n, accumulate ? 1 : 0);
  return launch_status();
}

ssgi_status ssgi_keyframe_of(int64_t frame, int32_t period, int64_t* keyframe, float* alpha) {
  if (frame < 0 || period < 1 || !keyframe || !alpha) return SSGI_ERR_INVALID_ARG;
  *keyframe = frame / period;
  *alpha = (float)(frame % period) / (float)period;
  return SSGI_OK;
}

}  // extern "C"
