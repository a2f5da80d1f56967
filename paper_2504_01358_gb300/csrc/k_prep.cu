// k_prep.cu -- per-frame and per-environment precomputation: the BRDF-integral table
// (Appendix C), the environment mip chain (Sec. 3.2, SampleEnvMap) and the hierarchical-Z
// pyramid used by the screen-space march (Sec. 3.3).  Stage bodies live in ssgi_ops.cuh.
#include "ssgi_ops.cuh"

namespace ssgi {

// ------------------------------------------------------------------------------------------
// BRDF table.  One warp per entry; lanes take strided Hammersley samples and reduce.
// ------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_brdf_lut(int N, int M, float* __restrict__ lut) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= N * N) return;
  const int i = warp / N, j = warp % N;
  const float rho = ((float)i + 0.5f) / (float)N;
  const float mu = ((float)j + 0.5f) / (float)N;
  const float3 v = f3(sqrtf(fmaxf(0.0f, 1.0f - mu * mu)), 0.0f, mu);
  const float3 n = f3(0.0f, 0.0f, 1.0f);
  const float g1v = ggx_G1(mu, rho);
  float A = 0.0f, B = 0.0f;
  for (int k = lane; k < M; k += 32) {
    const float xi0 = ((float)k + 0.5f) / (float)M;
    const float xi1 = (float)__brev((uint32_t)k) * (1.0f / 4294967296.0f);
    float nh;
    const float3 h = ggx_sample_h(n, rho, xi0, xi1, &nh);
    const float vh = dot3(v, h);
    const float lz = fmaf(2.0f * vh, nh, -mu);
    if (lz <= 0.0f || vh <= 0.0f || nh <= 0.0f) continue;
    const float w = ggx_G1(lz, rho) * g1v * vh / (nh * mu);
    const float fc = pow5(1.0f - vh);
    A += w * (1.0f - fc);
    B += w * fc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    A += __shfl_xor_sync(0xffffffffu, A, o);
    B += __shfl_xor_sync(0xffffffffu, B, o);
  }
  if (lane == 0) {
    lut[(i * N + j) * 2 + 0] = A / (float)M;
    lut[(i * N + j) * 2 + 1] = B / (float)M;
  }
}

__global__ void k_env_down(const float* __restrict__ src, int hs, int ws, float* __restrict__ dst) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (hs >> 1) * (ws >> 1) * 3) return;
  env_down_item(src, hs, ws, dst, t);
}

__global__ void __launch_bounds__(256) k_hiz_tile(const float* __restrict__ depth, int H, int W, HizInfo hz,
                                                  float* __restrict__ hiz) {
  __shared__ TileBuf s;
  hiz_tile_block(depth, H, W, hz, hiz, blockIdx.z, blockIdx.x, blockIdx.y, s);
}

__global__ void k_hiz_level(int V, HizInfo hz, int l, float* __restrict__ hiz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= V * hz.w[l] * hz.h[l]) return;
  hiz_level_item(hz, l, hiz, t);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" {

ssgi_status ssgi_build_brdf_lut(int32_t n, int32_t samples, float* lut_out, ssgi_stream_t stream) {
  if (!lut_out || n < 2 || n > 1024 || samples < 1 || samples > (1 << 20)) return SSGI_ERR_INVALID_ARG;
  const int warps = n * n;
  const int threads = 256;
  const int blocks = ceil_div((long long)warps * 32, threads);
  k_brdf_lut<<<blocks, threads, 0, (cudaStream_t)stream>>>(n, samples, lut_out);
  return launch_status();
}

ssgi_status ssgi_build_env_mips(const float* env, int32_t h, int32_t w, float* mips_out, ssgi_stream_t stream) {
  EnvInfo e;
  if (!env || !mips_out || make_env_dims(h, w, &e) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (env != mips_out) {
    if (cudaMemcpyAsync(mips_out, env, sizeof(float) * (size_t)h * w * 3, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return SSGI_ERR_CUDA;
  }
  for (int l = 1; l < e.levels; ++l) {
    const int n = e.h[l] * e.w[l] * 3;
    k_env_down<<<ceil_div(n, 256), 256, 0, s>>>(mips_out + e.off[l - 1], e.h[l - 1], e.w[l - 1], mips_out + e.off[l]);
    const ssgi_status st = launch_status();
    if (st != SSGI_OK) return st;
  }
  return SSGI_OK;
}

ssgi_status ssgi_build_hiz(const float* depth, ssgi_dims d, int32_t levels, float* hiz_out, ssgi_stream_t stream) {
  if (!depth || !dims_ok(d) || levels < 1 || levels > SSGI_MAX_HIZ_LEVELS) return SSGI_ERR_INVALID_ARG;
  if (levels == 1) return SSGI_OK;
  if (!hiz_out) return SSGI_ERR_INVALID_ARG;
  HizInfo hz;
  make_hiz_info(d, levels, &hz);
  cudaStream_t s = (cudaStream_t)stream;
  dim3 grid(ceil_div(d.width, kHizTile), ceil_div(d.height, kHizTile), d.views);
  k_hiz_tile<<<grid, 256, 0, s>>>(depth, d.height, d.width, hz, hiz_out);
  ssgi_status st = launch_status();
  for (int l = 6; l < levels && st == SSGI_OK; ++l) {
    const int n = d.views * hz.w[l] * hz.h[l];
    k_hiz_level<<<ceil_div(n, 256), 256, 0, s>>>(d.views, hz, l, hiz_out);
    st = launch_status();
  }
  return st;
}

}  // extern "C"
