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

// Environment mips in two launches: 32 x 32 texel tiles copied and reduced through level 5 in
// shared memory, then one block builds levels 6.. from level 5.
__global__ void __launch_bounds__(256) k_env_tiles(const float* env0, EnvInfo e, float* mips) {
  __shared__ TileBuf s;
  env_tile_block<kHizTile>(env0, e, mips, blockIdx.x, blockIdx.y, s);
}

__global__ void __launch_bounds__(256) k_env_upper(EnvInfo e, float* mips) { env_upper_block(e, mips); }

// Hi-Z in two launches: 32 x 32 tiles through level 5, then one block per view for levels 6..
__global__ void __launch_bounds__(256) k_hiz_tile(const float* __restrict__ depth, int H, int W, HizInfo hz,
                                                  float* __restrict__ hiz) {
  __shared__ TileBuf s;
  hiz_tile_block<kHizTile>(depth, H, W, hz, hiz, blockIdx.z, blockIdx.x, blockIdx.y, s);
}

__global__ void __launch_bounds__(256) k_hiz_upper(HizInfo hz, float* hiz) { hiz_upper_block(hz, blockIdx.x, hiz); }

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
  // tiles are exact: the sizes are powers of two (env may equal mips_out: level 0 is rewritten
  // with its own values)
  const dim3 grid(w / (w < kHizTile ? w : kHizTile), h / (h < kHizTile ? h : kHizTile));
  k_env_tiles<<<grid, 256, 0, s>>>(env, e, mips_out);
  ssgi_status st = launch_status();
  if (st == SSGI_OK && e.levels > 6) {
    k_env_upper<<<1, 256, 0, s>>>(e, mips_out);
    st = launch_status();
  }
  return st;
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
  if (st == SSGI_OK && levels > 6) {
    k_hiz_upper<<<d.views, 256, 0, s>>>(hz, hiz_out);
    st = launch_status();
  }
  return st;
}

}  // extern "C"
