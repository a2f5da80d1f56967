// k_normals.cu -- depth normals (Sec. 3.1: surface normals from the rendered depth buffer by
// finite differences, as in 2DGS).
//
// P(x, y) = d(x, y) z(x, y) is the camera-space point of the pixel centre at linear depth z.
// Per image direction the difference is central where both neighbours are foreground,
// one-sided where only one is, absent where neither is; n = normalize(dP/dy x dP/dx) (y down the
// image), flipped to face the camera, rotated to world space.  With a direction absent or a zero
// cross product n is the unit vector towards the camera; background pixels get (0, 0, 0).
//
// The differences are written as (d_r - d_l) z_l + d_r (z_r - z_l): the direction difference is
// exact ((r - l) / f in one component) and z_r - z_l is exact for nearby depths, so the FP32
// result keeps its relative accuracy where P_r - P_l would cancel.
#include "ssgi_ops.cuh"

namespace ssgi {

constexpr int kNormBX = 32, kNormBY = 8;

// Depth normal of foreground pixel (x, y) (z = its depth), the neighbours' depths read through
// zat(x, y) (+inf or another non-finite value, i.e. background, outside the image).  Every sum
// of products is written out (explicit fused or separate roundings), so the kernels that
// inline it produce the same bits.
template <class ZAt>
__device__ __forceinline__ float3 depth_normal(const DevCam& c, int x, int y, float z, ZAt zat) {
  const bool hl = !is_background(zat(x - 1, y)), hr = !is_background(zat(x + 1, y));
  const bool hu = !is_background(zat(x, y - 1)), hb = !is_background(zat(x, y + 1));
  const int l = hl ? x - 1 : x, r = hr ? x + 1 : x, u = hu ? y - 1 : y, b = hb ? y + 1 : y;
  const float3 dc = pix_dir_cam(c, x, y);
  const float3 P = dc * z;
  float3 n = P * (-1.0f / sqrtf(dot3_rn(P, P)));
  if (l != r && u != b) {
    const float zl = zat(l, y), zr = zat(r, y);
    const float zu = zat(x, u), zb = zat(x, b);
    const float3 dr = pix_dir_cam(c, r, y), db = pix_dir_cam(c, x, b);
    const float ex = zr - zl, ey = zb - zu;
    const float ax = (float)(r - l) / c.f, ay = (float)(b - u) / c.f;
    const float3 dPx = f3(fmaf(ax, zl, dr.x * ex), dr.y * ex, -ex);
    const float3 dPy = f3(db.x * ey, fmaf(-ay, zu, db.y * ey), -ey);
    // dP/dy x dP/dx; its x and y components in closed form (dr.y - db.y = (b - y) / f and
    // dr.x - db.x = (r - x) / f): the generic products cancel for surfaces seen at a grazing angle
    const float3 cr = f3(ex * fmaf(ey, (float)(b - y) / c.f, ay * zu), -ey * fmaf(ex, (float)(r - x) / c.f, ax * zl),
                         __fmaf_rn(dPy.x, dPx.y, -__fmul_rn(dPy.y, dPx.x)));
    const float cl2 = dot3_rn(cr, cr);
    if (cl2 > 0.0f) {
      n = cr * (1.0f / sqrtf(cl2));
      if (dot3_rn(n, P) > 0.0f) n = n * -1.0f;
    }
  }
  return cam_to_world(c, n);
}

__global__ void __launch_bounds__(kNormBX* kNormBY) k_depth_normals(Views vs, const float* __restrict__ depth,
                                                                    float* __restrict__ normal_out) {
  const int x = blockIdx.x * kNormBX + threadIdx.x, y = blockIdx.y * kNormBY + threadIdx.y, view = blockIdx.z;
  const int H = vs.H, W = vs.W;
  if (x >= W || y >= H) return;
  const float* dz = depth + (size_t)view * H * W;
  const size_t p = (size_t)view * H * W + (size_t)y * W + x;
  const float z = __ldg(dz + (size_t)y * W + x);
  if (is_background(z)) {
    st3(normal_out + 3 * p, f3(0.f, 0.f, 0.f));
    return;
  }
  auto zat = [&](int xx, int yy) {
    return (xx >= 0 && xx < W && yy >= 0 && yy < H) ? __ldg(dz + (size_t)yy * W + xx) : INFINITY;
  };
  st3(normal_out + 3 * p, depth_normal(vs.cam[view], x, y, z, zat));
}

// Depth normals and the Hi-Z pyramid's levels 1..5 from one read of depth (Sec. 3.1's depth
// normals fused into the pyramid's pass): a 32 x 32 tile with a one-pixel border in shared
// memory; normals of the tile's pixels from it (the same arithmetic as k_depth_normals, so the
// same bits), then the tile's reduction (hiz_tile_reduce, the same bits as k_hiz_tile).
__global__ void __launch_bounds__(256) k_hiz_normals_tile(Views vs, const float* __restrict__ depth, HizInfo hz,
                                                          float* __restrict__ hiz, float* __restrict__ normal_out) {
  __shared__ float sd[kHizTile + 2][kHizTile + 3];
  __shared__ TileBuf s;
  const int H = vs.H, W = vs.W, view = blockIdx.z;
  const int bx = blockIdx.x * kHizTile, by = blockIdx.y * kHizTile;
  const float* d0 = depth + (size_t)view * H * W;
  for (int k = threadIdx.x; k < (kHizTile + 2) * (kHizTile + 2); k += blockDim.x) {
    const int ty = k / (kHizTile + 2), tx = k % (kHizTile + 2);
    const int y = by + ty - 1, x = bx + tx - 1;
    sd[ty][tx] = (y >= 0 && y < H && x >= 0 && x < W) ? __ldg(d0 + (size_t)y * W + x) : INFINITY;
  }
  __syncthreads();
  const DevCam& c = vs.cam[view];
  auto zat = [&](int xx, int yy) { return sd[yy - by + 1][xx - bx + 1]; };
  for (int k = threadIdx.x; k < kHizTile * kHizTile; k += blockDim.x) {
    const int ty = k / kHizTile, tx = k % kHizTile;
    const int y = by + ty, x = bx + tx;
    const float z = sd[ty + 1][tx + 1];
    s[ty][tx] = z;
    if (y < H && x < W) {
      const size_t p = (size_t)view * H * W + (size_t)y * W + x;
      st3(normal_out + 3 * p, is_background(z) ? f3(0.f, 0.f, 0.f) : depth_normal(c, x, y, z, zat));
    }
  }
  __syncthreads();
  if (hz.levels > 1) hiz_tile_reduce<kHizTile>(H, W, hz, hiz, view, blockIdx.x, blockIdx.y, s);
}

__global__ void __launch_bounds__(256) k_hiz_normals_upper(HizInfo hz, float* hiz) {
  hiz_upper_block(hz, blockIdx.x, hiz);
}

}  // namespace ssgi

using namespace ssgi;

extern "C" ssgi_status ssgi_depth_normals(const float* depth, ssgi_dims d, const ssgi_camera* cams, float* normal_out,
                                          ssgi_stream_t stream) {
  if (!depth || !cams || !normal_out || !dims_ok(d)) return SSGI_ERR_INVALID_ARG;
  Views vs;
  if (make_views(cams, d, &vs) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  const dim3 grid(ceil_div(d.width, kNormBX), ceil_div(d.height, kNormBY), d.views);
  k_depth_normals<<<grid, dim3(kNormBX, kNormBY), 0, (cudaStream_t)stream>>>(vs, depth, normal_out);
  return launch_status();
}

extern "C" ssgi_status ssgi_build_hiz_normals(const float* depth, ssgi_dims d, const ssgi_camera* cams, int32_t levels,
                                              float* hiz_out, float* normal_out, ssgi_stream_t stream) {
  if (!depth || !cams || !normal_out || !dims_ok(d) || levels < 1 || levels > SSGI_MAX_HIZ_LEVELS)
    return SSGI_ERR_INVALID_ARG;
  if (levels > 1 && !hiz_out) return SSGI_ERR_INVALID_ARG;
  Views vs;
  if (make_views(cams, d, &vs) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  HizInfo hz;
  make_hiz_info(d, levels, &hz);
  cudaStream_t s = (cudaStream_t)stream;
  const dim3 grid(ceil_div(d.width, kHizTile), ceil_div(d.height, kHizTile), d.views);
  k_hiz_normals_tile<<<grid, 256, 0, s>>>(vs, depth, hz, hiz_out, normal_out);
  ssgi_status st = launch_status();
  if (st == SSGI_OK && levels > 6) {
    k_hiz_normals_upper<<<d.views, 256, 0, s>>>(hz, hiz_out);
    st = launch_status();
  }
  return st;
}
