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
#include "ssgi_internal.h"
#include "ssgi_device.cuh"

namespace ssgi {

constexpr int kNormBX = 32, kNormBY = 8;

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
  const DevCam& c = vs.cam[view];
  const int l = (x > 0 && !is_background(__ldg(dz + (size_t)y * W + x - 1))) ? x - 1 : x;
  const int r = (x + 1 < W && !is_background(__ldg(dz + (size_t)y * W + x + 1))) ? x + 1 : x;
  const int u = (y > 0 && !is_background(__ldg(dz + (size_t)(y - 1) * W + x))) ? y - 1 : y;
  const int b = (y + 1 < H && !is_background(__ldg(dz + (size_t)(y + 1) * W + x))) ? y + 1 : y;
  const float3 dc = pix_dir_cam(c, x, y);
  const float3 P = dc * z;
  float3 n = P * (-1.0f / sqrtf(dot3(P, P)));
  if (l != r && u != b) {
    const float zl = __ldg(dz + (size_t)y * W + l), zr = __ldg(dz + (size_t)y * W + r);
    const float zu = __ldg(dz + (size_t)u * W + x), zb = __ldg(dz + (size_t)b * W + x);
    const float3 dr = pix_dir_cam(c, r, y), db = pix_dir_cam(c, x, b);
    const float ex = zr - zl, ey = zb - zu;
    const float ax = (float)(r - l) / c.f, ay = (float)(b - u) / c.f;
    const float3 dPx = f3(fmaf(ax, zl, dr.x * ex), dr.y * ex, -ex);
    const float3 dPy = f3(db.x * ey, fmaf(-ay, zu, db.y * ey), -ey);
    // dP/dy x dP/dx; its x and y components in closed form (dr.y - db.y = (b - y) / f and
    // dr.x - db.x = (r - x) / f): the generic products cancel for surfaces seen at a grazing angle
    const float3 cr = f3(ex * fmaf(ey, (float)(b - y) / c.f, ay * zu), -ey * fmaf(ex, (float)(r - x) / c.f, ax * zl),
                         dPy.x * dPx.y - dPy.y * dPx.x);
    const float cl2 = dot3(cr, cr);
    if (cl2 > 0.0f) {
      n = cr * (1.0f / sqrtf(cl2));
      if (dot3(n, P) > 0.0f) n = n * -1.0f;
    }
  }
  st3(normal_out + 3 * p, cam_to_world(c, n));
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
