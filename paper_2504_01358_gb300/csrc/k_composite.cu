// k_composite.cu -- object insertion (Sec. 4 "Object Insertion"): an object's G-buffer, rendered
// on its own, merged into the scene's by depth comparison before the pyramid and shading passes.
// A pixel takes all five of the object's channels where the object's depth is strictly smaller
// than the scene's; ties and object background (+inf) keep the scene.  In place (outputs equal
// to the scene's planes) only the object's pixels are written.
#include "ssgi_internal.h"
#include "ssgi_device.cuh"

namespace ssgi {

struct CompositeArgs {
  const float *sd, *sn, *sa, *sr, *sm;  // scene
  const float *od, *on, *oa, *orr, *om; // object
  float *dd, *dn, *da, *dr, *dm;        // out
  uint8_t* mask;
  long long npx;
  bool in_place;
};

__global__ void __launch_bounds__(256) k_composite(CompositeArgs a) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.npx) return;
  const float zs = __ldg(a.sd + p), zo = __ldg(a.od + p);
  const bool win = zo < zs;
  if (a.mask) a.mask[p] = win ? 1 : 0;
  if (win) {
    a.dd[p] = zo;
    st3(a.dn + 3 * p, ld3(a.on + 3 * p));
    st3(a.da + 3 * p, ld3(a.oa + 3 * p));
    a.dr[p] = __ldg(a.orr + p);
    a.dm[p] = __ldg(a.om + p);
  } else if (!a.in_place) {
    a.dd[p] = zs;
    st3(a.dn + 3 * p, ld3(a.sn + 3 * p));
    st3(a.da + 3 * p, ld3(a.sa + 3 * p));
    a.dr[p] = __ldg(a.sr + p);
    a.dm[p] = __ldg(a.sm + p);
  }
}

}  // namespace ssgi

using namespace ssgi;

extern "C" ssgi_status ssgi_composite_gbuffer(const ssgi_gbuffer* scene, const ssgi_gbuffer* object, float* out_depth,
                                              float* out_normal, float* out_albedo, float* out_rough,
                                              float* out_metal, uint8_t* mask_out, ssgi_stream_t stream) {
  if (!scene || !object || gbuffer_ok(scene) != SSGI_OK || gbuffer_ok(object) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  if (scene->d.views != object->d.views || scene->d.height != object->d.height || scene->d.width != object->d.width)
    return SSGI_ERR_INVALID_ARG;
  if (!out_depth || !out_normal || !out_albedo || !out_rough || !out_metal) return SSGI_ERR_INVALID_ARG;
  const bool same = out_depth == scene->depth && out_normal == scene->normal && out_albedo == scene->albedo &&
                    out_rough == scene->rough && out_metal == scene->metal;
  const bool none = out_depth != scene->depth && out_normal != scene->normal && out_albedo != scene->albedo &&
                    out_rough != scene->rough && out_metal != scene->metal;
  if (!same && !none) return SSGI_ERR_INVALID_ARG;  // all planes in place, or none
  CompositeArgs a;
  a.sd = scene->depth; a.sn = scene->normal; a.sa = scene->albedo; a.sr = scene->rough; a.sm = scene->metal;
  a.od = object->depth; a.on = object->normal; a.oa = object->albedo; a.orr = object->rough; a.om = object->metal;
  a.dd = out_depth; a.dn = out_normal; a.da = out_albedo; a.dr = out_rough; a.dm = out_metal;
  a.mask = mask_out;
  a.npx = (long long)scene->d.views * scene->d.height * scene->d.width;
  a.in_place = same;
  k_composite<<<ceil_div(a.npx, 256), 256, 0, (cudaStream_t)stream>>>(a);
  return launch_status();
}
