// abi.cu -- status strings, size queries and argument validation of the SSGI C ABI.
#include <math.h>
#include <string.h>

#include "ssgi_internal.h"

namespace ssgi {

bool dims_ok(ssgi_dims d) {
  if (d.views < 1 || d.views > SSGI_MAX_VIEWS) return false;
  if (d.height < 1 || d.width < 1 || d.height > 16384 || d.width > 16384) return false;
  return (long long)d.views * d.height * d.width <= (1LL << 28);
}

ssgi_status make_views(const ssgi_camera* cams, ssgi_dims d, Views* out) {
  if (!cams || !dims_ok(d)) return SSGI_ERR_INVALID_ARG;
  out->V = d.views;
  out->H = d.height;
  out->W = d.width;
  for (int v = 0; v < d.views; ++v) {
    const ssgi_camera& c = cams[v];
    if (!(c.fov_y_rad > 0.0f && c.fov_y_rad < 3.1f) || !(c.z_near > 0.0f)) return SSGI_ERR_INVALID_ARG;
    DevCam& o = out->cam[v];
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) o.R[i * 3 + j] = c.cam_to_world[i * 4 + j];
      o.eye[i] = c.cam_to_world[i * 4 + 3];
    }
    o.f = (float)((d.height / 2.0) / tan((double)c.fov_y_rad / 2.0));
    o.cx = (float)(d.width / 2.0);
    o.cy = (float)(d.height / 2.0);
    o.znear = c.z_near;
  }
  return SSGI_OK;
}

ssgi_status make_env_dims(int32_t h, int32_t w, EnvInfo* out) {
  const int L = ssgi_env_levels(h, w);
  if (L < 1) return SSGI_ERR_INVALID_ARG;
  out->levels = L;
  int off = 0;
  for (int l = 0; l < L; ++l) {
    out->h[l] = h >> l;
    out->w[l] = w >> l;
    out->off[l] = off;
    off += out->h[l] * out->w[l] * 3;
  }
  out->total_floats = off;
  return SSGI_OK;
}

ssgi_status make_env(const ssgi_envmap* env, EnvInfo* out) {
  if (!env || !env->mips) return SSGI_ERR_INVALID_ARG;
  if (make_env_dims(env->h, env->w, out) != SSGI_OK) return SSGI_ERR_INVALID_ARG;
  if (env->levels != out->levels) return SSGI_ERR_INVALID_ARG;
  return SSGI_OK;
}

void make_hiz_info(ssgi_dims d, int levels, HizInfo* out) {
  out->levels = levels;
  int off = 0;
  out->off[0] = 0;
  out->w[0] = d.width;
  out->h[0] = d.height;
  for (int l = 1; l < levels; ++l) {
    out->off[l] = off;
    out->w[l] = lvl_dim(d.width, l);
    out->h[l] = lvl_dim(d.height, l);
    off += out->w[l] * out->h[l];
  }
  for (int l = levels; l < SSGI_MAX_HIZ_LEVELS; ++l) {
    out->off[l] = off;
    out->w[l] = 1;
    out->h[l] = 1;
  }
  out->per_view = off;
}

ssgi_status gbuffer_ok(const ssgi_gbuffer* g) {
  if (!g || !g->depth || !g->normal || !g->albedo || !g->rough || !g->metal) return SSGI_ERR_INVALID_ARG;
  if (!dims_ok(g->d)) return SSGI_ERR_INVALID_ARG;
  return SSGI_OK;
}

ssgi_status trace_params_ok(const ssgi_trace_params* p) {
  if (!p) return SSGI_ERR_INVALID_ARG;
  if (p->spp < 1 || p->spp > 1024 || p->max_steps < 0) return SSGI_ERR_INVALID_ARG;
  if (p->hiz_levels < 1 || p->hiz_levels > SSGI_MAX_HIZ_LEVELS) return SSGI_ERR_INVALID_ARG;
  if (!(p->thickness >= 0.0f) || !(p->max_distance > 0.0f)) return SSGI_ERR_INVALID_ARG;
  if (p->flags & ~(uint32_t)(SSGI_DIFFUSE_INDIRECT | SSGI_BRUTE_FORCE | SSGI_PATHWISE | SSGI_SRGB_LOSS | SSGI_SRGB_FINAL))
    return SSGI_ERR_INVALID_ARG;
  return SSGI_OK;
}

ssgi_status launch_status() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? SSGI_OK : SSGI_ERR_CUDA;
}

}  // namespace ssgi

extern "C" {

const char* ssgi_status_string(ssgi_status s) {
  switch (s) {
    case SSGI_OK: return "ok";
    case SSGI_ERR_INVALID_ARG: return "invalid argument";
    case SSGI_ERR_UNSUPPORTED: return "unsupported";
    case SSGI_ERR_CUDA: return "CUDA error";
    case SSGI_ERR_OOM: return "out of memory";
    case SSGI_ERR_BUDGET: return "over the device-memory budget";
    case SSGI_ERR_QUEUE_FULL: return "queue full";
    case SSGI_ERR_TIMEOUT: return "timed out";
    case SSGI_ERR_NOT_READY: return "not ready";
    case SSGI_ERR_CANCELLED: return "cancelled";
  }
  return "unknown status";
}

const char* ssgi_version(void) { return "ssgi 0.1 sm_103a"; }

int32_t ssgi_env_levels(int32_t h, int32_t w) {
  if (h < 1 || w < h) return -1;
  if ((h & (h - 1)) != 0 || (w & (w - 1)) != 0) return -1;
  int l = 0;
  while ((1 << l) < h) ++l;
  if (l + 1 > SSGI_MAX_ENV_LEVELS) return -1;
  if ((long long)h * w > (1LL << 26)) return -1;
  return l + 1;
}

size_t ssgi_env_mip_floats(int32_t h, int32_t w) {
  ssgi::EnvInfo e;
  if (ssgi::make_env_dims(h, w, &e) != SSGI_OK) return 0;
  return (size_t)e.total_floats;
}

size_t ssgi_hiz_floats(ssgi_dims d, int32_t levels) {
  if (!ssgi::dims_ok(d) || levels < 1 || levels > SSGI_MAX_HIZ_LEVELS) return 0;
  ssgi::HizInfo hz;
  ssgi::make_hiz_info(d, levels, &hz);
  return (size_t)hz.per_view * (size_t)d.views;
}

size_t ssgi_backward_workspace_bytes(ssgi_dims d, int32_t env_h, int32_t env_w) {
  if (!ssgi::dims_ok(d)) return 0;
  const size_t mf = ssgi_env_mip_floats(env_h, env_w);
  if (mf == 0) return 0;
  // g_c1: one RGB + pad (16 bytes) per pixel; the mip-chain gradient: one per texel
  const size_t px = (size_t)d.views * d.height * d.width;
  const size_t a = (px * 16 + 255) & ~(size_t)255;
  return a + ((mf / 3 * 16 + 255) & ~(size_t)255);
}

}  // extern "C"
