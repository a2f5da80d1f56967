// ssgi_internal.h -- host/device descriptors passed to the SSGI kernels by value, and the
// host-side validation helpers shared by the C-ABI entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ssgi.h"

namespace ssgi {

// Camera as the kernels use it: R row-major (world <- camera), focal length and principal
// point in pixels, near plane.
struct DevCam {
  float R[9];
  float eye[3];
  float f, cx, cy, znear;
};

struct Views {
  DevCam cam[SSGI_MAX_VIEWS];
  int V, H, W;
};

// Packed environment mip chain: per level height, width and float offset.
struct EnvInfo {
  int h[SSGI_MAX_ENV_LEVELS];
  int w[SSGI_MAX_ENV_LEVELS];
  int off[SSGI_MAX_ENV_LEVELS];
  int levels;
  int total_floats;
};

// Packed hierarchical-Z pyramid of one view: float offset and width of levels 1..L-1.
struct HizInfo {
  int off[SSGI_MAX_HIZ_LEVELS];
  int w[SSGI_MAX_HIZ_LEVELS];
  int h[SSGI_MAX_HIZ_LEVELS];
  int levels;
  int per_view;
};

inline int lvl_dim(int n, int l) { return (n + (1 << l) - 1) >> l; }

bool dims_ok(ssgi_dims d);
ssgi_status make_views(const ssgi_camera* cams, ssgi_dims d, Views* out);
ssgi_status make_env(const ssgi_envmap* env, EnvInfo* out);
ssgi_status make_env_dims(int32_t h, int32_t w, EnvInfo* out);
void make_hiz_info(ssgi_dims d, int levels, HizInfo* out);
ssgi_status gbuffer_ok(const ssgi_gbuffer* g);
ssgi_status trace_params_ok(const ssgi_trace_params* p);
ssgi_status launch_status();

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

}  // namespace ssgi
