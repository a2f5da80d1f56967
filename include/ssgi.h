/*
 * ssgi.h -- C ABI of the GB300 (sm_103a) screen-space global-illumination library.
 *
 * Method: "3D Gaussian Inverse Rendering with Approximated Global Illumination"
 * (arXiv 2504.01358).  The library implements the paper's data-parallel hot path on a
 * rasterised G-buffer:
 *   - direct split-sum shading from an environment map (Sec. 3.2 "Shading"),
 *   - Monte-Carlo screen-space ray tracing for one-bounce indirect light against a
 *     hierarchical-Z pyramid (Sec. 3.3, Appendix D),
 *   - the adjoint of both with the march frozen (backward pass for inverse rendering),
 *   - a continuous-batching serving loop (ssgi_serve_*).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Memory.  Every array pointer is a DEVICE pointer owned by the caller unless the argument
 *   says "host".  The library never frees or retains caller memory; the only device
 *   memory it allocates is a serving arena, inside ssgi_serve_create.  All arrays are
 *   dense, C-contiguous FP32 (int32 for hit indices), 4-byte aligned.
 * Streams.  Work is enqueued asynchronously on `stream` (a cudaStream_t; NULL = the legacy
 *   default stream).  A call returns after argument validation and launch; device-side
 *   faults surface as SSGI_ERR_CUDA from this or a later call.
 * Errors.  Every call returns an ssgi_status.  On any non-OK status nothing was enqueued
 *   unless the status is SSGI_ERR_CUDA from a launch, in which case earlier launches of the
 *   same call may have run.  ssgi_status_string() names a status.
 * Layouts.  G-buffer planes are [V,H,W] (depth, roughness, metallic) or [V,H,W,3] (normal,
 *   albedo); images c_d, c_s, c1, final are [V,H,W,3]; hit indices [V,H,W,spp].
 * Camera.  World is right-handed with y up.  cam_to_world is 3x4 row-major [R | eye]; the
 *   columns of R are the camera's right, up and back axes in world space (the camera looks
 *   down its -z).  Pinhole, vertical FOV, pixel (x, y) centre at (x + 0.5, y + 0.5), y down,
 *   focal length f = (H/2) / tan(fov_y/2), principal point (W/2, H/2).
 * Depth.  Linear depth (distance along the camera's forward axis).  A pixel whose depth is
 *   not finite and positive is background: it shows the environment in its view direction
 *   and casts no rays.
 * Environment.  Lat-long RGB map, h x w with h, w powers of two and w >= h; direction d maps
 *   to u = 0.5 + atan2(d.x, -d.z) / (2 pi), v = atan2(sqrt(d.x^2 + d.z^2), d.y) / pi (v = 0 is
 *   +y); texel (i, j) centre at ((j + 0.5)/w, (i + 0.5)/h); bilinear, u wraps, v clamps.
 *   The mip chain has levels = log2(h) + 1; level l is the 2x2 box mean of level l-1; all
 *   levels packed level 0 first, each [h>>l][w>>l][3].  lambda_max = levels - 1.
 * RNG.  Sample s of pixel p (row-major index within its view) of view v draws Philox4x32-10
 *   (Salmon et al., SC'11) with counter (p, s, 0, 0) and key (seed_lo, seed_hi ^ v);
 *   xi_k = (out_k >> 8) * 2^-24.
 */
#ifndef SSGI_H
#define SSGI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef void *ssgi_stream_t; /* cudaStream_t */

typedef enum {
  SSGI_OK = 0,
  SSGI_ERR_INVALID_ARG = 1, /* null pointer, bad size, unsupported combination of sizes */
  SSGI_ERR_UNSUPPORTED = 2, /* valid request this build cannot serve (e.g. too many views) */
  SSGI_ERR_CUDA = 3,        /* a CUDA call or launch failed */
  SSGI_ERR_OOM = 4,         /* an allocation inside ssgi_serve_create failed */
  SSGI_ERR_BUDGET = 5,      /* serving: request larger than the device-memory budget */
  SSGI_ERR_QUEUE_FULL = 6,  /* serving: no free queue entry */
  SSGI_ERR_TIMEOUT = 7,     /* a bounded wait ran out (host or device side) */
  SSGI_ERR_NOT_READY = 8,   /* serving: result not finished yet */
  SSGI_ERR_CANCELLED = 9    /* serving: request was cancelled or the server shut down */
} ssgi_status;

#define SSGI_MAX_VIEWS 32
#define SSGI_MAX_HIZ_LEVELS 16
#define SSGI_MAX_ENV_LEVELS 16

/* hit_idx codes: >= 0 is the hit pixel's row-major index within the view */
#define SSGI_HIT_MISS (-1)       /* left the screen, passed the near plane or ray length, or ran out of steps */
#define SSGI_HIT_INVALID (-2)    /* sample below the surface (n.v <= 0 or n.w <= 0): weight 0 */
#define SSGI_HIT_BACKGROUND (-3) /* background pixel: no rays */

/* ssgi_trace_params.flags */
#define SSGI_DIFFUSE_INDIRECT 1u /* also estimate diffuse indirect light from the same rays and add it to final */
#define SSGI_BRUTE_FORCE 2u      /* ignore the pyramid: walk every pixel, no step budget (reference mode) */
#define SSGI_PATHWISE 4u         /* backward only: pathwise gradients through the sampled directions */
#define SSGI_SRGB_LOSS 8u        /* fused step only: the L2 loss compares the sRGB image (ssgi_l2_loss_srgb) */
#define SSGI_SRGB_FINAL 16u      /* trace only: final_out receives the display image, ssgi_tonemap_srgb of the
                                    composite (Sec. 3.3), written by the trace itself; not for ssgi_step_fused */

typedef struct { int32_t views, height, width; } ssgi_dims;

/* One camera per view (host memory).  Same 14 floats as the input generator's record. */
typedef struct {
  float cam_to_world[12];
  float fov_y_rad;
  float z_near;
} ssgi_camera;

/* Device planes of a G-buffer (Sec. 3.2, eq:g-buffer): depth [V,H,W], normal [V,H,W,3]
 * (unit, world space), albedo [V,H,W,3] in [0,1], roughness [V,H,W] in [0,1] (GGX alpha,
 * eq:ndf), metallic [V,H,W] in [0,1]. */
typedef struct {
  const float *depth, *normal, *albedo, *rough, *metal;
  ssgi_dims d;
} ssgi_gbuffer;

/* Device environment mip chain (Sec. 3.2, SampleEnvMap), as built by ssgi_build_env_mips. */
typedef struct {
  const float *mips;
  int32_t h, w, levels;
} ssgi_envmap;

/* Trace parameters (Sec. 3.3; Appendix D's threshold and maxRayLength). */
typedef struct {
  int32_t spp;        /* rays per pixel, N_s (paper: 8) -- 1..1024 */
  int32_t max_steps;  /* march iterations (skip, refine or test) before a ray counts as a miss, >= 0 */
  int32_t hiz_levels; /* pyramid levels including level 0 = depth, 1..SSGI_MAX_HIZ_LEVELS */
  float thickness;    /* a hit needs the ray to pass behind the depth buffer by at most this (world units) */
  float max_distance; /* ray length in world units (> 0) */
  uint64_t seed;      /* RNG key */
  uint32_t flags;     /* SSGI_DIFFUSE_INDIRECT | SSGI_BRUTE_FORCE | SSGI_PATHWISE | SSGI_SRGB_LOSS | SSGI_SRGB_FINAL */
} ssgi_trace_params;

/* ---------------------------------------------------------------------------------------- */
/* Sizes (pure host functions; 0 / -1 on invalid input)                                      */
/* ---------------------------------------------------------------------------------------- */
const char *ssgi_status_string(ssgi_status s);
const char *ssgi_version(void);
/* number of mip levels of an h x w map, or -1 if h, w are not powers of two with w >= h */
int32_t ssgi_env_levels(int32_t h, int32_t w);
/* floats in the packed mip chain of an h x w RGB map */
size_t ssgi_env_mip_floats(int32_t h, int32_t w);
/* floats in the packed pyramid of all views: per view, levels 1..levels-1 of ceil(H/2^l) x
 * ceil(W/2^l) cells, level after level; views one after another */
size_t ssgi_hiz_floats(ssgi_dims d, int32_t levels);
/* bytes of scratch ssgi_backward needs */
size_t ssgi_backward_workspace_bytes(ssgi_dims d, int32_t env_h, int32_t env_w);

/* ---------------------------------------------------------------------------------------- */
/* Precomputation                                                                           */
/* ---------------------------------------------------------------------------------------- */
/* BRDF-integral table of the split sum (Sec. 3.2 "Shading", Appendix C): lut[(i*n + j)*2 + k]
 * for roughness (i + 0.5)/n and n.v = (j + 0.5)/n; k = 0 is A (F0 scale), k = 1 is B (bias),
 * so that int f_s cos = F0 A + B.  Monte-Carlo over `samples` GGX half vectors at Hammersley
 * points (xi0 = (k + 0.5)/samples, xi1 = radical inverse of k).  n in [2, 1024], samples in
 * [1, 1<<20].  Output: 2 n^2 floats. */
ssgi_status ssgi_build_brdf_lut(int32_t n, int32_t samples, float *lut_out, ssgi_stream_t stream);

/* Environment mip chain (Sec. 3.2, SampleEnvMap): env [h][w][3] -> mips_out
 * (ssgi_env_mip_floats(h, w) floats; level 0 is a copy of env). */
ssgi_status ssgi_build_env_mips(const float *env, int32_t h, int32_t w, float *mips_out, ssgi_stream_t stream);

/* Hierarchical-Z pyramid (McGuire & Mara 2014, cited in Sec. 3.3): level l cell (i, j) is
 * the minimum depth over the level-0 pixels [i 2^l, (i+1) 2^l) x [j 2^l, (j+1) 2^l) inside
 * the image.  depth [V,H,W] -> hiz_out (ssgi_hiz_floats(d, levels) floats).  levels in
 * [1, SSGI_MAX_HIZ_LEVELS]; levels == 1 writes nothing. */
ssgi_status ssgi_build_hiz(const float *depth, ssgi_dims d, int32_t levels, float *hiz_out, ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Forward                                                                                  */
/* ---------------------------------------------------------------------------------------- */
/* Direct shading (Sec. 3.2 "Shading"): per pixel v = unit vector to the camera,
 * r = 2 (v.n) n - v, lambda = log2(rho + 1) lambda_max, (A, B) = bilinear table lookup at
 * (rho, clamp(n.v, 1e-4, 1)), F0 = lerp(0.04, albedo, metallic) (Appendix B);
 *   c_s = L_E(r, lambda) (F0 A + B),  c_d = (1 - m) a L_E(n, lambda),  c1 = c_d + c_s.
 * Background pixels: c_d = c_s = 0, c1 = L_E(view direction, 0).
 * cams: host array of d.views cameras.  lut: 2 lut_n^2 floats from ssgi_build_brdf_lut.
 * Outputs [V,H,W,3]; c_s may be NULL. */
ssgi_status ssgi_shade_direct(const ssgi_gbuffer *g, const ssgi_camera *cams, const ssgi_envmap *env,
                              const float *lut, int32_t lut_n, float *c_d, float *c_s, float *c1,
                              ssgi_stream_t stream);

/* Monte-Carlo screen-space ray tracing (Sec. 3.3, Appendix D) and composite.  Per pixel and
 * sample: GGX half vector h (alpha = rho) around n, w = 2 (v.h) h - v; the screen-space
 * march finds the first pixel q != origin where the ray's depth interval over q reaches
 * behind depth(q) by at most `thickness` (hierarchical-Z skipping never changes that pixel);
 * L = c1[q] on a hit, else L_E(w, 0).  c_s' = 1/spp sum F G (v.h) / ((n.v)(n.h)) L (invalid
 * samples count as 0); final = c_d + c_s' (+ c_id with SSGI_DIFFUSE_INDIRECT, where
 * c_id = (1 - m) a / pi * 1/spp sum L (n.w) / p, p = D (n.h) / (4 v.h)).
 * hiz: ssgi_build_hiz output for p->hiz_levels (may be NULL when hiz_levels == 1 or with
 * SSGI_BRUTE_FORCE).  c1, c_d: ssgi_shade_direct outputs.  Outputs: final [V,H,W,3];
 * c_s_mc, c_id [V,H,W,3] and hit_idx [V,H,W,spp] are optional (NULL).  step_count (one
 * device uint64, optional) has the total number of march iterations of the call added to
 * it atomically (the caller zeroes it); this is the traversal work of the launch.  With
 * SSGI_SRGB_FINAL final holds the display image (the composite's output transform, clamp to
 * [0, 1] and the sRGB transfer function, equal to ssgi_tonemap_srgb of the linear final),
 * applied in the trace's own epilogue: no separate pass over the image. */
ssgi_status ssgi_trace_indirect(const ssgi_gbuffer *g, const ssgi_camera *cams, const float *hiz, const float *c1,
                                const float *c_d, const ssgi_envmap *env, const ssgi_trace_params *p,
                                float *c_s_mc, float *c_id, float *final_out, int32_t *hit_idx,
                                uint64_t *step_count, ssgi_stream_t stream);

/* L2 loss against a target: loss = mean((final - target)^2) over n floats, and
 * g_final = 2 (final - target) / n.  loss_out (one device float) may be NULL. */
ssgi_status ssgi_l2_loss(const float *final_in, const float *target, int64_t n, float *g_final, float *loss_out,
                         ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Backward (adjoint).  The paper's march is not differentiable (Sec. 5); the hits, the      */
/* sampled directions and the sampling pdf are frozen at their forward values ("replay"),  */
/* and the adjoint is exact for that replay function:                                       */
/*   per sample  f_s(w; theta) (n.w) / p_frozen * L(theta),  f_s = D F G / (4 (n.w)(n.v)).   */
/* With SSGI_PATHWISE in params->flags (an answer to the limitation stated in Sec. 5) each    */
/* sample's uniforms and hit index are frozen instead and its direction is re-drawn from the  */
/* current normal and roughness (reparameterised sampling): per sample                        */
/*   F G1(n.w) G1(n.v) (v.h) / ((n.v)(n.h)) * L,  h = h(n, rho, xi),  w = 2 (v.h) h - v,       */
/* L = c1 of the frozen hit pixel or the environment (mip 0) in the re-drawn direction; the  */
/* normal and roughness gradients then include d w / d{n, rho} (and the environment's        */
/* variation along it).  Albedo, metallic, c1 and texel gradients are the same in both modes. */
/* The forward ignores the flag.                                                              */
/* ---------------------------------------------------------------------------------------- */
/* Inputs: g_final = d loss / d final [V,H,W,3]; the forward's G-buffer, cameras, c1, env,
 * table, stored hit_idx [V,H,W,spp] and the same params.  Outputs (overwritten):
 * g_albedo [V,H,W,3], g_rough [V,H,W], g_metal [V,H,W], g_normal [V,H,W,3] and
 * g_env [h][w][3] (base level of the environment; the mip-chain adjoint is included).
 * workspace: >= ssgi_backward_workspace_bytes(d, env->h, env->w) bytes of device scratch,
 * 16-byte aligned, cleared by the call.  Pixels whose normal points exactly at a pole of
 * the lat-long map (+-y) get no gradient through the direction of that lookup (the map is
 * not differentiable there). */
ssgi_status ssgi_backward(const float *g_final, const ssgi_gbuffer *g, const ssgi_camera *cams, const float *c1,
                          const ssgi_envmap *env, const float *lut, int32_t lut_n, const int32_t *hit_idx,
                          const ssgi_trace_params *p, float *g_albedo, float *g_rough, float *g_metal,
                          float *g_normal, float *g_env, void *workspace, size_t ws_bytes, ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Fused inverse-rendering step: every stage above for all views of a frame in ONE launch     */
/* (env mips, Hi-Z, direct shading, trace with stored hits, L2 loss against `target`,         */
/* backward): one block per work item, phase after phase, each block of a phase waiting       */
/* (bounded) until the previous phase has finished; a trace tile's block also runs the        */
/* Monte-Carlo adjoint of its pixels.  Same per-pixel code as the separate calls, so final    */
/* and hit_idx equal theirs bit for bit and the gradients agree up to the order of atomic     */
/* additions.                                                                                 */
/* ---------------------------------------------------------------------------------------- */
/* workspace bytes of ssgi_step_fused (mips, pyramid, c_d, c1, g_final and the backward scratch) */
size_t ssgi_step_fused_workspace_bytes(ssgi_dims d, int32_t env_h, int32_t env_w, int32_t hiz_levels);
/* env: device base level [env_h][env_w][3]; target: device [V,H,W,3]; outputs: final_out
 * [V,H,W,3], hit_idx [V,H,W,spp], loss (one device float), gradients as ssgi_backward.
 * workspace: 256-byte aligned, >= ssgi_step_fused_workspace_bytes.  A block's wait for the
 * previous phase is bounded; if a block ever gives up waiting every later block stops and
 * ssgi_step_fused_check reports it (the outputs are then incomplete). */
ssgi_status ssgi_step_fused(const ssgi_gbuffer *g, const ssgi_camera *cams, const float *env, int32_t env_h,
                            int32_t env_w, const float *lut, int32_t lut_n, const float *target,
                            const ssgi_trace_params *p, float *final_out, int32_t *hit_idx, float *loss,
                            float *g_albedo, float *g_rough, float *g_metal, float *g_normal, float *g_env,
                            void *workspace, size_t ws_bytes, ssgi_stream_t stream);
/* Synchronous: *failed = 1 if a block of the last fused step on this workspace gave up waiting. */
ssgi_status ssgi_step_fused_check(const void *workspace, int32_t *failed);
/* How long a block of later ssgi_step_fused launches waits for the previous phase before it
 * gives up: `polls` polls of ~100 ns each; a negative value restores the default (2^26 polls,
 * several seconds).  Process-wide, read at each launch.  A short limit makes the step stop at
 * its first phase boundary with ssgi_step_fused_check reporting failure, as a stalled block
 * would (a test of the error path: the blocks return, nothing faults, and the next launch
 * starts clean). */
ssgi_status ssgi_step_fused_set_wait_limit(int64_t polls);
/* Synchronous: the durations (ns, from %globaltimer) of the last fused step's phases, each from
 * its first block's start to its last block's end, in order: pyramids (env mips + Hi-Z, with
 * the clears), direct shading, trace + loss + Monte-Carlo adjoint, direct adjoint, mip-chain
 * adjoint. */
#define SSGI_FUSED_PHASES 5
ssgi_status ssgi_step_fused_phase_ns(const void *workspace, uint64_t *ns);

/* ---------------------------------------------------------------------------------------- */
/* Serving: continuous batching of render requests (real-time relighting / material editing,  */
/* Sec. 4 "Editing"; the per-request work is steps mips -> Hi-Z -> direct -> trace above).     */
/*                                                                                            */
/* A server owns one device arena of hbm_budget_bytes (allocated by ssgi_serve_create; the    */
/* only allocation the library makes) and max_slots CUDA streams.  An engine thread admits    */
/* queued requests in arrival order whenever a slot is free and the arena has room for the   */
/* request's buffers, enqueues its copies and kernels on the slot's stream, and retires it    */
/* when its completion event fires; admitted requests of different slots run concurrently on  */
/* the device.  Scenes (G-buffer + camera + Hi-Z pyramid) can be made resident once and then  */
/* re-rendered by many requests with new environment maps or materials edits applied on the  */
/* host.  All waits are bounded; nothing on the device spins.                                 */
/* ---------------------------------------------------------------------------------------- */
typedef struct ssgi_server ssgi_server;

typedef struct {
  size_t hbm_budget_bytes; /* device arena size; requests and resident scenes are carved from it */
  int32_t max_slots;       /* requests on the GPU at once (1..64); each slot has its own stream */
  int32_t queue_capacity;  /* requests submitted but not yet admitted (>= 1) */
  int32_t lut_n, lut_samples; /* BRDF table built at create (0 = 64, 4096) */
} ssgi_serve_config;

/* One render request.  Host arrays must stay valid until the request completes; pinned host
 * memory lets its copies overlap other requests' kernels.  scene >= 0 renders a resident scene
 * (depth..metal, cams and d are then ignored); scene < 0 uploads the request's own G-buffer. */
typedef struct {
  int64_t scene;
  ssgi_dims d;                                      /* views, height, width */
  const float *depth, *normal, *albedo, *rough, *metal; /* host, layouts as ssgi_gbuffer */
  const ssgi_camera *cams;                          /* host, d.views cameras */
  const float *env;                                 /* host [env_h][env_w][3] */
  int32_t env_h, env_w;
  ssgi_trace_params params;
  float *final_out;                                 /* host [V,H,W,3], written on completion */
} ssgi_request;

typedef struct {
  uint64_t submitted, admitted, completed, cancelled, rejected;
  int32_t queued, in_flight, resident_scenes, pad_;
  size_t arena_bytes_in_use, arena_bytes_peak;
} ssgi_serve_stats;

/* Create a server: allocates the arena and builds the BRDF table on the current device.
 * SSGI_ERR_OOM if the arena cannot be allocated. */
ssgi_status ssgi_serve_create(const ssgi_serve_config *cfg, ssgi_server **out);
/* Upload a G-buffer (host arrays) and build its pyramid once; *scene receives its id.
 * Synchronous.  SSGI_ERR_BUDGET if the arena has no room for it now. */
ssgi_status ssgi_serve_scene_add(ssgi_server *s, ssgi_dims d, const float *depth, const float *normal,
                                 const float *albedo, const float *rough, const float *metal,
                                 const ssgi_camera *cams, int32_t hiz_levels, int64_t *scene);
/* Release a resident scene; SSGI_ERR_NOT_READY while requests that use it are queued or running. */
ssgi_status ssgi_serve_scene_remove(ssgi_server *s, int64_t scene);
/* Queue a request; *ticket identifies it.  SSGI_ERR_QUEUE_FULL when queue_capacity requests
 * wait; SSGI_ERR_BUDGET when the request alone is larger than the whole arena;
 * SSGI_ERR_INVALID_ARG for malformed requests (checked before anything is queued). */
ssgi_status ssgi_serve_submit(ssgi_server *s, const ssgi_request *req, uint64_t *ticket);
/* SSGI_OK once the request finished (final_out written; *latency_ms = submit to completion,
 * optional), SSGI_ERR_NOT_READY before, SSGI_ERR_CANCELLED if it was cancelled,
 * SSGI_ERR_CUDA if its work failed, SSGI_ERR_INVALID_ARG for an unknown or already
 * collected ticket.  A finished ticket is forgotten once OK/CANCELLED/CUDA is returned. */
ssgi_status ssgi_serve_poll(ssgi_server *s, uint64_t ticket, double *latency_ms);
/* Like poll, blocking up to timeout_ms; SSGI_ERR_TIMEOUT if the request is still unfinished. */
ssgi_status ssgi_serve_wait(ssgi_server *s, uint64_t ticket, uint32_t timeout_ms, double *latency_ms);
/* Cancel a request that has not been admitted yet; SSGI_ERR_NOT_READY if it is already running. */
ssgi_status ssgi_serve_cancel(ssgi_server *s, uint64_t ticket);
ssgi_status ssgi_serve_stats_get(ssgi_server *s, ssgi_serve_stats *out);
/* Stop: cancel queued requests, wait (bounded, timeout_ms) for running ones, free everything.
 * SSGI_ERR_TIMEOUT if running work did not finish in time (resources are then kept, not freed). */
ssgi_status ssgi_serve_destroy(ssgi_server *s, uint32_t timeout_ms);
/* Device bytes a request of these sizes needs in the arena (0 if the sizes are invalid). */
size_t ssgi_serve_request_bytes(ssgi_dims d, int32_t env_h, int32_t env_w, int32_t hiz_levels, int32_t resident);

/* ---------------------------------------------------------------------------------------- */
/* Allocation-free backward (no counterpart in the paper; an interface convenience)          */
/* ---------------------------------------------------------------------------------------- */
/* Largest scratch the allocation-free backward can use: 32 MiB.  That covers one 1600x900
 * view with a 256x512 environment (25.8 MB); see ssgi_backward_workspace_bytes. */
#define SSGI_BACKWARD_NOALLOC_MAX_BYTES (32u << 20)

/* Same computation, arguments and outputs as ssgi_backward, for callers that cannot allocate
 * device memory while they run -- a render or training loop held to a fixed per-frame memory
 * budget, a host application whose pool allocator owns all device memory, or code running where
 * a cudaMalloc would synchronise the device and stall other streams.  Instead of a caller
 * workspace it uses a scratch array of SSGI_BACKWARD_NOALLOC_MAX_BYTES that lives in the
 * library's device image: every GPU that loads the library keeps that memory until the process
 * exits.  It calls no cudaMalloc or cudaFree and no allocating library routine.
 *   - Every call looks up the array's device address with the caller's device current (no
 *     cached address outlives a cudaDeviceReset); the first call on a device also loads the
 *     library's module there, so make that first call before any stream capture.
 *   - Sizes whose workspace (ssgi_backward_workspace_bytes) exceeds the maximum return
 *     SSGI_ERR_UNSUPPORTED before anything is enqueued.
 *   - The scratch is cleared on `stream` at the start of every call and keeps the last call's
 *     contents afterwards.  All calls on a device share it: calls that may overlap on the GPU
 *     (different streams without ordering between them) race and give wrong results; order them
 *     on one stream or with events. */
ssgi_status ssgi_backward_noalloc(const float *g_final, const ssgi_gbuffer *g, const ssgi_camera *cams,
                                  const float *c1, const ssgi_envmap *env, const float *lut, int32_t lut_n,
                                  const int32_t *hit_idx, const ssgi_trace_params *p, float *g_albedo,
                                  float *g_rough, float *g_metal, float *g_normal, float *g_env,
                                  ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Output transform and keyframe lighting.                                                    */
/* Tone mapping + gamma to sRGB after the composite (Sec. 3.3; the paper names no operator):  */
/* clamp to [0, 1], then the sRGB transfer function of IEC 61966-2-1 (12.92 x up to 0.0031308, */
/* 1.055 x^(1/2.4) - 0.055 above).  Keyframe lighting (Sec. 4 implementation details): every   */
/* period-th frame (10 in the paper) has its own environment map, frames in between blend the */
/* two neighbouring keyframes linearly.  Arrays are device memory; all calls but               */
/* ssgi_keyframe_of are asynchronous on `stream`.                                              */
/* ---------------------------------------------------------------------------------------- */
/* srgb[i] = T(linear[i]) for n floats (may be the same array). */
ssgi_status ssgi_tonemap_srgb(const float *linear, float *srgb, int64_t n, ssgi_stream_t stream);
/* loss = mean((T(final) - target)^2) over n floats against an sRGB target, g_final = its gradient
 * with respect to the linear final (0 where final is clamped).  loss_out may be NULL. */
ssgi_status ssgi_l2_loss_srgb(const float *final_in, const float *target, int64_t n, float *g_final, float *loss_out,
                              ssgi_stream_t stream);
/* env_out = (1 - alpha) env_a + alpha env_b, maps [env_h][env_w][3], alpha in [0, 1]. */
ssgi_status ssgi_env_keyframe_lerp(const float *env_a, const float *env_b, float alpha, int32_t env_h, int32_t env_w,
                                   float *env_out, ssgi_stream_t stream);
/* Adjoint: g_a = (1 - alpha) g_env, g_b = alpha g_env (added to g_a, g_b when accumulate != 0,
 * so that gradients of many frames collect in the keyframes); g_a and g_b distinct. */
ssgi_status ssgi_env_keyframe_lerp_backward(const float *g_env, float alpha, int32_t env_h, int32_t env_w, float *g_a,
                                            float *g_b, int32_t accumulate, ssgi_stream_t stream);
/* Host: frame -> (keyframe k, alpha) with env(frame) = (1 - alpha) env_k + alpha env_{k+1}. */
ssgi_status ssgi_keyframe_of(int64_t frame, int32_t period, int64_t *keyframe, float *alpha);

/* ---------------------------------------------------------------------------------------- */
/* Object insertion (Sec. 4 "Object Insertion"): an object's G-buffer, rendered on its own,   */
/* merged into the scene's by depth comparison (before the pyramid and shading).  A pixel     */
/* takes all five of the object's channels where the object's depth is strictly smaller than  */
/* the scene's; ties and object background (+inf) keep the scene.  scene and object: device   */
/* G-buffers of the same dims.  out_*: device planes, either all equal to the scene's (in     */
/* place: only the object's pixels are written) or all distinct from them (a full copy); the  */
/* object's planes must not overlap them.  mask_out (nullable): [V,H,W] bytes, 1 where the    */
/* object won.  Asynchronous on `stream`.                                                      */
/* ---------------------------------------------------------------------------------------- */
ssgi_status ssgi_composite_gbuffer(const ssgi_gbuffer *scene, const ssgi_gbuffer *object, float *out_depth,
                                   float *out_normal, float *out_albedo, float *out_rough, float *out_metal,
                                   uint8_t *mask_out, ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Depth normals (Sec. 3.1 "depth normal": surface normals from the rendered depth buffer by  */
/* finite differences, as in 2DGS).  P(x, y) = camera-space point of the pixel centre at its  */
/* linear depth; per image direction a central difference where both neighbours are          */
/* foreground, one-sided where one is; n = normalize(dP/dy x dP/dx) (y down the image),       */
/* flipped to face the camera, in world space.  With no foreground neighbour in a direction   */
/* (or a zero cross product) n is the unit vector towards the camera; background pixels get   */
/* (0, 0, 0).  depth [V,H,W] and normal_out [V,H,W,3] are device arrays (distinct); cams: V    */
/* host records.  Asynchronous on `stream`.                                                    */
/* ---------------------------------------------------------------------------------------- */
ssgi_status ssgi_depth_normals(const float *depth, ssgi_dims d, const ssgi_camera *cams, float *normal_out,
                               ssgi_stream_t stream);
/* Depth normals and the Hi-Z pyramid in one pass over depth (the two above fused: the depth
 * normals of Sec. 3.1 computed while the pyramid's tiles are read, no second read of depth).
 * normal_out [V,H,W,3] equals ssgi_depth_normals' and hiz_out equals ssgi_build_hiz's for the
 * same arguments, bit for bit.  levels as for ssgi_build_hiz (hiz_out may be NULL with
 * levels == 1: normals only). */
ssgi_status ssgi_build_hiz_normals(const float *depth, ssgi_dims d, const ssgi_camera *cams, int32_t levels,
                                   float *hiz_out, float *normal_out, ssgi_stream_t stream);

/* ---------------------------------------------------------------------------------------- */
/* Measurement: a read-bandwidth probe.  Streams `bytes` of device memory at `buf` `reps` times */
/* through L2 only (16-byte loads that skip L1), from every SM.  Timed with events around it,  */
/* a buffer that fits in L2 gives the L2 read ceiling and a much larger one the HBM ceiling:   */
/* the rooflines of kernels whose working set lives in L2.  buf: device, 16-byte aligned;      */
/* bytes: a positive multiple of 16; reps >= 1; sink: one device word, written only in the    */
/* rare case that keeps the loads from being optimised away.  Asynchronous on `stream`.        */
/* ---------------------------------------------------------------------------------------- */
ssgi_status ssgi_read_bandwidth_probe(const void *buf, size_t bytes, int32_t reps, uint32_t *sink,
                                      ssgi_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* SSGI_H */
