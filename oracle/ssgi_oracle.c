/*
 * ssgi_oracle.c -- plain, slow, FP64 CPU oracle of the SSGI hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library (paper_2504_01358_gb300/) links, loads or
 * calls this file.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference
 * leg may use it.  It shares no code, header, table or constant generator with the CUDA path;
 * the two only agree on the data formats documented in include/ssgi.h.
 *
 * Paper: "3D Gaussian Inverse Rendering with Approximated Global Illumination" (arXiv 2504.01358).
 * Each function names the passage it follows.  Everything is computed in double precision from
 * FP32 inputs promoted to double (the caller hands in double arrays).  No blocking, fusion or
 * reordering beyond what the definitions state: direct shading for every pixel first, then the
 * per-sample trace, then the Monte-Carlo sum, then the composite.
 *
 * Readings of the paper that this file takes (the paper is silent or garbled there):
 *   - Fresnel (Appendix B, eq:fresnel) is Schlick's F0 + (1 - F0)(1 - w_o.h)^5; the printed
 *     parenthesis around the fifth power is read as a typo.
 *   - GGX alpha = rho exactly as printed (eq:ndf, eq:geometry); no rho^2 remap.
 *   - The BRDF-integral table (Appendix C) is F_s = F0 * A + B with F0 = lerp(0.04, a, m);
 *     "a" in the printed split is read as F0, and (1 - cos)^5 uses w_o.h.
 *   - The environment is a lat-long map with a 2x2 box-filter mip chain; lambda_max = #levels-1.
 *   - The march (Sec. 3.3 "Screen-space Ray Tracing", Appendix D) is a pixel-exact traversal of
 *     the screen-space segment with conservative hierarchical-Z skipping.  A hit is the first
 *     pixel q != origin where the ray's depth interval over q reaches behind depth(q) by at most
 *     `thickness` (the sign change of dz and the |d_ray - d_scene| < threshold test together).
 *     Misses (off screen, past the near plane or the ray length, budget exhausted) take the
 *     environment map at mip 0.  The origin pixel is never a hit.
 *   - The ray depth is view-space linear depth.
 *   - Hit radiance is c1 of the hit pixel (first-pass radiance, nearest pixel).
 *   - Backward: hits, sampled directions and the sampling pdf are frozen ("replay mode");
 *     the paper only states that the march is not differentiable (Sec. 5).
 *   - Pathwise backward (flag 4, answering the limitation stated in Sec. 5): the uniforms of
 *     every sample and its hit index are frozen, the direction is re-drawn from the current
 *     normal and roughness (reparameterised sampling), a hit keeps c1 of its frozen pixel and
 *     a miss looks the environment up in the new direction.  The sampling frame keeps the
 *     branch (sign of n.z) of the base normal, so the summand is smooth in n at n.z = 0.  Its n and rho derivatives are
 *     taken here by central differences of that per-sample function (the definition of the
 *     derivative, in FP64); everything else equals the replay adjoint at the base point.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846
#define OR_MAX_LEVELS 16

#define ORF_DIFFUSE_INDIRECT 1u
#define ORF_BRUTE_FORCE 2u
#define ORF_PATHWISE 4u
/* difference step of the pathwise n / rho derivatives and its form: 0 central, +1 forward,
 * -1 backward (orc_set_pathwise_step) */
static double g_pathwise_h = 1e-6;
static int g_pathwise_mode = 0;

/* ------------------------------------------------------------------------------------------ */
/* small vector helpers                                                                        */
/* ------------------------------------------------------------------------------------------ */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 ld3(const double *p) { return mk(p[0], p[1], p[2]); }

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3",   */
/* SC'11): 10 rounds of the 4x32 S-box with the published multipliers and Weyl key increments. */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniforms of sample s at pixel `pix` of view `view`: counter (pix, s, 0, 0), key
 * (seed_lo, seed_hi ^ view); xi_k = (out_k >> 8) * 2^-24, exact in float and double. */
static void sample_uniforms(uint64_t seed, int view, uint32_t pix, uint32_t s, double xi[2]) {
  uint32_t ctr[4] = {pix, s, 0u, 0u};
  uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32) ^ (uint32_t)view};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  xi[0] = (double)(o[0] >> 8) * (1.0 / 16777216.0);
  xi[1] = (double)(o[1] >> 8) * (1.0 / 16777216.0);
}

/* ------------------------------------------------------------------------------------------ */
/* Microfacet terms (Appendix B)                                                               */
/* ------------------------------------------------------------------------------------------ */
/* eq:ndf  D(h; rho, n) = rho^2 / (pi ((h.n)^2 (rho^2 - 1) + 1)^2) */
double orc_ggx_D(double nh, double rho) {
  double a2 = rho * rho;
  double den = nh * nh * (a2 - 1.0) + 1.0;
  return a2 / (OR_PI * den * den);
}

/* eq:geometry  G_GGX(z) = 2z / (z + sqrt(rho^2 + (1 - rho^2) z^2)) */
double orc_ggx_G1(double z, double rho) {
  double a2 = rho * rho;
  return 2.0 * z / (z + sqrt(a2 + (1.0 - a2) * z * z));
}

/* eq:fresnel (Schlick), per channel: F0 + (1 - F0)(1 - w_o.h)^5 */
double orc_fresnel(double F0, double vh) {
  double c = 1.0 - vh;
  double c5 = c * c * c * c * c;
  return F0 + (1.0 - F0) * c5;
}

/* F0 = lerp(0.04, a, m) (Appendix B, below eq:fresnel). */
static double f0_of(double a, double m) { return 0.04 * (1.0 - m) + a * m; }

/* GGX importance sample of the half vector (Sec. 3.3: directions "sampled from the GGX
 * distribution", Walter et al. 2007): cos^2(theta_h) = (1 - xi0) / (1 + (rho^2 - 1) xi0),
 * phi = 2 pi xi1, in the orthonormal basis of Duff et al. 2017 ("Building an Orthonormal
 * Basis, Revisited", JCGT 6(1)) around n. */
static v3 ggx_sample_h_frame(v3 n, double sgn, double rho, double xi0, double xi1);

void orc_ggx_sample_h(const double n_in[3], double rho, double xi0, double xi1, double h_out[3]) {
  v3 n = ld3(n_in);
  v3 h = ggx_sample_h_frame(n, (n.z >= 0.0) ? 1.0 : -1.0, rho, xi0, xi1);
  h_out[0] = h.x; h_out[1] = h.y; h_out[2] = h.z;
}

/* The same with the branch of the frame (the sign of n.z) given. */
static v3 ggx_sample_h_frame(v3 n, double sgn, double rho, double xi0, double xi1) {
  double a2 = rho * rho;
  double c2 = (1.0 - xi0) / (1.0 + (a2 - 1.0) * xi0);
  double ct = sqrt(c2);
  double st = sqrt(fmax(0.0, 1.0 - c2));
  double phi = 2.0 * OR_PI * xi1;
  double aa = -1.0 / (sgn + n.z);
  double bb = n.x * n.y * aa;
  v3 t1 = mk(1.0 + sgn * n.x * n.x * aa, sgn * bb, -sgn * n.x);
  v3 t2 = mk(bb, sgn + n.y * n.y * aa, -n.y);
  return add(add(scl(t1, st * cos(phi)), scl(t2, st * sin(phi))), scl(n, ct));
}

/* ------------------------------------------------------------------------------------------ */
/* Environment map: lat-long, 2x2 box-filter mip chain (Sec. 3.2, SampleEnvMap)               */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const double *mips; /* packed, level 0 first, each [h_l][w_l][3] */
  int levels;
  int h[OR_MAX_LEVELS], w[OR_MAX_LEVELS];
  long off[OR_MAX_LEVELS]; /* in doubles */
} env_t;

static int ilog2_exact(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return ((1 << l) == x) ? l : -1;
}

int orc_env_levels(int He, int We) {
  int lh = ilog2_exact(He), lw = ilog2_exact(We);
  if (lh < 0 || lw < 0 || We < He || lh + 1 > OR_MAX_LEVELS) return -1;
  return lh + 1;
}

long orc_env_mip_doubles(int He, int We) {
  int L = orc_env_levels(He, We);
  if (L < 0) return -1;
  long tot = 0;
  for (int l = 0; l < L; ++l) tot += (long)(He >> l) * (long)(We >> l) * 3;
  return tot;
}

static void env_init(env_t *e, const double *mips, int He, int We) {
  e->mips = mips;
  e->levels = orc_env_levels(He, We);
  long off = 0;
  for (int l = 0; l < e->levels; ++l) {
    e->h[l] = He >> l;
    e->w[l] = We >> l;
    e->off[l] = off;
    off += (long)e->h[l] * e->w[l] * 3;
  }
}

/* Level j texel = mean of its 2x2 children at level j-1, until the map is 1 texel high. */
void orc_build_env_mips(const double *env, int He, int We, double *mips) {
  env_t e;
  env_init(&e, mips, He, We);
  memcpy(mips, env, sizeof(double) * (size_t)He * We * 3);
  for (int l = 1; l < e.levels; ++l) {
    const double *src = mips + e.off[l - 1];
    double *dst = mips + e.off[l];
    int ws = e.w[l - 1];
    for (int i = 0; i < e.h[l]; ++i)
      for (int j = 0; j < e.w[l]; ++j)
        for (int c = 0; c < 3; ++c) {
          double s = src[((2 * i) * ws + 2 * j) * 3 + c] + src[((2 * i) * ws + 2 * j + 1) * 3 + c] +
                     src[((2 * i + 1) * ws + 2 * j) * 3 + c] + src[((2 * i + 1) * ws + 2 * j + 1) * 3 + c];
          dst[(i * e.w[l] + j) * 3 + c] = 0.25 * s;
        }
  }
}

/* Direction -> lat-long coordinates: u = 0.5 + atan2(d.x, -d.z) / (2 pi),
 * v = atan2(sqrt(d.x^2 + d.z^2), d.y) / pi  (v = 0 is straight up). */
static void dir_to_uv(v3 d, double *u, double *v) {
  *u = 0.5 + atan2(d.x, -d.z) / (2.0 * OR_PI);
  *v = atan2(sqrt(d.x * d.x + d.z * d.z), d.y) / OR_PI;
}

/* The four texels and bilinear weights of (u, v) at level l (texel centres; u wraps, v clamps). */
typedef struct { long idx[4]; double wt[4]; } bilin_t;

static int wrapi(int x, int n) { int r = x % n; return r < 0 ? r + n : r; }
static int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }

static bilin_t env_taps(const env_t *e, int l, double u, double v) {
  bilin_t b;
  int h = e->h[l], w = e->w[l];
  double x = u * w - 0.5, y = v * h - 0.5;
  double x0f = floor(x), y0f = floor(y);
  double tx = x - x0f, ty = y - y0f;
  int x0 = (int)x0f, y0 = (int)y0f;
  int c0 = wrapi(x0, w), c1 = wrapi(x0 + 1, w);
  int r0 = clampi(y0, 0, h - 1), r1 = clampi(y0 + 1, 0, h - 1);
  b.idx[0] = e->off[l] + ((long)r0 * w + c0) * 3; b.wt[0] = (1 - tx) * (1 - ty);
  b.idx[1] = e->off[l] + ((long)r0 * w + c1) * 3; b.wt[1] = tx * (1 - ty);
  b.idx[2] = e->off[l] + ((long)r1 * w + c0) * 3; b.wt[2] = (1 - tx) * ty;
  b.idx[3] = e->off[l] + ((long)r1 * w + c1) * 3; b.wt[3] = tx * ty;
  return b;
}

/* SampleEnvMap(d, lambda): bilinear at levels floor(lambda) and floor(lambda)+1, linear in lambda. */
static void env_lookup(const env_t *e, v3 d, double lam, double out[3]) {
  double lmax = (double)(e->levels - 1);
  if (lam < 0.0) lam = 0.0;
  if (lam > lmax) lam = lmax;
  int l0 = (int)floor(lam);
  int l1 = l0 + 1 < e->levels ? l0 + 1 : l0;
  double t = lam - (double)l0;
  double u, v;
  dir_to_uv(d, &u, &v);
  out[0] = out[1] = out[2] = 0.0;
  bilin_t b0 = env_taps(e, l0, u, v), b1 = env_taps(e, l1, u, v);
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 3; ++c)
      out[c] += (1.0 - t) * b0.wt[k] * e->mips[b0.idx[k] + c] + t * b1.wt[k] * e->mips[b1.idx[k] + c];
}

void orc_env_lookup(const double *mips, int He, int We, const double d[3], double lam, double out[3]) {
  env_t e;
  env_init(&e, mips, He, We);
  env_lookup(&e, ld3(d), lam, out);
}

/* ------------------------------------------------------------------------------------------ */
/* BRDF-integral table (Sec. 3.2 "Shading", Appendix C)                                       */
/* ------------------------------------------------------------------------------------------ */
static double radical_inverse2(uint32_t k) {
  uint32_t r = 0;
  for (int i = 0; i < 32; ++i) { r = (r << 1) | (k & 1u); k >>= 1; }
  return (double)r * (1.0 / 4294967296.0);
}

/* Table entry (i, j): rho_i = (i + 0.5)/N, mu_j = (j + 0.5)/N (mu = n.v).  The two integrals of
 * Appendix C, A = int f_s/F (1 - (1 - w_o.h)^5) cos and B = int f_s/F (1 - w_o.h)^5 cos, by
 * Monte-Carlo with M GGX-importance-sampled half vectors at Hammersley points
 * (xi0 = (k + 0.5)/M, xi1 = radical inverse of k).  With h ~ D(h)(n.h), the estimator of
 * f_s cos / pdf is G (v.h) / ((n.h)(n.v)) times the Fresnel factor.  lut[(i*N + j)*2 + {0,1}]. */
void orc_build_lut(int N, int M, double *lut) {
  for (int i = 0; i < N; ++i) {
    double rho = (i + 0.5) / N;
    for (int j = 0; j < N; ++j) {
      double mu = (j + 0.5) / N;
      v3 v = mk(sqrt(fmax(0.0, 1.0 - mu * mu)), 0.0, mu);
      double n_up[3] = {0.0, 0.0, 1.0};
      double A = 0.0, B = 0.0;
      for (int k = 0; k < M; ++k) {
        double hh[3];
        orc_ggx_sample_h(n_up, rho, (k + 0.5) / M, radical_inverse2((uint32_t)k), hh);
        v3 h = ld3(hh);
        double vh = dot(v, h);
        v3 l = sub(scl(h, 2.0 * vh), v);
        if (l.z <= 0.0 || vh <= 0.0 || h.z <= 0.0) continue;
        double w = orc_ggx_G1(l.z, rho) * orc_ggx_G1(mu, rho) * vh / (h.z * mu);
        double c = 1.0 - vh;
        double fc = c * c * c * c * c;
        A += w * (1.0 - fc);
        B += w * fc;
      }
      lut[(i * N + j) * 2 + 0] = A / M;
      lut[(i * N + j) * 2 + 1] = B / M;
    }
  }
}

/* Bilinear lookup at (rho, mu), texel centres, clamped to the table. */
typedef struct { double A, B, dA_drho, dB_drho, dA_dmu, dB_dmu; } lutv_t;

static lutv_t lut_sample(const double *lut, int N, double rho, double mu) {
  lutv_t r;
  double x = mu * N - 0.5, y = rho * N - 0.5;
  int xin = (x > 0.0 && x < N - 1.0), yin = (y > 0.0 && y < N - 1.0);
  if (x < 0.0) x = 0.0;
  if (x > N - 1.0) x = N - 1.0;
  if (y < 0.0) y = 0.0;
  if (y > N - 1.0) y = N - 1.0;
  int x0 = (int)floor(x), y0 = (int)floor(y);
  if (x0 > N - 2) x0 = N - 2;
  if (y0 > N - 2) y0 = N - 2;
  double tx = x - x0, ty = y - y0;
  double v[2][2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int c = 0; c < 2; ++c) v[a][b][c] = lut[((y0 + a) * N + (x0 + b)) * 2 + c];
  double out[2], dx[2], dy[2];
  for (int c = 0; c < 2; ++c) {
    out[c] = (1 - ty) * ((1 - tx) * v[0][0][c] + tx * v[0][1][c]) + ty * ((1 - tx) * v[1][0][c] + tx * v[1][1][c]);
    dx[c] = (1 - ty) * (v[0][1][c] - v[0][0][c]) + ty * (v[1][1][c] - v[1][0][c]);
    dy[c] = (1 - tx) * (v[1][0][c] - v[0][0][c]) + tx * (v[1][1][c] - v[0][1][c]);
  }
  r.A = out[0]; r.B = out[1];
  r.dA_dmu = xin ? dx[0] * N : 0.0; r.dB_dmu = xin ? dx[1] * N : 0.0;
  r.dA_drho = yin ? dy[0] * N : 0.0; r.dB_drho = yin ? dy[1] * N : 0.0;
  return r;
}

void orc_lut_sample(const double *lut, int N, double rho, double mu, double out[2]) {
  lutv_t r = lut_sample(lut, N, rho, mu);
  out[0] = r.A; out[1] = r.B;
}

/* ------------------------------------------------------------------------------------------ */
/* Hierarchical-Z pyramid (McGuire & Mara 2014, cited in Sec. 3.3): level k cell (i, j) is the  */
/* minimum depth over the level-0 pixels it covers (ceil-div sizes).  Level 0 is the depth      */
/* buffer itself; the output holds levels 1..levels-1 of each view, packed level after level.   */
/* ------------------------------------------------------------------------------------------ */
static int lvl_dim(int n, int l) { return (n + (1 << l) - 1) >> l; }

long orc_hiz_floats_per_view(int H, int W, int levels) {
  long tot = 0;
  for (int l = 1; l < levels; ++l) tot += (long)lvl_dim(H, l) * lvl_dim(W, l);
  return tot;
}

void orc_build_hiz(const double *depth, int V, int H, int W, int levels, double *hiz) {
  long per = orc_hiz_floats_per_view(H, W, levels);
  for (int v = 0; v < V; ++v) {
    const double *d0 = depth + (long)v * H * W;
    long off = 0;
    for (int l = 1; l < levels; ++l) {
      int hl = lvl_dim(H, l), wl = lvl_dim(W, l), s = 1 << l;
      double *dst = hiz + (long)v * per + off;
      for (int i = 0; i < hl; ++i)
        for (int j = 0; j < wl; ++j) {
          double m = INFINITY;
          for (int y = i * s; y < (i + 1) * s && y < H; ++y)
            for (int x = j * s; x < (j + 1) * s && x < W; ++x) {
              double z = d0[(long)y * W + x];
              if (z < m) m = z;
            }
          dst[(long)i * wl + j] = m;
        }
      off += (long)hl * wl;
    }
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Camera (pinhole, vertical FOV, y down in pixels)                                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  double R[3][3]; /* columns: camera right, up, back in world */
  v3 eye;
  double f, cx, cy, znear;
  int H, W;
} cam_t;

static cam_t cam_init(const double *rec, int H, int W) {
  cam_t c;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) c.R[i][j] = rec[i * 4 + j];
  c.eye = mk(rec[3], rec[7], rec[11]);
  c.f = (H / 2.0) / tan(rec[12] / 2.0);
  c.cx = W / 2.0;
  c.cy = H / 2.0;
  c.znear = rec[13];
  c.H = H; c.W = W;
  return c;
}

/* Camera-space direction through the centre of pixel (x, y), forward component 1. */
static v3 pix_dir_cam(const cam_t *c, int x, int y) {
  return mk((x + 0.5 - c->cx) / c->f, -(y + 0.5 - c->cy) / c->f, -1.0);
}
static v3 cam_to_world_dir(const cam_t *c, v3 d) {
  return mk(c->R[0][0] * d.x + c->R[0][1] * d.y + c->R[0][2] * d.z,
            c->R[1][0] * d.x + c->R[1][1] * d.y + c->R[1][2] * d.z,
            c->R[2][0] * d.x + c->R[2][1] * d.y + c->R[2][2] * d.z);
}
static v3 world_to_cam_dir(const cam_t *c, v3 d) {
  return mk(c->R[0][0] * d.x + c->R[1][0] * d.y + c->R[2][0] * d.z,
            c->R[0][1] * d.x + c->R[1][1] * d.y + c->R[2][1] * d.z,
            c->R[0][2] * d.x + c->R[1][2] * d.y + c->R[2][2] * d.z);
}

static int is_background(double z) { return !(isfinite(z) && z > 0.0); }

/* ------------------------------------------------------------------------------------------ */
/* Direct shading (Sec. 3.2 "Shading"):                                                        */
/*   v = direction to the camera, r = 2 (v.n) n - v, lambda = log2(rho + 1) lambda_max,         */
/*   c_s = L_E(r, lambda) (F0 A + B),  c_d = (1 - m) a L_E(n, lambda),  c1 = c_d + c_s.         */
/* (A, B) from the table at (rho, clamp(n.v, 1e-4, 1)).  Background pixels (depth not finite)  */
/* take the environment at mip 0 in the view direction as c1, with c_d = c_s = 0.               */
/* ------------------------------------------------------------------------------------------ */
void orc_shade_direct(int V, int H, int W, const double *depth, const double *normal, const double *albedo,
                      const double *rough, const double *metal, const double *cams, const double *mips, int He,
                      int We, const double *lut, int lut_n, double *cd, double *cs, double *c1) {
  env_t e;
  env_init(&e, mips, He, We);
  double lmax = (double)(e.levels - 1);
  for (int v = 0; v < V; ++v) {
    cam_t cam = cam_init(cams + 14 * v, H, W);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        long p = ((long)v * H + y) * W + x;
        v3 d = cam_to_world_dir(&cam, pix_dir_cam(&cam, x, y));
        double outd[3] = {0, 0, 0}, outs[3] = {0, 0, 0}, o1[3];
        if (is_background(depth[p])) {
          env_lookup(&e, d, 0.0, o1);
        } else {
          v3 vv = scl(d, -1.0 / len(d));
          v3 n = ld3(normal + 3 * p);
          double nv = dot(n, vv);
          double mu = nv < 1e-4 ? 1e-4 : (nv > 1.0 ? 1.0 : nv);
          v3 r = sub(scl(n, 2.0 * nv), vv);
          double rho = rough[p], m = metal[p];
          double lam = log2(rho + 1.0) * lmax;
          lutv_t ab = lut_sample(lut, lut_n, rho, mu);
          double Er[3], En[3];
          env_lookup(&e, r, lam, Er);
          env_lookup(&e, n, lam, En);
          for (int c = 0; c < 3; ++c) {
            double a = albedo[3 * p + c];
            outs[c] = Er[c] * (f0_of(a, m) * ab.A + ab.B);
            outd[c] = (1.0 - m) * a * En[c];
            o1[c] = outd[c] + outs[c];
          }
        }
        for (int c = 0; c < 3; ++c) {
          if (cd) cd[3 * p + c] = outd[c];
          if (cs) cs[3 * p + c] = outs[c];
          c1[3 * p + c] = o1[c];
        }
      }
  }
}


/* ------------------------------------------------------------------------------------------ */
/* Screen-space march (Sec. 3.3: dz changes sign where the ray passes behind the depth buffer; */
/* Appendix D's |d_ray - d_scene| < threshold), walked pixel by pixel with conservative        */
/* hierarchical-Z skipping.                                                                    */
/*                                                                                             */
/* The ray o + t w (camera space) is clipped to z >= z_near and t <= max_distance and projected */
/* to the screen segment P(s) = P0 + s (P1 - P0), s in [0, 1], along which 1/z is linear in s.  */
/* The traversal state is a level-0 pixel (ix, iy) entered at parameter s, and a level L.       */
/* Each iteration looks at the level-L cell holding (ix, iy): the ray's depth interval over    */
/* [s, min(s_exit, 1)] is compared with the cell's minimum depth.  Entirely in front: skip the  */
/* cell and go up a level.  Otherwise, above level 0: go down a level.  At level 0: hit if the  */
/* interval also reaches no deeper than depth + thickness, else step to the next pixel.        */
/* Leaving a cell through its x side (ties go to x) enters the pixel across that side, on the  */
/* row of the exit point clamped to the cell's rows (and symmetrically for y).                 */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  const cam_t *cam;
  const double *depth;   /* this view's level 0 */
  const double *hiz;     /* this view's levels 1..L-1 (NULL when levels == 1) */
  long hoff[OR_MAX_LEVELS];
  int hw[OR_MAX_LEVELS];
  int levels, max_steps; /* max_steps < 0: unbounded */
  double thickness, max_distance;
} march_t;

static void upd_margin(double *mg, double val) {
  if (!mg) return;
  val = fabs(val);
  if (val < *mg) *mg = val;
}

typedef struct { double P0x, P0y, Dx, Dy; } seg_t;

/* Exit parameters of the level-L cell holding pixel (ix, iy) through its x and y sides. */
static void cell_exit(const seg_t *g, int ix, int iy, int L, double *sx, double *sy) {
  int S = 1 << L;
  int cxl = ix >> L, cyl = iy >> L;
  *sx = INFINITY;
  *sy = INFINITY;
  if (g->Dx > 0.0) *sx = ((double)(cxl + 1) * S - g->P0x) / g->Dx;
  else if (g->Dx < 0.0) *sx = ((double)cxl * S - g->P0x) / g->Dx;
  if (g->Dy > 0.0) *sy = ((double)(cyl + 1) * S - g->P0y) / g->Dy;
  else if (g->Dy < 0.0) *sy = ((double)cyl * S - g->P0y) / g->Dy;
}

/* Move (ix, iy) to the pixel entered when the ray leaves the level-L cell. */
static void cell_step(const seg_t *g, int L, double sx, double sy, int *ix, int *iy, double *s, double *margin) {
  int S = 1 << L;
  int cxl = *ix >> L, cyl = *iy >> L;
  if (isfinite(sx) && isfinite(sy)) upd_margin(margin, (sx - sy) / fmax(fabs(sx), fabs(sy)));
  if (sx <= sy) {
    int nix = g->Dx > 0.0 ? (cxl + 1) * S : cxl * S - 1;
    double py = g->P0y + sx * g->Dy;
    double fy = floor(py);
    double lo = (double)(cyl * S), hi = (double)(cyl * S + S - 1);
    if (S > 1 && fy > lo && fy < hi) upd_margin(margin, py - floor(py + 0.5));
    *iy = (int)(fy < lo ? lo : (fy > hi ? hi : fy));
    *ix = nix;
    *s = sx;
  } else {
    int niy = g->Dy > 0.0 ? (cyl + 1) * S : cyl * S - 1;
    double px = g->P0x + sy * g->Dx;
    double fx = floor(px);
    double lo = (double)(cxl * S), hi = (double)(cxl * S + S - 1);
    if (S > 1 && fx > lo && fx < hi) upd_margin(margin, px - floor(px + 0.5));
    *ix = (int)(fx < lo ? lo : (fx > hi ? hi : fx));
    *iy = niy;
    *s = sy;
  }
}

/* Trace from pixel (x, y) at linear depth z0 along the camera-space direction w.  Returns the
 * hit pixel's linear index in the view (>= 0) or -1 for a miss.  *iters counts loop
 * iterations (skip, refine or level-0 test); *margin (optional) receives the smallest
 * relative slack of any decision taken, a diagnostic for rounding-order disagreements. */
static int march(const march_t *M, int x, int y, double z0, v3 w, int *iters, double *margin) {
  const cam_t *c = M->cam;
  int H = c->H, W = c->W;
  *iters = 0;
  v3 o = scl(pix_dir_cam(c, x, y), z0);
  double wz = -w.z; /* forward component of the direction */
  double t_end = M->max_distance;
  if (wz < 0.0) {
    double tn = (c->znear - z0) / wz;
    if (tn < t_end) t_end = tn;
  }
  if (!(t_end > 0.0)) return -1;
  v3 X1 = add(o, scl(w, t_end));
  double z1 = -X1.z;
  seg_t g;
  g.P0x = x + 0.5;
  g.P0y = y + 0.5;
  g.Dx = (c->cx + c->f * X1.x / z1) - g.P0x;
  g.Dy = (c->cy - c->f * X1.y / z1) - g.P0y;
  double k0 = 1.0 / z0, dk = 1.0 / z1 - k0;

  int ix = x, iy = y, L = 0;
  double s = 0.0, sx, sy;
  /* leave the origin pixel: it is never tested */
  cell_exit(&g, ix, iy, 0, &sx, &sy);
  {
    double se = sx <= sy ? sx : sy;
    if (isfinite(se)) upd_margin(margin, se - 1.0);
    if (!(se < 1.0)) return -1;
  }
  cell_step(&g, 0, sx, sy, &ix, &iy, &s, margin);

  for (;;) {
    if (ix < 0 || ix >= W || iy < 0 || iy >= H) return -1;
    if (M->max_steps >= 0 && *iters >= M->max_steps) return -1;
    ++*iters;
    cell_exit(&g, ix, iy, L, &sx, &sy);
    double se = sx <= sy ? sx : sy;
    double sb = se < 1.0 ? se : 1.0;
    double za = 1.0 / (k0 + s * dk), zb = 1.0 / (k0 + sb * dk);
    double zlo = za < zb ? za : zb, zhi = za < zb ? zb : za;
    double hz = (L == 0) ? M->depth[(long)iy * W + ix]
                         : M->hiz[M->hoff[L] + (long)(iy >> L) * M->hw[L] + (ix >> L)];
    if (isfinite(hz)) upd_margin(margin, (zhi - hz) / hz);
    if (zhi < hz) {
      /* the whole cell lies behind the ray: skip it and go up a level */
      if (isfinite(se)) upd_margin(margin, se - 1.0);
      if (!(se < 1.0)) return -1;
      cell_step(&g, L, sx, sy, &ix, &iy, &s, margin);
      if (L + 1 < M->levels) ++L;
    } else if (L > 0) {
      --L; /* something in this cell may be hit: refine */
    } else {
      upd_margin(margin, (zlo - (hz + M->thickness)) / (hz + M->thickness));
      if (zlo <= hz + M->thickness) return iy * W + ix;
      /* the ray passes behind this pixel by more than the thickness: next pixel */
      if (isfinite(se)) upd_margin(margin, se - 1.0);
      if (!(se < 1.0)) return -1;
      cell_step(&g, 0, sx, sy, &ix, &iy, &s, margin);
    }
  }
}

static void march_init(march_t *M, const cam_t *cam, const double *depth_v, const double *hiz_v, int levels,
                       int max_steps, double thickness, double max_distance) {
  M->cam = cam;
  M->depth = depth_v;
  M->hiz = hiz_v;
  M->levels = levels;
  M->max_steps = max_steps;
  M->thickness = thickness;
  M->max_distance = max_distance;
  long off = 0;
  for (int l = 1; l < levels; ++l) {
    M->hoff[l] = off;
    M->hw[l] = lvl_dim(cam->W, l);
    off += (long)lvl_dim(cam->H, l) * lvl_dim(cam->W, l);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* One sample's geometry: GGX half vector, reflected direction and validity (Sec. 3.3)          */
/* ------------------------------------------------------------------------------------------ */
/* ------------------------------------------------------------------------------------------ */
/* Depth normals (Sec. 3.1, "depth normal": surface normals from the rendered depth buffer by   */
/* finite differences, as in 2DGS).  P(x, y) = d(x, y) z(x, y) is the camera-space point of the */
/* pixel centre at linear depth z.  Per direction the difference is central where both         */
/* neighbours are foreground, one-sided where one is, absent where neither is.  The normal is   */
/* normalize(dP/dy x dP/dx) (y down the image), flipped to face the camera, in world space.     */
/* With a direction absent, or a zero cross product, it is the unit vector towards the camera.  */
/* Background pixels get (0, 0, 0).                                                             */
/* ------------------------------------------------------------------------------------------ */
void orc_depth_normals(int V, int H, int W, const double *depth, const double *cams, double *normal_out) {
  for (int v = 0; v < V; ++v) {
    cam_t cam = cam_init(cams + 14 * v, H, W);
    const double *dz = depth + (long)v * H * W;
#pragma omp parallel for schedule(static)
    for (int rem = 0; rem < H * W; ++rem) {
      int y = rem / W, x = rem % W;
      double *out = normal_out + 3 * ((long)v * H * W + rem);
      out[0] = out[1] = out[2] = 0.0;
      if (is_background(dz[rem])) continue;
      v3 P = scl(pix_dir_cam(&cam, x, y), dz[rem]);
      int l = (x > 0 && !is_background(dz[rem - 1])) ? x - 1 : x;
      int r = (x + 1 < W && !is_background(dz[rem + 1])) ? x + 1 : x;
      int u = (y > 0 && !is_background(dz[rem - W])) ? y - 1 : y;
      int b = (y + 1 < H && !is_background(dz[rem + W])) ? y + 1 : y;
      v3 n = scl(P, -1.0 / len(P));
      if (l != r && u != b) {
        v3 dPx = sub(scl(pix_dir_cam(&cam, r, y), dz[y * W + r]), scl(pix_dir_cam(&cam, l, y), dz[y * W + l]));
        v3 dPy = sub(scl(pix_dir_cam(&cam, x, b), dz[b * W + x]), scl(pix_dir_cam(&cam, x, u), dz[u * W + x]));
        v3 c = mk(dPy.y * dPx.z - dPy.z * dPx.y, dPy.z * dPx.x - dPy.x * dPx.z, dPy.x * dPx.y - dPy.y * dPx.x);
        double cl = len(c);
        if (cl > 0.0) {
          n = scl(c, 1.0 / cl);
          if (dot(n, P) > 0.0) n = scl(n, -1.0);
        }
      }
      v3 nw = cam_to_world_dir(&cam, n);
      out[0] = nw.x; out[1] = nw.y; out[2] = nw.z;
    }
  }
}

typedef struct {
  v3 h, w;            /* half vector, sampled direction (world) */
  double vh, nh, nw;  /* at the sampling normal */
  int valid;
} smp_t;

static smp_t make_sample_frame(v3 n, double sgn, v3 vv, double nv, double rho, const double xi[2]) {
  smp_t r;
  r.h = ggx_sample_h_frame(n, sgn, rho, xi[0], xi[1]);
  r.vh = dot(vv, r.h);
  r.w = sub(scl(r.h, 2.0 * r.vh), vv);
  r.nh = dot(n, r.h);
  r.nw = dot(n, r.w);
  r.valid = (nv > 0.0) && (r.nw > 0.0) && (r.vh > 0.0) && (r.nh > 0.0);
  return r;
}

static smp_t make_sample(v3 n, v3 vv, double nv, double rho, const double xi[2]) {
  return make_sample_frame(n, (n.z >= 0.0) ? 1.0 : -1.0, vv, nv, rho, xi);
}

/* ------------------------------------------------------------------------------------------ */
/* Trace + Monte-Carlo + composite (Sec. 3.3):                                                 */
/*   c_s' = 1/N_s sum_i f_s L_i (w_i.n) / p_GGX(w_i) = 1/N_s sum_i F G (v.h) / ((n.v)(n.h)) L_i  */
/*   L_i = c1[hit] or, on a miss, the environment at mip 0 in direction w_i;                    */
/*   final = c_d + c_s'.  Invalid samples (n.v <= 0, n.w <= 0) count as zero in the average.    */
/* Optional diffuse-indirect channel (flag 1): c_id = (1-m) a / pi * 1/N_s sum L_i (n.w)/p_i,   */
/* p_i = D (n.h) / (4 v.h), added to final.                                                     */
/* ------------------------------------------------------------------------------------------ */
static int levels_ok(int levels) { return levels >= 1 && levels <= OR_MAX_LEVELS; }

/* hit_idx codes */
#define OR_MISS (-1)
#define OR_INVALID (-2)
#define OR_BACKGROUND (-3)

int orc_trace(int V, int H, int W, const double *depth, const double *normal, const double *albedo,
              const double *rough, const double *metal, const double *cams, const double *mips, int He, int We,
              const double *hiz, const double *c1, const double *cd, int spp, int max_steps, int hiz_levels,
              double thickness, double max_distance, uint64_t seed, uint32_t flags, const int64_t *pix_list,
              long n_pix, double *cs_mc, double *final_out, double *cid_out, int32_t *hit_idx, int32_t *iters_out,
              double *margin_out) {
  if (!levels_ok(hiz_levels) || spp < 1) return -1;
  env_t e;
  env_init(&e, mips, He, We);
  int brute = (flags & ORF_BRUTE_FORCE) != 0;
  int levels = brute ? 1 : hiz_levels;
  int msteps = brute ? -1 : max_steps;
  long per = orc_hiz_floats_per_view(H, W, hiz_levels);
  long total = pix_list ? n_pix : (long)V * H * W;
  cam_t *camv = (cam_t *)malloc(sizeof(cam_t) * (size_t)V);
  for (int v = 0; v < V; ++v) camv[v] = cam_init(cams + 14 * v, H, W);

#pragma omp parallel for schedule(dynamic, 64)
  for (long k = 0; k < total; ++k) {
    long p = pix_list ? pix_list[k] : k;
    int v = (int)(p / ((long)H * W));
    int rem = (int)(p % ((long)H * W));
    int y = rem / W, x = rem % W;
    const cam_t *cam = &camv[v];
    march_t M;
    march_init(&M, cam, depth + (long)v * H * W, hiz ? hiz + (long)v * per : NULL, levels, msteps, thickness,
               max_distance);
    double acc[3] = {0, 0, 0}, accd[3] = {0, 0, 0};
    double z0 = depth[p];
    if (is_background(z0)) {
      for (int s = 0; s < spp; ++s) {
        if (hit_idx) hit_idx[k * spp + s] = OR_BACKGROUND;
        if (iters_out) iters_out[k * spp + s] = 0;
        if (margin_out) margin_out[k * spp + s] = INFINITY;
      }
      for (int c = 0; c < 3; ++c) {
        if (cs_mc) cs_mc[3 * k + c] = 0.0;
        if (cid_out) cid_out[3 * k + c] = 0.0;
        final_out[3 * k + c] = c1[3 * p + c];
      }
      continue;
    }
    v3 d = cam_to_world_dir(cam, pix_dir_cam(cam, x, y));
    v3 vv = scl(d, -1.0 / len(d));
    v3 n = ld3(normal + 3 * p);
    double nv = dot(n, vv);
    double rho = rough[p], m = metal[p];
    for (int s = 0; s < spp; ++s) {
      double xi[2];
      sample_uniforms(seed, v, (uint32_t)rem, (uint32_t)s, xi);
      smp_t sm = make_sample(n, vv, nv, rho, xi);
      double mg = INFINITY;
      upd_margin(&mg, nv);
      upd_margin(&mg, sm.nw);
      upd_margin(&mg, sm.vh);
      upd_margin(&mg, sm.nh);
      int it = 0, q = OR_INVALID;
      if (sm.valid) {
        q = march(&M, x, y, z0, world_to_cam_dir(cam, sm.w), &it, &mg);
        double Li[3];
        if (q >= 0) {
          const double *src = c1 + 3 * ((long)v * H * W + q);
          Li[0] = src[0]; Li[1] = src[1]; Li[2] = src[2];
        } else {
          env_lookup(&e, sm.w, 0.0, Li);
        }
        double G = orc_ggx_G1(sm.nw, rho) * orc_ggx_G1(nv, rho);
        for (int c = 0; c < 3; ++c) {
          double F = orc_fresnel(f0_of(albedo[3 * p + c], m), sm.vh);
          acc[c] += F * G * sm.vh / (nv * sm.nh) * Li[c];
        }
        if (flags & ORF_DIFFUSE_INDIRECT) {
          double pdf = orc_ggx_D(sm.nh, rho) * sm.nh / (4.0 * sm.vh);
          if (pdf > 0.0 && isfinite(pdf))
            for (int c = 0; c < 3; ++c) accd[c] += (1.0 - m) * albedo[3 * p + c] / OR_PI * Li[c] * sm.nw / pdf;
        }
      }
      if (hit_idx) hit_idx[k * spp + s] = q;
      if (iters_out) iters_out[k * spp + s] = it;
      if (margin_out) margin_out[k * spp + s] = mg;
    }
    for (int c = 0; c < 3; ++c) {
      double csm = acc[c] / spp, cid = accd[c] / spp;
      if (cs_mc) cs_mc[3 * k + c] = csm;
      if (cid_out) cid_out[3 * k + c] = cid;
      final_out[3 * k + c] = cd[3 * p + c] + csm + ((flags & ORF_DIFFUSE_INDIRECT) ? cid : 0.0);
    }
  }
  free(camv);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Pathwise (reparameterised) form of one Monte-Carlo summand (Sec. 3.3 estimator): with the   */
/* sample's uniforms xi and hit index q fixed, the half vector and direction are drawn from the */
/* given normal n and roughness rho, the weight is the cancelled f_s (n.w) / p_GGX(w) =          */
/* F G1(n.w) G1(n.v) (v.h) / ((n.v)(n.h)) at those same n and rho, L = c1 of the frozen hit     */
/* pixel (c1q) or the environment at mip 0 in the new direction.  spec and cid receive the      */
/* specular summand F K L and the diffuse-indirect summand (1-m) a / pi L (n.w) / p per channel;  */
/* returns 0 (and zeros) when the re-drawn sample is invalid.  sgn fixes the branch of the     */
/* sampling frame (the sign of the base normal's z) so that the summand is smooth in n.        */
/* ------------------------------------------------------------------------------------------ */
static int pathwise_summand(v3 n, double sgn, double rho, v3 vv, const double xi[2], const double a[3], double m,
                            int q, const double *c1q, const env_t *e, uint32_t flags, double spec[3], double cid[3]) {
  double nv = dot(n, vv);
  smp_t sm = make_sample_frame(n, sgn, vv, nv, rho, xi);
  for (int c = 0; c < 3; ++c) spec[c] = cid[c] = 0.0;
  if (!sm.valid) return 0;
  double L[3];
  if (q >= 0) {
    L[0] = c1q[0]; L[1] = c1q[1]; L[2] = c1q[2];
  } else {
    env_lookup(e, sm.w, 0.0, L);
  }
  double K = orc_ggx_G1(sm.nw, rho) * orc_ggx_G1(nv, rho) * sm.vh / (nv * sm.nh);
  for (int c = 0; c < 3; ++c) spec[c] = K * orc_fresnel(f0_of(a[c], m), sm.vh) * L[c];
  if (flags & ORF_DIFFUSE_INDIRECT) {
    double pdf = orc_ggx_D(sm.nh, rho) * sm.nh / (4.0 * sm.vh);
    if (pdf > 0.0 && isfinite(pdf))
      for (int c = 0; c < 3; ++c) cid[c] = (1.0 - m) * a[c] / OR_PI * L[c] * sm.nw / pdf;
  }
  return 1;
}

/* ------------------------------------------------------------------------------------------ */
/* Replay forward: the forward pass with the samples, their validity, the sampling pdf and the */
/* hit pixels frozen at a base parameter set, evaluated at another parameter set.  Per sample   */
/*   contribution = f_s(w; eval) (n.w) / p(w; base) * L(eval),  f_s = D F G / (4 (n.w)(n.v)),   */
/* so that at eval == base it equals the forward pass.  This is the function whose derivative  */
/* the backward pass computes (the march itself is not differentiable, Sec. 5).                 */
/* Pixels whose base roughness is 0 (delta lobe) keep the cancelled form G (v.h)/((n.v)(n.h)). */
/* With flag 4 (pathwise) a sample valid at the base is re-drawn at the evaluation normal and  */
/* roughness instead (pathwise_summand); its hit index stays frozen.                           */
/* ------------------------------------------------------------------------------------------ */
int orc_replay_final(int V, int H, int W, const double *depth, const double *cams, int He, int We,
                     const double *lut, int lut_n, int spp, uint64_t seed, uint32_t flags,
                     const double *normal_b, const double *rough_b,
                     const double *normal_e, const double *albedo_e, const double *rough_e, const double *metal_e,
                     const double *env_e, const int32_t *hit_idx, double *final_out) {
  long np = (long)V * H * W;
  long nm = orc_env_mip_doubles(He, We);
  if (nm < 0) return -1;
  double *mips = (double *)malloc(sizeof(double) * (size_t)nm);
  double *cd = (double *)malloc(sizeof(double) * (size_t)np * 3);
  double *c1 = (double *)malloc(sizeof(double) * (size_t)np * 3);
  orc_build_env_mips(env_e, He, We, mips);
  orc_shade_direct(V, H, W, depth, normal_e, albedo_e, rough_e, metal_e, cams, mips, He, We, lut, lut_n, cd, NULL, c1);
  env_t e;
  env_init(&e, mips, He, We);
  for (int v = 0; v < V; ++v) {
    cam_t cam = cam_init(cams + 14 * v, H, W);
#pragma omp parallel for schedule(dynamic, 64)
    for (int rem = 0; rem < H * W; ++rem) {
      long p = (long)v * H * W + rem;
      int y = rem / W, x = rem % W;
      if (is_background(depth[p])) {
        for (int c = 0; c < 3; ++c) final_out[3 * p + c] = c1[3 * p + c];
        continue;
      }
      v3 d = cam_to_world_dir(&cam, pix_dir_cam(&cam, x, y));
      v3 vv = scl(d, -1.0 / len(d));
      v3 nb = ld3(normal_b + 3 * p), ne = ld3(normal_e + 3 * p);
      double nvb = dot(nb, vv), nve = dot(ne, vv);
      double rb = rough_b[p], re = rough_e[p], m = metal_e[p];
      double acc[3] = {0, 0, 0}, accd[3] = {0, 0, 0};
      for (int s = 0; s < spp; ++s) {
        double xi[2];
        sample_uniforms(seed, v, (uint32_t)rem, (uint32_t)s, xi);
        smp_t sm = make_sample(nb, vv, nvb, rb, xi);
        if (!sm.valid) continue;
        int q = hit_idx[p * spp + s];
        if (flags & ORF_PATHWISE) {  /* direction re-drawn at the evaluation point */
          double spec[3], cidv[3];
          const double *c1q = q >= 0 ? c1 + 3 * ((long)v * H * W + q) : NULL;
          pathwise_summand(ne, nb.z >= 0.0 ? 1.0 : -1.0, re, vv, xi, albedo_e + 3 * p, m, q, c1q, &e, flags, spec,
                           cidv);
          for (int c = 0; c < 3; ++c) {
            acc[c] += spec[c];
            accd[c] += cidv[c];
          }
          continue;
        }
        double Li[3];
        if (q >= 0) {
          const double *src = c1 + 3 * ((long)v * H * W + q);
          Li[0] = src[0]; Li[1] = src[1]; Li[2] = src[2];
        } else {
          env_lookup(&e, sm.w, 0.0, Li);
        }
        double nwe = dot(ne, sm.w), nhe = dot(ne, sm.h);
        double G = orc_ggx_G1(nwe, re) * orc_ggx_G1(nve, re);
        double K;
        double pdf_b = orc_ggx_D(sm.nh, rb) * sm.nh / (4.0 * sm.vh);
        if (rb > 0.0) K = orc_ggx_D(nhe, re) * G / (4.0 * nve * pdf_b);
        else K = G * sm.vh / (nve * nhe);
        for (int c = 0; c < 3; ++c) {
          double F = orc_fresnel(f0_of(albedo_e[3 * p + c], m), sm.vh);
          acc[c] += K * F * Li[c];
        }
        if ((flags & ORF_DIFFUSE_INDIRECT) && pdf_b > 0.0 && isfinite(pdf_b))
          for (int c = 0; c < 3; ++c) accd[c] += (1.0 - m) * albedo_e[3 * p + c] / OR_PI * Li[c] * nwe / pdf_b;
      }
      for (int c = 0; c < 3; ++c)
        final_out[3 * p + c] = cd[3 * p + c] + acc[c] / spp + ((flags & ORF_DIFFUSE_INDIRECT) ? accd[c] / spp : 0.0);
    }
  }
  free(mips);
  free(cd);
  free(c1);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* Adjoint of the replay forward (the backward pass): d loss / d {albedo, roughness, metallic,  */
/* normal, environment base texels} given d loss / d final.                                    */
/* ------------------------------------------------------------------------------------------ */

/* d ln G1(z; rho) / dz and / drho */
static void dlnG1(double z, double rho, double *dz, double *drho) {
  double a2 = rho * rho;
  double s = sqrt(a2 + (1.0 - a2) * z * z);
  *dz = 1.0 / z - (1.0 + (1.0 - a2) * z / s) / (z + s);
  *drho = -(rho * (1.0 - z * z) / s) / (z + s);
}

/* d ln D(c; rho) / dc and / drho, c = n.h */
static void dlnD(double c, double rho, double *dc, double *drho) {
  double a2 = rho * rho;
  double den = c * c * (a2 - 1.0) + 1.0;
  *dc = -4.0 * c * (a2 - 1.0) / den;
  *drho = 2.0 / rho - 4.0 * rho * c * c / den;
}

/* Scatter g (per channel) through the bilinear taps of level l, and return d/dx, d/dy of the
 * bilinear value contracted with g. */
static void bilin_adj(const env_t *e, int l, double u, double v, const double g[3], double wscale, double *gm,
                      double *gx, double *gy) {
  int h = e->h[l], w = e->w[l];
  double x = u * w - 0.5, y = v * h - 0.5;
  double tx = x - floor(x), ty = y - floor(y);
  bilin_t b = env_taps(e, l, u, v);
  *gx = 0.0;
  *gy = 0.0;
  for (int c = 0; c < 3; ++c) {
    double T00 = e->mips[b.idx[0] + c], T01 = e->mips[b.idx[1] + c];
    double T10 = e->mips[b.idx[2] + c], T11 = e->mips[b.idx[3] + c];
    *gx += g[c] * ((1 - ty) * (T01 - T00) + ty * (T11 - T10));
    *gy += g[c] * ((1 - tx) * (T10 - T00) + tx * (T11 - T01));
    if (gm)
      for (int k = 0; k < 4; ++k) {
#pragma omp atomic
        gm[b.idx[k] + c] += wscale * b.wt[k] * g[c];
      }
  }
}

/* Adjoint of SampleEnvMap(d, lambda): accumulates texel gradients into gm (all mip levels,
 * packed like the mips) and returns d/d(direction) and d/dlambda. */
static void env_lookup_adj(const env_t *e, v3 d, double lam, const double g[3], double *gm, v3 *gd, double *glam) {
  double lmax = (double)(e->levels - 1);
  int inside = (lam > 0.0 && lam < lmax);
  if (lam < 0.0) lam = 0.0;
  if (lam > lmax) lam = lmax;
  int l0 = (int)floor(lam);
  int l1 = l0 + 1 < e->levels ? l0 + 1 : l0;
  double t = lam - (double)l0;
  double u, v;
  dir_to_uv(d, &u, &v);
  double gx0, gy0, gx1, gy1;
  bilin_adj(e, l0, u, v, g, 1.0 - t, gm, &gx0, &gy0);
  bilin_adj(e, l1, u, v, g, t, gm, &gx1, &gy1);
  double gu = (1.0 - t) * gx0 * e->w[l0] + t * gx1 * e->w[l1];
  double gv = (1.0 - t) * gy0 * e->h[l0] + t * gy1 * e->h[l1];
  /* d lambda: difference of the two bilinear values */
  *glam = 0.0;
  if (inside && l1 != l0) {
    bilin_t b0 = env_taps(e, l0, u, v), b1 = env_taps(e, l1, u, v);
    for (int c = 0; c < 3; ++c) {
      double v0 = 0.0, v1 = 0.0;
      for (int k = 0; k < 4; ++k) {
        v0 += b0.wt[k] * e->mips[b0.idx[k] + c];
        v1 += b1.wt[k] * e->mips[b1.idx[k] + c];
      }
      *glam += g[c] * (v1 - v0);
    }
  }
  /* chain through u(d), v(d) */
  double q2 = d.x * d.x + d.z * d.z, q = sqrt(q2);
  *gd = mk(0, 0, 0);
  if (q2 > 0.0) {
    double r2 = q2 + d.y * d.y;
    double dux = -d.z / (2.0 * OR_PI * q2), duz = d.x / (2.0 * OR_PI * q2);
    double dvx = d.y * d.x / (q * r2 * OR_PI), dvz = d.y * d.z / (q * r2 * OR_PI), dvy = -q / (r2 * OR_PI);
    *gd = mk(gu * dux + gv * dvx, gv * dvy, gu * duz + gv * dvz);
  }
}

int orc_backward(int V, int H, int W, const double *depth, const double *normal, const double *albedo,
                 const double *rough, const double *metal, const double *cams, const double *mips, int He, int We,
                 const double *lut, int lut_n, const double *c1, const int32_t *hit_idx, const double *g_final,
                 int spp, uint64_t seed, uint32_t flags, double *g_albedo, double *g_rough, double *g_metal,
                 double *g_normal, double *g_env) {
  env_t e;
  env_init(&e, mips, He, We);
  long np = (long)V * H * W;
  long nm = orc_env_mip_doubles(He, We);
  double lmax = (double)(e.levels - 1);
  double *g_c1 = (double *)calloc((size_t)np * 3, sizeof(double));
  double *g_mips = (double *)calloc((size_t)nm, sizeof(double));

  /* (1) per receiver pixel: adjoint of the Monte-Carlo sum with frozen samples and hits */
  for (int v = 0; v < V; ++v) {
    cam_t cam = cam_init(cams + 14 * v, H, W);
#pragma omp parallel for schedule(dynamic, 64)
    for (int rem = 0; rem < H * W; ++rem) {
      long p = (long)v * H * W + rem;
      int y = rem / W, x = rem % W;
      g_albedo[3 * p] = g_albedo[3 * p + 1] = g_albedo[3 * p + 2] = 0.0;
      g_normal[3 * p] = g_normal[3 * p + 1] = g_normal[3 * p + 2] = 0.0;
      g_rough[p] = 0.0;
      g_metal[p] = 0.0;
      if (is_background(depth[p])) continue;
      v3 d = cam_to_world_dir(&cam, pix_dir_cam(&cam, x, y));
      v3 vv = scl(d, -1.0 / len(d));
      v3 n = ld3(normal + 3 * p);
      double nv = dot(n, vv);
      double rho = rough[p], m = metal[p];
      double ga[3] = {0, 0, 0}, gr = 0.0, gmt = 0.0;
      v3 gn = mk(0, 0, 0);
      for (int s = 0; s < spp; ++s) {
        double xi[2];
        sample_uniforms(seed, v, (uint32_t)rem, (uint32_t)s, xi);
        smp_t sm = make_sample(n, vv, nv, rho, xi);
        if (!sm.valid) continue;
        int q = hit_idx[p * spp + s];
        double Li[3];
        if (q >= 0) {
          const double *src = c1 + 3 * ((long)v * H * W + q);
          Li[0] = src[0]; Li[1] = src[1]; Li[2] = src[2];
        } else {
          env_lookup(&e, sm.w, 0.0, Li);
        }
        double K = orc_ggx_G1(sm.nw, rho) * orc_ggx_G1(nv, rho) * sm.vh / (nv * sm.nh);
        double fc = pow(1.0 - sm.vh, 5.0);
        double gL[3], gK = 0.0;
        for (int c = 0; c < 3; ++c) {
          double a = albedo[3 * p + c];
          double F = orc_fresnel(f0_of(a, m), sm.vh);
          double gC = g_final[3 * p + c] / spp;
          gL[c] = gC * K * F;
          double gF = gC * K * Li[c];
          ga[c] += gF * m * (1.0 - fc);
          gmt += gF * (a - 0.04) * (1.0 - fc);
          gK += gC * F * Li[c];
        }
        const int pathwise = (flags & ORF_PATHWISE) != 0;
        if (pathwise) {
          /* d/d{n, rho} of the pathwise summand contracted with g_final / N: central differences */
          const double hstep = g_pathwise_h;
          double gCv[3];
          for (int c = 0; c < 3; ++c) gCv[c] = g_final[3 * p + c] / spp;
          const double *c1q = q >= 0 ? c1 + 3 * ((long)v * H * W + q) : NULL;
          double dth[4];
          for (int k = 0; k < 4; ++k) {
            double fpm[2];
            for (int sg = 0; sg < 2; ++sg) {
              double dlt = sg == 0 ? (g_pathwise_mode < 0 ? 0.0 : hstep) : (g_pathwise_mode > 0 ? 0.0 : -hstep);
              v3 nn = n;
              double rr = rho;
              if (k == 0) nn.x += dlt;
              else if (k == 1) nn.y += dlt;
              else if (k == 2) nn.z += dlt;
              else rr += dlt;
              double spec[3], cidv[3];
              pathwise_summand(nn, n.z >= 0.0 ? 1.0 : -1.0, rr, vv, xi, albedo + 3 * p, m, q, c1q, &e, flags,
                               spec, cidv);
              fpm[sg] = 0.0;
              for (int c = 0; c < 3; ++c) fpm[sg] += gCv[c] * (spec[c] + cidv[c]);
            }
            dth[k] = (fpm[0] - fpm[1]) / (g_pathwise_mode == 0 ? 2.0 * hstep : hstep);
          }
          gn = add(gn, mk(dth[0], dth[1], dth[2]));
          gr += dth[3];
        }
        /* d ln K with K = D(n.h) G1(n.w) G1(n.v) / (4 (n.v) p_frozen) */
        double dgw_z, dgw_r, dgv_z, dgv_r;
        dlnG1(sm.nw, rho, &dgw_z, &dgw_r);
        dlnG1(nv, rho, &dgv_z, &dgv_r);
        double dlnK_r = dgw_r + dgv_r;
        v3 dlnK_n = add(scl(sm.w, dgw_z), scl(vv, dgv_z - 1.0 / nv));
        if (rho > 0.0) {
          double dd_c, dd_r;
          dlnD(sm.nh, rho, &dd_c, &dd_r);
          dlnK_r += dd_r;
          dlnK_n = add(dlnK_n, scl(sm.h, dd_c));
        }
        double gKK = gK * K;
        if (!pathwise) {
          gr += gKK * dlnK_r;
          gn = add(gn, scl(dlnK_n, gKK));
        }
        if (flags & ORF_DIFFUSE_INDIRECT) {
          double pdf = orc_ggx_D(sm.nh, rho) * sm.nh / (4.0 * sm.vh);
          if (pdf > 0.0 && isfinite(pdf)) {
            for (int c = 0; c < 3; ++c) {
              double a = albedo[3 * p + c];
              double gC = g_final[3 * p + c] / spp;
              ga[c] += gC * (1.0 - m) / OR_PI * Li[c] * sm.nw / pdf;
              gmt -= gC * a / OR_PI * Li[c] * sm.nw / pdf;
              if (!pathwise) gn = add(gn, scl(sm.w, gC * (1.0 - m) * a / OR_PI * Li[c] / pdf));
              gL[c] += gC * (1.0 - m) * a / OR_PI * sm.nw / pdf;
            }
          }
        }
        if (q >= 0) {
          double *dst = g_c1 + 3 * ((long)v * H * W + q);
          for (int c = 0; c < 3; ++c) {
#pragma omp atomic
            dst[c] += gL[c];
          }
        } else {
          double u, vt, gx, gy;
          dir_to_uv(sm.w, &u, &vt);
          bilin_adj(&e, 0, u, vt, gL, 1.0, g_mips, &gx, &gy);
        }
      }
      for (int c = 0; c < 3; ++c) g_albedo[3 * p + c] = ga[c];
      g_rough[p] = gr;
      g_metal[p] = gmt;
      g_normal[3 * p] = gn.x; g_normal[3 * p + 1] = gn.y; g_normal[3 * p + 2] = gn.z;
    }
  }

  /* (2) per pixel: adjoint of the direct shading with d/dc_d = g_final + g_c1, d/dc_s = g_c1 */
  for (int v = 0; v < V; ++v) {
    cam_t cam = cam_init(cams + 14 * v, H, W);
#pragma omp parallel for schedule(dynamic, 64)
    for (int rem = 0; rem < H * W; ++rem) {
      long p = (long)v * H * W + rem;
      int y = rem / W, x = rem % W;
      v3 d = cam_to_world_dir(&cam, pix_dir_cam(&cam, x, y));
      double gcd[3], gcs[3];
      for (int c = 0; c < 3; ++c) {
        gcd[c] = g_final[3 * p + c] + g_c1[3 * p + c];
        gcs[c] = g_c1[3 * p + c];
      }
      if (is_background(depth[p])) {
        double u, vt, gx, gy;
        dir_to_uv(d, &u, &vt);
        bilin_adj(&e, 0, u, vt, gcd, 1.0, g_mips, &gx, &gy);
        continue;
      }
      v3 vv = scl(d, -1.0 / len(d));
      v3 n = ld3(normal + 3 * p);
      double nv = dot(n, vv);
      double mu = nv < 1e-4 ? 1e-4 : (nv > 1.0 ? 1.0 : nv);
      v3 r = sub(scl(n, 2.0 * nv), vv);
      double rho = rough[p], m = metal[p];
      double lam = log2(rho + 1.0) * lmax;
      lutv_t ab = lut_sample(lut, lut_n, rho, mu);
      double Er[3], En[3];
      env_lookup(&e, r, lam, Er);
      env_lookup(&e, n, lam, En);
      double gEn[3], gEr[3], gA = 0.0, gB = 0.0, gm_ = 0.0;
      for (int c = 0; c < 3; ++c) {
        double a = albedo[3 * p + c];
        double F0 = f0_of(a, m);
        g_albedo[3 * p + c] += gcd[c] * (1.0 - m) * En[c] + gcs[c] * Er[c] * ab.A * m;
        gm_ += -gcd[c] * a * En[c] + gcs[c] * Er[c] * ab.A * (a - 0.04);
        gEn[c] = gcd[c] * (1.0 - m) * a;
        gEr[c] = gcs[c] * (F0 * ab.A + ab.B);
        gA += gcs[c] * Er[c] * F0;
        gB += gcs[c] * Er[c];
      }
      v3 gdn, gdr;
      double gl1, gl2;
      env_lookup_adj(&e, n, lam, gEn, g_mips, &gdn, &gl1);
      env_lookup_adj(&e, r, lam, gEr, g_mips, &gdr, &gl2);
      double gnv = 0.0;
      if (nv > 1e-4 && nv < 1.0) gnv += gA * ab.dA_dmu + gB * ab.dB_dmu;
      /* r = 2 (n.v) n - v */
      v3 gn = add(gdn, add(scl(vv, 2.0 * dot(gdr, n)), scl(gdr, 2.0 * nv)));
      gn = add(gn, scl(vv, gnv));
      double gr = gA * ab.dA_drho + gB * ab.dB_drho + (gl1 + gl2) * lmax / ((rho + 1.0) * log(2.0));
      g_rough[p] += gr;
      g_metal[p] += gm_;
      g_normal[3 * p] += gn.x; g_normal[3 * p + 1] += gn.y; g_normal[3 * p + 2] += gn.z;
    }
  }

  /* (3) adjoint of the 2x2 box-filter mip chain, top level down: each child gets 1/4 */
  for (int l = e.levels - 1; l >= 1; --l) {
    const double *src = g_mips + e.off[l];
    double *dst = g_mips + e.off[l - 1];
    int wd = e.w[l - 1];
    for (int i = 0; i < e.h[l]; ++i)
      for (int j = 0; j < e.w[l]; ++j)
        for (int c = 0; c < 3; ++c) {
          double g = 0.25 * src[((long)i * e.w[l] + j) * 3 + c];
          dst[((long)(2 * i) * wd + 2 * j) * 3 + c] += g;
          dst[((long)(2 * i) * wd + 2 * j + 1) * 3 + c] += g;
          dst[((long)(2 * i + 1) * wd + 2 * j) * 3 + c] += g;
          dst[((long)(2 * i + 1) * wd + 2 * j + 1) * 3 + c] += g;
        }
  }
  memcpy(g_env, g_mips, sizeof(double) * (size_t)He * We * 3);
  free(g_c1);
  free(g_mips);
  return 0;
}

/* ------------------------------------------------------------------------------------------ */
/* threading control for timing                                                                */
/* ------------------------------------------------------------------------------------------ */
/* Step (default 1e-6) and form (0 central, default; +1 forward; -1 backward) of the
 * differences of the pathwise derivatives.  Where the per-sample function is not
 * differentiable (a sample on a bilinear texel-centre kink of the map, or on the edge of
 * validity where the summand reaches 0 with a nonzero slope) the difference depends on the
 * step and the one-sided differences disagree; comparing them finds those points. */
void orc_set_pathwise_step(double h, int mode) {
  if (h > 0.0) g_pathwise_h = h;
  g_pathwise_mode = mode < 0 ? -1 : (mode > 0 ? 1 : 0);
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
