/*
 * FP64 CPU oracle for the VRSplat rasterizer hot path (arXiv 2505.10144).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the CPU-baseline leg of the
 * benchmark call this library; the product path (the CUDA library and its Python
 * binding) never does, and shares no code, header or constant with it.
 *
 * Everything is written as the plain definition, in double precision, for reading:
 *
 *   - 3D Gaussian G(x) = exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)), Sigma = R S S^T R^T   (Eq. 1)
 *   - Optimal Projection: each Gaussian is projected onto the tangent plane of the unit
 *     sphere around the camera centre o, perpendicular to mu - o                    (Sec. 4.2)
 *   - front-to-back blending C = sum_i c_i a_i prod_{j<i} (1 - a_j), a = sigma G_2D  (Eq. 2)
 *   - per-pixel order by the depth of each Gaussian's maximum response along the ray
 *     (StopThePop, Sec. 4.1), ties broken by Gaussian index
 *   - tile culling on the optimal plane: a Gaussian/tile pair is dropped when the largest
 *     alpha over the tile's quadrilateral is below 1/255; the maximum is the projected
 *     mean when it lies inside, else on an edge, found in closed form           (Eq. 4)
 *   - single-pass foveation: 32x32 tiles (16x16 as a tuning option), focus tiles at full
 *     resolution, periphery tiles shaded on 2x2 pixel groups, hybrid tiles blended by
 *     the continuous mask                                                        (Sec. 4.3)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - camera: OpenCV axes, world->camera [R|t], pixel centres at (x+0.5, y+0.5);
 *   - near cull at view z < near_z (0.2), alpha clamp 0.99, transmittance stop 1e-4,
 *     background given by the caller (black by default);
 *   - dilation 0.3 px^2 expressed on the tangent plane as 0.3/(fx fy) I;
 *   - tangent-plane basis e1 = (u_z, 0, -u_x)/|.|, e2 = u x e1 (camera frame); every
 *     result is invariant to this choice;
 *   - depth t* = v^T Sigma^-1 (mu - o) / v^T Sigma^-1 v with v = K^-1 (px, py, 1), i.e. the
 *     camera-z of the point of maximum response along the pixel's ray;
 *   - tile key = t* on the ray through the tile maximum x^ projected back to the image;
 *     Eq. 4's line parameter is clamped to the edge segment;
 *   - hierarchical resort = a cascade of three min-windows (4x4-sample block, 2x2-sample
 *     block, per sample), membership of a block = kept at any still-active sample of it,
 *     keys = t* at the block centre; window mode = the cascade with k1 = k2 = 0; the
 *     exact order = the cascade with unbounded windows.  This function is "parity
 *     unpinned" against the paper (only its invariants are pinned).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_ALPHA_MIN (1.0 / 255.0)
#define OG_ALPHA_MAX 0.99
#define OG_T_STOP 1e-4
#define OG_DILATION_PX2 0.3

/* relative margins of the marginal-sample rule (set from og_opts for each render) */
static double g_margin_alpha = 1e-4, g_margin_stop = 1e-4, g_margin_tie = 1e-5;

/* Gaussian parameters in SoA layout (double, so that finite differences can perturb
 * them below float32 resolution; the product's float32 inputs convert exactly). */
typedef struct {
  const double *mean, *log_scale, *quat, *opacity_logit, *sh;
  int64_t n;
  int sh_degree;
} og_scene;

typedef struct {
  double w2c[12];
  double fx, fy, cx, cy;
  int width, height;
  double near_z;
} og_camera;

typedef struct {
  int mode;      /* 0 exact, 1 window (k3), 2 hierarchical (k1, k2, k3), 3 global sort by view-space z
                  * of the mean, 4 global sort by distance |mu - o| (the popping orders of 3DGS
                  * and Mini-Splatting, Sec. 3): blend every tile list in its order */
  int k1, k2, k3;
  int key_tile;  /* side of the square tiles the sort keys use: 16 or 32 */
  int foveated;  /* 0 plain (every pixel a sample), 1 single-pass foveated */
  int tile_cull; /* 1: Eq. 4 pair culling; 0: bounding rectangle only */
  int brute;     /* 1: no tiles at all, every Gaussian a candidate of every sample */
  double gaze_x, gaze_y, radius, band;
  double bg[3];
  /* margins of the FP32-vs-FP64 comparison rule: a sample is marginal when a decision
   * falls within these relative distances of its threshold */
  double margin_alpha, margin_stop, margin_tie;
  /* visibility culling (Sec. 4.3): [H][W] bytes, nonzero where the pixel is visible in
   * the headset; NULL = every pixel visible.  A key tile with no visible pixel gets no
   * Gaussian/tile instances, and its pixels output the background. */
  const uint8_t* visible;
  /* 1: also enumerate the outcome sets (og_out.alt, og_out.unchecked): every result that
   * the marginal decisions of a pixel's samples allow, for the FP32-vs-FP64 comparison */
  int outcomes;
  /* 1: render only the Gaussians whose mean lies at a world-space distance d from
   * dist_ref with dist_min <= d < dist_max (the near or the far layer of the stereo
   * reuse of distant content, Sec. 7) */
  int dist_cull;
  double dist_ref[3], dist_min, dist_max;
} og_opts;

typedef struct {
  double *image;      /* [3][H][W] composited output */
  double *full;       /* [4][H][W]: C rgb and T of full-res samples (NaN elsewhere) */
  double *low;        /* [4][H/2][W/2]: C rgb and T of group samples (NaN elsewhere) */
  double *lowimg;     /* [3][H/2][W/2]: the half-resolution image that is upsampled */
  uint8_t *marginal;  /* [H][W]: 1 where an FP32 renderer may legitimately differ */
  uint8_t *tile_class;/* [nty][ntx]: 0 focus/plain, 1 hybrid, 2 periphery; + 4 when invisible */
  int32_t *order;     /* gids in blend order, samples concatenated */
  int64_t *order_off; /* [H*W + (H/2)*(W/2) + 1] */
  int64_t max_order;
  int64_t n_order;    /* out */
  int64_t stats[8];   /* out: valid, instances, evaluated, kept, blended, marginal px, samples,
                       * unchecked px */
  /* outcome sets (og_opts.outcomes): for each pixel, the other valid composited values
   * alt[alt_off[k] .. alt_off[k + 1]) (rgb triples), and unchecked[k] = 1 where the
   * valid values are too many to enumerate.  alt_off and alt are malloc'd by og_render
   * and released with og_free. */
  uint8_t* unchecked; /* [H][W], caller-owned, may be NULL */
  int64_t* alt_off;   /* out: [H*W + 1] */
  double* alt;        /* out: [n_alt][3] */
  double* alt4;       /* out, plain renders only: [n_alt][4], the (C rgb, T) of each alternative */
  int64_t n_alt;
} og_out;

/* ------------------------------------------------------------------ projection ---- */

typedef struct {
  int valid;
  double mu[3];        /* camera-space mean (camera centre at the origin) */
  double d, u[3];      /* distance and unit direction to the mean */
  double E[2][3];      /* orthonormal basis of the tangent plane */
  double Sc[3][3];     /* camera-space covariance */
  double Sci[3][3];    /* its inverse R S^-2 R^T */
  double Sp[2][2];     /* tangent-plane covariance incl. dilation */
  double A[2][2];      /* conic = Sp^-1 */
  double sigma, r2;    /* opacity and cutoff: alpha >= 1/255  <=>  q <= r2 */
  double rgb[3];
  double bbox[4];      /* xmin, ymin, xmax, ymax of the alpha >= 1/255 region (pixels) */
  int bounded;
} og_proj;

/* Real spherical-harmonics basis, degrees 0..3, in the sign convention of 3DGS. */
void og_sh_basis(int degree, const double dir[3], double Y[16]) {
  const double pi = 3.14159265358979323846;
  const double x = dir[0], y = dir[1], z = dir[2];
  const double s = 1.0 / sqrt(pi);
  for (int k = 0; k < 16; ++k) Y[k] = 0.0;
  Y[0] = 0.5 * s;
  if (degree < 1) return;
  const double c1 = 0.5 * sqrt(3.0) * s;
  Y[1] = -c1 * y;
  Y[2] = c1 * z;
  Y[3] = -c1 * x;
  if (degree < 2) return;
  Y[4] = 0.5 * sqrt(15.0) * s * x * y;
  Y[5] = -0.5 * sqrt(15.0) * s * y * z;
  Y[6] = 0.25 * sqrt(5.0) * s * (2 * z * z - x * x - y * y);
  Y[7] = -0.5 * sqrt(15.0) * s * x * z;
  Y[8] = 0.25 * sqrt(15.0) * s * (x * x - y * y);
  if (degree < 3) return;
  Y[9] = -0.25 * sqrt(35.0 / 2.0) * s * y * (3 * x * x - y * y);
  Y[10] = 0.5 * sqrt(105.0) * s * x * y * z;
  Y[11] = -0.25 * sqrt(21.0 / 2.0) * s * y * (4 * z * z - x * x - y * y);
  Y[12] = 0.25 * sqrt(7.0) * s * z * (2 * z * z - 3 * x * x - 3 * y * y);
  Y[13] = -0.25 * sqrt(21.0 / 2.0) * s * x * (4 * z * z - x * x - y * y);
  Y[14] = 0.25 * sqrt(105.0) * s * z * (x * x - y * y);
  Y[15] = -0.25 * sqrt(35.0 / 2.0) * s * x * (x * x - 3 * y * y);
}

static void mat3_mul(const double a[3][3], const double b[3][3], double c[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int k = 0; k < 3; ++k) s += a[i][k] * b[k][j];
      c[i][j] = s;
    }
}

static int all_finite(const double* v, int n) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(v[i])) return 0;
  return 1;
}

/* camera ray through continuous pixel position (px, py): K^-1 (px, py, 1) */
static void pixel_ray(const og_camera* c, double px, double py, double v[3]) {
  v[0] = (px - c->cx) / c->fx;
  v[1] = (py - c->cy) / c->fy;
  v[2] = 1.0;
}

/* t*(v): parameter of the maximum of the 3D Gaussian along the ray t v (camera frame) */
static double tstar_ray(const og_proj* p, const double v[3]) {
  double num = 0, den = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      num += v[i] * p->Sci[i][j] * p->mu[j];
      den += v[i] * p->Sci[i][j] * v[j];
    }
  return num / den;
}

static void conic_bbox(og_proj* p, const og_camera* c) {
  /* Rays x with sample alpha >= 1/255 form the cone (E x)^T A (E x) <= r2 (u.x)^2,
   * u.x > 0.  Its image in pixel space is the conic p~^T C p~ <= 0, C = K^-T Q K^-1. */
  double Q[3][3], Ki[3][3] = {{1.0 / c->fx, 0, -c->cx / c->fx}, {0, 1.0 / c->fy, -c->cy / c->fy}, {0, 0, 1}};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0;
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) s += p->E[a][i] * p->A[a][b] * p->E[b][j];
      Q[i][j] = s - p->r2 * p->u[i] * p->u[j];
    }
  double KiT[3][3], T1[3][3], C[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) KiT[i][j] = Ki[j][i];
  mat3_mul(KiT, Q, T1);
  mat3_mul(T1, Ki, C);
  double det2 = C[0][0] * C[1][1] - C[0][1] * C[1][0];
  p->bounded = 0;
  p->bbox[0] = 0;
  p->bbox[1] = 0;
  p->bbox[2] = c->width;
  p->bbox[3] = c->height;
  if (C[0][0] > 0 && det2 > 0) {
    /* ellipse: (p - p0)^T C2 (p - p0) <= -k */
    double i00 = C[1][1] / det2, i01 = -C[0][1] / det2, i11 = C[0][0] / det2;
    double p0x = -(i00 * C[0][2] + i01 * C[1][2]);
    double p0y = -(i01 * C[0][2] + i11 * C[1][2]);
    double k = C[2][2] + C[0][2] * p0x + C[1][2] * p0y;
    if (k <= 0) {
      double hx = sqrt(-k * i00), hy = sqrt(-k * i11);
      p->bbox[0] = p0x - hx;
      p->bbox[1] = p0y - hy;
      p->bbox[2] = p0x + hx;
      p->bbox[3] = p0y + hy;
      p->bounded = 1;
    }
  }
}

/* Optimal-Projection preprocessing of Gaussian i for camera c (Sec. 4.2, Eq. 1).
 * Gaussians with opacity below sigma_min are culled (1/255 by definition: no alpha can
 * reach the cut; a little lower when the outcome sets need those within the margin). */
static int og_project_min(const og_scene* sc, int64_t i, const og_camera* c, og_proj* p, double sigma_min);

int og_project(const og_scene* sc, int64_t i, const og_camera* c, og_proj* p) {
  return og_project_min(sc, i, c, p, OG_ALPHA_MIN);
}

static int og_project_min(const og_scene* sc, int64_t i, const og_camera* c, og_proj* p, double sigma_min) {
  memset(p, 0, sizeof *p);
  const int64_t n = sc->n;
  double m[3] = {sc->mean[i], sc->mean[n + i], sc->mean[2 * n + i]};
  double ls[3] = {sc->log_scale[i], sc->log_scale[n + i], sc->log_scale[2 * n + i]};
  double q[4] = {sc->quat[i], sc->quat[n + i], sc->quat[2 * n + i], sc->quat[3 * n + i]};
  double logit = sc->opacity_logit[i];
  if (!all_finite(m, 3) || !all_finite(ls, 3) || !all_finite(q, 4) || !isfinite(logit)) return 0;
  double Rw[3][3], t[3];
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) Rw[r][k] = c->w2c[4 * r + k];
    t[r] = c->w2c[4 * r + 3];
  }
  for (int r = 0; r < 3; ++r) p->mu[r] = Rw[r][0] * m[0] + Rw[r][1] * m[1] + Rw[r][2] * m[2] + t[r];
  if (!(p->mu[2] >= c->near_z)) return 0;
  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0)) return 0;
  double w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
  double R[3][3] = {{1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)},
                    {2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)},
                    {2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)}};
  double Rc[3][3];
  mat3_mul(Rw, R, Rc); /* rotation of the Gaussian's axes into the camera frame */
  double s2[3], si2[3];
  for (int k = 0; k < 3; ++k) {
    s2[k] = exp(2 * ls[k]);
    si2[k] = exp(-2 * ls[k]);
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0, si = 0;
      for (int k = 0; k < 3; ++k) {
        s += Rc[a][k] * s2[k] * Rc[b][k];
        si += Rc[a][k] * si2[k] * Rc[b][k];
      }
      p->Sc[a][b] = s;
      p->Sci[a][b] = si;
    }
  if (!all_finite(&p->Sc[0][0], 9) || !all_finite(&p->Sci[0][0], 9)) return 0;
  p->sigma = 1.0 / (1.0 + exp(-logit));
  if (!(p->sigma >= sigma_min)) return 0;
  p->r2 = 2.0 * log(255.0 * p->sigma);
  p->d = sqrt(p->mu[0] * p->mu[0] + p->mu[1] * p->mu[1] + p->mu[2] * p->mu[2]);
  for (int k = 0; k < 3; ++k) p->u[k] = p->mu[k] / p->d;
  double rho = sqrt(p->u[0] * p->u[0] + p->u[2] * p->u[2]);
  p->E[0][0] = p->u[2] / rho;
  p->E[0][1] = 0;
  p->E[0][2] = -p->u[0] / rho;
  p->E[1][0] = p->u[1] * p->E[0][2] - p->u[2] * p->E[0][1];
  p->E[1][1] = p->u[2] * p->E[0][0] - p->u[0] * p->E[0][2];
  p->E[1][2] = p->u[0] * p->E[0][1] - p->u[1] * p->E[0][0];
  double dil = OG_DILATION_PX2 / (c->fx * c->fy);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += p->E[a][k] * p->Sc[k][l] * p->E[b][l];
      p->Sp[a][b] = s / (p->d * p->d) + (a == b ? dil : 0.0);
    }
  double det = p->Sp[0][0] * p->Sp[1][1] - p->Sp[0][1] * p->Sp[1][0];
  p->A[0][0] = p->Sp[1][1] / det;
  p->A[1][1] = p->Sp[0][0] / det;
  p->A[0][1] = p->A[1][0] = -p->Sp[0][1] / det;
  /* colour from SH along the world-space viewing direction (mu - o)/|mu - o| */
  double dirw[3];
  for (int k = 0; k < 3; ++k) dirw[k] = Rw[0][k] * p->u[0] + Rw[1][k] * p->u[1] + Rw[2][k] * p->u[2];
  double Y[16];
  og_sh_basis(sc->sh_degree, dirw, Y);
  int K = (sc->sh_degree + 1) * (sc->sh_degree + 1);
  for (int ch = 0; ch < 3; ++ch) {
    double v = 0.5;
    for (int k = 0; k < K; ++k) v += Y[k] * sc->sh[((int64_t)k * 3 + ch) * n + i];
    p->rgb[ch] = v > 0 ? v : 0.0;
  }
  conic_bbox(p, c);
  p->valid = 1;
  return 1;
}

/* alpha and depth of Gaussian p at the sample position (px, py).  Returns 1 when the pair
 * is kept (alpha >= 1/255 and the ray meets the tangent plane in front of o). */
static int og_eval(const og_proj* p, const og_camera* c, double px, double py, double* alpha,
                   double* tstar, double* sg) {
  double v[3];
  pixel_ray(c, px, py, v);
  double w = p->u[0] * v[0] + p->u[1] * v[1] + p->u[2] * v[2];
  *sg = 0;
  if (!(w > 0)) return 0;
  double s0 = (p->E[0][0] * v[0] + p->E[0][1] * v[1] + p->E[0][2] * v[2]) / w;
  double s1 = (p->E[1][0] * v[0] + p->E[1][1] * v[1] + p->E[1][2] * v[2]) / w;
  double q = p->A[0][0] * s0 * s0 + 2 * p->A[0][1] * s0 * s1 + p->A[1][1] * s1 * s1;
  *sg = p->sigma * exp(-0.5 * q);
  if (!(*sg >= OG_ALPHA_MIN)) return 0;
  *alpha = *sg < OG_ALPHA_MAX ? *sg : OG_ALPHA_MAX;
  *tstar = tstar_ray(p, v);
  return 1;
}

/* Eq. 4: maximum of the plane Gaussian (conic A, centre 0) on the segment P + t D,
 * t clamped to [0, 1].  Returns the exponent q = x^T A x at the maximum point. */
static double edge_min_q(const double A[2][2], const double P[2], const double D[2], double* tout) {
  double AP0 = A[0][0] * P[0] + A[0][1] * P[1], AP1 = A[1][0] * P[0] + A[1][1] * P[1];
  double AD0 = A[0][0] * D[0] + A[0][1] * D[1], AD1 = A[1][0] * D[0] + A[1][1] * D[1];
  double dAd = D[0] * AD0 + D[1] * AD1;
  double t = dAd > 0 ? -(D[0] * AP0 + D[1] * AP1) / dAd : 0.0;
  if (t < 0) t = 0;
  if (t > 1) t = 1;
  double X0 = P[0] + t * D[0], X1 = P[1] + t * D[1];
  *tout = t;
  return A[0][0] * X0 * X0 + 2 * A[0][1] * X0 * X1 + A[1][1] * X1 * X1;
}

/* exported for the Eq. 4 pin: out = {t, q} */
void og_edge_max(const double A4[4], const double P[2], const double D[2], double out[2]) {
  double A[2][2] = {{A4[0], A4[1]}, {A4[2], A4[3]}};
  out[1] = edge_min_q(A, P, D, &out[0]);
}

/* Tile culling on the optimal plane (Sec. 4.2, Eq. 4).  The quad spans the sample
 * positions [x0, x1] x [y0, y1].  Returns 1 when the pair is kept; *key = t* on the ray
 * through the maximum point projected back to the image. */
static int og_tile_keep_r(const og_proj* p, const og_camera* c, double x0, double y0, double x1, double y1,
                          double relax, double* key, double* qmin_out);

static int og_tile_keep(const og_proj* p, const og_camera* c, double x0, double y0, double x1,
                        double y1, double* key, double* qmin_out) {
  return og_tile_keep_r(p, c, x0, y0, x1, y1, 0.0, key, qmin_out);
}

/* og_tile_keep with the cut moved up by relax: keeps the pair while qmin <= r2 + relax */
static int og_tile_keep_r(const og_proj* p, const og_camera* c, double x0, double y0, double x1, double y1,
                          double relax, double* key, double* qmin_out) {
  const double cx[4] = {x0, x1, x1, x0}, cy[4] = {y0, y0, y1, y1};
  double S[4][2];
  *key = p->mu[2];
  *qmin_out = 0;
  for (int k = 0; k < 4; ++k) {
    double v[3];
    pixel_ray(c, cx[k], cy[k], v);
    double w = p->u[0] * v[0] + p->u[1] * v[1] + p->u[2] * v[2];
    if (!(w > 0)) return 1; /* quad not bounded on the plane: keep, key at the mean */
    S[k][0] = (p->E[0][0] * v[0] + p->E[0][1] * v[1] + p->E[0][2] * v[2]) / w;
    S[k][1] = (p->E[1][0] * v[0] + p->E[1][1] * v[1] + p->E[1][2] * v[2]) / w;
  }
  int pos = 0, neg = 0;
  for (int k = 0; k < 4; ++k) {
    int l = (k + 1) & 3;
    double cr = (S[l][0] - S[k][0]) * (0 - S[k][1]) - (S[l][1] - S[k][1]) * (0 - S[k][0]);
    if (cr > 0) pos = 1;
    if (cr < 0) neg = 1;
  }
  if (!(pos && neg)) return 1; /* projected mean inside the quad: maximum at the mean */
  double qmin = INFINITY, X[2] = {0, 0};
  for (int k = 0; k < 4; ++k) {
    int l = (k + 1) & 3;
    double D[2] = {S[l][0] - S[k][0], S[l][1] - S[k][1]}, t;
    double q = edge_min_q(p->A, S[k], D, &t);
    if (q < qmin) {
      qmin = q;
      X[0] = S[k][0] + t * D[0];
      X[1] = S[k][1] + t * D[1];
    }
  }
  *qmin_out = qmin;
  if (!(qmin <= p->r2 + relax)) return 0;
  double y[3];
  for (int k = 0; k < 3; ++k) y[k] = p->u[k] + p->E[0][k] * X[0] + p->E[1][k] * X[1];
  if (y[2] > 0) {
    double v[3] = {y[0] / y[2], y[1] / y[2], 1.0};
    *key = tstar_ray(p, v);
  }
  return 1;
}

/* ------------------------------------------------------------- exported single ops ---- */

/* out: valid, mu[3], d, u[3], E[6], Sc[9], Sci[9], Sp[4], A[4], sigma, r2, rgb[3], bbox[4],
 * bounded  (52 doubles) */
int og_project_one(const og_scene* sc, int64_t i, const og_camera* c, double* out) {
  og_proj p;
  int v = og_project(sc, i, c, &p);
  double* o = out;
  *o++ = v;
  for (int k = 0; k < 3; ++k) *o++ = p.mu[k];
  *o++ = p.d;
  for (int k = 0; k < 3; ++k) *o++ = p.u[k];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 3; ++k) *o++ = p.E[a][k];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) *o++ = p.Sc[a][k];
  for (int a = 0; a < 3; ++a)
    for (int k = 0; k < 3; ++k) *o++ = p.Sci[a][k];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 2; ++k) *o++ = p.Sp[a][k];
  for (int a = 0; a < 2; ++a)
    for (int k = 0; k < 2; ++k) *o++ = p.A[a][k];
  *o++ = p.sigma;
  *o++ = p.r2;
  for (int k = 0; k < 3; ++k) *o++ = p.rgb[k];
  for (int k = 0; k < 4; ++k) *o++ = p.bbox[k];
  *o++ = p.bounded;
  return v;
}

/* out: kept, alpha, tstar, sigma*G */
int og_eval_one(const og_scene* sc, int64_t i, const og_camera* c, double px, double py, double* out) {
  og_proj p;
  out[0] = out[1] = out[2] = out[3] = 0;
  if (!og_project(sc, i, c, &p)) return 0;
  double a = 0, t = 0, sg = 0;
  int k = og_eval(&p, c, px, py, &a, &t, &sg);
  out[0] = k;
  out[1] = a;
  out[2] = t;
  out[3] = sg;
  return k;
}

/* out: keep, key, qmin */
int og_tile_one(const og_scene* sc, int64_t i, const og_camera* c, double x0, double y0, double x1,
                double y1, double* out) {
  og_proj p;
  out[0] = out[1] = out[2] = 0;
  if (!og_project(sc, i, c, &p)) return 0;
  double key, qmin;
  int k = og_tile_keep(&p, c, x0, y0, x1, y1, &key, &qmin);
  out[0] = k;
  out[1] = key;
  out[2] = qmin;
  return k;
}

/* Local-affine (EWA) projection as in 3DGS, used only by the pins (Eq. 3):
 * out = mean2d[2], cov2d[3] (xx, xy, yy) including the 0.3 px^2 dilation. */
int og_ewa_one(const og_scene* sc, int64_t i, const og_camera* c, double* out) {
  og_proj p;
  if (!og_project(sc, i, c, &p)) return 0;
  double x = p.mu[0], y = p.mu[1], z = p.mu[2];
  double J[2][3] = {{c->fx / z, 0, -c->fx * x / (z * z)}, {0, c->fy / z, -c->fy * y / (z * z)}};
  double S[2][2];
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      double s = 0;
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) s += J[a][k] * p.Sc[k][l] * J[b][l];
      S[a][b] = s;
    }
  out[0] = c->fx * x / z + c->cx;
  out[1] = c->fy * y / z + c->cy;
  out[2] = S[0][0] + OG_DILATION_PX2;
  out[3] = S[0][1];
  out[4] = S[1][1] + OG_DILATION_PX2;
  return 1;
}

/* ------------------------------------------------------------------ rendering ---- */

typedef struct {
  double key;
  int32_t gid;
} went;

static int went_less(went a, went b) { return a.key < b.key || (a.key == b.key && a.gid < b.gid); }

typedef struct {
  went* e;
  int n, cap;
} window;

/* ---- decisions within the comparison margins ------------------------------------
 * An FP32 renderer may legitimately take a decision the other way when its FP64 value
 * lies within the comparison rule's margin of the threshold.  Each such decision gets
 * an identity, so that a run can record it and a re-run can be told to flip it:
 *   OG_DEC_KEEP  alpha of (sample idx, Gaussian g1) against 1/255
 *   OG_DEC_STOP  transmittance test of (sample idx, Gaussian g1) against 1e-4
 *   OG_DEC_WTIE  order of Gaussians g1 < g2 in window idx of a hierarchical block
 *   OG_DEC_STIE  order of Gaussians g1 < g2 in the tile's sorted stream
 * The alpha clamp at 0.99 is continuous in sigma G, so it decides nothing here. */
enum { OG_DEC_KEEP = 0, OG_DEC_STOP = 1, OG_DEC_WTIE = 2, OG_DEC_STIE = 3 };

typedef struct {
  int type, idx;
  int32_t g1, g2;
} dec;

typedef struct {
  dec* d;
  int n, cap;
} decset;

static int dec_eq(dec a, dec b) { return a.type == b.type && a.idx == b.idx && a.g1 == b.g1 && a.g2 == b.g2; }

static int decset_find(const decset* s, dec x) {
  if (!s) return -1;
  for (int k = 0; k < s->n; ++k)
    if (dec_eq(s->d[k], x)) return k;
  return -1;
}

static void decset_add(decset* s, dec x) {
  if (!s || decset_find(s, x) >= 0) return;
  if (s->n == s->cap) {
    s->cap = s->cap ? 2 * s->cap : 16;
    s->d = (dec*)realloc(s->d, sizeof(dec) * s->cap);
  }
  s->d[s->n++] = x;
}

/* records decision x in `seen` and returns 1 when this run is told to flip it */
static int decide(const decset* forced, decset* seen, dec x) {
  decset_add(seen, x);
  return decset_find(forced, x) >= 0;
}

static dec tie_dec(int type, int idx, int32_t a, int32_t b) {
  return (dec){type, idx, a < b ? a : b, a < b ? b : a};
}

/* ---- outcome sets ---------------------------------------------------------------
 * The valid results of one sample: (C rgb, T) of every combination of its marginal
 * decisions, distinct values only.  A sample with more than OG_MAX_OUTCOMES distinct
 * results, or whose combinations cannot be enumerated within the limits below, is
 * "unchecked". */
#define OG_MAX_OUTCOMES 64
#define OG_MAX_LEAVES 4096    /* paths of one sample's walk (exact and global orders) */
#define OG_MAX_GROUP 4        /* near-tied pairs whose orders are enumerated */
#define OG_MAX_BLOCK_DECISIONS 64
#define OG_MAX_SAMPLE_DECISIONS 6
#define OG_MAX_PIXEL_COMBOS 4096
#define OG_SAME 1e-13         /* results closer than this are one result */

typedef struct {
  double v[4];
} outcome;

static int outcome_add(outcome** arr, int* n, const double C[3], double T) {
  for (int k = 0; k < *n; ++k)
    if (fabs((*arr)[k].v[0] - C[0]) <= OG_SAME && fabs((*arr)[k].v[1] - C[1]) <= OG_SAME &&
        fabs((*arr)[k].v[2] - C[2]) <= OG_SAME && fabs((*arr)[k].v[3] - T) <= OG_SAME)
      return 1;
  if (*n >= OG_MAX_OUTCOMES) return 0;
  if (*n % 8 == 0) *arr = (outcome*)realloc(*arr, sizeof(outcome) * (*n + 8));
  (*arr)[*n] = (outcome){{C[0], C[1], C[2], T}};
  ++*n;
  return 1;
}

typedef struct {
  double C[3], T;
  int done, marginal, active_sample;
  int32_t* gids;
  int ng, capg;
  outcome* alt; /* every distinct valid result (nalt >= 2), or NULL: the nominal one only */
  int nalt;
  int unchecked;
} sample;

static void sample_push(sample* s, int32_t g) {
  if (s->ng == s->capg) {
    s->capg = s->capg ? 2 * s->capg : 16;
    s->gids = (int32_t*)realloc(s->gids, sizeof(int32_t) * s->capg);
  }
  s->gids[s->ng++] = g;
}

/* front-to-back blending step (Eq. 2) with the 3DGS stopping rule */
static void blend(sample* s, double alpha, const double rgb[3], int32_t g) {
  if (s->done) return;
  double test = s->T * (1.0 - alpha);
  if (fabs(test - OG_T_STOP) < g_margin_stop * OG_T_STOP) s->marginal = 1;
  if (test < OG_T_STOP) {
    s->done = 1;
    return;
  }
  for (int c = 0; c < 3; ++c) s->C[c] += alpha * s->T * rgb[c];
  s->T = test;
  sample_push(s, g);
}

static int near_alpha_min(double sg) { return fabs(sg - OG_ALPHA_MIN) < g_margin_alpha * OG_ALPHA_MIN; }

static void mark_threshold(sample* s, double sg) {
  if (near_alpha_min(sg) || fabs(sg - OG_ALPHA_MAX) < g_margin_alpha * OG_ALPHA_MAX) s->marginal = 1;
}

/* og_eval that also returns alpha and t* of a pair below the cut (ray in front of o),
 * for the runs that keep a pair whose keep decision is within the margin */
static int eval_full(const og_proj* p, const og_camera* c, double px, double py, double* alpha, double* tstar,
                     double* sg) {
  int k = og_eval(p, c, px, py, alpha, tstar, sg);
  if (!k && *sg > 0) {
    double v[3];
    pixel_ray(c, px, py, v);
    *alpha = *sg < OG_ALPHA_MAX ? *sg : OG_ALPHA_MAX;
    *tstar = tstar_ray(p, v);
  }
  return k;
}

/* ---- one sample's outcome walk (exact and global orders) ------------------------
 * cand: the sample's kept pairs and the pairs whose keep decision is within the margin,
 * in blend order; key is what orders them (t* for the exact order, the list key for the
 * global orders).  Pairs whose keys are within the tie margin form groups whose every
 * order is valid.  The walk follows every combination of group order, keep decision
 * and stop decision and collects the distinct (C, T) it ends with. */
typedef struct {
  double key, alpha;
  const double* rgb;
  int32_t gid;
  int kept, amb;
} cand;

static int cand_cmp(const void* a, const void* b) {
  const cand *x = (const cand*)a, *y = (const cand*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->gid > y->gid) - (x->gid < y->gid);
}

typedef struct {
  const cand* c;
  int n;
  const int* gend; /* gend[j]: end of the tie group that starts at j */
  outcome* out;
  int nout, overflow, leaves;
} walker;

static void walk_leaf(walker* w, double T, const double C[3]) {
  if (w->overflow) return;
  if (++w->leaves > OG_MAX_LEAVES || !outcome_add(&w->out, &w->nout, C, T)) w->overflow = 1;
}

static void walk_groups(walker* w, int j, double T, const double C[3]);

static void walk_perm(walker* w, const int* perm, int g, int pos, int jnext, double T, const double C[3]) {
  if (w->overflow) return;
  if (pos == g) {
    walk_groups(w, jnext, T, C);
    return;
  }
  const cand* c = &w->c[perm[pos]];
  for (int keep = 0; keep <= 1; ++keep) {
    if (!c->amb && keep != c->kept) continue;
    if (!keep) {
      walk_perm(w, perm, g, pos + 1, jnext, T, C);
      continue;
    }
    double test = T * (1.0 - c->alpha);
    int amb_stop = fabs(test - OG_T_STOP) < g_margin_stop * OG_T_STOP;
    int stop = test < OG_T_STOP;
    if (stop || amb_stop) walk_leaf(w, T, C); /* stop before this pair */
    if (!stop || amb_stop) {
      double C2[3];
      for (int ch = 0; ch < 3; ++ch) C2[ch] = C[ch] + c->alpha * T * c->rgb[ch];
      walk_perm(w, perm, g, pos + 1, jnext, test, C2);
    }
  }
}

/* all orders of g <= OG_MAX_GROUP items, lexicographic (the identity first) */
static int permutations(int g, int out[][OG_MAX_GROUP]) {
  int n = 0, a[OG_MAX_GROUP];
  for (int k = 0; k < g; ++k) a[k] = k;
  for (;;) {
    for (int k = 0; k < g; ++k) out[n][k] = a[k];
    ++n;
    int i = g - 2;
    while (i >= 0 && a[i] > a[i + 1]) --i;
    if (i < 0) return n;
    int j = g - 1;
    while (a[j] < a[i]) --j;
    int t = a[i];
    a[i] = a[j];
    a[j] = t;
    for (int l = i + 1, r = g - 1; l < r; ++l, --r) {
      t = a[l];
      a[l] = a[r];
      a[r] = t;
    }
  }
}

static void walk_groups(walker* w, int j, double T, const double C[3]) {
  if (w->overflow) return;
  if (j >= w->n) {
    walk_leaf(w, T, C);
    return;
  }
  const int g = w->gend[j] - j;
  if (g > OG_MAX_GROUP) {
    w->overflow = 1;
    return;
  }
  int perms[24][OG_MAX_GROUP];
  const int np = permutations(g, perms);
  for (int p = 0; p < np && !w->overflow; ++p) {
    int perm[OG_MAX_GROUP];
    for (int k = 0; k < g; ++k) perm[k] = j + perms[p][k];
    walk_perm(w, perm, g, 0, j + g, T, C);
  }
}

/* outcome set of one sample from its candidates in blend order (sorted by key, gid) */
static void sample_outcomes(sample* s, const cand* c, int n) {
  int* gend = (int*)malloc(sizeof(int) * (n ? n : 1));
  for (int j = n - 1; j >= 0; --j)
    gend[j] = (j + 1 < n && fabs(c[j + 1].key - c[j].key) < g_margin_tie * fabs(c[j + 1].key)) ? gend[j + 1] : j + 1;
  walker w = {c, n, gend, NULL, 0, 0, 0};
  const double C0[3] = {0, 0, 0};
  walk_groups(&w, 0, 1.0, C0);
  free(gend);
  if (w.overflow) {
    s->unchecked = 1;
    free(w.out);
  } else if (w.nout > 1) {
    s->alt = w.out;
    s->nalt = w.nout;
  } else {
    free(w.out);
  }
}

/* ---- hierarchical blocks --------------------------------------------------------- */

typedef struct {
  const og_proj* P;
  const og_camera* cam;
  sample* s[16];
  double px[16], py[16];
  double c4[2], c2[4][2];
  window L1, L2[4], L3[16];
  int k1, k2, k3;
  int tie;
  double last_key; /* tile key of the previous stream entry that was a block member */
  int32_t last_gid;
  int has_last;
  int64_t evals, kept;
  const decset* forced; /* decisions this run takes the other way */
  decset* seen;         /* decisions within the margins this run met (may be NULL) */
  int record;           /* nominal run: keep blend orders */
} hblock;

/* window indices in decision identities: L1 0, L2 1 + b, L3 5 + i */
static int win_less(hblock* B, int widx, went a, went b) {
  int less = went_less(a, b);
  if (B->forced && B->forced->n && decset_find(B->forced, tie_dec(OG_DEC_WTIE, widx, a.gid, b.gid)) >= 0)
    less = !less;
  return less;
}

static void win_push(hblock* B, int widx, window* w, went x, int* tie) {
  if (w->n == w->cap) {
    w->cap = w->cap ? 2 * w->cap : 16;
    w->e = (went*)realloc(w->e, sizeof(went) * w->cap);
  }
  int j = w->n++;
  while (j > 0 && win_less(B, widx, x, w->e[j - 1])) {
    w->e[j] = w->e[j - 1];
    --j;
  }
  w->e[j] = x;
  double tol = g_margin_tie * fabs(x.key);
  for (int nb = j - 1; nb <= j + 1; nb += 2)
    if (nb >= 0 && nb < w->n && fabs(w->e[nb].key - x.key) < tol) {
      *tie = 1;
      decide(B->forced, B->seen, tie_dec(OG_DEC_WTIE, widx, x.gid, w->e[nb].gid));
    }
}

static went win_pop(window* w) {
  went m = w->e[0];
  memmove(w->e, w->e + 1, sizeof(went) * (w->n - 1));
  w->n--;
  return m;
}

/* keep decision of Gaussian g at sample i (0 for a missing or finished sample);
 * *amb (optional) reports a decision within the margin */
static int keep_at(hblock* B, int i, int32_t g, double* a, double* t, int* amb, int count) {
  if (!B->s[i] || B->s[i]->done) return 0;
  double sg;
  if (count) B->evals++;
  int k = eval_full(&B->P[g], B->cam, B->px[i], B->py[i], a, t, &sg);
  mark_threshold(B->s[i], sg);
  int near = near_alpha_min(sg);
  if (amb) *amb = near;
  if (near && decide(B->forced, B->seen, (dec){OG_DEC_KEEP, i, g, 0})) k = !k;
  return k;
}

/* membership of a block = kept at any active sample; it can flip in FP32 only when every
 * keep decision behind it is marginal */
typedef struct {
  int sure, unsure;
} vote;

static void vote_add(vote* v, int kept, int flip) {
  if (kept && !flip) v->sure = 1;
  if (flip) v->unsure = 1;
}

static int vote_result(hblock* B, vote v, int any) {
  if (!v.sure && v.unsure) B->tie = 1;
  return any;
}

static void blend_at(hblock* B, int i, int32_t g) {
  double a, t;
  sample* s = B->s[i];
  if (!s || s->done) return;
  if (!keep_at(B, i, g, &a, &t, NULL, 0)) return;
  double test = s->T * (1.0 - a);
  int stop = test < OG_T_STOP;
  if (fabs(test - OG_T_STOP) < g_margin_stop * OG_T_STOP) {
    s->marginal = 1;
    if (decide(B->forced, B->seen, (dec){OG_DEC_STOP, i, g, 0})) stop = !stop;
  }
  if (stop) {
    s->done = 1;
    return;
  }
  for (int c = 0; c < 3; ++c) s->C[c] += a * s->T * B->P[g].rgb[c];
  s->T = test;
  if (B->record) sample_push(s, g);
}

static void to_L3(hblock* B, int b, int32_t g) {
  int bx = (b & 1) * 2, by = (b >> 1) * 2;
  for (int j = 0; j < 4; ++j) {
    int i = (by + (j >> 1)) * 4 + bx + (j & 1);
    double a, t;
    if (!keep_at(B, i, g, &a, &t, NULL, 1)) continue;
    if (B->record) B->kept++;
    int tie = 0;
    win_push(B, 5 + i, &B->L3[i], (went){t, g}, &tie);
    if (tie) B->s[i]->marginal = 1;
    if (B->L3[i].n > B->k3) blend_at(B, i, win_pop(&B->L3[i]).gid);
  }
}

static void to_L2(hblock* B, int32_t g) {
  for (int b = 0; b < 4; ++b) {
    int bx = (b & 1) * 2, by = (b >> 1) * 2, any = 0;
    vote vt = {0, 0};
    for (int j = 0; j < 4; ++j) {
      double a, t;
      int f = 0, k = keep_at(B, (by + (j >> 1)) * 4 + bx + (j & 1), g, &a, &t, &f, 1);
      if (k) any = 1;
      vote_add(&vt, k, f);
    }
    if (!vote_result(B, vt, any)) continue;
    double v[3];
    pixel_ray(B->cam, B->c2[b][0], B->c2[b][1], v);
    win_push(B, 1 + b, &B->L2[b], (went){tstar_ray(&B->P[g], v), g}, &B->tie);
    if (B->L2[b].n > B->k2) to_L3(B, b, win_pop(&B->L2[b]).gid);
  }
}

static void stream_entry(hblock* B, int32_t g, double tile_key) {
  int any = 0;
  vote vt = {0, 0};
  for (int i = 0; i < 16; ++i) {
    double a, t;
    int f = 0, k = keep_at(B, i, g, &a, &t, &f, 1);
    if (k) any = 1;
    vote_add(&vt, k, f);
  }
  if (!vote_result(B, vt, any)) return;
  /* FP32 keys may swap near-tied members of the stream */
  if (B->has_last && fabs(tile_key - B->last_key) < g_margin_tie * fabs(tile_key)) {
    B->tie = 1;
    decide(B->forced, B->seen, tie_dec(OG_DEC_STIE, 0, g, B->last_gid));
  }
  B->last_key = tile_key;
  B->last_gid = g;
  B->has_last = 1;
  double v[3];
  pixel_ray(B->cam, B->c4[0], B->c4[1], v);
  win_push(B, 0, &B->L1, (went){tstar_ray(&B->P[g], v), g}, &B->tie);
  if (B->L1.n > B->k1) to_L2(B, win_pop(&B->L1).gid);
}

static void flush_block(hblock* B) {
  while (B->L1.n) to_L2(B, win_pop(&B->L1).gid);
  for (int b = 0; b < 4; ++b)
    while (B->L2[b].n) to_L3(B, b, win_pop(&B->L2[b]).gid);
  for (int i = 0; i < 16; ++i)
    while (B->L3[i].n) blend_at(B, i, win_pop(&B->L3[i]).gid);
}

typedef struct {
  int32_t gid;
  double key;
} tentry;

static int tentry_cmp(const void* a, const void* b) {
  const tentry *x = (const tentry*)a, *y = (const tentry*)b;
  if (x->key < y->key) return -1;
  if (x->key > y->key) return 1;
  return (x->gid > y->gid) - (x->gid < y->gid);
}

/* tile visibility: a key tile is visible when any of its pixels is (all tiles when the
 * mask is NULL); returns a calloc'd [ntiles] array of 0/1 */
static uint8_t* tile_visibility(const uint8_t* visible, int W, int H, int T) {
  const int ntx = (W + T - 1) / T, nty = (H + T - 1) / T;
  uint8_t* tv = (uint8_t*)calloc((size_t)ntx * nty, 1);
  for (int ty = 0; ty < nty; ++ty)
    for (int tx = 0; tx < ntx; ++tx) {
      int any = visible == NULL;
      for (int y = ty * T; y < (ty + 1) * T && y < H && !any; ++y)
        for (int x = tx * T; x < (tx + 1) * T && x < W; ++x)
          if (visible[(int64_t)y * W + x]) {
            any = 1;
            break;
          }
      tv[ty * ntx + tx] = (uint8_t)any;
    }
  return tv;
}

/* Gaussian/tile instances after the bounding rectangle and (optionally) Eq. 4 culling,
 * on visible tiles only (tvis NULL: all), sorted per tile by (key, gid): the stream every
 * sample of the tile reads.  cnt gets ntiles + 1 prefix offsets.  relax > 0 also keeps
 * the pairs whose Eq. 4 exponent is above the cut r2 by at most relax: their largest
 * alpha over the tile is below 1/255 but within the margin, so an FP32 renderer may keep
 * them at a sample there (they change no FP64 result).  slack (optional, malloc'd into
 * *slack) gets qmin - r2 per entry in list order (0 for a pair kept without Eq. 4). */
static tentry* build_lists(const og_proj* P, int64_t n, const og_camera* cam, int T, int tile_cull,
                           const uint8_t* tvis, int key_mode, double relax, int64_t* cnt, double** slack) {
  const int W = cam->width, H = cam->height;
  const int ntx = (W + T - 1) / T, nty = (H + T - 1) / T, ntiles = ntx * nty;
  tentry* lists = NULL;
  double* sl = NULL;
  for (int pass = 0; pass < 2; ++pass) {
    int64_t* fill = pass ? (int64_t*)calloc(ntiles, sizeof(int64_t)) : NULL;
    for (int64_t i = 0; i < n; ++i) {
      if (!P[i].valid) continue;
      const double* bb = P[i].bbox;
      int tx0 = (int)ceil((bb[0] + 0.5) / T - 1), tx1 = (int)floor((bb[2] - 0.5) / T);
      int ty0 = (int)ceil((bb[1] + 0.5) / T - 1), ty1 = (int)floor((bb[3] - 0.5) / T);
      if (relax > 0 && P[i].bounded) { /* the relaxed cone is a little wider than the bbox */
        tx0 = (int)floor(bb[0] / T) - 1;
        ty0 = (int)floor(bb[1] / T) - 1;
        tx1 = (int)floor(bb[2] / T) + 1;
        ty1 = (int)floor(bb[3] / T) + 1;
      }
      if (tx0 < 0) tx0 = 0;
      if (ty0 < 0) ty0 = 0;
      if (tx1 > ntx - 1) tx1 = ntx - 1;
      if (ty1 > nty - 1) ty1 = nty - 1;
      for (int ty = ty0; ty <= ty1; ++ty)
        for (int tx = tx0; tx <= tx1; ++tx) {
          double key = P[i].mu[2], qmin = 0;
          if (tvis && !tvis[ty * ntx + tx]) continue;
          if (tile_cull) {
            double x0 = tx * T + 0.5, y0 = ty * T + 0.5;
            double x1 = fmin((tx + 1) * T, W) - 0.5, y1 = fmin((ty + 1) * T, H) - 0.5;
            if (!og_tile_keep_r(&P[i], cam, x0, y0, x1, y1, relax, &key, &qmin)) continue;
          }
          /* global orders: one key per Gaussian */
          if (key_mode == 3) key = P[i].mu[2];
          if (key_mode == 4) key = sqrt(P[i].mu[0] * P[i].mu[0] + P[i].mu[1] * P[i].mu[1] + P[i].mu[2] * P[i].mu[2]);
          int t = ty * ntx + tx;
          if (!pass) {
            cnt[t + 1]++;
          } else {
            int64_t at = cnt[t] + fill[t]++;
            lists[at] = (tentry){(int32_t)i, key};
            if (sl) sl[at] = qmin > 0 ? qmin - P[i].r2 : 0.0;
          }
        }
    }
    if (!pass) {
      for (int t = 0; t < ntiles; ++t) cnt[t + 1] += cnt[t];
      lists = (tentry*)malloc(sizeof(tentry) * (cnt[ntiles] ? cnt[ntiles] : 1));
      if (slack) sl = (double*)malloc(sizeof(double) * (cnt[ntiles] ? cnt[ntiles] : 1));
    } else {
      free(fill);
    }
  }
  if (sl) {
    /* sort the entries of each tile together with their slack */
    typedef struct {
      tentry e;
      double slack;
    } tslack;
    int64_t tot = cnt[ntiles];
    tslack* tmp = (tslack*)malloc(sizeof(tslack) * (tot ? tot : 1));
    for (int64_t j = 0; j < tot; ++j) tmp[j] = (tslack){lists[j], sl[j]};
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < ntiles; ++t) qsort(tmp + cnt[t], cnt[t + 1] - cnt[t], sizeof(tslack), tentry_cmp);
    for (int64_t j = 0; j < tot; ++j) {
      lists[j] = tmp[j].e;
      sl[j] = tmp[j].slack;
    }
    free(tmp);
    *slack = sl;
  } else {
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < ntiles; ++t) qsort(lists + cnt[t], cnt[t + 1] - cnt[t], sizeof(tentry), tentry_cmp);
  }
  return lists;
}

typedef struct {
  double t, alpha;
  int32_t gid;
} kpair;

static int kpair_cmp(const void* a, const void* b) {
  const kpair *x = (const kpair*)a, *y = (const kpair*)b;
  if (x->t < y->t) return -1;
  if (x->t > y->t) return 1;
  return (x->gid > y->gid) - (x->gid < y->gid);
}

/* exact order at one sample: every kept candidate sorted by (t*, gid), then Eq. 2.
 * With outcomes, also the sample's outcome set over its marginal decisions. */
static void render_exact(const og_proj* P, const og_camera* cam, const int32_t* cand_ids, int64_t nc,
                         double px, double py, sample* s, int outcomes, int64_t* evals, int64_t* kept) {
  kpair* kp = (kpair*)malloc(sizeof(kpair) * (nc ? nc : 1));
  cand* ca = outcomes ? (cand*)malloc(sizeof(cand) * (nc ? nc : 1)) : NULL;
  int64_t nk = 0, na = 0;
  for (int64_t j = 0; j < nc; ++j) {
    double a, t, sg;
    ++*evals;
    int k = eval_full(&P[cand_ids[j]], cam, px, py, &a, &t, &sg);
    mark_threshold(s, sg);
    if (k) kp[nk++] = (kpair){t, a, cand_ids[j]};
    if (ca && (k || near_alpha_min(sg))) ca[na++] = (cand){t, a, P[cand_ids[j]].rgb, cand_ids[j], k, near_alpha_min(sg)};
  }
  *kept += nk;
  qsort(kp, nk, sizeof(kpair), kpair_cmp);
  for (int64_t j = 0; j < nk; ++j) {
    if (j > 0 && fabs(kp[j].t - kp[j - 1].t) < g_margin_tie * fabs(kp[j].t)) s->marginal = 1;
    blend(s, kp[j].alpha, P[kp[j].gid].rgb, kp[j].gid);
    if (s->done) {
      /* the pair after the stop could have come first among near-ties */
      if (j + 1 < nk && fabs(kp[j + 1].t - kp[j].t) < g_margin_tie * fabs(kp[j].t)) s->marginal = 1;
      break;
    }
  }
  free(kp);
  if (ca) {
    qsort(ca, na, sizeof(cand), cand_cmp);
    sample_outcomes(s, ca, (int)na);
    free(ca);
  }
}

/* One 4x4 block of samples of the hierarchical (or window) order: its geometry, its
 * tile's stream and its windows. */
typedef struct {
  const og_proj* P;
  const og_camera* cam;
  double px[16], py[16], c4[2], c2[4][2];
  const tentry* list;
  int64_t nlist;
  int k1, k2, k3;
} blockdef;

/* Runs the block's cascade over its stream on the samples s[16] (NULL where there is
 * none), taking the decisions in `forced` the other way and recording in `seen` the
 * decisions within the margins that it meets. */
static void run_block(const blockdef* bd, sample* s[16], const decset* forced, decset* seen, int record,
                      int64_t* evals, int64_t* kept, int* tie) {
  hblock B;
  memset(&B, 0, sizeof B);
  B.P = bd->P;
  B.cam = bd->cam;
  B.k1 = bd->k1;
  B.k2 = bd->k2;
  B.k3 = bd->k3;
  B.forced = forced;
  B.seen = seen;
  B.record = record;
  for (int i = 0; i < 16; ++i) {
    B.s[i] = s[i];
    B.px[i] = bd->px[i];
    B.py[i] = bd->py[i];
  }
  memcpy(B.c4, bd->c4, sizeof B.c4);
  memcpy(B.c2, bd->c2, sizeof B.c2);
  /* forced stream ties: the two entries swap places in the stream */
  const tentry* L = bd->list;
  tentry* cp = NULL;
  for (int f = 0; forced && f < forced->n; ++f) {
    if (forced->d[f].type != OG_DEC_STIE) continue;
    if (!cp) {
      cp = (tentry*)malloc(sizeof(tentry) * (bd->nlist ? bd->nlist : 1));
      memcpy(cp, bd->list, sizeof(tentry) * bd->nlist);
      L = cp;
    }
    int64_t a = -1, b = -1;
    for (int64_t j = 0; j < bd->nlist; ++j) {
      if (cp[j].gid == forced->d[f].g1) a = j;
      if (cp[j].gid == forced->d[f].g2) b = j;
    }
    if (a >= 0 && b >= 0) {
      tentry t = cp[a];
      cp[a] = cp[b];
      cp[b] = t;
    }
  }
  for (int64_t j = 0; j < bd->nlist; ++j) {
    int all_done = 1;
    for (int i = 0; i < 16; ++i)
      if (B.s[i] && !B.s[i]->done) all_done = 0;
    if (all_done) break;
    stream_entry(&B, L[j].gid, L[j].key);
  }
  flush_block(&B);
  free(cp);
  if (evals) *evals += B.evals;
  if (kept) *kept += B.kept;
  if (tie) *tie = B.tie;
  free(B.L1.e);
  for (int b = 0; b < 4; ++b) free(B.L2[b].e);
  for (int i = 0; i < 16; ++i) free(B.L3[i].e);
}

typedef struct {
  uint64_t mask;
  double v[16][4];
} brun;

/* Outcome sets of a block's samples.  The nominal run met the decisions `seen`.  Each
 * is flipped alone first; a sample's relevant decisions are those whose flip alone
 * changes its result, and every combination of them (at most OG_MAX_SAMPLE_DECISIONS)
 * is run.  Runs are shared between samples by the set of flips. */
static void block_outcomes(const blockdef* bd, sample* S16[16], const decset* seen) {
  const int nd = seen->n;
  if (nd == 0) return;
  if (nd > OG_MAX_BLOCK_DECISIONS) {
    for (int i = 0; i < 16; ++i)
      if (S16[i]) S16[i]->unchecked = 1;
    return;
  }
  brun* runs = NULL;
  int nruns = 0, capruns = 0;
  uint32_t aff[OG_MAX_BLOCK_DECISIONS];
  double nom[16][4];
  for (int i = 0; i < 16; ++i)
    if (S16[i]) {
      for (int c = 0; c < 3; ++c) nom[i][c] = S16[i]->C[c];
      nom[i][3] = S16[i]->T;
    }
  decset F = {0};
  /* returns the index of the run with flips `mask` (run on first use) */
#define OG_RUN(maskv, idxout)                                                      \
  do {                                                                             \
    int found_ = -1;                                                               \
    for (int r_ = 0; r_ < nruns; ++r_)                                             \
      if (runs[r_].mask == (maskv)) found_ = r_;                                   \
    if (found_ < 0) {                                                              \
      if (nruns == capruns) {                                                      \
        capruns = capruns ? 2 * capruns : 64;                                      \
        runs = (brun*)realloc(runs, sizeof(brun) * capruns);                       \
      }                                                                            \
      F.n = 0;                                                                     \
      for (int d_ = 0; d_ < nd; ++d_)                                              \
        if (((maskv) >> d_) & 1) decset_add(&F, seen->d[d_]);                      \
      sample loc_[16];                                                             \
      sample* lp_[16];                                                             \
      memset(loc_, 0, sizeof loc_);                                                \
      for (int i_ = 0; i_ < 16; ++i_) {                                            \
        loc_[i_].T = 1.0;                                                          \
        lp_[i_] = S16[i_] ? &loc_[i_] : NULL;                                      \
      }                                                                            \
      run_block(bd, lp_, &F, NULL, 0, NULL, NULL, NULL);                           \
      runs[nruns].mask = (maskv);                                                  \
      for (int i_ = 0; i_ < 16; ++i_) {                                            \
        for (int c_ = 0; c_ < 3; ++c_) runs[nruns].v[i_][c_] = loc_[i_].C[c_];     \
        runs[nruns].v[i_][3] = loc_[i_].T;                                         \
      }                                                                            \
      found_ = nruns++;                                                            \
    }                                                                              \
    (idxout) = found_;                                                             \
  } while (0)
  for (int d = 0; d < nd; ++d) {
    int r;
    OG_RUN(1ull << d, r);
    aff[d] = 0;
    for (int i = 0; i < 16; ++i) {
      if (!S16[i]) continue;
      for (int c = 0; c < 4; ++c)
        if (fabs(runs[r].v[i][c] - nom[i][c]) > OG_SAME) aff[d] |= 1u << i;
    }
  }
  for (int i = 0; i < 16; ++i) {
    if (!S16[i]) continue;
    int R[OG_MAX_BLOCK_DECISIONS], nr = 0;
    for (int d = 0; d < nd; ++d)
      if ((aff[d] >> i) & 1) R[nr++] = d;
    if (nr == 0) continue;
    if (nr > OG_MAX_SAMPLE_DECISIONS) {
      S16[i]->unchecked = 1;
      continue;
    }
    outcome* out = NULL;
    int nout = 0, ok = outcome_add(&out, &nout, nom[i], nom[i][3]);
    for (uint32_t sub = 1; ok && sub < (1u << nr); ++sub) {
      uint64_t mask = 0;
      for (int k = 0; k < nr; ++k)
        if ((sub >> k) & 1) mask |= 1ull << R[k];
      int r;
      OG_RUN(mask, r);
      ok = outcome_add(&out, &nout, runs[r].v[i], runs[r].v[i][3]);
    }
    if (!ok) {
      S16[i]->unchecked = 1;
      free(out);
    } else if (nout > 1) {
      S16[i]->alt = out;
      S16[i]->nalt = nout;
    } else {
      free(out);
    }
  }
#undef OG_RUN
  free(F.d);
  free(runs);
}

static double fovea_weight(const og_opts* o, double px, double py) {
  double dx = px - o->gaze_x, dy = py - o->gaze_y;
  double w = (o->radius + o->band - sqrt(dx * dx + dy * dy)) / o->band;
  return w < 0 ? 0 : (w > 1 ? 1 : w);
}

/* tile class from the distances of the tile's pixel centres to the gaze point */
static int classify_tile(const og_opts* o, const og_camera* c, int tx, int ty, int T) {
  double x0 = tx * T + 0.5, y0 = ty * T + 0.5;
  double x1 = fmin((tx + 1) * T, c->width) - 0.5, y1 = fmin((ty + 1) * T, c->height) - 0.5;
  double nx = fmin(fmax(o->gaze_x, x0), x1), ny = fmin(fmax(o->gaze_y, y0), y1);
  double dmin = hypot(nx - o->gaze_x, ny - o->gaze_y);
  double fx = fmax(fabs(x0 - o->gaze_x), fabs(x1 - o->gaze_x));
  double fy = fmax(fabs(y0 - o->gaze_y), fabs(y1 - o->gaze_y));
  double dmax = hypot(fx, fy);
  if (dmax <= o->radius) return 0;
  if (dmin >= o->radius + o->band) return 2;
  return 1;
}

/* The samples an output pixel reads and their weights: the pixel's own sample (plain
 * and focus tiles); its sample at weight w and the four samples of its 2x2 group at
 * (1 - w) / 4 (hybrid tiles); the four bilinear taps of the half-resolution image, each
 * a group sample or the mean of four full-resolution samples (periphery tiles).  None
 * for a pixel of an invisible tile (the background). */
typedef struct {
  int64_t k;
  double w;
} tap;

static int add_tap(tap* t, int n, int64_t k, double w) {
  for (int j = 0; j < n; ++j)
    if (t[j].k == k) {
      t[j].w += w;
      return n;
    }
  t[n] = (tap){k, w};
  return n + 1;
}

static int low_taps(const sample* S, int W, int W2, int64_t nfull, int gx, int gy, double w, tap* t, int n) {
  int64_t g = nfull + (int64_t)gy * W2 + gx;
  if (S[g].active_sample) return add_tap(t, n, g, w);
  for (int j = 0; j < 4; ++j) n = add_tap(t, n, (int64_t)(2 * gy + (j >> 1)) * W + 2 * gx + (j & 1), 0.25 * w);
  return n;
}

static int pixel_taps(const og_opts* o, const og_camera* cam, const sample* S, const uint8_t* cls, const uint8_t* tvis,
                      int T, int x, int y, tap* t) {
  const int W = cam->width, H = cam->height, W2 = W / 2, H2 = H / 2, ntx = (W + T - 1) / T;
  const int64_t nfull = (int64_t)W * H, k = (int64_t)y * W + x;
  const int tl = (y / T) * ntx + x / T;
  if (!tvis[tl]) return 0;
  int c = cls[tl];
  if (!o->foveated || c == 0) return add_tap(t, 0, k, 1.0);
  if (c == 1) {
    double w = fovea_weight(o, x + 0.5, y + 0.5);
    int n = add_tap(t, 0, k, w);
    return low_taps(S, W, W2, nfull, x / 2, y / 2, 1 - w, t, n);
  }
  double ux = (x + 0.5) / 2 - 0.5, uy = (y + 0.5) / 2 - 0.5;
  int x0 = (int)floor(ux), y0 = (int)floor(uy);
  double fx = ux - x0, fy = uy - y0;
  int xa = x0 < 0 ? 0 : (x0 > W2 - 1 ? W2 - 1 : x0), xb = x0 + 1 > W2 - 1 ? W2 - 1 : x0 + 1;
  int ya = y0 < 0 ? 0 : (y0 > H2 - 1 ? H2 - 1 : y0), yb = y0 + 1 > H2 - 1 ? H2 - 1 : y0 + 1;
  if (xb < 0) xb = 0;
  if (yb < 0) yb = 0;
  int n = 0;
  n = low_taps(S, W, W2, nfull, xa, ya, (1 - fx) * (1 - fy), t, n);
  n = low_taps(S, W, W2, nfull, xb, ya, fx * (1 - fy), t, n);
  n = low_taps(S, W, W2, nfull, xa, yb, (1 - fx) * fy, t, n);
  n = low_taps(S, W, W2, nfull, xb, yb, fx * fy, t, n);
  return n;
}

void og_free(void* p) { free(p); }

int og_render(const og_scene* sc, const og_camera* cam, const og_opts* o, og_out* out) {
  const int W = cam->width, H = cam->height, T = o->key_tile;
  if (W <= 0 || H <= 0 || T <= 0 || T % 4) return -1;
  /* foveation classifies the key tiles (32x32 as in Sec. 4.3, or 16x16); periphery tiles
   * hold whole 2x2 groups, and their 4x4 blocks of groups stay inside one tile */
  if (o->foveated && ((T != 32 && T != 16) || W % 2 || H % 2)) return -1;
  if (o->brute && o->mode != 0) return -1;
  if (o->mode < 0 || o->mode > 4) return -1;
  const int ntx = (W + T - 1) / T, nty = (H + T - 1) / T, ntiles = ntx * nty;
  const int64_t n = sc->n;
  const int W2 = W / 2, H2 = H / 2;
  const int64_t nfull = (int64_t)W * H, nsamp = nfull + (int64_t)W2 * H2;
  memset(out->stats, 0, sizeof out->stats);
  g_margin_alpha = o->margin_alpha;
  g_margin_stop = o->margin_stop;
  g_margin_tie = o->margin_tie;

  og_proj* P = (og_proj*)malloc(sizeof(og_proj) * (n ? n : 1));
  int64_t nvalid = 0;
  /* with outcome sets, Gaussians whose opacity is within the alpha margin below 1/255
   * are kept too: an FP32 renderer may keep them, at alpha within the margin of the cut
   * (they change no FP64 result, as no sample keeps them) */
  const double sigma_min = o->outcomes ? OG_ALPHA_MIN * (1.0 - o->margin_alpha) : OG_ALPHA_MIN;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : nvalid)
  for (int64_t i = 0; i < n; ++i) {
    int v = og_project_min(sc, i, cam, &P[i], sigma_min);
    if (v && o->dist_cull) {
      double dd = 0;
      for (int k = 0; k < 3; ++k) {
        double e = sc->mean[k * n + i] - o->dist_ref[k];
        dd += e * e;
      }
      const double d = sqrt(dd);
      if (!(d >= o->dist_min && d < o->dist_max)) P[i].valid = v = 0;
    }
    nvalid += v && P[i].sigma >= OG_ALPHA_MIN;
  }
  out->stats[0] = nvalid;

  /* tile classes */
  uint8_t* cls = (uint8_t*)calloc(ntiles, 1);
  if (o->foveated)
    for (int ty = 0; ty < nty; ++ty)
      for (int tx = 0; tx < ntx; ++tx) cls[ty * ntx + tx] = (uint8_t)classify_tile(o, cam, tx, ty, T);

  /* visibility culling: invisible key tiles get no instances */
  uint8_t* tvis = tile_visibility(o->visible, W, H, T);
  if (out->tile_class) /* class, with 4 added for a tile without visible pixels */
    for (int t = 0; t < ntiles; ++t) out->tile_class[t] = (uint8_t)(cls[t] | (tvis[t] ? 0 : 4));
  /* tile lists sorted by (key, gid): the stream each sample reads */
  int64_t* cnt = (int64_t*)calloc(ntiles + 1, sizeof(int64_t));
  tentry* lists = NULL;
  int32_t* brute_ids = NULL;
  if (o->brute) {
    brute_ids = (int32_t*)malloc(sizeof(int32_t) * (n ? n : 1));
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i)
      if (P[i].valid) brute_ids[m++] = (int32_t)i;
    nvalid = m;
  } else {
    /* with outcome sets, the lists also hold the pairs that only a decision within the
     * alpha margin keeps: their largest alpha over the tile is below the cut by less
     * than the margin (sigma G > (1 - m) / 255  <=>  q < r2 - 2 ln(1 - m)) */
    double relax = o->outcomes ? -2.0 * log1p(-o->margin_alpha) : 0.0;
    double* slack = NULL;
    lists = build_lists(P, n, cam, T, o->tile_cull, tvis, o->mode, relax, cnt, o->outcomes ? &slack : NULL);
    int64_t ninst = cnt[ntiles];
    if (slack) {
      ninst = 0;
      for (int64_t j = 0; j < cnt[ntiles]; ++j) ninst += slack[j] <= 0;
      free(slack);
    }
    out->stats[1] = ninst;
  }
  if (o->brute) out->stats[1] = 0;

  sample* S = (sample*)calloc(nsamp, sizeof(sample));
  for (int64_t k = 0; k < nsamp; ++k) S[k].T = 1.0;
  /* which samples exist: full-res pixels of focus/hybrid/plain tiles, groups of periphery tiles */
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int c = cls[(y / T) * ntx + x / T];
      if (!tvis[(y / T) * ntx + x / T]) continue; /* no sample renders: C = 0, T = 1 */
      if (c != 2) S[(int64_t)y * W + x].active_sample = 1;
      else if (!(x & 1) && !(y & 1)) S[nfull + (int64_t)(y / 2) * W2 + x / 2].active_sample = 1;
    }

  int64_t evals = 0, kept = 0;
  if (o->mode == 0) {
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : evals, kept)
    for (int64_t k = 0; k < nsamp; ++k) {
      if (!S[k].active_sample) continue;
      double px, py;
      int sx, sy;
      if (k < nfull) {
        sx = (int)(k % W);
        sy = (int)(k / W);
        px = sx + 0.5;
        py = sy + 0.5;
      } else {
        int64_t g = k - nfull;
        sx = (int)(g % W2) * 2;
        sy = (int)(g / W2) * 2;
        px = sx + 1.0;
        py = sy + 1.0;
      }
      const int32_t* cand;
      int64_t nc;
      int32_t* tmp = NULL;
      if (o->brute) {
        cand = brute_ids;
        nc = nvalid;
      } else {
        int t = (sy / T) * ntx + sx / T;
        nc = cnt[t + 1] - cnt[t];
        tmp = (int32_t*)malloc(sizeof(int32_t) * (nc ? nc : 1));
        for (int64_t j = 0; j < nc; ++j) tmp[j] = lists[cnt[t] + j].gid;
        cand = tmp;
      }
      render_exact(P, cam, cand, nc, px, py, &S[k], o->outcomes, &evals, &kept);
      free(tmp);
    }
  } else if (o->mode == 3 || o->mode == 4) {
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : evals, kept)
    for (int64_t k = 0; k < nsamp; ++k) {
      if (!S[k].active_sample) continue;
      int sx, sy;
      double px, py;
      if (k < nfull) {
        sx = (int)(k % W);
        sy = (int)(k / W);
        px = sx + 0.5;
        py = sy + 0.5;
      } else {
        int64_t g = k - nfull;
        sx = (int)(g % W2) * 2;
        sy = (int)(g / W2) * 2;
        px = sx + 1.0;
        py = sy + 1.0;
      }
      const int t = (sy / T) * ntx + sx / T;
      double last_key = -INFINITY;
      for (int64_t j = cnt[t]; j < cnt[t + 1] && !S[k].done; ++j) {
        double a, ts, sg;
        ++evals;
        const int32_t gid = lists[j].gid;
        const int keep = og_eval(&P[gid], cam, px, py, &a, &ts, &sg);
        mark_threshold(&S[k], sg);
        if (!keep) continue;
        ++kept;
        /* an FP32 key may order two near-equal keys the other way */
        if (fabs(lists[j].key - last_key) < g_margin_tie * fabs(lists[j].key)) S[k].marginal = 1;
        last_key = lists[j].key;
        blend(&S[k], a, P[gid].rgb, gid);
      }
      if (o->outcomes) {
        /* outcome set: the list order, near-equal keys in either order */
        int64_t nc = cnt[t + 1] - cnt[t], na = 0;
        cand* ca = (cand*)malloc(sizeof(cand) * (nc ? nc : 1));
        for (int64_t j = cnt[t]; j < cnt[t + 1]; ++j) {
          double a, ts, sg;
          const int32_t gid = lists[j].gid;
          const int keep = eval_full(&P[gid], cam, px, py, &a, &ts, &sg);
          if (keep || near_alpha_min(sg)) ca[na++] = (cand){lists[j].key, a, P[gid].rgb, gid, keep, near_alpha_min(sg)};
        }
        sample_outcomes(&S[k], ca, (int)na);
        free(ca);
      }
    }
  } else {
    int k1 = o->mode == 1 ? 0 : o->k1, k2 = o->mode == 1 ? 0 : o->k2, k3 = o->k3;
    /* independent 4x4 sample blocks of the full-res grid and of the group grid */
    int nbx = (W + 3) / 4, nby = (H + 3) / 4, nbx2 = (W2 + 3) / 4, nby2 = (H2 + 3) / 4;
    int64_t nb_full = (int64_t)nbx * nby, nb_all = nb_full + (int64_t)nbx2 * nby2;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : evals, kept)
    for (int64_t bi = 0; bi < nb_all; ++bi) {
      blockdef bd;
      memset(&bd, 0, sizeof bd);
      bd.P = P;
      bd.cam = cam;
      bd.k1 = k1;
      bd.k2 = k2;
      bd.k3 = k3;
      sample* bs[16] = {NULL};
      int lowgrid = bi >= nb_full;
      int bx, by, any = 0, tile = -1;
      if (!lowgrid) {
        bx = (int)(bi % nbx) * 4;
        by = (int)(bi / nbx) * 4;
      } else {
        bx = (int)((bi - nb_full) % nbx2) * 4;
        by = (int)((bi - nb_full) / nbx2) * 4;
      }
      for (int i = 0; i < 16; ++i) {
        int sx = bx + (i & 3), sy = by + (i >> 2);
        int64_t k;
        if (!lowgrid) {
          if (sx >= W || sy >= H) continue;
          k = (int64_t)sy * W + sx;
          bd.px[i] = sx + 0.5;
          bd.py[i] = sy + 0.5;
          tile = (sy / T) * ntx + sx / T;
        } else {
          if (sx >= W2 || sy >= H2) continue;
          k = nfull + (int64_t)sy * W2 + sx;
          bd.px[i] = 2 * sx + 1.0;
          bd.py[i] = 2 * sy + 1.0;
          tile = ((2 * sy) / T) * ntx + (2 * sx) / T;
        }
        if (S[k].active_sample) {
          bs[i] = &S[k];
          any = 1;
        }
      }
      if (!any) continue;
      if (!lowgrid) {
        bd.c4[0] = bx + 2.0;
        bd.c4[1] = by + 2.0;
        for (int b = 0; b < 4; ++b) {
          bd.c2[b][0] = bx + (b & 1) * 2 + 1.0;
          bd.c2[b][1] = by + (b >> 1) * 2 + 1.0;
        }
      } else {
        bd.c4[0] = 2 * bx + 4.0;
        bd.c4[1] = 2 * by + 4.0;
        for (int b = 0; b < 4; ++b) {
          bd.c2[b][0] = 2 * (bx + (b & 1) * 2) + 2.0;
          bd.c2[b][1] = 2 * (by + (b >> 1) * 2) + 2.0;
        }
      }
      bd.list = lists + cnt[tile];
      bd.nlist = cnt[tile + 1] - cnt[tile];
      decset seen = {0};
      int tie = 0;
      int64_t be = 0, bk = 0;
      run_block(&bd, bs, NULL, o->outcomes ? &seen : NULL, 1, &be, &bk, &tie);
      evals += be;
      kept += bk;
      /* a block-level decision within the margins marks every sample of the block */
      if (tie)
        for (int i = 0; i < 16; ++i)
          if (bs[i]) bs[i]->marginal = 1;
      if (o->outcomes) block_outcomes(&bd, bs, &seen);
      free(seen.d);
    }
  }
  out->stats[2] = evals;
  out->stats[3] = kept;

  /* per-sample outputs */
  double bg[3] = {o->bg[0], o->bg[1], o->bg[2]};
  double* lowimg = (double*)calloc((size_t)3 * (W2 > 0 ? W2 : 1) * (H2 > 0 ? H2 : 1), sizeof(double));
  uint8_t* lowmarg = (uint8_t*)calloc((size_t)(W2 > 0 ? W2 : 1) * (H2 > 0 ? H2 : 1), 1);
  if (out->full)
    for (int64_t k = 0; k < 4 * nfull; ++k) out->full[k] = NAN;
  if (out->low)
    for (int64_t k = 0; k < 4 * (int64_t)W2 * H2; ++k) out->low[k] = NAN;
  for (int64_t k = 0; k < nsamp; ++k) {
    if (!S[k].active_sample) continue;
    if (k < nfull) {
      if (out->full) {
        for (int c = 0; c < 3; ++c) out->full[c * nfull + k] = S[k].C[c];
        out->full[3 * nfull + k] = S[k].T;
      }
    } else if (out->low) {
      int64_t g = k - nfull, ng = (int64_t)W2 * H2;
      for (int c = 0; c < 3; ++c) out->low[c * ng + g] = S[k].C[c];
      out->low[3 * ng + g] = S[k].T;
    }
  }
  /* half-resolution image: group samples in periphery tiles, 2x2 means elsewhere */
  if (o->foveated) {
    for (int gy = 0; gy < H2; ++gy)
      for (int gx = 0; gx < W2; ++gx) {
        int64_t g = (int64_t)gy * W2 + gx;
        sample* sg = &S[nfull + g];
        if (sg->active_sample) {
          for (int c = 0; c < 3; ++c) lowimg[c * W2 * H2 + g] = sg->C[c] + sg->T * bg[c];
          lowmarg[g] = (uint8_t)sg->marginal;
        } else {
          for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int j = 0; j < 4; ++j) {
              sample* sp = &S[(int64_t)(2 * gy + (j >> 1)) * W + 2 * gx + (j & 1)];
              s += sp->C[c] + sp->T * bg[c];
            }
            lowimg[c * W2 * H2 + g] = 0.25 * s;
          }
          for (int j = 0; j < 4; ++j)
            if (S[(int64_t)(2 * gy + (j >> 1)) * W + 2 * gx + (j & 1)].marginal) lowmarg[g] = 1;
        }
      }
    if (out->lowimg) memcpy(out->lowimg, lowimg, sizeof(double) * 3 * W2 * H2);
  }
  int64_t nmarg = 0;
  for (int y = 0; y < H; ++y)
    for (int x = 0; x < W; ++x) {
      int64_t k = (int64_t)y * W + x;
      int c = cls[(y / T) * ntx + x / T];
      int marg = 0;
      double v[3];
      if (!tvis[(y / T) * ntx + x / T]) {
        for (int ch = 0; ch < 3; ++ch) v[ch] = bg[ch];
      } else if (!o->foveated || c == 0) {
        for (int ch = 0; ch < 3; ++ch) v[ch] = S[k].C[ch] + S[k].T * bg[ch];
        marg = S[k].marginal;
      } else if (c == 1) {
        double w = fovea_weight(o, x + 0.5, y + 0.5);
        int64_t g = (int64_t)(y / 2) * W2 + x / 2;
        for (int ch = 0; ch < 3; ++ch)
          v[ch] = w * (S[k].C[ch] + S[k].T * bg[ch]) + (1 - w) * lowimg[ch * W2 * H2 + g];
        marg = S[k].marginal || lowmarg[g];
      } else {
        /* bilinear upsampling with clamp-to-edge, half-pixel aligned */
        double ux = (x + 0.5) / 2 - 0.5, uy = (y + 0.5) / 2 - 0.5;
        int x0 = (int)floor(ux), y0 = (int)floor(uy);
        double fx = ux - x0, fy = uy - y0;
        int xa = x0 < 0 ? 0 : (x0 > W2 - 1 ? W2 - 1 : x0), xb = x0 + 1 > W2 - 1 ? W2 - 1 : x0 + 1;
        int ya = y0 < 0 ? 0 : (y0 > H2 - 1 ? H2 - 1 : y0), yb = y0 + 1 > H2 - 1 ? H2 - 1 : y0 + 1;
        if (xb < 0) xb = 0;
        if (yb < 0) yb = 0;
        for (int ch = 0; ch < 3; ++ch) {
          const double* L = lowimg + (int64_t)ch * W2 * H2;
          double top = (1 - fx) * L[ya * W2 + xa] + fx * L[ya * W2 + xb];
          double bot = (1 - fx) * L[yb * W2 + xa] + fx * L[yb * W2 + xb];
          v[ch] = (1 - fy) * top + fy * bot;
        }
        marg = lowmarg[ya * W2 + xa] || lowmarg[ya * W2 + xb] || lowmarg[yb * W2 + xa] || lowmarg[yb * W2 + xb];
      }
      for (int ch = 0; ch < 3; ++ch) out->image[ch * nfull + k] = v[ch];
      if (out->marginal) out->marginal[k] = (uint8_t)marg;
      nmarg += marg;
    }
  out->stats[5] = nmarg;

  /* outcome sets of the composited pixels: every combination of the valid results of
   * the samples a pixel reads, through the same composite (its taps and weights) */
  out->alt_off = NULL;
  out->alt = NULL;
  out->alt4 = NULL;
  out->n_alt = 0;
  if (o->outcomes) {
    int64_t cap = 0, nalt = 0, nunchk = 0;
    double* alt = NULL;
    double* alt4 = NULL; /* plain renders: the one sample's (C, T) of each alternative */
    int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (nfull + 1));
    for (int y = 0; y < H; ++y)
      for (int x = 0; x < W; ++x) {
        int64_t k = (int64_t)y * W + x;
        off[k] = nalt;
        tap tp[32];
        int nt = pixel_taps(o, cam, S, cls, tvis, T, x, y, tp);
        int unchk = 0;
        int64_t combos = 1;
        for (int j = 0; j < nt; ++j) {
          if (S[tp[j].k].unchecked) unchk = 1;
          if (S[tp[j].k].nalt > 1) combos *= S[tp[j].k].nalt;
          if (combos > OG_MAX_PIXEL_COMBOS) unchk = 1;
        }
        if (out->unchecked) out->unchecked[k] = (uint8_t)unchk;
        nunchk += unchk;
        if (unchk || combos == 1) continue;
        int pick[32] = {0};
        int64_t first = nalt;
        for (int64_t c = 0; c < combos; ++c) {
          double v[3] = {0, 0, 0};
          for (int j = 0; j < nt; ++j) {
            const sample* sp = &S[tp[j].k];
            const double* r = sp->nalt > 1 ? sp->alt[pick[j]].v : NULL;
            for (int ch = 0; ch < 3; ++ch) {
              double Cc = r ? r[ch] : sp->C[ch], Tt = r ? r[3] : sp->T;
              v[ch] += tp[j].w * (Cc + Tt * bg[ch]);
            }
          }
          int dup = 0;
          for (int64_t a = first; a < nalt && !dup; ++a)
            dup = fabs(alt[3 * a] - v[0]) <= OG_SAME && fabs(alt[3 * a + 1] - v[1]) <= OG_SAME &&
                  fabs(alt[3 * a + 2] - v[2]) <= OG_SAME;
          if (!dup) {
            if (nalt == cap) {
              cap = cap ? 2 * cap : 1024;
              alt = (double*)realloc(alt, sizeof(double) * 3 * cap);
              if (!o->foveated) alt4 = (double*)realloc(alt4, sizeof(double) * 4 * cap);
            }
            for (int ch = 0; ch < 3; ++ch) alt[3 * nalt + ch] = v[ch];
            if (!o->foveated) { /* one tap of weight 1: the sample itself */
              const sample* sp = &S[tp[0].k];
              const double* r = sp->nalt > 1 ? sp->alt[pick[0]].v : NULL;
              for (int q = 0; q < 4; ++q) alt4[4 * nalt + q] = r ? r[q] : (q < 3 ? sp->C[q] : sp->T);
            }
            ++nalt;
          }
          /* next combination (mixed radix over the taps with several results) */
          for (int j = 0; j < nt; ++j) {
            if (S[tp[j].k].nalt <= 1) continue;
            if (++pick[j] < S[tp[j].k].nalt) break;
            pick[j] = 0;
          }
        }
      }
    off[nfull] = nalt;
    out->alt_off = off;
    out->alt = alt;
    out->alt4 = alt4;
    out->n_alt = nalt;
    out->stats[7] = nunchk;
  }

  /* blend orders for the gradient oracle */
  int64_t tot = 0, blended = 0;
  for (int64_t k = 0; k < nsamp; ++k) {
    if (out->order_off) out->order_off[k] = tot;
    if (out->order && tot + S[k].ng <= out->max_order)
      memcpy(out->order + tot, S[k].gids, sizeof(int32_t) * S[k].ng);
    tot += S[k].ng;
    blended += S[k].ng;
    if (S[k].active_sample) out->stats[6]++;
  }
  if (out->order_off) out->order_off[nsamp] = tot;
  out->n_order = tot;
  out->stats[4] = blended;

  for (int64_t k = 0; k < nsamp; ++k) {
    free(S[k].gids);
    free(S[k].alt);
  }
  free(S);
  free(lowimg);
  free(lowmarg);
  free(lists);
  free(brute_ids);
  free(cnt);
  free(cls);
  free(tvis);
  free(P);
  return 0;
}

/* Tile lists as the oracle builds them, for list-level comparisons:
 * counts[ntiles] (always), and when gids/keys are given (sized >= total) the sorted
 * lists concatenated by tile, with (slack, optional) qmin - r2 of each entry's Eq. 4
 * test.  relax > 0 adds the entries with 0 < qmin - r2 <= relax (a largest alpha over
 * the tile within the margin below 1/255).  Returns the total number of entries. */
int64_t og_tile_lists(const og_scene* sc, const og_camera* cam, int T, int tile_cull, const uint8_t* visible,
                      double relax, int64_t* counts, int32_t* gids, double* keys, double* slack, int64_t cap) {
  const int W = cam->width, H = cam->height;
  const int ntx = (W + T - 1) / T, nty = (H + T - 1) / T, ntiles = ntx * nty;
  const int64_t n = sc->n;
  og_proj* P = (og_proj*)malloc(sizeof(og_proj) * (n ? n : 1));
#pragma omp parallel for schedule(dynamic, 1024)
  for (int64_t i = 0; i < n; ++i) og_project(sc, i, cam, &P[i]);
  int64_t* cnt = (int64_t*)calloc(ntiles + 1, sizeof(int64_t));
  uint8_t* tvis = tile_visibility(visible, W, H, T);
  double* sl = NULL;
  tentry* lists = build_lists(P, n, cam, T, tile_cull, tvis, 0, relax, cnt, &sl);
  free(tvis);
  for (int t = 0; t < ntiles; ++t) counts[t] = cnt[t + 1] - cnt[t];
  int64_t tot = cnt[ntiles];
  if (gids && keys && cap >= tot)
    for (int64_t j = 0; j < tot; ++j) {
      gids[j] = lists[j].gid;
      keys[j] = lists[j].key;
      if (slack) slack[j] = sl[j];
    }
  free(sl);
  free(lists);
  free(cnt);
  free(P);
  return tot;
}

int og_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
