// Optimal-Projection preprocessing (Sec. 4.2), tile culling on the optimal plane (Eq. 4)
// and Gaussian/tile key duplication (Sec. 3 tile-based rasterization, Sec. 4.3 32x32
// tiles).  One thread per Gaussian reads its 59 parameters once and loops over every
// view of its scene, so the parameter traffic of a batch of views is paid once.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace vrs {

namespace {

// real spherical-harmonics constants (3DGS sign convention): 1/(2 sqrt(pi)),
// sqrt(3)/(2 sqrt(pi)), and the degree-2/3 normalisations
constexpr float kY0 = 0.28209479177387814f;
constexpr float kY1 = 0.4886025119029199f;
constexpr float kY2a = 1.0925484305920792f;
constexpr float kY2b = 0.31539156525252005f;
constexpr float kY2c = 0.5462742152960396f;
constexpr float kY3a = 0.5900435899266435f;
constexpr float kY3b = 2.890611442640554f;
constexpr float kY3c = 0.4570457994644658f;
constexpr float kY3d = 0.3731763325901154f;
constexpr float kY3e = 1.445305721320277f;

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float Y[16]) {
  Y[0] = kY0;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

__device__ __forceinline__ bool finite3(float a, float b, float c) { return isfinite(a) && isfinite(b) && isfinite(c); }

}  // namespace

// Optimal projection of Gaussian i into view vp.  Writes the 96-byte record and a
// conservative pixel bounding box of its alpha >= 1/255 region.  Returns false when the
// Gaussian is culled (non-finite, behind near_z, opacity < 1/255, degenerate).
__device__ bool project_gaussian(const SceneDev& s, long long i, const ViewParams& vp, float4 rec[6],
                                 float4& bb) {
  const long long n = s.n;
  const float m0 = s.mean[i], m1 = s.mean[n + i], m2 = s.mean[2 * n + i];
  const float l0 = s.ls[i], l1 = s.ls[n + i], l2 = s.ls[2 * n + i];
  float qw = s.quat[i], qx = s.quat[n + i], qy = s.quat[2 * n + i], qz = s.quat[3 * n + i];
  const float logit = s.logit[i];
  if (!finite3(m0, m1, m2) || !finite3(l0, l1, l2) || !finite3(qw, qx, qy) || !isfinite(qz) || !isfinite(logit))
    return false;
  {  // the view's layer: distance of the mean from the layer reference
    const float e0 = m0 - vp.dist_ref[0], e1 = m1 - vp.dist_ref[1], e2 = m2 - vp.dist_ref[2];
    const float dd = sqrtf(fmaf(e0, e0, fmaf(e1, e1, e2 * e2)));
    if (!(dd >= vp.dist_min && dd < vp.dist_max)) return false;
  }
  const float* R = vp.R;
  const float mx = fmaf(R[0], m0, fmaf(R[1], m1, fmaf(R[2], m2, vp.t[0])));
  const float my = fmaf(R[3], m0, fmaf(R[4], m1, fmaf(R[5], m2, vp.t[1])));
  const float mz = fmaf(R[6], m0, fmaf(R[7], m1, fmaf(R[8], m2, vp.t[2])));
  if (!(mz >= vp.near_z)) return false;
  const float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  if (!(qn > 0.f)) return false;
  const float iq = 1.f / qn;
  qw *= iq; qx *= iq; qy *= iq; qz *= iq;
  float G[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
  float Rc[9];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) Rc[3 * a + b] = R[3 * a] * G[b] + R[3 * a + 1] * G[3 + b] + R[3 * a + 2] * G[6 + b];
  const float s2[3] = {expf(2.f * l0), expf(2.f * l1), expf(2.f * l2)};
  const float si2[3] = {expf(-2.f * l0), expf(-2.f * l1), expf(-2.f * l2)};
  float Sc[6], Si[6];  // xx xy xz yy yz zz
  {
    const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const float* ra = Rc + 3 * ia[e];
      const float* rb = Rc + 3 * ib[e];
      Sc[e] = ra[0] * s2[0] * rb[0] + ra[1] * s2[1] * rb[1] + ra[2] * s2[2] * rb[2];
      Si[e] = ra[0] * si2[0] * rb[0] + ra[1] * si2[1] * rb[1] + ra[2] * si2[2] * rb[2];
    }
  }
#pragma unroll
  for (int e = 0; e < 6; ++e)
    if (!isfinite(Sc[e]) || !isfinite(Si[e])) return false;
  const float sigma = 1.f / (1.f + expf(-logit));
  if (!(sigma >= kAlphaMin)) return false;
  const float lg2s = log2f(sigma);
  const float d = sqrtf(mx * mx + my * my + mz * mz);
  const float ux = mx / d, uy = my / d, uz = mz / d;
  const float rho = sqrtf(ux * ux + uz * uz);
  const float e1x = uz / rho, e1z = -ux / rho;  // e1y = 0
  const float e2x = uy * e1z, e2y = uz * e1x - ux * e1z, e2z = -uy * e1x;
  // Sigma_p = E Sc E^T / d^2 + dilation
  auto quad = [&](float ax, float ay, float az, float bx, float by, float bz) {
    return ax * (Sc[0] * bx + Sc[1] * by + Sc[2] * bz) + ay * (Sc[1] * bx + Sc[3] * by + Sc[4] * bz) +
           az * (Sc[2] * bx + Sc[4] * by + Sc[5] * bz);
  };
  const float id2 = 1.f / (d * d);
  const float dil = kDilationPx2 / (vp.fx * vp.fy);
  const float p00 = quad(e1x, 0.f, e1z, e1x, 0.f, e1z) * id2 + dil;
  const float p01 = quad(e1x, 0.f, e1z, e2x, e2y, e2z) * id2;
  const float p11 = quad(e2x, e2y, e2z, e2x, e2y, e2z) * id2 + dil;
  const float det = p00 * p11 - p01 * p01;
  if (!(det > 0.f)) return false;
  {
    // every kept ray lies within angle atan(rho) of u, rho = r sqrt(lambda_max(Sigma_p)),
    // r^2 = 2 ln(255 sigma); drop the Gaussian when that cone misses a side of the view
    // frustum (extended by one pixel)
    const float r2 = 2.f * logf(255.f * sigma);
    const float hm = 0.5f * (p00 + p11), hd = 0.5f * (p00 - p11);
    const float lmax = hm + sqrtf(hd * hd + p01 * p01);
    const float rho = sqrtf(fmaxf(r2, 0.f) * lmax) * 1.001f + 1e-6f;
    const float sin_t = rho * rsqrtf(1.f + rho * rho);
    const float tl = (vp.cx + 1.f) / vp.fx, tr = (vp.W - vp.cx + 1.f) / vp.fx;
    const float tt = (vp.cy + 1.f) / vp.fy, tb = (vp.H - vp.cy + 1.f) / vp.fy;
    if ((ux + tl * uz) * rsqrtf(1.f + tl * tl) < -sin_t) return false;
    if ((-ux + tr * uz) * rsqrtf(1.f + tr * tr) < -sin_t) return false;
    if ((uy + tt * uz) * rsqrtf(1.f + tt * tt) < -sin_t) return false;
    if ((-uy + tb * uz) * rsqrtf(1.f + tb * tb) < -sin_t) return false;
  }
  const float idet = kHalfLog2e / det;
  const float A00 = p11 * idet, A01 = -p01 * idet, A11 = p00 * idet;
  const float ifx = 1.f / vp.fx, ify = 1.f / vp.fy;
  const float h00 = e1x * ifx, h01 = 0.f, h10 = e2x * ifx, h11 = e2y * ify, h20 = ux * ifx, h21 = uy * ify;
  const float h22 = 1.f / uz;
  const float pmx = fmaf(vp.fx, mx / mz, vp.cx), pmy = fmaf(vp.fy, my / mz, vp.cy);
  // depth form, normalised so that den(pm) = 1 and t*(pm) = z of the mean
  const float svx = Si[0] * mx + Si[1] * my + Si[2] * mz;
  const float svy = Si[1] * mx + Si[3] * my + Si[4] * mz;
  const float svz = Si[2] * mx + Si[4] * my + Si[5] * mz;
  const float den0 = (mx * svx + my * svy + mz * svz) / (mz * mz);
  if (!(den0 > 0.f) || !isfinite(den0)) return false;
  const float iden = 1.f / den0;
  const float n0 = svx * ifx * iden, n1 = svy * ify * iden;
  const float m00 = Si[0] * ifx * ifx * iden, m01x2 = 2.f * Si[1] * ifx * ify * iden, m11 = Si[3] * ify * ify * iden;
  const float m02x2 = 2.f * n0 / mz, m12x2 = 2.f * n1 / mz;
  // colour along the world-space viewing direction R^T u
  const float dx = R[0] * ux + R[3] * uy + R[6] * uz;
  const float dy = R[1] * ux + R[4] * uy + R[7] * uz;
  const float dz = R[2] * ux + R[5] * uy + R[8] * uz;
  float Y[16];
  sh_basis(s.deg, dx, dy, dz, Y);
  const int K = (s.deg + 1) * (s.deg + 1);
  float col[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    float v = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k)
      if (k < K) v = fmaf(Y[k], s.sh[((long long)k * 3 + c) * n + i], v);
    col[c] = fmaxf(v, 0.f);
  }
  rec[0] = make_float4(pmx, pmy, h00, h01);
  rec[1] = make_float4(h10, h11, h20, h21);
  rec[2] = make_float4(h22, A00, 2.f * A01, A11);
  rec[3] = make_float4(lg2s, n0, n1, mz);
  rec[4] = make_float4(m00, m01x2, m11, m02x2);
  rec[5] = make_float4(m12x2, col[0], col[1], col[2]);
  // bounding box: the cone (a, b) A' (a, b)^T <= cut w^2 seen as a conic in (dx, dy)
  const float cut = lg2s + kLog2_255;
  const float mA0x = A00 * h00 + A01 * h10, mA1x = A01 * h00 + A11 * h10;
  const float mA0y = A00 * h01 + A01 * h11, mA1y = A01 * h01 + A11 * h11;
  const float c00 = h00 * mA0x + h10 * mA1x - cut * h20 * h20;
  const float c01 = h01 * mA0x + h11 * mA1x - cut * h20 * h21;
  const float c11 = h01 * mA0y + h11 * mA1y - cut * h21 * h21;
  const float cx = -cut * h22 * h20, cy = -cut * h22 * h21, c33 = -cut * h22 * h22;
  const float cdet = c00 * c11 - c01 * c01;
  bb = make_float4(0.f, 0.f, (float)vp.W, (float)vp.H);
  if (c00 > 0.f && cdet > 1e-6f * c00 * c11) {
    const float i00 = c11 / cdet, i01 = -c01 / cdet, i11 = c00 / cdet;
    const float p0x = -(i00 * cx + i01 * cy), p0y = -(i01 * cx + i11 * cy);
    const float k = c33 + cx * p0x + cy * p0y;
    if (k < 0.f) {
      const float hx = sqrtf(-k * i00) * 1.01f + 1.f, hy = sqrtf(-k * i11) * 1.01f + 1.f;
      const float bx = pmx + p0x, by = pmy + p0y;
      if (isfinite(bx) && isfinite(by) && isfinite(hx) && isfinite(hy))
        bb = make_float4(fmaxf(bx - hx, -1e7f), fmaxf(by - hy, -1e7f), fminf(bx + hx, 1e7f), fminf(by + hy, 1e7f));
    }
  }
  return true;
}

// Eq. 4 on the optimal plane.  The sample quad [x0, x1] x [y0, y1] maps to a convex
// quadrilateral on the Gaussian's tangent plane; the plane maximum is the projected
// mean if it lies inside, otherwise the best of the closed-form edge maxima (line
// parameter clamped to the segment).  Returns true when the pair is kept; *key is the
// depth t* on the ray through the maximum point projected back to the image.
// Not inlined: the count pass and the emit pass run the same machine code, so they
// make the same decisions.
struct Keep {
  bool keep;
  float key;
};

__device__ __noinline__ Keep tile_keep(float4 f0, float4 f1, float4 f2, float4 f3, float4 f4, float m12x2, float x0,
                                       float y0, float x1, float y1) {
  const float cxs[4] = {x0, x1, x1, x0}, cys[4] = {y0, y0, y1, y1};
  float S0[4], S1[4];
  Keep res{true, f3.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float dx = cxs[k] - f0.x, dy = cys[k] - f0.y;
    const float a = fmaf(f0.z, dx, f0.w * dy);
    const float b = fmaf(f1.x, dx, f1.y * dy);
    const float w = fmaf(f1.z, dx, fmaf(f1.w, dy, f2.x));
    if (!(w > 0.f)) return res;  // quad not bounded on the plane
    S0[k] = a / w;
    S1[k] = b / w;
  }
  bool pos = false, neg = false;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int l = (k + 1) & 3;
    const float cr = (S0[l] - S0[k]) * (-S1[k]) - (S1[l] - S1[k]) * (-S0[k]);
    pos |= cr > 0.f;
    neg |= cr < 0.f;
  }
  if (!(pos && neg)) return res;  // projected mean inside: maximum at the mean
  const float A00 = f2.y, A01 = 0.5f * f2.z, A11 = f2.w;
  float qmin = INFINITY, X0 = 0.f, X1 = 0.f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int l = (k + 1) & 3;
    const float Px = S0[k], Py = S1[k], Dx = S0[l] - S0[k], Dy = S1[l] - S1[k];
    const float APx = A00 * Px + A01 * Py, APy = A01 * Px + A11 * Py;
    const float ADx = A00 * Dx + A01 * Dy, ADy = A01 * Dx + A11 * Dy;
    const float dAd = Dx * ADx + Dy * ADy;
    float t = dAd > 0.f ? -(Dx * APx + Dy * APy) / dAd : 0.f;
    t = fminf(fmaxf(t, 0.f), 1.f);
    const float Xx = Px + t * Dx, Xy = Py + t * Dy;
    const float q = Xx * (A00 * Xx + A01 * Xy) + Xy * (A01 * Xx + A11 * Xy);
    if (q < qmin) {
      qmin = q;
      X0 = Xx;
      X1 = Xy;
    }
  }
  const float cut = f3.x + kLog2_255;
  if (!(qmin <= cut * 1.0001f + 1e-5f)) return Keep{false, f3.w};  // a hair conservative vs FP64
  // back-project X to the image: solve a - X0 w = 0, b - X1 w = 0 for (dx, dy)
  const float a00 = f0.z - X0 * f1.z, a01 = f0.w - X0 * f1.w;
  const float a10 = f1.x - X1 * f1.z, a11 = f1.y - X1 * f1.w;
  const float r0 = X0 * f2.x, r1 = X1 * f2.x;
  const float dt = a00 * a11 - a01 * a10;
  if (dt != 0.f) {
    const float dx = (r0 * a11 - a01 * r1) / dt, dy = (a00 * r1 - a10 * r0) / dt;
    const float w = fmaf(f1.z, dx, fmaf(f1.w, dy, f2.x));
    if (w > 0.f && isfinite(dx) && isfinite(dy)) {
      const float num = fmaf(f3.y, dx, fmaf(f3.z, dy, f3.w));
      const float den = fmaf(dx, fmaf(f4.x, dx, fmaf(f4.y, dy, f4.w)), fmaf(dy, fmaf(f4.z, dy, m12x2), 1.0f));
      const float kk = num / den;
      if (isfinite(kk)) res.key = kk;
    }
  }
  return res;
}

__device__ __forceinline__ void tile_span(const float4& bb, const ViewParams& vp, int T, int& tx0, int& tx1,
                                          int& ty0, int& ty1) {
  tx0 = max((int)ceilf((bb.x + 0.5f) / T - 1.f), 0);
  ty0 = max((int)ceilf((bb.y + 0.5f) / T - 1.f), 0);
  tx1 = min((int)floorf((bb.z - 0.5f) / T), vp.ntx - 1);
  ty1 = min((int)floorf((bb.w - 0.5f) / T), vp.nty - 1);
}

__device__ __forceinline__ void tile_quad(int tx, int ty, int T, const ViewParams& vp, float& x0, float& y0,
                                          float& x1, float& y1) {
  x0 = tx * T + 0.5f;
  y0 = ty * T + 0.5f;
  x1 = (float)min((tx + 1) * T, vp.W) - 0.5f;
  y1 = (float)min((ty + 1) * T, vp.H) - 0.5f;
}

struct Span {
  int tx0, ty0, nx, nt;
};

__device__ __forceinline__ Span make_span(const float4& bb, const ViewParams& vp, int T, bool ok) {
  Span sp{0, 0, 0, 0};
  if (!ok) return sp;
  int tx0, tx1, ty0, ty1;
  tile_span(bb, vp, T, tx0, tx1, ty0, ty1);
  if (tx1 < tx0 || ty1 < ty0) return sp;
  sp.tx0 = tx0;
  sp.ty0 = ty0;
  sp.nx = tx1 - tx0 + 1;
  sp.nt = sp.nx * (ty1 - ty0 + 1);
  return sp;
}

// The count pass also keeps the sort keys of a Gaussian's first kKeyCache kept tiles
// (view-local tile << 32 | depth bits, row-major order of the rectangle), so the emit
// pass copies them for every Gaussian with at most that many instances instead of
// testing its tiles again; the whole warp re-tests the tiles of the larger ones.  Only
// the slots a Gaussian fills are written and read (the cache takes 256 B of address
// space per (view, Gaussian)).  Duplication of the VR stereo frame with 8 / 16 / 32
// slots: 0.122 / 0.065 / 0.045 ms; the re-tests of larger Gaussians, one warp per
// Gaussian, were most of its time.
constexpr int kKeyCache = kKeyCacheSlots;
__device__ __forceinline__ unsigned long long local_key(int tile, float key) {
  return ((unsigned long long)(unsigned)tile << 32) | float_order_bits(key);
}

// Sort key of the global orders (Sec. 3): key_mode 3 = view-space z of the mean (3DGS),
// 4 = its distance from the camera centre (Mini-Splatting), recovered from the record's
// projected mean and z; otherwise the Eq. 4 tile key.
__device__ __forceinline__ float order_key(int key_mode, float tile_key, const float4& f0, const float4& f3,
                                           const ViewParams& vp) {
  if (key_mode == 3) return f3.w;
  if (key_mode == 4) {
    const float mz = f3.w, mx = (f0.x - vp.cx) * mz / vp.fx, my = (f0.y - vp.cy) * mz / vp.fy;
    return sqrtf(mx * mx + my * my + mz * mz);
  }
  return tile_key;
}

// The count pass works in two phases per view.  Each thread projects its Gaussian (record,
// rectangle, span of key tiles).  Then the warp flattens the (Gaussian, tile) pairs of its
// 32 Gaussians into one list and tests 32 of them per step, one per lane: a lane finds
// its pair's Gaussian by a binary search over the warp's running tile counts and reads
// that Gaussian's record (written in the first phase) from memory.  Every lane works
// whatever the tile counts of the Gaussians, so few and many tiles, and culled
// Gaussians, cost no idle lanes.  Kept tiles are counted per Gaussian in shared memory,
// and ranked within their Gaussian in tile order for the key cache.
// parameter rows a Gaussian's projection reads: mean 3, log-scale 3, quaternion 4,
// opacity logit 1, and 3 per SH coefficient of the scene's degree
__host__ __device__ inline int param_rows(int deg) { return 11 + 3 * (deg + 1) * (deg + 1); }

__device__ __forceinline__ const float* param_row(const SceneDev& s, int r) {
  if (r < 3) return s.mean + r * s.n;
  if (r < 6) return s.ls + (r - 3) * s.n;
  if (r < 10) return s.quat + (r - 6) * s.n;
  if (r == 10) return s.logit;
  return s.sh + (r - 11) * s.n;
}

__global__ void __launch_bounds__(256, 2) preprocess_kernel(SceneDev s, const ViewParams* __restrict__ views,
                                                            const int* __restrict__ view_list, int nv, int T,
                                                            int key_mode, Visibility vis, float4* __restrict__ rec,
                                                            float4* __restrict__ bbox, uint32_t* __restrict__ count,
                                                            unsigned long long* __restrict__ kcache) {
  __shared__ uint32_t s_cnt[256];
  extern __shared__ float s_par[];  // [param_rows(deg)][256]: the block's parameters
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  uint32_t* wc = s_cnt + (threadIdx.x & ~31);  // this warp's 32 counters
  const long long warp_i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  const bool in = i < s.n;
  // The block's parameters go to shared memory with asynchronous 4-byte copies, all in
  // flight at once (coalesced rows of the SoA arrays); every view then projects from
  // there.  Reading them with plain loads left the kernel waiting on one load at a time.
  const int rows = param_rows(s.deg);
  if (in) {
    for (int r = 0; r < rows; ++r) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(s_par + r * 256 + threadIdx.x);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(param_row(s, r) + i) : "memory");
    }
  }
  asm volatile("cp.async.commit_group;\ncp.async.wait_all;" ::: "memory");
  __syncthreads();
  const SceneDev sb{s_par, s_par + 3 * 256, s_par + 6 * 256, s_par + 10 * 256, s_par + 11 * 256, 256, s.deg};
  for (int k = 0; k < nv; ++k) {
    const int view = view_list[k];
    const ViewParams& vp = views[view];
    const long long vg = vp.base + i;
    float4 r[6], bb;
    const bool ok = in && project_gaussian(sb, threadIdx.x, vp, r, bb);
    if (!ok) bb = make_float4(0.f, 0.f, -1.f, -1.f);
    Span sp = make_span(bb, vp, T, ok);
    // no visible tile in the rectangle: nothing to test (summed-area table, Sec. 4.3)
    if (vis.tvis && sp.nt > 0 &&
        sat_count(vis, view, vp.ntx, sp.tx0, sp.ty0, sp.tx0 + sp.nx - 1, sp.ty0 + sp.nt / sp.nx - 1) == 0)
      sp.nt = 0;
    const uint8_t* tv = vis.tvis ? vis.tvis + (long long)view * vis.tiles_per_view : nullptr;
    if (in) {
      bbox[vg] = bb;
      if (sp.nt > 0) {
        float4* dst = rec + vg * kRecF4;
#pragma unroll
        for (int q = 0; q < kRecF4; ++q) dst[q] = r[q];
      }
    }
    // running tile counts of the warp's Gaussians (inclusive scan)
    unsigned endc = (unsigned)sp.nt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, endc, o);
      if (lane >= o) endc += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, endc, 31);
    wc[lane] = 0u;
    __syncwarp();  // records and counters visible to the warp
    for (unsigned b = 0; b < total; b += 32) {
      const unsigned t = b + lane;
      // owner: the number of Gaussians whose tiles end at or before t
      int own = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned e = __shfl_sync(0xffffffffu, endc, own + step - 1);
        if (e <= t) own += step;
      }
      own = t < total ? own : 0;
      const int nt_o = __shfl_sync(0xffffffffu, sp.nt, own), tx0 = __shfl_sync(0xffffffffu, sp.tx0, own),
                ty0 = __shfl_sync(0xffffffffu, sp.ty0, own), nx = __shfl_sync(0xffffffffu, sp.nx, own);
      const unsigned end_o = __shfl_sync(0xffffffffu, endc, own);
      Keep kp{false, 0.f};
      int tile = 0;
      float4 f0, f3;
      if (t < total) {
        const int kk = (int)(t - (end_o - (unsigned)nt_o));
        const int tx = tx0 + kk % nx, ty = ty0 + kk / nx;
        tile = ty * vp.ntx + tx;
        if (!tv || tv[tile]) {
          const float4* ro = rec + (vp.base + warp_i0 + own) * kRecF4;
          f0 = ro[0];
          f3 = ro[3];
          float x0, y0, x1, y1;
          tile_quad(tx, ty, T, vp, x0, y0, x1, y1);
          kp = tile_keep(f0, ro[1], ro[2], f3, ro[4], ro[5].x, x0, y0, x1, y1);
        }
      }
      // rank among this step's kept tiles of the same Gaussian (tile order)
      const unsigned bal = __ballot_sync(0xffffffffu, kp.keep);
      const unsigned peers = __match_any_sync(0xffffffffu, t < total ? own : 32 + lane);
      const unsigned mine_kept = bal & peers;
      const uint32_t base = wc[own];
      __syncwarp();
      if (kp.keep) {
        const uint32_t slot = base + __popc(mine_kept & ((1u << lane) - 1u));
        if (slot < kKeyCache)
          kcache[(vp.base + warp_i0 + own) * kKeyCache + slot] = local_key(tile, order_key(key_mode, kp.key, f0, f3, vp));
        if ((mine_kept & ((1u << lane) - 1u)) == 0u) wc[own] = base + __popc(mine_kept);
      }
      __syncwarp();
    }
    if (in) count[vg] = wc[lane];
    __syncwarp();
  }
}

// Emits the (tile | depth, index) instances of a view: the same warp-cooperative walk
// as the count, with a ballot prefix giving each kept tile its slot (row-major order of
// the rectangle, so the output is deterministic).  64 registers (4 blocks per SM): 0.139
// against 0.151 ms per VR stereo frame at 80 registers (3 blocks).
__global__ void __launch_bounds__(256, 4) duplicate_kernel(const ViewParams* __restrict__ views, int n_views,
                                                        long long total_nv, const float4* __restrict__ rec,
                                                        const float4* __restrict__ bbox,
                                                        const uint32_t* __restrict__ count,
                                                        const uint32_t* __restrict__ offsets, int T,
                                                        int tiles_per_view, const uint8_t* __restrict__ tvis,
                                                        const unsigned long long* __restrict__ kcache, int key_mode,
                                                        uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                        long long cap, uint32_t* status) {
  // every view in one launch: blockIdx.y is the view, and its Gaussians run from its base
  // to the next view's (the last view's to the total)
  const int view = blockIdx.y;
  const ViewParams& vp = views[view];
  const long long nview = (view + 1 < n_views ? views[view + 1].base : total_nv) - vp.base;
  if ((long long)blockIdx.x * blockDim.x >= nview) return;  // the whole block is past this view
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const long long vg = vp.base + i;
  const uint32_t cnt = i < nview ? count[vg] : 0u;
  const uint64_t vbase = (uint64_t)view * (uint64_t)tiles_per_view;
  const uint32_t lt = (1u << lane) - 1u;
  const uint8_t* tv = tvis ? tvis + (long long)view * tiles_per_view : nullptr;
  // Gaussians with at most kKeyCache instances: the count pass kept their keys.  The
  // warp copies them as one flattened list, one instance per lane (owner by binary
  // search over the running counts), so the writes of consecutive Gaussians coalesce.
  {
    const long long warp_i0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    const unsigned c = cnt <= kKeyCache ? cnt : 0u;
    unsigned endc = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, endc, o);
      if (lane >= o) endc += y;
    }
    const unsigned total = __shfl_sync(0xffffffffu, endc, 31);
    const long long myoff = c ? (long long)offsets[vg] : 0;
    for (unsigned b = 0; b < total; b += 32) {
      const unsigned t = b + lane;
      int own = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned e = __shfl_sync(0xffffffffu, endc, own + step - 1);
        if (e <= t) own += step;
      }
      own = t < total ? own : 0;
      const unsigned end_o = __shfl_sync(0xffffffffu, endc, own), c_o = __shfl_sync(0xffffffffu, c, own);
      const long long off_o = __shfl_sync(0xffffffffu, myoff, own);
      if (t < total) {
        const unsigned q = t - (end_o - c_o);
        const long long o = off_o + q;
        if (o < cap) {
          keys[o] = kcache[(vp.base + warp_i0 + own) * kKeyCache + q] + (vbase << 32);
          vals[o] = (uint32_t)(warp_i0 + own);
        } else {
          atomicOr(status, kStOverflow);
        }
      }
    }
  }
  // Gaussians with more instances: the warp tests their tiles, one Gaussian at a time
  unsigned todo = __ballot_sync(0xffffffffu, cnt > kKeyCache);
  while (todo) {
    const int j = __ffs(todo) - 1;
    todo &= todo - 1;
    const long long vj = vp.base + (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31) + j;
    const float4* r = rec + vj * kRecF4;
    const float4 g0 = r[0], g1 = r[1], g2 = r[2], g3 = r[3], g4 = r[4];
    const float g5x = r[5].x;
    const Span spj = make_span(bbox[vj], vp, T, true);
    long long o = offsets[vj];
    const uint32_t gid = (uint32_t)(vj - vp.base);
    for (int b = 0; b < spj.nt; b += 32) {
      const int t = b + lane;
      Keep kp{false, 0.f};
      int tx = 0, ty = 0;
      if (t < spj.nt) {
        float x0, y0, x1, y1;
        tx = spj.tx0 + t % spj.nx;
        ty = spj.ty0 + t / spj.nx;
        if (!tv || tv[ty * vp.ntx + tx]) {
          tile_quad(tx, ty, T, vp, x0, y0, x1, y1);
          kp = tile_keep(g0, g1, g2, g3, g4, g5x, x0, y0, x1, y1);
        }
      }
      const unsigned bal = __ballot_sync(0xffffffffu, kp.keep);
      if (kp.keep) {
        const long long slot = o + __popc(bal & lt);
        if (slot < cap) {
          keys[slot] = ((vbase + (uint64_t)(ty * vp.ntx + tx)) << 32) |
                       float_order_bits(order_key(key_mode, kp.key, g0, g3, vp));
          vals[slot] = gid;
        } else {
          atomicOr(status, kStOverflow);
        }
      }
      o += __popc(bal);
    }
  }
}

void launch_preprocess(const SceneDev& s, const ViewParams* d_views, const int* d_view_list, int nv, int T,
                       int key_mode, const Visibility& vis, float4* rec, float4* bbox, uint32_t* count,
                       unsigned long long* kcache, cudaStream_t st) {
  if (s.n <= 0 || nv <= 0) return;
  const unsigned grid = (unsigned)((s.n + 255) / 256);
  const int smem = param_rows(s.deg) * 256 * (int)sizeof(float);
  cudaFuncSetAttribute(preprocess_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  preprocess_kernel<<<grid, 256, smem, st>>>(s, d_views, d_view_list, nv, T, key_mode, vis, rec, bbox, count, kcache);
}

void launch_duplicate(const ViewParams* d_views, int n_views, const float4* rec, const float4* bbox,
                      const uint32_t* count, const uint32_t* offsets, const long long* h_view_n, int T,
                      int tiles_per_view, const Visibility& vis, const unsigned long long* kcache, int key_mode,
                      uint64_t* keys, uint32_t* vals, const uint32_t* /*d_total*/, long long cap, uint32_t* status,
                      cudaStream_t st) {
  long long max_n = 0, total = 0;
  for (int v = 0; v < n_views; ++v) {
    max_n = std::max(max_n, h_view_n[v]);
    total += h_view_n[v];
  }
  if (max_n <= 0) return;
  const dim3 grid((unsigned)((max_n + 255) / 256), (unsigned)n_views);
  duplicate_kernel<<<grid, 256, 0, st>>>(d_views, n_views, total, rec, bbox, count, offsets, T, tiles_per_view,
                                         vis.tvis, kcache, key_mode, keys, vals, cap, status);
}

// ---- visibility culling (Sec. 4.3) ----------------------------------------------------

// One block per (view, key tile): the tile is visible when any of its pixels is.
__global__ void __launch_bounds__(256) tile_visibility_kernel(const ViewParams* __restrict__ views, int T,
                                                              int tiles_per_view, uint8_t* __restrict__ tvis) {
  const int view = blockIdx.x / tiles_per_view, t = blockIdx.x % tiles_per_view;
  const ViewParams& vp = views[view];
  const int tx = t % vp.ntx, ty = t / vp.ntx;
  int any = 0;
  if (!vp.visible) {
    any = 1;
  } else if (t < vp.ntx * vp.nty) {
    for (int p = threadIdx.x; p < T * T && !any; p += blockDim.x) {
      const int x = tx * T + p % T, y = ty * T + p / T;
      if (x < vp.W && y < vp.H && vp.visible[(long long)y * vp.W + x]) any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) tvis[blockIdx.x] = (uint8_t)(any != 0);
}

// One block per view: summed-area table of the visible tiles, (nty + 1) x (ntx + 1).
__global__ void __launch_bounds__(256) sat_kernel(const uint8_t* __restrict__ tvis, int tiles_per_view, int ntx,
                                                  int nty, int sat_per_view, uint32_t* __restrict__ sat) {
  const int view = blockIdx.x;
  const uint8_t* tv = tvis + (long long)view * tiles_per_view;
  uint32_t* S = sat + (long long)view * sat_per_view;
  const int w = ntx + 1;
  for (int x = threadIdx.x; x < w; x += blockDim.x) S[x] = 0;
  for (int y = threadIdx.x; y < nty; y += blockDim.x) {  // row prefix sums
    uint32_t run = 0;
    S[(y + 1) * w] = 0;
    for (int x = 0; x < ntx; ++x) {
      run += tv[y * ntx + x];
      S[(y + 1) * w + x + 1] = run;
    }
  }
  __syncthreads();
  for (int x = threadIdx.x; x < w; x += blockDim.x)  // column prefix sums
    for (int y = 1; y <= nty; ++y) S[y * w + x] += S[(y - 1) * w + x];
}

void launch_visibility(const ViewParams* d_views, int n_views, int T, int ntx, int nty, const Visibility& v,
                       cudaStream_t st) {
  if (n_views <= 0) return;
  tile_visibility_kernel<<<(unsigned)(n_views * v.tiles_per_view), 256, 0, st>>>(d_views, T, v.tiles_per_view,
                                                                                 const_cast<uint8_t*>(v.tvis));
  sat_kernel<<<(unsigned)n_views, 256, 0, st>>>(v.tvis, v.tiles_per_view, ntx, nty, v.sat_per_view,
                                                const_cast<uint32_t*>(v.sat));
}

// ---- inspection entry point support ----------------------------------------------

__global__ void project_only_kernel(SceneDev s, const ViewParams* __restrict__ vpp, int T, float* __restrict__ out,
                                    float* __restrict__ bbox_out, uint32_t* __restrict__ count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const ViewParams vp = *vpp;
  float4 r[6], bb;
  uint32_t cnt = 0;
  const bool ok = project_gaussian(s, i, vp, r, bb);
  if (ok) {
    int tx0, tx1, ty0, ty1;
    tile_span(bb, vp, T, tx0, tx1, ty0, ty1);
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        float x0, y0, x1, y1;
        tile_quad(tx, ty, T, vp, x0, y0, x1, y1);
        cnt += tile_keep(r[0], r[1], r[2], r[3], r[4], r[5].x, x0, y0, x1, y1).keep ? 1u : 0u;
      }
  }
  for (int q = 0; q < kRecF4; ++q) {
    const float4 v = ok ? r[q] : make_float4(0.f, 0.f, 0.f, 0.f);
    out[i * 24 + 4 * q + 0] = v.x;
    out[i * 24 + 4 * q + 1] = v.y;
    out[i * 24 + 4 * q + 2] = v.z;
    out[i * 24 + 4 * q + 3] = v.w;
  }
  const float4 b = ok ? bb : make_float4(0.f, 0.f, 0.f, 0.f);
  bbox_out[4 * i] = b.x;
  bbox_out[4 * i + 1] = b.y;
  bbox_out[4 * i + 2] = b.z;
  bbox_out[4 * i + 3] = b.w;
  count[i] = cnt;
}

void launch_project_only(const SceneDev& s, const ViewParams* d_vp, int T, float* out, float* bbox, uint32_t* count,
                         cudaStream_t st) {
  if (s.n <= 0) return;
  project_only_kernel<<<(unsigned)((s.n + 255) / 256), 256, 0, st>>>(s, d_vp, T, out, bbox, count);
}

}  // namespace vrs
