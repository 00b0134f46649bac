// Backward of the render (fine-tuning through the StopThePop + Optimal-Projection
// rasterizer, Sec. 4.1 / 4.2): composite backward (focus, hybrid blend, bilinear
// periphery) to per-sample dL/dC, and the chain from per-(view, Gaussian) record
// gradients back to the Gaussian parameters.  Sorting, culling, windowing and the depth
// t* are piecewise constant and carry no gradient.
#include <algorithm>

#include "common.cuh"

namespace vrs {

namespace {

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

// SH basis (3DGS convention) and its gradient with respect to the direction
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16], float dY[16][3]) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    Y[k] = 0.f;
    dY[k][0] = dY[k][1] = dY[k][2] = 0.f;
  }
  Y[0] = kY0;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  dY[1][1] = -kY1;
  Y[2] = kY1 * z;
  dY[2][2] = kY1;
  Y[3] = -kY1 * x;
  dY[3][0] = -kY1;
  if (deg < 2) return;
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  dY[4][0] = kY2a * y;
  dY[4][1] = kY2a * x;
  Y[5] = -kY2a * y * z;
  dY[5][1] = -kY2a * z;
  dY[5][2] = -kY2a * y;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  dY[6][0] = -2.f * kY2b * x;
  dY[6][1] = -2.f * kY2b * y;
  dY[6][2] = 4.f * kY2b * z;
  Y[7] = -kY2a * x * z;
  dY[7][0] = -kY2a * z;
  dY[7][2] = -kY2a * x;
  Y[8] = kY2c * (xx - yy);
  dY[8][0] = 2.f * kY2c * x;
  dY[8][1] = -2.f * kY2c * y;
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  dY[9][0] = -kY3a * 6.f * x * y;
  dY[9][1] = -kY3a * (3.f * xx - 3.f * yy);
  Y[10] = kY3b * x * y * z;
  dY[10][0] = kY3b * y * z;
  dY[10][1] = kY3b * x * z;
  dY[10][2] = kY3b * x * y;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  dY[11][0] = kY3c * 2.f * x * y;
  dY[11][1] = -kY3c * (4.f * zz - xx - 3.f * yy);
  dY[11][2] = -kY3c * 8.f * y * z;
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  dY[12][0] = -kY3d * 6.f * x * z;
  dY[12][1] = -kY3d * 6.f * y * z;
  dY[12][2] = kY3d * (6.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  dY[13][0] = -kY3c * (4.f * zz - 3.f * xx - yy);
  dY[13][1] = kY3c * 2.f * x * y;
  dY[13][2] = -kY3c * 8.f * x * z;
  Y[14] = kY3e * z * (xx - yy);
  dY[14][0] = kY3e * 2.f * x * z;
  dY[14][1] = -kY3e * 2.f * y * z;
  dY[14][2] = kY3e * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
  dY[15][0] = -kY3a * (3.f * xx - 3.f * yy);
  dY[15][1] = kY3a * 6.f * x * y;
}

// Per pixel: dL/dout -> dL/d(sample value) for focus and plain pixels, the w-weighted
// share of hybrid pixels, and the (1 - w) share that goes to the pixel's 2x2 average.
__global__ void composite_bwd_pixels(const ViewParams* __restrict__ views, int n_views, const uint8_t* __restrict__ cls,
                                     int tiles_per_view, int T, int fovea_mode, const float* __restrict__ dout, int W,
                                     int H, float4* __restrict__ dfull, float4* __restrict__ dhyb) {
  const long long HW = (long long)W * H, total = HW * n_views;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int view = (int)(i / HW);
    const long long r = i % HW;
    const int y = (int)(r / W), x = (int)(r % W);
    const float* g = dout + (long long)view * 3 * HW + r;
    const float g0 = g[0], g1 = g[HW], g2 = g[2 * HW];
    if (fovea_mode == 0) {
      dfull[i] = make_float4(g0, g1, g2, 0.f);
      continue;
    }
    const ViewParams& vp = views[view];
    const int c = cls[(long long)view * tiles_per_view + (y / T) * vp.ntx + x / T];
    if (c == kClassFocus) {
      dfull[i] = make_float4(g0, g1, g2, 0.f);
      dhyb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else if (c == kClassHybrid) {
      const float dx = x + 0.5f - vp.gaze_x, dy = y + 0.5f - vp.gaze_y;
      const float w = fminf(fmaxf((vp.radius + vp.band - sqrtf(dx * dx + dy * dy)) / vp.band, 0.f), 1.f);
      dfull[i] = make_float4(w * g0, w * g1, w * g2, 0.f);
      dhyb[i] = make_float4((1.f - w) * g0, (1.f - w) * g1, (1.f - w) * g2, 0.f);
    } else {
      dfull[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      dhyb[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Per 2x2 group: gathers the bilinear weights of every periphery pixel that reads the
// group (deterministic, no atomics); periphery groups receive it as their sample
// gradient, focus / hybrid groups pass it (and the hybrid averages) to their 4 pixels.
__global__ void composite_bwd_groups(const ViewParams* __restrict__ views, int n_views, const uint8_t* __restrict__ cls,
                                     int tiles_per_view, int T, const float* __restrict__ dout, int W, int H,
                                     float4* __restrict__ dfull, const float4* __restrict__ dhyb,
                                     float4* __restrict__ dlow) {
  const int W2 = W / 2, H2 = H / 2;
  const long long HW = (long long)W * H, HW2 = (long long)W2 * H2, total = HW2 * n_views;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    const int view = (int)(i / HW2);
    const long long r = i % HW2;
    const int gy = (int)(r / W2), gx = (int)(r % W2);
    const ViewParams& vp = views[view];
    const uint8_t* vc = cls + (long long)view * tiles_per_view;
    const float* g = dout + (long long)view * 3 * HW;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int y = max(2 * gy - 2, 0); y <= min(2 * gy + 3, H - 1); ++y) {
      const float uy = (y + 0.5f) * 0.5f - 0.5f;
      const int y0 = (int)floorf(uy);
      const float fy = uy - y0;
      const int ya = min(max(y0, 0), H2 - 1), yb = min(max(y0 + 1, 0), H2 - 1);
      const float wy = (ya == gy ? 1.f - fy : 0.f) + (yb == gy ? fy : 0.f);
      if (wy == 0.f) continue;
      for (int x = max(2 * gx - 2, 0); x <= min(2 * gx + 3, W - 1); ++x) {
        if (vc[(y / T) * vp.ntx + x / T] != kClassPeriphery) continue;
        const float ux = (x + 0.5f) * 0.5f - 0.5f;
        const int x0 = (int)floorf(ux);
        const float fx = ux - x0;
        const int xa = min(max(x0, 0), W2 - 1), xb = min(max(x0 + 1, 0), W2 - 1);
        const float wx = (xa == gx ? 1.f - fx : 0.f) + (xb == gx ? fx : 0.f);
        const float wgt = wx * wy;
        if (wgt == 0.f) continue;
        const long long p = (long long)y * W + x;
        s0 = fmaf(wgt, g[p], s0);
        s1 = fmaf(wgt, g[HW + p], s1);
        s2 = fmaf(wgt, g[2 * HW + p], s2);
      }
    }
    if (vc[((2 * gy) / T) * vp.ntx + (2 * gx) / T] == kClassPeriphery) {
      dlow[i] = make_float4(s0, s1, s2, 0.f);
    } else {
      const long long base = (long long)view * HW + (long long)(2 * gy) * W + 2 * gx;
      const long long px[4] = {base, base + 1, base + W, base + W + 1};
      float h0 = s0, h1 = s1, h2 = s2;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float4 hv = dhyb[px[k]];
        h0 += hv.x;
        h1 += hv.y;
        h2 += hv.z;
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float4 v = dfull[px[k]];
        v.x = fmaf(0.25f, h0, v.x);
        v.y = fmaf(0.25f, h1, v.y);
        v.z = fmaf(0.25f, h2, v.z);
        dfull[px[k]] = v;
      }
    }
  }
}

// Record gradients -> parameter gradients (chain through the Optimal Projection of
// project_gaussian: pm, plane map rows [E; u] K^-1, conic A' = 0.5 log2(e) Sigma_p^-1,
// log2 sigma, SH colour).  One thread per Gaussian sums over the views of its scene.
__global__ void __launch_bounds__(128) preprocess_bwd_kernel(SceneDev s, const ViewParams* __restrict__ views,
                                                              const int* __restrict__ view_list, int nv,
                                                              const uint32_t* __restrict__ count,
                                                              const float* __restrict__ grad_rec,
                                                              vrs_gaussian_grads out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const long long n = s.n;
  const float mw[3] = {s.mean[i], s.mean[n + i], s.mean[2 * n + i]};
  const float ls[3] = {s.ls[i], s.ls[n + i], s.ls[2 * n + i]};
  const float q4[4] = {s.quat[i], s.quat[n + i], s.quat[2 * n + i], s.quat[3 * n + i]};
  const float qn = sqrtf(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
  if (!(qn > 0.f) || !isfinite(qn)) return;
  const float qw = q4[0] / qn, qx = q4[1] / qn, qy = q4[2] / qn, qz = q4[3] / qn;
  const float G[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy),
                      2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx),
                      2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)};
  const float s2[3] = {expf(2.f * ls[0]), expf(2.f * ls[1]), expf(2.f * ls[2])};
  const float sigma = 1.f / (1.f + expf(-s.logit[i]));
  const int K = (s.deg + 1) * (s.deg + 1);
  float gmw[3] = {0.f, 0.f, 0.f}, gs2[3] = {0.f, 0.f, 0.f}, gG[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float glogit = 0.f;
  float gsh[16][3];
#pragma unroll
  for (int k = 0; k < 16; ++k) gsh[k][0] = gsh[k][1] = gsh[k][2] = 0.f;
  bool any = false;
  for (int kv = 0; kv < nv; ++kv) {
    const ViewParams& vp = views[view_list[kv]];
    const long long vg = vp.base + i;
    if (count[vg] == 0) continue;
    any = true;
    const float* gr = grad_rec + vg * 16;
    float gv[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) gv[k] = gr[k];
    const float* R = vp.R;
    const float mx = fmaf(R[0], mw[0], fmaf(R[1], mw[1], fmaf(R[2], mw[2], vp.t[0])));
    const float my = fmaf(R[3], mw[0], fmaf(R[4], mw[1], fmaf(R[5], mw[2], vp.t[1])));
    const float mz = fmaf(R[6], mw[0], fmaf(R[7], mw[1], fmaf(R[8], mw[2], vp.t[2])));
    const float d = sqrtf(mx * mx + my * my + mz * mz);
    const float u[3] = {mx / d, my / d, mz / d};
    const float rho = sqrtf(u[0] * u[0] + u[2] * u[2]);
    const float e1[3] = {u[2] / rho, 0.f, -u[0] / rho};
    const float e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
    float Rc[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) Rc[3 * a + b] = R[3 * a] * G[b] + R[3 * a + 1] * G[3 + b] + R[3 * a + 2] * G[6 + b];
    float Sc[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        Sc[3 * a + b] = Rc[3 * a] * s2[0] * Rc[3 * b] + Rc[3 * a + 1] * s2[1] * Rc[3 * b + 1] +
                        Rc[3 * a + 2] * s2[2] * Rc[3 * b + 2];
    const float* E[2] = {e1, e2};
    float ScE[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) ScE[a][r] = Sc[3 * r] * E[a][0] + Sc[3 * r + 1] * E[a][1] + Sc[3 * r + 2] * E[a][2];
    const float id2 = 1.f / (d * d);
    const float dil = kDilationPx2 / (vp.fx * vp.fy);
    float Pm[2][2];  // Sigma_p - dilation
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) Pm[a][b] = (E[a][0] * ScE[b][0] + E[a][1] * ScE[b][1] + E[a][2] * ScE[b][2]) * id2;
    const float p00 = Pm[0][0] + dil, p01 = Pm[0][1], p11 = Pm[1][1] + dil;
    const float det = p00 * p11 - p01 * p01;
    const float Ai[2][2] = {{p11 / det, -p01 / det}, {-p01 / det, p00 / det}};  // Sigma_p^-1
    // ---- colour
    float gu[3] = {0.f, 0.f, 0.f}, gm[3] = {0.f, 0.f, 0.f};
    {
      const float dx = R[0] * u[0] + R[3] * u[1] + R[6] * u[2];
      const float dy = R[1] * u[0] + R[4] * u[1] + R[7] * u[2];
      const float dz = R[2] * u[0] + R[5] * u[1] + R[8] * u[2];
      float Y[16], dY[16][3];
      sh_basis_grad(s.deg, dx, dy, dz, Y, dY);
      float gdir[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float v = 0.5f;
#pragma unroll
        for (int k = 0; k < 16; ++k)
          if (k < K) v = fmaf(Y[k], s.sh[((long long)k * 3 + c) * n + i], v);
        const float gc = v > 0.f ? gv[13 + c] : 0.f;
        if (gc == 0.f) continue;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          if (k >= K) continue;
          gsh[k][c] += Y[k] * gc;
          const float shv = s.sh[((long long)k * 3 + c) * n + i] * gc;
          gdir[0] += dY[k][0] * shv;
          gdir[1] += dY[k][1] * shv;
          gdir[2] += dY[k][2] * shv;
        }
      }
      // dir = R^T u  ->  dL/du = R dL/ddir
#pragma unroll
      for (int a = 0; a < 3; ++a) gu[a] += R[3 * a] * gdir[0] + R[3 * a + 1] * gdir[1] + R[3 * a + 2] * gdir[2];
    }
    // ---- opacity: log2 sigma = -log2(1 + e^-logit)
    glogit += gv[12] * (1.f - sigma) / kLn2;
    // ---- conic A' = k Sigma_p^-1  ->  dL/dSigma_p = -k Ai G_A' Ai
    const float GA[2][2] = {{gv[9], gv[10]}, {gv[10], gv[11]}};
    float T1[2][2], GP[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) T1[a][b] = Ai[a][0] * GA[0][b] + Ai[a][1] * GA[1][b];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) GP[a][b] = -kHalfLog2e * (T1[a][0] * Ai[0][b] + T1[a][1] * Ai[1][b]);
    // Sigma_p = E Sc E^T / d^2 + dil
    float gSc[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c2 = 0; c2 < 3; ++c2) {
        float acc = 0.f;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int b = 0; b < 2; ++b) acc += GP[a][b] * E[a][r] * E[b][c2];
        gSc[3 * r + c2] = acc * id2;
      }
    float ge[2][3];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int r = 0; r < 3; ++r) ge[a][r] = 2.f * id2 * (GP[a][0] * ScE[0][r] + GP[a][1] * ScE[1][r]);
    float gd = 0.f;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) gd += GP[a][b] * Pm[a][b];
    gd *= -2.f / d;
    // ---- plane-map rows: h00 = e1x/fx, h10 = e2x/fx, h11 = e2y/fy, h20 = ux/fx, h21 = uy/fy, h22 = 1/uz
    ge[0][0] += gv[2] / vp.fx;
    ge[1][0] += gv[4] / vp.fx;
    ge[1][1] += gv[5] / vp.fy;
    gu[0] += gv[6] / vp.fx;
    gu[1] += gv[7] / vp.fy;
    gu[2] += -gv[8] / (u[2] * u[2]);
    // ---- projected mean pm = (fx mx/mz + cx, fy my/mz + cy)
    gm[0] += gv[0] * vp.fx / mz;
    gm[1] += gv[1] * vp.fy / mz;
    gm[2] += -(gv[0] * vp.fx * mx + gv[1] * vp.fy * my) / (mz * mz);
    // ---- e2 = u x e1
    gu[0] += e1[1] * ge[1][2] - e1[2] * ge[1][1];
    gu[1] += e1[2] * ge[1][0] - e1[0] * ge[1][2];
    gu[2] += e1[0] * ge[1][1] - e1[1] * ge[1][0];
    ge[0][0] += ge[1][1] * u[2] - ge[1][2] * u[1];
    ge[0][1] += ge[1][2] * u[0] - ge[1][0] * u[2];
    ge[0][2] += ge[1][0] * u[1] - ge[1][1] * u[0];
    // ---- e1 = (uz, 0, -ux) / rho
    {
      const float t = (ge[0][0] * u[0] + ge[0][2] * u[2]) / (rho * rho * rho);
      gu[0] += -u[2] * t;
      gu[2] += u[0] * t;
    }
    // ---- u = m / d, d = |m|
    const float ug = u[0] * gu[0] + u[1] * gu[1] + u[2] * gu[2];
#pragma unroll
    for (int a = 0; a < 3; ++a) gm[a] += (gu[a] - u[a] * ug) / d + u[a] * gd;
    // ---- m = R mw + t
#pragma unroll
    for (int a = 0; a < 3; ++a) gmw[a] += R[a] * gm[0] + R[3 + a] * gm[1] + R[6 + a] * gm[2];
    // ---- Sc = Rc diag(s2) Rc^T, Rc = R G
    float gRc[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        gRc[3 * a + k] =
            2.f * s2[k] * (gSc[3 * a] * Rc[k] + gSc[3 * a + 1] * Rc[3 + k] + gSc[3 * a + 2] * Rc[6 + k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      float acc = 0.f;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) acc += Rc[3 * a + k] * gSc[3 * a + b] * Rc[3 * b + k];
      gs2[k] += acc;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) gG[3 * a + b] += R[a] * gRc[b] + R[3 + a] * gRc[3 + b] + R[6 + a] * gRc[6 + b];
  }
  if (!any) return;
  // quaternion (normalised) from dL/dG
  const float gw = 2.f * (-qz * gG[1] + qy * gG[2] + qz * gG[3] - qx * gG[5] - qy * gG[6] + qx * gG[7]);
  const float gx = 2.f * (qy * gG[1] + qz * gG[2] + qy * gG[3] - 2.f * qx * gG[4] - qw * gG[5] + qz * gG[6] +
                          qw * gG[7] - 2.f * qx * gG[8]);
  const float gy = 2.f * (-2.f * qy * gG[0] + qx * gG[1] + qw * gG[2] + qx * gG[3] + qz * gG[5] - qw * gG[6] +
                          qz * gG[7] - 2.f * qy * gG[8]);
  const float gz = 2.f * (-2.f * qz * gG[0] - qw * gG[1] + qx * gG[2] + qw * gG[3] - 2.f * qz * gG[4] + qy * gG[5] +
                          qx * gG[6] + qy * gG[7]);
  const float dotq = qw * gw + qx * gx + qy * gy + qz * gz;
  out.quat[i] += (gw - qw * dotq) / qn;
  out.quat[n + i] += (gx - qx * dotq) / qn;
  out.quat[2 * n + i] += (gy - qy * dotq) / qn;
  out.quat[3 * n + i] += (gz - qz * dotq) / qn;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    out.mean[a * n + i] += gmw[a];
    out.log_scale[a * n + i] += 2.f * s2[a] * gs2[a];
  }
  out.opacity_logit[i] += glogit;
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    if (k >= K) continue;
#pragma unroll
    for (int c = 0; c < 3; ++c) out.sh[((long long)k * 3 + c) * n + i] += gsh[k][c];
  }
}

unsigned grid_for(long long n, int per = 16) {
  return (unsigned)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * per);
}

}  // namespace

void launch_composite_backward(const ViewParams* views, int n_views, const uint8_t* tile_class, int tiles_per_view,
                               int T, int fovea_mode, const float* dout, int W, int H, float4* dfull, float4* dhyb,
                               float4* dlow, cudaStream_t st) {
  const long long HW = (long long)W * H;
  composite_bwd_pixels<<<grid_for(HW * n_views), 256, 0, st>>>(views, n_views, tile_class, tiles_per_view, T,
                                                               fovea_mode, dout, W, H, dfull, dhyb);
  if (fovea_mode != 0)
    composite_bwd_groups<<<grid_for(HW / 4 * n_views), 256, 0, st>>>(views, n_views, tile_class, tiles_per_view, T,
                                                                      dout, W, H, dfull, dhyb, dlow);
}

void launch_preprocess_backward(const SceneDev& s, const ViewParams* d_views, const int* d_view_list, int nv,
                                const uint32_t* count, const float* grad_rec, const vrs_gaussian_grads& g,
                                cudaStream_t st) {
  if (s.n <= 0 || nv <= 0) return;
  preprocess_bwd_kernel<<<(unsigned)((s.n + 127) / 128), 128, 0, st>>>(s, d_views, d_view_list, nv, count, grad_rec, g);
}

}  // namespace vrs
