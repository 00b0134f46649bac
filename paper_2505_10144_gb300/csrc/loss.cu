// Fine-tuning loss (Sec. 5: 3DGS-style objective) 0.8 L1 + 0.2 (1 - SSIM) and its image
// gradient, plus the Adam update.  SSIM (Wang et al. 2004): 11x11 Gaussian window,
// sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, zero padding, mean over pixels and channels.
// All five window statistics come from two separable passes; the gradient is the
// adjoint (the same symmetric filter) of three per-pixel partial-derivative maps.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace vrs {

namespace {

constexpr int kWin = 11;
constexpr int kR = 5;
constexpr float kC1 = 0.0001f;
constexpr float kC2 = 0.0009f;

struct Win {
  float g[kWin];
};

Win make_window() {
  Win w;
  double s = 0, v[kWin];
  for (int k = 0; k < kWin; ++k) {
    const double x = k - kR;
    v[k] = exp(-x * x / (2.0 * 1.5 * 1.5));
    s += v[k];
  }
  for (int k = 0; k < kWin; ++k) w.g[k] = (float)(v[k] / s);
  return w;
}

// horizontal pass of x, y, x^2, y^2, xy over every plane (image * channel)
__global__ void ssim_h_kernel(const float* __restrict__ x, const float* __restrict__ y, long long planes, int H, int W,
                              Win w, float* __restrict__ out /*[5][planes][H][W]*/) {
  const long long HW = (long long)H * W, tot = planes * HW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long pl = i / HW;
    const int r = (int)((i % HW) / W), c = (int)(i % W);
    const float* xr = x + pl * HW + (long long)r * W;
    const float* yr = y + pl * HW + (long long)r * W;
    float a = 0, b = 0, aa = 0, bb = 0, ab = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int cc = c + k - kR;
      if (cc < 0 || cc >= W) continue;
      const float xv = xr[cc], yv = yr[cc], g = w.g[k];
      a = fmaf(g, xv, a);
      b = fmaf(g, yv, b);
      aa = fmaf(g, xv * xv, aa);
      bb = fmaf(g, yv * yv, bb);
      ab = fmaf(g, xv * yv, ab);
    }
    out[i] = a;
    out[tot + i] = b;
    out[2 * tot + i] = aa;
    out[3 * tot + i] = bb;
    out[4 * tot + i] = ab;
  }
}

// vertical pass, SSIM map and its partial derivatives; accumulates sum S and sum |x - y|
__global__ void ssim_v_kernel(const float* __restrict__ hbuf, const float* __restrict__ x, const float* __restrict__ y,
                              long long planes, int H, int W, Win w, float* __restrict__ dmaps /*[3][planes][H][W]*/,
                              double* __restrict__ sums) {
  const long long HW = (long long)H * W, tot = planes * HW;
  double ls = 0, l1 = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long pl = i / HW;
    const int r = (int)((i % HW) / W), c = (int)(i % W);
    float m[5] = {0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int rr = r + k - kR;
      if (rr < 0 || rr >= H) continue;
      const long long j = pl * HW + (long long)rr * W + c;
      const float g = w.g[k];
#pragma unroll
      for (int q = 0; q < 5; ++q) m[q] = fmaf(g, hbuf[q * tot + j], m[q]);
    }
    const float m1 = m[0], m2 = m[1];
    const float A1 = 2.f * m1 * m2 + kC1, A2 = 2.f * (m[4] - m1 * m2) + kC2;
    const float B1 = m1 * m1 + m2 * m2 + kC1, B2 = (m[2] - m1 * m1) + (m[3] - m2 * m2) + kC2;
    const float iB = 1.f / (B1 * B2);
    const float S = A1 * A2 * iB;
    ls += S;
    l1 += fabsf(x[i] - y[i]);
    if (dmaps) {
      dmaps[i] = 2.f * m2 * (A2 - A1) * iB - 2.f * m1 * S * (1.f / B1 - 1.f / B2);  // dS/dm1
      dmaps[tot + i] = -S / B2;                                                       // dS/dm11
      dmaps[2 * tot + i] = 2.f * A1 * iB;                                             // dS/dm12
    }
  }
  // block reduction of the two sums
  __shared__ double sh[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    ls += __shfl_xor_sync(0xffffffffu, ls, o);
    l1 += __shfl_xor_sync(0xffffffffu, l1, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = ls;
    sh[1][wid] = l1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      a += sh[0][k];
      b += sh[1][k];
    }
    atomicAdd(&sums[0], a);
    atomicAdd(&sums[1], b);
  }
}

__global__ void grad_h_kernel(const float* __restrict__ dmaps, long long planes, int H, int W, Win w,
                              float* __restrict__ out) {
  const long long HW = (long long)H * W, tot = planes * HW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long rowbase = i - (i % W);
    const int c = (int)(i % W);
    float a = 0, b = 0, e = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int cc = c + k - kR;
      if (cc < 0 || cc >= W) continue;
      const float g = w.g[k];
      a = fmaf(g, dmaps[rowbase + cc], a);
      b = fmaf(g, dmaps[tot + rowbase + cc], b);
      e = fmaf(g, dmaps[2 * tot + rowbase + cc], e);
    }
    out[i] = a;
    out[tot + i] = b;
    out[2 * tot + i] = e;
  }
}

__global__ void grad_v_kernel(const float* __restrict__ hbuf, const float* __restrict__ x, const float* __restrict__ y,
                              long long planes, int H, int W, Win w, float scale_l1, float scale_ssim,
                              float* __restrict__ grad) {
  const long long HW = (long long)H * W, tot = planes * HW;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
    const long long pl = i / HW;
    const int r = (int)((i % HW) / W), c = (int)(i % W);
    float a = 0, b = 0, e = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int rr = r + k - kR;
      if (rr < 0 || rr >= H) continue;
      const long long j = pl * HW + (long long)rr * W + c;
      const float g = w.g[k];
      a = fmaf(g, hbuf[j], a);
      b = fmaf(g, hbuf[tot + j], b);
      e = fmaf(g, hbuf[2 * tot + j], e);
    }
    const float xv = x[i], yv = y[i];
    const float dS = a + 2.f * xv * b + yv * e;
    const float sg = xv > yv ? 1.f : (xv < yv ? -1.f : 0.f);
    grad[i] = scale_l1 * sg - scale_ssim * dS;
  }
}

__global__ void loss_finalize_kernel(const double* __restrict__ sums, double count, float* __restrict__ loss) {
  *loss = (float)(0.8 * sums[1] / count + 0.2 * (1.0 - sums[0] / count));
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, long long n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

unsigned grid_for(long long n) {
  return (unsigned)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 16);
}

}  // namespace

size_t loss_scratch_bytes(int n, int H, int W) {
  const size_t tot = (size_t)n * 3 * H * W;
  return tot * sizeof(float) * 8 + 64;
}

vrs_status loss_l1_ssim_impl(const float* img, const float* tgt, int n, int H, int W, float* loss, float* grad,
                             void* scratch, size_t scratch_bytes, cudaStream_t st) {
  const long long planes = 3ll * n, tot = planes * H * W;
  if (scratch_bytes < loss_scratch_bytes(n, H, W)) return VRS_ERR_CAPACITY;
  double* sums = reinterpret_cast<double*>(scratch);
  float* hbuf = reinterpret_cast<float*>(reinterpret_cast<char*>(scratch) + 64);  // 5 planes
  float* dmaps = hbuf + 5 * tot;                                                  // 3 planes
  const Win w = make_window();
  cudaMemsetAsync(sums, 0, 2 * sizeof(double), st);
  ssim_h_kernel<<<grid_for(tot), 256, 0, st>>>(img, tgt, planes, H, W, w, hbuf);
  ssim_v_kernel<<<grid_for(tot), 256, 0, st>>>(hbuf, img, tgt, planes, H, W, w, grad ? dmaps : nullptr, sums);
  loss_finalize_kernel<<<1, 1, 0, st>>>(sums, (double)tot, loss);
  if (grad) {
    grad_h_kernel<<<grid_for(tot), 256, 0, st>>>(dmaps, planes, H, W, w, hbuf);
    grad_v_kernel<<<grid_for(tot), 256, 0, st>>>(hbuf, img, tgt, planes, H, W, w, (float)(0.8 / tot),
                                                 (float)(0.2 / tot), grad);
  }
  return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}

}  // namespace vrs

extern "C" vrs_status vrs_adam_step(float* d_param, const float* d_grad, float* d_m, float* d_v, int64_t n, float lr,
                                    float beta1, float beta2, float eps, int step, void* stream) {
  if (n < 0 || step < 1 || (n > 0 && (!d_param || !d_grad || !d_m || !d_v))) return VRS_ERR_INVALID;
  if (n == 0) return VRS_OK;
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  vrs::adam_kernel<<<vrs::grid_for(n), 256, 0, (cudaStream_t)stream>>>(d_param, d_grad, d_m, d_v, n, lr, beta1, beta2,
                                                                      eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
