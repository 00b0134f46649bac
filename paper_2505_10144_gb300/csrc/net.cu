// Learned periphery reconstruction (the workload's replacement for Sec. 4.3's
// nearest-neighbour upsampling + 3x3 blur):
//   y = x + conv3(relu(conv2(relu(conv1(xin))))),  x = bilinear x2 of the half-resolution
//   image, xin = bf16(x), 3 -> 32 -> 32 -> 3 channels, 3x3 kernels, zero padding 1.
// Weights and activations are BF16 (round to nearest even), accumulation FP32.  Hidden
// activations are rounded after bias and ReLU.
//
// Parameters: one float32 buffer of kNetParams values, OIHW:
//   w1[32][3][3][3] b1[32] w2[32][32][3][3] b2[32] w3[3][32][3][3] b3[3]
// (float master weights; every kernel rounds them to BF16 when it loads them).
//
// Two kinds of kernels:
//  - training (any image size, activations saved for the backward): direct 3x3
//    convolutions in FP32 SIMT arithmetic on BF16 values, plus the data and weight
//    gradients;
//  - inference on the periphery tiles of a rendered frame: one fused tensor-core kernel
//    per 32x32 tile (mma.sync m16n8k16 bf16 -> f32, ldmatrix, swizzled shared memory),
//    all three layers in shared memory, reading the half-resolution image directly.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace vrs {

constexpr int kNetCh = 32;
constexpr int kW1 = 0, kB1 = 864, kW2 = 896, kB2 = 10112, kW3 = 10144, kB3 = 11008, kNetParams = 11011;

namespace {

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint16_t bf16bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ float bits2f(uint16_t u) {
  return __uint_as_float(((uint32_t)u) << 16);
}

// ------------------------------------------------------------------ training kernels

// One CTA = 16x16 output pixels of one image; input tile with a one-pixel halo in
// shared memory, weights in shared memory (BF16 values as float).  LAYER 1 reads the
// float input x (rounded to BF16), layers 2-3 read saved BF16 activations.  Layers 1-2
// write BF16(relu(.)), layer 3 writes x + conv + b3 in float.
template <int CIN, int COUT, int LAYER>
__global__ void __launch_bounds__(256) conv_fwd_kernel(const float* __restrict__ params, const float* __restrict__ x,
                                                       const uint16_t* __restrict__ act_in,
                                                       uint16_t* __restrict__ act_out, float* __restrict__ y, int H,
                                                       int W) {
  extern __shared__ __align__(16) float smf[];
  float(*in_s)[18][18] = reinterpret_cast<float(*)[18][18]>(smf);
  float(*w_s)[CIN * 9] = reinterpret_cast<float(*)[CIN * 9]>(smf + CIN * 324);
  float* b_s = smf + CIN * 324 + COUT * CIN * 9;
  const int woff = LAYER == 1 ? kW1 : (LAYER == 2 ? kW2 : kW3);
  const int boff = LAYER == 1 ? kB1 : (LAYER == 2 ? kB2 : kB3);
  for (int k = threadIdx.x; k < COUT * CIN * 9; k += 256) w_s[k / (CIN * 9)][k % (CIN * 9)] = bf16r(params[woff + k]);
  if (threadIdx.x < COUT) b_s[threadIdx.x] = params[boff + threadIdx.x];
  const int img = blockIdx.z;
  const int ox = blockIdx.x * 16, oy = blockIdx.y * 16;
  const long long HW = (long long)H * W;
  for (int k = threadIdx.x; k < CIN * 324; k += 256) {
    const int c = k / 324, r = k % 324, iy = oy - 1 + r / 18, ix = ox - 1 + r % 18;
    float v = 0.f;
    if (iy >= 0 && iy < H && ix >= 0 && ix < W) {
      const long long idx = ((long long)img * CIN + c) * HW + (long long)iy * W + ix;
      v = LAYER == 1 ? bf16r(x[idx]) : bits2f(act_in[idx]);
    }
    in_s[c][r / 18][r % 18] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int px = ox + tx, py = oy + ty;
  float acc[COUT];
#pragma unroll
  for (int o = 0; o < COUT; ++o) acc[o] = b_s[o];
  for (int c = 0; c < CIN; ++c)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float v = in_s[c][ty + k / 3][tx + k % 3];
#pragma unroll
      for (int o = 0; o < COUT; ++o) acc[o] = fmaf(w_s[o][c * 9 + k], v, acc[o]);
    }
  if (px >= W || py >= H) return;
  const long long p = (long long)py * W + px;
#pragma unroll
  for (int o = 0; o < COUT; ++o) {
    const long long idx = ((long long)img * COUT + o) * HW + p;
    if (LAYER == 3)
      y[idx] = x[idx] + acc[o];
    else
      act_out[idx] = bf16bits(fmaxf(acc[o], 0.f));
  }
}

// dIn = conv_transpose(dOut, W), then the ReLU mask of the input activation (layers 2,
// 3 inputs are post-ReLU BF16 activations: mask = act > 0).
template <int CIN, int COUT>
__global__ void __launch_bounds__(256) conv_bwd_data_kernel(const float* __restrict__ params, int woff,
                                                            const float* __restrict__ dout,
                                                            const uint16_t* __restrict__ act_in,
                                                            float* __restrict__ din, int H, int W) {
  extern __shared__ __align__(16) float smf[];
  float(*d_s)[18][18] = reinterpret_cast<float(*)[18][18]>(smf);
  float(*w_s)[CIN * 9] = reinterpret_cast<float(*)[CIN * 9]>(smf + COUT * 324);
  for (int k = threadIdx.x; k < COUT * CIN * 9; k += 256) w_s[k / (CIN * 9)][k % (CIN * 9)] = bf16r(params[woff + k]);
  const int img = blockIdx.z;
  const int ox = blockIdx.x * 16, oy = blockIdx.y * 16;
  const long long HW = (long long)H * W;
  for (int k = threadIdx.x; k < COUT * 324; k += 256) {
    const int c = k / 324, r = k % 324, iy = oy - 1 + r / 18, ix = ox - 1 + r % 18;
    float v = 0.f;
    if (iy >= 0 && iy < H && ix >= 0 && ix < W) v = dout[((long long)img * COUT + c) * HW + (long long)iy * W + ix];
    d_s[c][r / 18][r % 18] = v;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int px = ox + tx, py = oy + ty;
  if (px >= W || py >= H) return;
  float acc[CIN];
#pragma unroll
  for (int c = 0; c < CIN; ++c) acc[c] = 0.f;
  // in(q) feeds out(q - (ky - 1, kx - 1)) with weight w[o][c][ky][kx]
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float g = d_s[o][ty + 2 - k / 3][tx + 2 - k % 3];
#pragma unroll
      for (int c = 0; c < CIN; ++c) acc[c] = fmaf(w_s[o][c * 9 + k], g, acc[c]);
    }
  const long long p = (long long)py * W + px;
#pragma unroll
  for (int c = 0; c < CIN; ++c) {
    const long long idx = ((long long)img * CIN + c) * HW + p;
    din[idx] = act_in[idx] != 0 ? acc[c] : 0.f;
  }
}

// dW[o][c][k] += sum over pixels of dOut[o](p) in[c](p + k - 1); dB[o] += sum dOut[o](p).
// Persistent CTAs over 16x16 tiles; one shared-memory accumulator per weight, flushed with
// one global atomic per weight per CTA.
template <int CIN, int COUT, int LAYER>
__global__ void __launch_bounds__(256) conv_bwd_weight_kernel(const float* __restrict__ x,
                                                              const uint16_t* __restrict__ act_in,
                                                              const float* __restrict__ dout, int n_images, int H,
                                                              int W, float* __restrict__ dparams) {
  extern __shared__ __align__(16) float smf[];
  float(*in_s)[18][18] = reinterpret_cast<float(*)[18][18]>(smf);
  float(*d_s)[16][16] = reinterpret_cast<float(*)[16][16]>(smf + CIN * 324);
  float* acc_s = smf + CIN * 324 + COUT * 256;
  const int nw = COUT * CIN * 9;
  for (int k = threadIdx.x; k < nw + COUT; k += 256) acc_s[k] = 0.f;
  const int tiles_x = (W + 15) / 16, tiles_y = (H + 15) / 16;
  const long long n_tiles = (long long)tiles_x * tiles_y * n_images;
  const long long HW = (long long)H * W;
  for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int img = (int)(t / (tiles_x * tiles_y));
    const int r0 = (int)(t % (tiles_x * tiles_y));
    const int ox = (r0 % tiles_x) * 16, oy = (r0 / tiles_x) * 16;
    __syncthreads();
    for (int k = threadIdx.x; k < CIN * 324; k += 256) {
      const int c = k / 324, r = k % 324, iy = oy - 1 + r / 18, ix = ox - 1 + r % 18;
      float v = 0.f;
      if (iy >= 0 && iy < H && ix >= 0 && ix < W) {
        const long long idx = ((long long)img * CIN + c) * HW + (long long)iy * W + ix;
        v = LAYER == 1 ? bf16r(x[idx]) : bits2f(act_in[idx]);
      }
      in_s[c][r / 18][r % 18] = v;
    }
    for (int k = threadIdx.x; k < COUT * 256; k += 256) {
      const int o = k / 256, r = k % 256, iy = oy + r / 16, ix = ox + r % 16;
      d_s[o][r / 16][r % 16] = (iy < H && ix < W) ? dout[((long long)img * COUT + o) * HW + (long long)iy * W + ix] : 0.f;
    }
    __syncthreads();
    for (int wi = threadIdx.x; wi < nw + COUT; wi += 256) {
      float s = 0.f;
      if (wi < nw) {
        const int o = wi / (CIN * 9), c = (wi / 9) % CIN, k = wi % 9, ky = k / 3, kx = k % 3;
        for (int yy = 0; yy < 16; ++yy)
#pragma unroll 4
          for (int xx = 0; xx < 16; ++xx) s = fmaf(d_s[o][yy][xx], in_s[c][yy + ky][xx + kx], s);
      } else {
        const int o = wi - nw;
        for (int r = 0; r < 256; ++r) s += d_s[o][r / 16][r % 16];
      }
      acc_s[wi] += s;
    }
  }
  __syncthreads();
  const int woff = LAYER == 1 ? kW1 : (LAYER == 2 ? kW2 : kW3);
  const int boff = LAYER == 1 ? kB1 : (LAYER == 2 ? kB2 : kB3);
  for (int k = threadIdx.x; k < nw; k += 256) atomicAdd(&dparams[woff + k], acc_s[k]);
  for (int k = threadIdx.x; k < COUT; k += 256) atomicAdd(&dparams[boff + k], acc_s[nw + k]);
}

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long n, double* sum,
                           float* __restrict__ dy, float scale) {
  double s = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * d;
    if (dy) dy[i] = scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
}

__global__ void mse_finalize_kernel(const double* sum, long long n, float* loss) { *loss = (float)(*sum / (double)n); }

// ------------------------------------------------------------------ fused tensor-core inference

constexpr int kT = 32;                 // output tile
constexpr int kGx = kT + 6;            // input grid (halo 3)
constexpr int kG1 = kT + 4;            // conv1 output grid
constexpr int kG2 = kT + 2;            // conv2 output grid
constexpr int kW1Stride = 88;          // conv1 K = 9 taps x 8 channels = 72, padded to 80 (+8 pad)
constexpr int kWStride = 296;          // conv2 / conv3 K = 288 (+8 pad, conflict-free ldmatrix rows)
constexpr int kSmW1 = 32 * kW1Stride * 2;
constexpr int kSmW2 = 32 * kWStride * 2;
constexpr int kSmW3 = 8 * kWStride * 2;
constexpr int kSmBias = 80 * 4;
constexpr int kSmA = kG2 * kG2 * 64;   // x tile (38^2 x 16 B) then conv2 output (34^2 x 64 B)
constexpr int kSmB = kG1 * kG1 * 64;   // conv1 output
constexpr int kOffW1 = 0, kOffW2 = kOffW1 + kSmW1, kOffW3 = kOffW2 + kSmW2, kOffBias = kOffW3 + kSmW3;
constexpr int kOffA = kOffBias + kSmBias, kOffB = kOffA + kSmA;
constexpr int kNetSmem = kOffB + kSmB;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x2(uint32_t addr, uint32_t& r0, uint32_t& r1) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float c[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// 64-byte activation rows, 16-byte chunks swizzled so that eight consecutive positions
// hit eight different bank groups
__device__ __forceinline__ int act_off(int pos, int chunk) { return pos * 64 + ((chunk ^ ((pos >> 1) & 3)) << 4); }

__device__ __forceinline__ void bilinear_x(const float* __restrict__ L, int W2, int H2, long long HW2, int x, int y,
                                           float v[3]) {
  const float ux = (x + 0.5f) * 0.5f - 0.5f, uy = (y + 0.5f) * 0.5f - 0.5f;
  const int x0 = (int)floorf(ux), y0 = (int)floorf(uy);
  const float fx = ux - x0, fy = uy - y0;
  const int xa = min(max(x0, 0), W2 - 1), xb = min(max(x0 + 1, 0), W2 - 1);
  const int ya = min(max(y0, 0), H2 - 1), yb = min(max(y0 + 1, 0), H2 - 1);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* Lc = L + c * HW2;
    const float top = (1.f - fx) * Lc[ya * W2 + xa] + fx * Lc[ya * W2 + xb];
    const float bot = (1.f - fx) * Lc[yb * W2 + xa] + fx * Lc[yb * W2 + xb];
    v[c] = (1.f - fy) * top + fy * bot;
  }
}

// implicit-GEMM 3x3 conv, 32 input channels in swizzled 64-byte rows (grid gin wide),
// outputs on a gout x gout grid, NT n8 tiles; epilogue functor per (m, channel pair)
template <int NT, class Epi>
__device__ __forceinline__ void conv32_mma(uint32_t in_base, int gin, int gout, uint32_t w_base, Epi epi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int M = gout * gout, mtiles = (M + 15) / 16;
  for (int mt = warp; mt < mtiles; mt += kBlock / 32) {
    float acc[NT][4];
#pragma unroll
    for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
    int m = mt * 16 + (lane & 15);
    if (m >= M) m = M - 1;
    const int oi = m / gout, oj = m % gout;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap) {
      const int pos = (oi + tap / 3) * gin + oj + tap % 3;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t a0, a1, a2, a3;
        ldsm_x4(in_base + act_off(pos, 2 * h + (lane >> 4)), a0, a1, a2, a3);
        const int k0 = tap * 32 + h * 16;
#pragma unroll
        for (int n = 0; n < NT; ++n) {
          uint32_t b0, b1;
          const int nrow = n * 8 + (lane & 7), kk = k0 + ((lane >> 3) & 1) * 8;
          ldsm_x2(w_base + (nrow * kWStride + kk) * 2, b0, b1);
          mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
        }
      }
    }
    const int r0 = mt * 16 + (lane >> 2), c0 = 2 * (lane & 3);
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      epi(r0, n * 8 + c0, acc[n][0], acc[n][1]);
      epi(r0 + 8, n * 8 + c0, acc[n][2], acc[n][3]);
    }
  }
}

__global__ void __launch_bounds__(kBlock, 1) net_periphery_kernel(const float* __restrict__ params,
                                                                  const float* __restrict__ low,
                                                                  float* __restrict__ out,
                                                                  const uint8_t* __restrict__ tile_class,
                                                                  const ViewParams* __restrict__ views, int n_views,
                                                                  int tiles_per_view, int W, int H) {
  extern __shared__ __align__(128) unsigned char sm[];
  uint16_t* w1s = reinterpret_cast<uint16_t*>(sm + kOffW1);
  uint16_t* w2s = reinterpret_cast<uint16_t*>(sm + kOffW2);
  uint16_t* w3s = reinterpret_cast<uint16_t*>(sm + kOffW3);
  float* bias = reinterpret_cast<float*>(sm + kOffBias);
  unsigned char* A = sm + kOffA;
  unsigned char* B = sm + kOffB;
  // weights to BF16, K-major rows: conv1 k = tap * 8 + c, conv2/3 k = tap * 32 + c
  for (int k = threadIdx.x; k < 32 * kW1Stride; k += kBlock) {
    const int n = k / kW1Stride, kk = k % kW1Stride, tap = kk / 8, c = kk % 8;
    w1s[k] = (tap < 9 && c < 3) ? bf16bits(params[kW1 + (n * 3 + c) * 9 + tap]) : (uint16_t)0;
  }
  for (int k = threadIdx.x; k < 32 * kWStride; k += kBlock) {
    const int n = k / kWStride, kk = k % kWStride, tap = kk / 32, c = kk % 32;
    w2s[k] = kk < 288 ? bf16bits(params[kW2 + (n * 32 + c) * 9 + tap]) : (uint16_t)0;
  }
  for (int k = threadIdx.x; k < 8 * kWStride; k += kBlock) {
    const int n = k / kWStride, kk = k % kWStride, tap = kk / 32, c = kk % 32;
    w3s[k] = (n < 3 && kk < 288) ? bf16bits(params[kW3 + (n * 32 + c) * 9 + tap]) : (uint16_t)0;
  }
  if (threadIdx.x < 32) bias[threadIdx.x] = params[kB1 + threadIdx.x];
  if (threadIdx.x < 32) bias[32 + threadIdx.x] = params[kB2 + threadIdx.x];
  if (threadIdx.x < 3) bias[64 + threadIdx.x] = params[kB3 + threadIdx.x];
  const int W2 = W / 2, H2 = H / 2;
  const long long HW = (long long)W * H, HW2 = (long long)W2 * H2;
  const long long n_tiles = (long long)n_views * tiles_per_view;
  const int lane = threadIdx.x & 31;
  for (long long tg = blockIdx.x; tg < n_tiles; tg += gridDim.x) {
    if (tile_class[tg] != kClassPeriphery) continue;
    const int view = (int)(tg / tiles_per_view), t = (int)(tg % tiles_per_view);
    const ViewParams& vp = views[view];
    const int ox = (t % vp.ntx) * kT, oy = (t / vp.ntx) * kT;
    const float* L = low + (long long)view * 3 * HW2;
    __syncthreads();  // previous tile done with A / B
    // x tile (halo 3), BF16, 8 channels per position (3 used)
    for (int p = threadIdx.x; p < kGx * kGx; p += kBlock) {
      const int gx = ox - 3 + p % kGx, gy = oy - 3 + p / kGx;
      float v[3] = {0.f, 0.f, 0.f};
      if (gx >= 0 && gx < W && gy >= 0 && gy < H) bilinear_x(L, W2, H2, HW2, gx, gy, v);
      uint4 q;
      q.x = (uint32_t)bf16bits(v[0]) | ((uint32_t)bf16bits(v[1]) << 16);
      q.y = (uint32_t)bf16bits(v[2]);
      q.z = q.w = 0u;
      *reinterpret_cast<uint4*>(A + p * 16) = q;
    }
    __syncthreads();
    // conv1 (K = 80: taps t = 2 step + {0, 1}, 8 channels each) -> B, 36 x 36
    {
      const int warp = threadIdx.x >> 5;
      const int M = kG1 * kG1, mtiles = M / 16;
      const uint32_t abase = smem_u32(A), wbase = smem_u32(w1s);
      for (int mt = warp; mt < mtiles; mt += kBlock / 32) {
        float acc[4][4];
#pragma unroll
        for (int n = 0; n < 4; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
        const int m = mt * 16 + (lane & 15), oi = m / kG1, oj = m % kG1;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
          const int tap = min(2 * step + (lane >> 4), 8);
          const int pos = (oi + tap / 3) * kGx + oj + tap % 3;
          uint32_t a0, a1, a2, a3;
          ldsm_x4(abase + pos * 16, a0, a1, a2, a3);
#pragma unroll
          for (int n = 0; n < 4; ++n) {
            uint32_t b0, b1;
            const int nrow = n * 8 + (lane & 7), kk = step * 16 + ((lane >> 3) & 1) * 8;
            ldsm_x2(wbase + (nrow * kW1Stride + kk) * 2, b0, b1);
            mma_bf16(acc[n], a0, a1, a2, a3, b0, b1);
          }
        }
        const int r0 = mt * 16 + (lane >> 2), c0 = 2 * (lane & 3);
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int mm = r0 + 8 * hh, ch = n * 8 + c0;
            const int gx = ox - 2 + mm % kG1, gy = oy - 2 + mm / kG1;
            const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
            const float v0 = in ? fmaxf(acc[n][2 * hh] + bias[ch], 0.f) : 0.f;
            const float v1 = in ? fmaxf(acc[n][2 * hh + 1] + bias[ch + 1], 0.f) : 0.f;
            *reinterpret_cast<uint32_t*>(B + act_off(mm, ch >> 3) + (ch & 7) * 2) =
                (uint32_t)bf16bits(v0) | ((uint32_t)bf16bits(v1) << 16);
          }
      }
    }
    __syncthreads();
    // conv2 -> A (34 x 34)
    conv32_mma<4>(smem_u32(B), kG1, kG2, smem_u32(w2s), [&](int mm, int ch, float c0v, float c1v) {
      if (mm >= kG2 * kG2) return;
      const int gx = ox - 1 + mm % kG2, gy = oy - 1 + mm / kG2;
      const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
      const float v0 = in ? fmaxf(c0v + bias[32 + ch], 0.f) : 0.f;
      const float v1 = in ? fmaxf(c1v + bias[32 + ch + 1], 0.f) : 0.f;
      *reinterpret_cast<uint32_t*>(A + act_off(mm, ch >> 3) + (ch & 7) * 2) =
          (uint32_t)bf16bits(v0) | ((uint32_t)bf16bits(v1) << 16);
    });
    __syncthreads();
    // conv3 -> out (32 x 32): residual on the float bilinear input
    conv32_mma<1>(smem_u32(A), kG2, kT, smem_u32(w3s), [&](int mm, int ch, float c0v, float c1v) {
      const int gx = ox + mm % kT, gy = oy + mm / kT;
      if (gx >= W || gy >= H || ch >= 3) return;
      float v[3];
      bilinear_x(L, W2, H2, HW2, gx, gy, v);
      float* o = out + (long long)view * 3 * HW + (long long)gy * W + gx;
      o[(long long)ch * HW] = v[ch] + c0v + bias[64 + ch];
      if (ch + 1 < 3) o[(long long)(ch + 1) * HW] = v[ch + 1] + c1v + bias[64 + ch + 1];
    });
  }
}

unsigned grid_for(long long n) {
  return (unsigned)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 16);
}

}  // namespace

template <int CIN, int COUT, int LAYER>
void launch_conv_fwd(dim3 grid, const float* params, const float* x, const uint16_t* ain, uint16_t* aout, float* y,
                     int H, int W, cudaStream_t st) {
  const int smem = (CIN * 324 + COUT * CIN * 9 + COUT) * 4;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv_fwd_kernel<CIN, COUT, LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  conv_fwd_kernel<CIN, COUT, LAYER><<<grid, 256, smem, st>>>(params, x, ain, aout, y, H, W);
}

template <int CIN, int COUT>
void launch_conv_bwd_data(dim3 grid, const float* params, int woff, const float* dout, const uint16_t* ain, float* din,
                          int H, int W, cudaStream_t st) {
  const int smem = (COUT * 324 + COUT * CIN * 9) * 4;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv_bwd_data_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  conv_bwd_data_kernel<CIN, COUT><<<grid, 256, smem, st>>>(params, woff, dout, ain, din, H, W);
}

template <int CIN, int COUT, int LAYER>
void launch_conv_bwd_weight(unsigned grid, const float* x, const uint16_t* ain, const float* dout, int B, int H, int W,
                            float* dparams, cudaStream_t st) {
  const int smem = (CIN * 324 + COUT * 256 + COUT * CIN * 9 + COUT) * 4;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(conv_bwd_weight_kernel<CIN, COUT, LAYER>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr = true;
  }
  conv_bwd_weight_kernel<CIN, COUT, LAYER><<<grid, 256, smem, st>>>(x, ain, dout, B, H, W, dparams);
}

// training forward: y[B][3][H][W], acts[B][2][32][H][W] (BF16 bits; a1 then a2)
void net_forward_train(const float* params, const float* x, int B, int H, int W, float* y, uint16_t* acts,
                       uint16_t* tmp_a1, uint16_t* tmp_a2, cudaStream_t st) {
  const dim3 grid((W + 15) / 16, (H + 15) / 16, B);
  uint16_t* a1 = acts ? acts : tmp_a1;
  uint16_t* a2 = acts ? acts + (size_t)B * 32 * H * W : tmp_a2;
  launch_conv_fwd<3, 32, 1>(grid, params, x, nullptr, a1, nullptr, H, W, st);
  launch_conv_fwd<32, 32, 2>(grid, params, nullptr, a1, a2, nullptr, H, W, st);
  launch_conv_fwd<32, 3, 3>(grid, params, x, a2, nullptr, y, H, W, st);
}

// training backward: dparams += d<dy, y>/dparams (BF16 rounding passes gradients straight
// through; ReLU masks from the saved activations); scratch: 2 x [B][32][H][W] floats
void net_backward_train(const float* params, const float* x, const uint16_t* acts, const float* dy, int B, int H,
                        int W, float* dparams, float* dz2, float* dz1, cudaStream_t st) {
  const dim3 grid((W + 15) / 16, (H + 15) / 16, B);
  const uint16_t* a1 = acts;
  const uint16_t* a2 = acts + (size_t)B * 32 * H * W;
  const long long tiles = (long long)((W + 15) / 16) * ((H + 15) / 16) * B;
  const unsigned wgrid = (unsigned)std::min<long long>(tiles, (long long)device_sm_count() * 2);
  launch_conv_bwd_weight<32, 3, 3>(wgrid, nullptr, a2, dy, B, H, W, dparams, st);
  launch_conv_bwd_data<32, 3>(grid, params, kW3, dy, a2, dz2, H, W, st);
  launch_conv_bwd_weight<32, 32, 2>(wgrid, nullptr, a1, dz2, B, H, W, dparams, st);
  launch_conv_bwd_data<32, 32>(grid, params, kW2, dz2, a1, dz1, H, W, st);
  launch_conv_bwd_weight<3, 32, 1>(wgrid, x, nullptr, dz1, B, H, W, dparams, st);
}

void net_mse(const float* y, const float* t, long long n, float* loss, float* dy, double* scratch, cudaStream_t st) {
  cudaMemsetAsync(scratch, 0, sizeof(double), st);
  mse_kernel<<<grid_for(n), 256, 0, st>>>(y, t, n, scratch, dy, (float)(2.0 / (double)n));
  mse_finalize_kernel<<<1, 1, 0, st>>>(scratch, n, loss);
}

void net_periphery(const float* params, const float* low, float* out, const uint8_t* tile_class,
                   const ViewParams* views, int n_views, int tiles_per_view, int W, int H, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(net_periphery_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kNetSmem);
    attr = true;
  }
  const long long n = (long long)n_views * tiles_per_view;
  const unsigned grid = (unsigned)std::min<long long>(n, (long long)device_sm_count());
  net_periphery_kernel<<<grid, kBlock, kNetSmem, st>>>(params, low, out, tile_class, views, n_views, tiles_per_view, W,
                                                       H);
}

int net_smem_bytes() { return kNetSmem; }

}  // namespace vrs
