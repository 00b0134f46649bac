// Training kernels of the learned periphery network, on the 5th-generation tensor cores.
//
// The network (net.cuh): y = x + conv3(relu(conv2(relu(conv1(bf16(x)))))), 3x3 kernels,
// zero padding 1, BF16 weights and activations, FP32 accumulation.  Training runs it on
// whole images (batches of crops) and back-propagates an output gradient dy:
//   dz2 = [a2 > 0] conv_T(dy, w3),   dz1 = [a1 > 0] conv_T(dz2, w2),
//   dw3 = sum_p a2 (x) dy,   dw2 = sum_p a1 (x) dz2,   dw1 = sum_p bf16(x) (x) dz1,
//   db  = sum_p of the layer's output gradient,
// where conv_T, the transposed convolution, is a 3x3 convolution with the kernel flipped
// and its channel roles swapped, and (x) pairs every tap and input channel with every
// output channel.  Every contraction is tcgen05.mma, BF16 x BF16 -> FP32 in tensor
// memory; the gradients dy, dz2 and dz1 are rounded to BF16 (nearest even) where they
// enter a contraction, as in mixed-precision training.
//
// Two kernels:
//  - conv_tc_kernel: one 3x3 convolution as an implicit GEMM, D[position][out channel] =
//    sum over taps and input channels.  One CTA per 32 x 12 output tile.  The input grid
//    with its one-pixel halo (34 x 14 positions) is the A operand, one row per position:
//    64-byte rows with the 64-byte swizzle for 32 channels, 32-byte rows with the 32-byte
//    swizzle for 3 channels padded to 16.  Tap (dy, dx) shifts the A start by dy * 34 + dx
//    rows: the outputs are computed on the rows of the input grid, and the two wrapped
//    columns of each row are discarded.  Its epilogues are the forward layers (bias and
//    ReLU, or the residual output) and the data gradients (the ReLU mask of the saved
//    activation).
//  - wgrad_tc_kernel: the weight and bias gradients of one layer, D[(tap, in channel) or
//    the bias row][out channel], K running over pixels.  Each chunk of 64 pixels of an
//    image row stages the layer input's three rows and the output gradient with 16-byte
//    asynchronous copies (double-buffered: the next chunk's copies are in flight while
//    this one is built), then builds the im2col matrix of the input (one row per tap and
//    input channel, plus a row of ones whose product is the bias gradient) and the
//    gradient matrix, both K-major without swizzle, by transposing the pixel-major staged
//    rows in shared memory.  The CTA's accumulators in tensor memory collect all its
//    chunks, and one atomic add per gradient value and CTA ends it.
// Activations and hidden-layer gradients are pixel-major BF16 ([B][H][W][32]); the
// weights are packed once per call into the B-operand planes (pack_weights_kernel).
// Both hold 128 tensor-memory columns and ask for at least kTcSmemFloor bytes of shared
// memory, so that at most four CTAs share an SM and their 4 x 128 columns fit its 512;
// the launchers check the residency from the device's shared memory and refuse a launch
// that could oversubscribe tensor memory.
// Every mbarrier wait is bounded: a thread that gives up raises kStTimeout in the status
// word, and the block waits for its committed MMAs before it frees tensor memory.
#include <algorithm>

#include "common.cuh"
#include "net.cuh"

namespace vrs {

namespace {

constexpr int kTcThreads = 256;  // eight warps: the MMA issuers are lanes 0 of warps 0 - 3
constexpr int kTmemCols = 128;
constexpr int kTcSmemFloor = 56 * 1024;

// ------------------------------------------------------------------ convolution layer

constexpr int kCT = 32;                                     // output tile width
constexpr int kCH = 12;                                     // output tile height
constexpr int kCG = kCT + 2;                                // input grid width
constexpr int kCGH = kCH + 2;                               // input grid height
constexpr int kCPos = kCG * kCGH;                           // input positions (476)
constexpr int kCMt = (kCH * kCG + 127) / 128;               // M tiles (408 rows -> 4)
constexpr int kCRows = (kCMt * 128 + 2 * kCG + 2 + 7) / 8 * 8;  // A rows read (584)
constexpr int kCOffB = kCRows * 64;                         // weights, after the A rows
constexpr int kCOffBias = kCOffB + 9 * 4 * 32 * 16;
constexpr int kCOffBar = kCOffBias + 32 * 4;                // full[kCMt], abort, TMEM address
constexpr int kCSmem = kCOffBar + 8 * kCMt + 8;
static_assert(kCMt * 32 <= kTmemCols && kCMt <= kTcThreads / 32, "accumulators of 32 columns, one issuing warp each");
static_assert(kCSmem <= kTcSmemFloor, "convolution tile does not fit the shared-memory floor");

enum { kEpiRelu = 0, kEpiResid = 1, kEpiMask = 2 };

// The B operands of the five convolutions, packed once per call from the float master
// weights: BF16 planes [tap][8 input channels][n][8], zero beyond the real channels.
// Layouts: 0 conv1, 1 conv2, 2 conv3 (forward); 3 conv_T through w3, 4 conv_T through w2.
constexpr int kPackBytes = 9 * 4 * 32 * 16;  // the largest layout (18 KB)
constexpr int kPackLayouts = 5;
struct PackSpec {
  int woff, cin, nreal, nout, transposed;
};
__host__ __device__ inline PackSpec pack_spec(int l) {
  switch (l) {
    case 0: return {kW1, 3, 32, 32, 0};
    case 1: return {kW2, 32, 32, 32, 0};
    case 2: return {kW3, 32, 3, 16, 0};
    case 3: return {kW3, 3, 32, 32, 1};
    default: return {kW2, 32, 32, 32, 1};
  }
}

__global__ void __launch_bounds__(256) pack_weights_kernel(const float* __restrict__ params,
                                                           uint16_t* __restrict__ packed) {
  const PackSpec ps = pack_spec(blockIdx.y);
  const int pl_per_tap = ps.cin == 32 ? 4 : 2;
  uint16_t* out = packed + (size_t)blockIdx.y * (kPackBytes / 2);
  for (int i = blockIdx.x * 256 + threadIdx.x; i < 9 * pl_per_tap * ps.nout * 8; i += gridDim.x * 256) {
    const int e = i & 7, n = (i >> 3) % ps.nout, pl = (i >> 3) / ps.nout;
    const int t = pl / pl_per_tap, ci = (pl % pl_per_tap) * 8 + e;
    float w = 0.f;
    if (n < ps.nreal && ci < ps.cin)
      w = ps.transposed ? params[ps.woff + (ci * ps.nreal + n) * 9 + (8 - t)] : params[ps.woff + (n * ps.cin + ci) * 9 + t];
    out[i] = bf16bits(w);
  }
}

struct ConvArgs {
  const float* params;    // network parameters (OIHW), for the bias
  const uint16_t* wpack;  // this convolution's packed B operand (pack_weights_kernel)
  int boff;               // bias (boff < 0: none)
  const float* in_f32;    // 3 input channels: float [B][3][H][W], rounded to BF16
  const uint16_t* in_bf;  // 32 input channels: BF16 [B][H][W][32]
  const float* xres;      // kEpiResid: float [B][3][H][W], added to the output
  float* out_f32;         // kEpiResid: float [B][3][H][W]
  const uint16_t* mask;   // kEpiMask: saved activation, BF16 [B][H][W][32]; > 0 keeps
  uint16_t* out_nhwc;     // BF16 [B][H][W][32]
  int H, W;
  uint32_t* status;
};

// CIN input channels (3 or 32), NOUT MMA columns (32, or 16 for the 3 outputs of conv3)
template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(kTcThreads) conv_tc_kernel(ConvArgs a) {
  constexpr int RB = CIN == 32 ? 64 : 32;  // bytes per A row
  constexpr int PL = CIN == 32 ? 4 : 2;    // weight planes (8 input channels) per tap
  constexpr int KH = CIN == 32 ? 2 : 1;    // MMAs (K = 16) per tap
  constexpr int NREAL = NOUT == 32 ? 32 : 3;
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t sm0 = smem_u32(sm);
  float* bias = reinterpret_cast<float*>(sm + kCOffBias);
  volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(sm + kCOffBar + 8 * kCMt);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kCOffBar + 8 * kCMt + 4);
  const uint32_t bar_full = sm0 + kCOffBar;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ox = blockIdx.x * kCT, oy = blockIdx.y * kCH, img = blockIdx.z;
  const int H = a.H, W = a.W;
  const long long HW = (long long)H * W;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int mt = 0; mt < kCMt; ++mt)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full + 8u * mt), "r"(1));
    *abort = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights: the packed B planes, 16-byte asynchronous copies in flight with the input's
  for (int i = tid; i < 9 * PL * NOUT / 8 * 8; i += kTcThreads) cp_async16(sm0 + kCOffB + 16u * i, a.wpack + 8 * i, 16u);
  if (tid < 32) bias[tid] = (a.boff >= 0 && tid < NREAL) ? a.params[a.boff + tid] : 0.f;
  // A: the input grid, zero outside the image and in the rows past the grid
  if (CIN == 32) {
    // 16-byte asynchronous copies, all in flight together; zero-filled outside the image
    for (int i = tid; i < kCRows * 4; i += kTcThreads) {
      const int p = i >> 2, q = i & 3;
      const uint16_t* src = a.in_bf;
      uint32_t bytes = 0u;
      if (p < kCPos) {
        const int gy = oy - 1 + p / kCG, gx = ox - 1 + p % kCG;
        if (gy >= 0 && gy < H && gx >= 0 && gx < W) {
          src = a.in_bf + (((long long)img * H + gy) * W + gx) * 32 + 8 * q;
          bytes = 16u;
        }
      }
      const uint32_t row = (uint32_t)p * 64u;
      const uint32_t sw = ((sm0 + row) >> 7) & 3u;  // 64-byte swizzle of this row
      cp_async16(sm0 + row + ((q ^ sw) << 4), src, bytes);
    }
    cp_async_wait_all();
  } else {
    // every position's three values loaded first, then converted and stored
    constexpr int kPer = (kCRows + kTcThreads - 1) / kTcThreads;
    float v[kPer][3];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int p = tid + k * kTcThreads;
      const int gy = oy - 1 + p / kCG, gx = ox - 1 + p % kCG;
      const bool in = p < kCPos && gy >= 0 && gy < H && gx >= 0 && gx < W;
#pragma unroll
      for (int c = 0; c < 3; ++c) v[k][c] = in ? a.in_f32[((long long)img * 3 + c) * HW + (long long)gy * W + gx] : 0.f;
    }
    cp_async_wait_all();
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int p = tid + k * kTcThreads;
      if (p >= kCRows) break;
      const float f[8] = {v[k][0], v[k][1], v[k][2], 0.f, 0.f, 0.f, 0.f, 0.f};
      const uint32_t row = (uint32_t)p * 32u;
      const uint32_t sw = ((sm0 + row) >> 7) & 1u;  // 32-byte swizzle: the halves swap
      *reinterpret_cast<uint4*>(sm + row + (sw << 4)) = pack8(f);
      *reinterpret_cast<uint4*>(sm + row + ((1u ^ sw) << 4)) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  if (lane == 0 && warp < kCMt) {
    // lane 0 of warp w issues M tile w: a thread's tcgen05.mma waits for its previous one,
    // so one issuer per M tile keeps four in flight
    const uint32_t id = umma_idesc(128, NOUT);
    const uint64_t a0 = CIN == 32 ? umma_desc_sw(sm0, 512, 4) : umma_desc_sw(sm0, 256, 6);
    const uint64_t b0 = umma_desc(sm0 + kCOffB, NOUT * 16);
    // start-address offsets in 16-byte units: a row is RB / 16 units, the second K half
    // of a 64-byte row 2 units, a weight plane NOUT units
    for (int mt = warp; mt < kCMt; mt += kCMt) {
      for (int t = 0; t < 9; ++t) {
        const int dy = t / 3, dx = t % 3;
#pragma unroll
        for (int h = 0; h < KH; ++h)
          umma(tmem + 32u * mt, a0 + (uint64_t)((mt * 128 + dy * kCG + dx) * (RB / 16) + 2 * h),
               b0 + (uint64_t)((t * PL + 2 * h) * NOUT), id, (t | h) != 0);
      }
      umma_commit(bar_full + 8u * mt);
    }
  }
  // epilogue: warp w reads tensor-memory lanes 32 (w & 3) .. + 31, the rows of its
  // quarter; the two warp quads take alternate M tiles
  bool ok = true;
  for (int mt = warp >> 2; mt < kCMt; mt += 2) {
    ok = mbar_wait(bar_full + 8u * mt, 0u, abort);
    if (!__all_sync(0xffffffffu, ok)) {
      ok = false;
      break;
    }
    tc_fence_after();
    const int m = mt * 128 + (warp & 3) * 32 + lane;
    const int oi = m / kCG, oj = m - (m / kCG) * kCG;
    const int gy = oy + oi, gx = ox + oj;
    const bool st = oi < kCH && oj < kCT && gy < H && gx < W;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + 32u * mt;
    const long long pix = ((long long)img * H + gy) * W + gx;
    if (NOUT == 32) {
      float v[32];
      tmem_ld32(taddr, v);
      if (st) {
        if (EPI == kEpiRelu) {
#pragma unroll
          for (int c = 0; c < 32; ++c) v[c] = fmaxf(v[c] + bias[c], 0.f);
        } else {
          const uint4* mk = reinterpret_cast<const uint4*>(a.mask + pix * 32);
          uint32_t mw[16];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint4 u = mk[q];
            mw[4 * q] = u.x;
            mw[4 * q + 1] = u.y;
            mw[4 * q + 2] = u.z;
            mw[4 * q + 3] = u.w;
          }
#pragma unroll
          for (int c = 0; c < 32; ++c)  // a positive BF16 value keeps the gradient
            v[c] = (int16_t)(uint16_t)(mw[c >> 1] >> (16 * (c & 1))) > 0 ? v[c] : 0.f;
        }
        uint4* o = reinterpret_cast<uint4*>(a.out_nhwc + pix * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) o[q] = pack8(v + 8 * q);
      }
    } else {
      float v[4];
      tmem_ld4(taddr, v);
      if (st) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const long long o = ((long long)img * 3 + c) * HW + (long long)gy * W + gx;
          a.out_f32[o] = a.xres[o] + v[c] + bias[c];
        }
      }
    }
  }
  if (!ok) atomicOr(a.status, kStTimeout);
  if (lane == 0 && *abort) {
    // a wait gave up: the committed MMAs finish (bounded waits that ignore the abort
    // flag) before tensor memory is freed
    uint32_t none = 0u;
    if (warp < kCMt) mbar_wait(bar_full + 8u * warp, 0u, &none);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// ------------------------------------------------------------------ weight gradients

constexpr int kWgThreads = 256;    // eight warps share each chunk's staging and im2col build
constexpr int kWK = 64;            // pixels per chunk (the MMAs' K)
constexpr int kWStage = kWK + 16;  // staged pixels per input row: x0 - 8 .. x0 + 71
constexpr int kWRow = kWStage + 8; // 3-channel input: staged row stride in elements (176 bytes)

struct WgradArgs {
  const uint16_t* a_bf;  // 32 input channels: the layer's input, BF16 [B][H][W][32]
  const float* a_f32;    // 3 input channels: float [B][3][H][W], rounded to BF16
  const uint16_t* g_bf;  // 32 output channels: the output gradient, BF16 [B][H][W][32]
  const float* g_f32;    // 3 output channels: float [B][3][H][W], rounded to BF16
  float* dparams;        // += dw[o][ci][t] at woff and db[o] at boff
  int woff, boff;
  int B, H, W;
  uint32_t* status;
};

template <int CIN, int NOUT>
struct WgradLayout {
  static constexpr int NREAL = NOUT == 32 ? 32 : 3;
  static constexpr int MROWS = 9 * CIN + 1;  // (tap, input channel) rows, then the bias row
  static constexpr int MT = (MROWS + 127) / 128;
  static constexpr int MPAD = MT * 128;
  static constexpr int LBOA = MPAD * 16;  // A: 8 planes (8 pixels each) of MPAD rows of 16 bytes
  static constexpr int LBOG = NOUT * 16;  // G: 8 planes of NOUT rows
  static constexpr int OFF_G = 8 * LBOA;
  // two staging buffers (chunks alternate; the next chunk's loads are in flight while the
  // current one is built): the output gradient (32 channels), [kWK pixels][32] BF16, and
  // the input rows y - 1 .. y + 1, [3][kWStage pixels][32] (32 channels) or [3][3][kWRow]
  // (3 channels), BF16
  static constexpr int GS_BYTES = NOUT == 32 ? kWK * 64 : 0;
  static constexpr int S_BYTES = CIN == 32 ? 3 * kWStage * 64 : 3 * 3 * kWRow * 2;
  static constexpr int OFF_GS = OFF_G + 8 * LBOG;
  static constexpr int OFF_S = OFF_GS + 2 * GS_BYTES;
  static constexpr int OFF_BAR = OFF_S + 2 * S_BYTES;
  static constexpr int SMEM = OFF_BAR + 16;  // done, abort, TMEM address
  static constexpr int REQ = SMEM > kTcSmemFloor ? SMEM : kTcSmemFloor;
  static_assert(MT * 32 <= kTmemCols, "accumulators of 32 columns");
};

__device__ __forceinline__ uint4 load8_f32(const float* plane, int gy, int xs, int H, int W) {
  float v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int x = xs + k;
    v[k] = (gy >= 0 && gy < H && x >= 0 && x < W) ? plane[(long long)gy * W + x] : 0.f;
  }
  return pack8(v);
}

// 8 BF16 values at stride 32 (one channel of 8 consecutive pixels of a pixel-major tile)
__device__ __forceinline__ uint4 gather8(const uint16_t* p) {
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) w[k] = (uint32_t)p[64 * k] | ((uint32_t)p[64 * k + 32] << 16);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

template <int CIN, int NOUT>
__global__ void __launch_bounds__(kWgThreads) wgrad_tc_kernel(WgradArgs a) {
  using L = WgradLayout<CIN, NOUT>;
  constexpr int NREAL = L::NREAL;
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t sm0 = smem_u32(sm);
  uint16_t* stg = reinterpret_cast<uint16_t*>(sm + L::OFF_S);
  uint16_t* gstg = reinterpret_cast<uint16_t*>(sm + L::OFF_GS);
  volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(sm + L::OFF_BAR + 8);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + L::OFF_BAR + 12);
  const uint32_t bar_done = sm0 + L::OFF_BAR;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int H = a.H, W = a.W;
  const long long HW = (long long)H * W;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    // one commit per M tile and chunk (lane 0 of warp mt issues M tile mt)
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_done), "r"(L::MT));
    *abort = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // A and G start at zero (rows past the real ones stay zero); the bias row of A is ones
  for (int i = tid; i < L::OFF_GS / 16; i += kWgThreads) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0u, 0u, 0u, 0u);
  __syncthreads();
  if (tid < 8) {
    const uint32_t one2 = 0x3F803F80u;  // two BF16 ones
    *reinterpret_cast<uint4*>(sm + tid * L::LBOA + (9 * CIN) * 16) = make_uint4(one2, one2, one2, one2);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int cpr = (W + kWK - 1) / kWK;
  const long long n_chunks = (long long)a.B * H * cpr;
  uint32_t n_issued = 0;
  bool ok = true;
  // stage chunk ch into buffer b: 16-byte asynchronous copies, one commit group per chunk
  auto stage = [&](long long ch, int b) {
    const long long row = ch / cpr;
    const int x0 = (int)(ch - row * cpr) * kWK;
    const int img = (int)(row / H), y = (int)(row - (long long)img * H);
    uint16_t* sb = stg + b * (L::S_BYTES / 2);
    if (CIN == 32) {
      for (int i = tid; i < 3 * kWStage * 4; i += kWgThreads) {
        const int q = i & 3, e = (i >> 2) % kWStage, r = (i >> 2) / kWStage;
        const int gy = y - 1 + r, gx = x0 - 8 + e;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        cp_async16(smem_u32(sb) + 16u * i, in ? a.a_bf + (((long long)img * H + gy) * W + gx) * 32 + 8 * q : a.a_bf,
                   in ? 16u : 0u);
      }
    } else {
      for (int i = tid; i < 3 * 3 * (kWStage / 8); i += kWgThreads) {
        const int u = i % (kWStage / 8), rc = i / (kWStage / 8);
        const int c = rc % 3, r = rc / 3;
        *reinterpret_cast<uint4*>(sb + rc * kWRow + 8 * u) =
            load8_f32(a.a_f32 + ((long long)img * 3 + c) * HW, y - 1 + r, x0 - 8 + 8 * u, H, W);
      }
    }
    if (NOUT == 32) {
      uint16_t* gsb = gstg + b * (L::GS_BYTES / 2);
      for (int i = tid; i < kWK * 4; i += kWgThreads) {
        const int q = i & 3, e = i >> 2, gx = x0 + e;
        const bool in = gx < W;
        cp_async16(smem_u32(gsb) + 16u * i, in ? a.g_bf + (((long long)img * H + y) * W + gx) * 32 + 8 * q : a.g_bf,
                   in ? 16u : 0u);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  if ((long long)blockIdx.x < n_chunks) stage(blockIdx.x, 0);
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long row = ch / cpr;
    const int x0 = (int)(ch - row * cpr) * kWK;
    const int img = (int)(row / H), y = (int)(row - (long long)img * H);
    const int b = (int)(n_issued & 1u);
    // the next chunk's loads go to the other buffer, which the previous chunk's build has
    // finished reading (a barrier separates them)
    if (ch + gridDim.x < n_chunks)
      stage(ch + gridDim.x, b ^ 1);
    else
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this chunk's group
    const uint16_t* sb = stg + b * (L::S_BYTES / 2);
    const uint16_t* gsb = gstg + b * (L::GS_BYTES / 2);
    // the previous chunk's MMAs have read A and G
    if (n_issued > 0) ok = mbar_wait(bar_done, (n_issued - 1u) & 1u, abort);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    // G: rows o, 8-pixel groups
    for (int i = tid; i < NREAL * 8; i += kWgThreads) {
      const int o = i % NREAL, gq = i / NREAL;
      uint4* d = reinterpret_cast<uint4*>(sm + L::OFF_G + gq * L::LBOG + o * 16);
      if (NOUT == 32)
        *d = gather8(gsb + (8 * gq) * 32 + o);
      else
        *d = load8_f32(a.g_f32 + ((long long)img * 3 + o) * HW, y, x0 + 8 * gq, H, W);
    }
    // A: im2col row m = t * CIN + c holds input channel c at pixel x + dx - 1 of row
    // y + dy - 1: staged pixels e = 8 gq + 7 + dx .. + 7 (staged pixel 0 = x0 - 8)
    // (each thread takes whole rows: the tap and channel once, then the 8 pixel groups)
    for (int m = tid; m < 9 * CIN; m += kWgThreads) {
      const int t = m / CIN, c = m - (m / CIN) * CIN;
      const int dy = t / 3, dx = t - (t / 3) * 3;
      unsigned char* dst = sm + m * 16;
      if (CIN == 32) {
        const uint16_t* src = sb + (dy * kWStage + 7 + dx) * 32 + c;
#pragma unroll
        for (int gq = 0; gq < 8; ++gq)
          *reinterpret_cast<uint4*>(dst + gq * L::LBOA) = gather8(src + gq * 8 * 32);
      } else {
        const uint16_t* rw = sb + (dy * 3 + c) * kWRow + 7 + dx;
#pragma unroll
        for (int gq = 0; gq < 8; ++gq) {
          uint32_t w[4];
#pragma unroll
          for (int k = 0; k < 4; ++k) w[k] = (uint32_t)rw[8 * gq + 2 * k] | ((uint32_t)rw[8 * gq + 2 * k + 1] << 16);
          *reinterpret_cast<uint4*>(dst + gq * L::LBOA) = make_uint4(w[0], w[1], w[2], w[3]);
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    if (lane == 0 && warp < L::MT) {
      tc_fence_after();
      const uint32_t id = umma_idesc(128, NOUT);
      const int mt = warp;
#pragma unroll
      for (int ks = 0; ks < kWK / 16; ++ks)
        umma(tmem + 32u * mt, umma_desc(sm0 + mt * 2048 + 2 * ks * L::LBOA, L::LBOA),
             umma_desc(sm0 + L::OFF_G + 2 * ks * L::LBOG, L::LBOG), id, (n_issued > 0 || ks > 0) ? 1u : 0u);
      umma_commit(bar_done);
    }
    ++n_issued;
  }
  // the last chunk's MMAs, then the accumulators to the parameter gradients
  if (ok && n_issued > 0) ok = mbar_wait(bar_done, (n_issued - 1u) & 1u, abort);
  ok = __syncthreads_and(ok);
  if (ok && n_issued > 0) {
    tc_fence_after();
    // warp w reads tensor-memory lanes 32 (w & 3) .. + 31; the two warp quads take
    // alternate M tiles
#pragma unroll 1
    for (int mt = warp >> 2; mt < L::MT; mt += 2) {
      const int m = mt * 128 + (warp & 3) * 32 + lane;
      const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + 32u * mt;
      float v[32];
      if (NOUT == 32)
        tmem_ld32(taddr, v);
      else
        tmem_ld4(taddr, v);
      if (m < 9 * CIN) {
        const int t = m / CIN, c = m - (m / CIN) * CIN;
#pragma unroll
        for (int o = 0; o < NREAL; ++o) atomicAdd(&a.dparams[a.woff + (o * CIN + c) * 9 + t], v[o]);
      } else if (m == 9 * CIN) {
#pragma unroll
        for (int o = 0; o < NREAL; ++o) atomicAdd(&a.dparams[a.boff + o], v[o]);
      }
    }
  }
  cp_async_wait_all();  // a prefetch left in flight by an early exit lands before the block ends
  if (!ok) {
    if (tid == 0) atomicOr(a.status, kStTimeout);
    // the committed MMAs finish (bounded, ignoring the abort flag) before tensor memory
    // is freed
    uint32_t none = 0u;
    if (tid == 0 && n_issued > 0) mbar_wait(bar_done, (n_issued - 1u) & 1u, &none);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// CTAs of `smem` bytes of dynamic shared memory that fit on one SM (its shared memory over
// the CTA's share plus the per-CTA reservation); the training kernels' residency is bound
// by shared memory (their registers allow more)
int ctas_by_smem(std::atomic<int>* memo, int smem) {
  return per_device_memo(memo, [smem] {
    int dev = 0, per_sm = 0, reserved = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
    const int n = per_sm / (smem + reserved);
    return n > 0 ? n : 1;
  });
}

// true when at most 512 / kTmemCols CTAs can be resident on an SM, so that no
// tcgen05.alloc has to wait for another CTA's columns
bool tmem_fits(int ctas_per_sm) { return ctas_per_sm * kTmemCols <= 512; }

template <int CIN, int NOUT, int EPI>
bool launch_conv(const ConvArgs& a, int B, cudaStream_t st) {
  static std::atomic<int> smem_set[kMemoDevices], res[kMemoDevices];
  auto k = conv_tc_kernel<CIN, NOUT, EPI>;
  ensure_dynamic_smem(smem_set, k, kTcSmemFloor);
  if (!tmem_fits(ctas_by_smem(res, kTcSmemFloor))) return false;
  const dim3 grid((a.W + kCT - 1) / kCT, (a.H + kCH - 1) / kCH, B);
  k<<<grid, kTcThreads, kTcSmemFloor, st>>>(a);
  return true;
}

template <int CIN, int NOUT>
bool launch_wgrad(const WgradArgs& a, cudaStream_t st) {
  using L = WgradLayout<CIN, NOUT>;
  static std::atomic<int> smem_set[kMemoDevices], res[kMemoDevices];
  auto k = wgrad_tc_kernel<CIN, NOUT>;
  ensure_dynamic_smem(smem_set, k, L::REQ);
  const int per_sm = ctas_by_smem(res, L::REQ);
  if (!tmem_fits(per_sm)) return false;
  const long long chunks = (long long)a.B * a.H * ((a.W + kWK - 1) / kWK);
  const unsigned grid = (unsigned)std::min<long long>(chunks, (long long)device_sm_count() * per_sm);
  k<<<grid, kWgThreads, L::REQ, st>>>(a);
  return true;
}

}  // namespace

// packed B operands of the five convolutions: kPackLayouts x kPackBytes of scratch
size_t net_train_pack_bytes() { return (size_t)kPackLayouts * kPackBytes; }

// training forward: y [B][3][H][W]; acts (BF16 [B][2][H][W][32], a1 then a2, pixel-major)
// receives the hidden activations for the backward, or, when null, a12 (scratch of the
// same size) holds them; wpack: net_train_pack_bytes() of scratch
bool net_forward_train(const float* params, const float* x, int B, int H, int W, float* y, uint16_t* acts,
                       uint16_t* a12, uint16_t* wpack, uint32_t* status, cudaStream_t st) {
  const long long plane = (long long)B * H * W * 32;
  uint16_t* a1 = acts ? acts : a12;
  uint16_t* a2 = a1 + plane;
  pack_weights_kernel<<<dim3(8, kPackLayouts), 256, 0, st>>>(params, wpack);
  ConvArgs c{};
  c.params = params;
  c.H = H;
  c.W = W;
  c.status = status;
  c.wpack = wpack;
  c.boff = kB1;
  c.in_f32 = x;
  c.out_nhwc = a1;
  if (!launch_conv<3, 32, kEpiRelu>(c, B, st)) return false;
  c.wpack = wpack + kPackBytes / 2;
  c.boff = kB2;
  c.in_f32 = nullptr;
  c.in_bf = a1;
  c.out_nhwc = a2;
  if (!launch_conv<32, 32, kEpiRelu>(c, B, st)) return false;
  c.wpack = wpack + 2 * (kPackBytes / 2);
  c.boff = kB3;
  c.in_bf = a2;
  c.out_nhwc = nullptr;
  c.xres = x;
  c.out_f32 = y;
  return launch_conv<32, 16, kEpiResid>(c, B, st);
}

// training backward: dparams += d<dy, y>/dparams for the forward that wrote acts;
// scratch: dz2, dz1 BF16 [B][H][W][32], wpack as above
bool net_backward_train(const float* params, const float* x, const uint16_t* acts, const float* dy, int B, int H,
                        int W, float* dparams, uint16_t* dz2, uint16_t* dz1, uint16_t* wpack, uint32_t* status,
                        cudaStream_t st) {
  const long long plane = (long long)B * H * W * 32;
  const uint16_t* a1 = acts;
  const uint16_t* a2 = acts + plane;
  pack_weights_kernel<<<dim3(8, kPackLayouts), 256, 0, st>>>(params, wpack);
  ConvArgs c{};
  c.params = params;
  c.H = H;
  c.W = W;
  c.status = status;
  c.boff = -1;
  c.wpack = wpack + 3 * (kPackBytes / 2);  // dz2 = [a2 > 0] conv_T(dy, w3)
  c.in_f32 = dy;
  c.mask = a2;
  c.out_nhwc = dz2;
  if (!launch_conv<3, 32, kEpiMask>(c, B, st)) return false;
  c.wpack = wpack + 4 * (kPackBytes / 2);  // dz1 = [a1 > 0] conv_T(dz2, w2)
  c.in_f32 = nullptr;
  c.in_bf = dz2;
  c.mask = a1;
  c.out_nhwc = dz1;
  if (!launch_conv<32, 32, kEpiMask>(c, B, st)) return false;
  WgradArgs g{};
  g.dparams = dparams;
  g.B = B;
  g.H = H;
  g.W = W;
  g.status = status;
  g.woff = kW3;
  g.boff = kB3;
  g.a_bf = a2;
  g.g_f32 = dy;
  if (!launch_wgrad<32, 16>(g, st)) return false;
  g.woff = kW2;
  g.boff = kB2;
  g.a_bf = a1;
  g.g_f32 = nullptr;
  g.g_bf = dz2;
  if (!launch_wgrad<32, 32>(g, st)) return false;
  g.woff = kW1;
  g.boff = kB1;
  g.a_bf = nullptr;
  g.a_f32 = x;
  g.g_bf = dz1;
  return launch_wgrad<3, 32>(g, st);
}

}  // namespace vrs
