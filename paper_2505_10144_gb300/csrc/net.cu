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
// This file holds the inference on the periphery tiles of a rendered frame: one fused
// kernel, all three layers of a 32x32 tile in shared memory as implicit GEMMs on the
// tensor cores (tcgen05.mma, BF16 -> FP32 accumulators in tensor memory), reading the
// half-resolution image directly; and the MSE loss.  The training kernels (any image
// size, activations saved for the backward, data and weight gradients) are in
// net_train.cu.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "net.cuh"

namespace vrs {



namespace {

__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, long long n, double* sum,
                           float* __restrict__ dy, float scale) {
  double s = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    s += (double)d * d;
    if (dy) dy[i] = scale * d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  // one atomic per block (one per warp serialised on the single address)
  __shared__ double ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    atomicAdd(sum, t);
  }
}

__global__ void mse_finalize_kernel(const double* sum, long long n, float* loss) { *loss = (float)(*sum / (double)n); }

// ------------------------------------------------------------------ fused tensor-core inference
//
// One CTA of 128 threads per SM walks the periphery tiles of the frame.  Per 32x32 output
// tile, the three convolutions run as implicit GEMMs on the 5th-generation tensor cores:
// tcgen05.mma (BF16 x BF16 -> FP32, M = 128 output positions, N = 32 or 16 channels,
// K = 16 per instruction), operands in shared memory, accumulators in tensor memory.
//
// Activations are the A operand, K-major, one row per grid position: 64-byte rows (32
// channels) with the 64-byte swizzle for the conv2 and conv3 inputs, 32-byte rows with the
// 32-byte swizzle for the conv1 input, whose row p holds x(p) and x(p + 1) (8 channels
// each, 3 used).  A 3x3 tap (dy, dx) is a shift of the A start by dy * grid_width + dx
// rows, and the swizzle keeps every row an aligned, conflict-free read.  Each layer
// computes its outputs on the rows of its input grid (row width = input width): the
// rightmost outputs of a row wrap around and are discarded, and in exchange every tap is
// one uniform shift.  Weights are the B operand, K-major without swizzle: planes of 8 input
// channels x N output channels, 16 bytes per output channel.  conv1 has one instruction
// per tap pair (dy, 2j), (dy, 2j + 1); tap (dy, 3) has zero weights.
//
// Warp roles.  Warps 16-19 issue: lane 0 of MMA warp k starts the MMAs of the M tiles
// numbered k mod 4 (in issue order) and commits each tile to its accumulator's "full"
// mbarrier.  A single issuing thread waits out each tcgen05.mma before the next, which
// left the tensor cores idle most of the time; four issuers keep several M tiles in
// flight (measured on the VR stereo frame: 1.57 / 1.08 / 0.98 ms for 1 / 2 / 4 issuers,
// 1.97 ms for the mma.sync kernel this one replaced).  Warps 0-15 load the input tile
// and run the epilogues in four groups of four warps: group g takes the M tiles numbered
// g mod 4, and warp w reads tensor-memory lanes 32 (w & 3) .. + 31, the rows of its
// quarter, all 32 channels.  kAcc tensor-memory accumulators of 32 columns rotate, so the
// issuers run up to kAcc M tiles ahead of the epilogues.  Handshakes, all on mbarriers (no
// block-wide barrier inside the tile loop):
//   full[b]  the MMAs into accumulator b completed (tcgen05.commit);
//   empty[b] the four warps of the group that took its last tile have read accumulator b;
//   ready    the sixteen epilogue warps have written a layer's input (x, conv1 output or
//            conv2 output) and fenced it for the tensor cores.
// Every wait is bounded.  A thread that gives up sets kStTimeout in *status and a flag in
// shared memory that ends every other wait at once, so the block leaves together.

constexpr int kT = 32;                    // output tile
constexpr int kGx = kT + 6;               // conv1 input grid (halo 3): 38 x 38
constexpr int kG1 = kT + 4;               // conv1 output / conv2 input grid: 36 x 36
constexpr int kG2 = kT + 2;               // conv2 output / conv3 input grid: 34 x 34
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = kEpiWarps * 32;      // warps 0-15
constexpr int kIssuers = 4;                      // MMA warps (a divisor of kAcc)
constexpr int kNetThreads = kEpiThreads + 32 * kIssuers;
constexpr int kMt1 = (kG1 * kGx + 127) / 128;  // 11 M tiles of conv1 (36 rows of 38)
constexpr int kMt2 = (kG2 * kG1 + 127) / 128;  // 10 M tiles of conv2 (34 rows of 36)
constexpr int kMt3 = (kT * kG2 + 127) / 128;   // 9 M tiles of conv3 (32 rows of 34)
// positions a plane must hold: the last M tile's rows plus the largest tap shift
constexpr int kPosX = kMt1 * 128 + 2 * kGx + 3;   // 1487 (dx up to 3: zero-weight tap)
constexpr int kPos1 = kMt2 * 128 + 2 * kG1 + 2;   // 1354
constexpr int kPos2 = kMt3 * 128 + 2 * kG2 + 2;   // 1222
constexpr int kRowsX = (kPosX + 7) / 8 * 8;  // conv1 input rows of 32 bytes
constexpr int kRows1 = (kPos1 + 7) / 8 * 8;  // conv2 input rows of 64 bytes
constexpr int kRows2 = (kPos2 + 7) / 8 * 8;  // conv3 input rows of 64 bytes
constexpr int kSmW1 = 12 * 32 * 16;       // 6 MMAs x 2 K halves x [32 n][16 B]
constexpr int kSmW2 = 36 * 32 * 16;       // 9 taps x 4 channel slices x [32 n][16 B]
constexpr int kSmW3 = 36 * 16 * 16;       // 9 taps x 4 slices x [16 n][16 B] (3 real outputs)
constexpr int kSmR0 = ((kRows2 * 64 > kRowsX * 32 ? kRows2 * 64 : kRowsX * 32) + 1023) / 1024 * 1024;  // x rows, then conv2 output
constexpr int kSmR1 = kRows1 * 64;        // conv1 output
constexpr int kOffW1 = 0, kOffW2 = kOffW1 + kSmW1, kOffW3 = kOffW2 + kSmW2, kOffR0 = kOffW3 + kSmW3;
// kOffXres: float bilinear input of the 32 x 32 outputs; kOffLow: the half-resolution
// patch (21 x 21 pixels, 3 channels, clamped to the image) the tile's bilinear input reads
constexpr int kLowP = 21;
constexpr int kOffR1 = kOffR0 + kSmR0, kOffXres = kOffR1 + kSmR1, kOffLow = kOffXres + kT * kT * 12;
constexpr int kOffBias = kOffLow + 3 * kLowP * kLowP * 4 + 4, kOffBar = kOffBias + 80 * 4;
constexpr int kAcc = 8;  // tensor-memory accumulators of 32 columns (a multiple of 4, a power of two)
constexpr int kEpiGroups = kEpiWarps / 4;  // epilogue groups of four warps (one per lane quarter)
static_assert(kAcc % kIssuers == 0 && kAcc % kEpiGroups == 0, "accumulators per MMA warp and epilogue group");
// barrier area: full[kAcc], empty[kAcc], ready, then the abort flag and the TMEM address
constexpr int kBarReady = 16 * kAcc, kBarAbort = kBarReady + 8, kBarTslot = kBarReady + 12;
constexpr int kNetSmem = kOffBar + kBarReady + 16;
static_assert(kNetSmem <= 227 * 1024, "net tile does not fit in shared memory");
static_assert((kOffR0 | kOffR1) % 1024 == 0 && (kOffW2 | kOffW3) % 16 == 0, "operand alignment");
// bilinear x2 upsample (half-pixel aligned, clamped to the edge) at full-resolution pixel
// (x, y), read from the shared half-resolution patch P: patch column j, row i hold the
// image's column clamp(px0 + j), row clamp(py0 + i), so the taps x0 - px0 and x0 - px0 + 1
// are the clamped taps x0 and x0 + 1
__device__ __forceinline__ void bilinear_patch(const float* __restrict__ P, int px0, int py0, int x, int y,
                                               float v[3]) {
  const float ux = (x + 0.5f) * 0.5f - 0.5f, uy = (y + 0.5f) * 0.5f - 0.5f;
  const int x0 = (int)floorf(ux), y0 = (int)floorf(uy);
  const float fx = ux - x0, fy = uy - y0;
  const int xa = x0 - px0, ya = y0 - py0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* Pc = P + c * kLowP * kLowP;
    const float top = (1.f - fx) * Pc[ya * kLowP + xa] + fx * Pc[ya * kLowP + xa + 1];
    const float bot = (1.f - fx) * Pc[(ya + 1) * kLowP + xa] + fx * Pc[(ya + 1) * kLowP + xa + 1];
    v[c] = (1.f - fy) * top + fy * bot;
  }
}

// the MMAs of one M tile of one layer into accumulator d (issued by one thread).  A tap
// or a channel slice moves an operand's start by whole 16-byte units, so each MMA's
// descriptors are the layer's base descriptors plus an offset in the start-address field
// (every shared-memory address here is below 2^18, so the 14-bit field cannot carry).
__device__ __forceinline__ void issue_tile(int layer, int mt, uint32_t d, uint32_t sm0) {
  if (layer == 1) {
    const uint32_t id = umma_idesc(128, 32);
    // rows of 32 bytes: row p holds x(p) and x(p + 1), so one instruction covers taps
    // (dy, 2j) and (dy, 2j + 1) from row p + dy * kGx + 2j
    const uint64_t a0 = umma_desc_sw(sm0 + kOffR0, 256, 6) + (uint64_t)(mt * 128 * 2);
    const uint64_t b0 = umma_desc(sm0 + kOffW1, 512);
#pragma unroll
    for (int q = 0; q < 6; ++q) {  // q = 2 dy + j
      const int dy = q >> 1, j = q & 1;
      umma(d, a0 + (uint64_t)((dy * kGx + 2 * j) * 2), b0 + (uint64_t)(q * 64), id, q > 0);
    }
  } else {
    const int gin = layer == 2 ? kG1 : kG2;
    const uint32_t bplane = layer == 2 ? 512u : 256u;
    const uint32_t id = umma_idesc(128, layer == 2 ? 32 : 16);
    // rows of 64 bytes (32 channels); tap (dy, dx) starts dy * gin + dx rows further, and
    // the second K half 32 bytes into the row
    const uint64_t a0 = umma_desc_sw(sm0 + (layer == 2 ? kOffR1 : kOffR0), 512, 4) + (uint64_t)(mt * 128 * 4);
    const uint64_t b0 = umma_desc(sm0 + (layer == 2 ? kOffW2 : kOffW3), bplane);
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int dy = t / 3, dx = t % 3;
#pragma unroll
      for (int h = 0; h < 2; ++h)
        umma(d, a0 + (uint64_t)((dy * gin + dx) * 4 + 2 * h),
             b0 + (uint64_t)((t * 4 + 2 * h) * (int)(bplane >> 4)), id, (t | h) != 0);
    }
  }
}

// failure-detection check: phase 0 of a fresh mbarrier never completes (nothing arrives),
// so the kernel's bounded wait gives up after `limit` polls and raises kStTimeout
__global__ void mbar_timeout_kernel(uint32_t* status, int limit) {
  __shared__ uint64_t bar;
  __shared__ uint32_t abort;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    abort = 0u;
  }
  __syncthreads();
  const bool ok = mbar_wait(smem_u32(&bar), 0u, &abort, limit);
  if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
}

__global__ void __launch_bounds__(kNetThreads, 1) net_periphery_kernel(const float* __restrict__ params,
                                                                       const float* __restrict__ low,
                                                                       float* __restrict__ out,
                                                                       const uint8_t* __restrict__ tile_class,
                                                                       const ViewParams* __restrict__ views,
                                                                       int n_views, int tiles_per_view, int W, int H,
                                                                       uint32_t* __restrict__ status) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* bias = reinterpret_cast<float*>(sm + kOffBias);
  float* xres = reinterpret_cast<float*>(sm + kOffXres);
  volatile uint32_t* abort = reinterpret_cast<volatile uint32_t*>(sm + kOffBar + kBarAbort);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + kOffBar + kBarTslot);
  const uint32_t sm0 = smem_u32(sm);
  const uint32_t bar_full = sm0 + kOffBar, bar_empty = bar_full + 8 * kAcc, bar_ready = sm0 + kOffBar + kBarReady;
  const int tid = threadIdx.x, warp = tid >> 5;
  // every operand byte starts defined (plane tails are read by discarded rows only)
  for (int i = tid; i < (kOffBias - kOffR0) / 16; i += kNetThreads)
    reinterpret_cast<uint4*>(sm + kOffR0)[i] = make_uint4(0u, 0u, 0u, 0u);
  // weights to BF16 planes [slice][n][8 channels]
  for (int i = tid; i < 12 * 32 * 8; i += kNetThreads) {  // conv1: plane 2q + half, q = 2 dy + j
    const int e = i & 7, n = (i >> 3) & 31, pl = i >> 8;
    const int q = pl >> 1, dy = q >> 1, dx = 2 * (q & 1) + (pl & 1);
    const float w = (dx < 3 && e < 3) ? params[kW1 + (n * 3 + e) * 9 + dy * 3 + dx] : 0.f;
    reinterpret_cast<uint16_t*>(sm + kOffW1)[i] = bf16bits(w);
  }
  for (int i = tid; i < 36 * 32 * 8; i += kNetThreads) {  // conv2: plane 4 t + slice
    const int e = i & 7, n = (i >> 3) & 31, pl = i >> 8;
    const int t = pl >> 2, c = (pl & 3) * 8 + e;
    reinterpret_cast<uint16_t*>(sm + kOffW2)[i] = bf16bits(params[kW2 + (n * 32 + c) * 9 + t]);
  }
  for (int i = tid; i < 36 * 16 * 8; i += kNetThreads) {  // conv3: 16 output rows, 3 real
    const int e = i & 7, n = (i >> 3) & 15, pl = i >> 7;
    const int t = pl >> 2, c = (pl & 3) * 8 + e;
    reinterpret_cast<uint16_t*>(sm + kOffW3)[i] = bf16bits(n < 3 ? params[kW3 + (n * 32 + c) * 9 + t] : 0.f);
  }
  if (tid < 32) bias[tid] = params[kB1 + tid];
  if (tid < 32) bias[32 + tid] = params[kB2 + tid];
  if (tid < 3) bias[64 + tid] = params[kB3 + tid];
  if (tid == 0) {
    for (int b = 0; b < kAcc; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_full + 8u * b), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_empty + 8u * b), "r"(4));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_ready), "r"(kEpiWarps));
    *abort = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == kEpiWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(32 * kAcc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const int W2 = W / 2, H2 = H / 2;
  const long long HW = (long long)W * H, HW2 = (long long)W2 * H2;
  const long long n_tiles = (long long)n_views * tiles_per_view;
  bool ok = true;
  if (warp >= kEpiWarps) {
    // ---- MMA warps: lane 0 of MMA warp k issues the M tiles numbered k mod kIssuers, in
    // the epilogue warps' tile order (each accumulator is always fed by the same warp)
    const uint32_t k = (uint32_t)(warp - kEpiWarps);
    if ((tid & 31) == 0) {
      uint32_t cnt = 0, ph_empty = 0, ph_ready = 0;
      uint32_t nc[kAcc];  // commits into each accumulator
#pragma unroll
      for (int b = 0; b < kAcc; ++b) nc[b] = 0u;
      for (long long tg = blockIdx.x; tg < n_tiles && ok; tg += gridDim.x) {
        if (tile_class[tg] != kClassPeriphery) continue;
        for (int layer = 1; layer <= 3 && ok; ++layer) {
          ok = mbar_wait(bar_ready, ph_ready, abort);  // the layer's input is in shared memory
          ph_ready ^= 1u;
          tc_fence_after();
          const int nt = layer == 1 ? kMt1 : (layer == 2 ? kMt2 : kMt3);
          for (int mt = 0; mt < nt && ok; ++mt, ++cnt) {
            if (cnt % kIssuers != k) continue;
            const uint32_t b = cnt & (kAcc - 1u);
            // accumulator b is free once its previous tile was read (the first use of each
            // accumulator waits on the phase before the first, which counts as complete)
            ok = mbar_wait(bar_empty + 8u * b, ((ph_empty >> b) & 1u) ^ 1u, abort);
            ph_empty ^= 1u << b;
            tc_fence_after();
            if (ok) {
              issue_tile(layer, mt, tmem + 32u * b, sm0);
              umma_commit(bar_full + 8u * b);
#pragma unroll
              for (int a = 0; a < kAcc; ++a) nc[a] += (uint32_t)a == b ? 1u : 0u;
            }
          }
        }
      }
      if (!ok || *abort) {
        // the block gave up: the MMAs already committed finish (bounded waits that ignore
        // the abort flag) before their accumulators are released
        uint32_t none = 0u;
#pragma unroll
        for (int b = 0; b < kAcc; ++b)
          if (nc[b]) mbar_wait(bar_full + 8u * b, (nc[b] - 1u) & 1u, &none);
      }
    }
  } else {
    // ---- epilogue warps 0-15
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const int group = warp >> 2;  // takes the M tiles numbered group mod kEpiGroups
    float* patch = reinterpret_cast<float*>(sm + kOffLow);
    uint32_t cnt = 0, ph_full = 0;
    // the next periphery tile of this block at or after tg
    auto next_tile = [&](long long tg) {
      while (tg < n_tiles && tile_class[tg] != kClassPeriphery) tg += gridDim.x;
      return tg;
    };
    // the half-resolution patch under tile tg and its halo, this thread's values of it
    // (loads issued now, consumed when the tile starts)
    constexpr int kPatchPer = (3 * kLowP * kLowP + kEpiThreads - 1) / kEpiThreads;
    auto load_patch = [&](long long tg, float pf[kPatchPer]) {
      if (tg >= n_tiles) return;
      const int view = (int)(tg / tiles_per_view), t = (int)(tg % tiles_per_view);
      const int ntx = views[view].ntx;
      const int px0 = (t % ntx) * (kT / 2) - 2, py0 = (t / ntx) * (kT / 2) - 2;
      const float* L = low + (long long)view * 3 * HW2;
#pragma unroll
      for (int u = 0; u < kPatchPer; ++u) {
        const int i = tid + u * kEpiThreads;
        if (i < 3 * kLowP * kLowP) {
          const int c = i / (kLowP * kLowP), r = (i / kLowP) % kLowP, j = i % kLowP;
          const int gy = min(max(py0 + r, 0), H2 - 1), gx = min(max(px0 + j, 0), W2 - 1);
          pf[u] = L[c * HW2 + (long long)gy * W2 + gx];
        }
      }
    };
    float pf[kPatchPer];
    long long tg = next_tile(blockIdx.x);
    load_patch(tg, pf);
    for (; tg < n_tiles && ok;) {
      const int view = (int)(tg / tiles_per_view), t = (int)(tg % tiles_per_view);
      const ViewParams& vp = views[view];
      const int ox = (t % vp.ntx) * kT, oy = (t / vp.ntx) * kT;
      const int px0 = ox / 2 - 2, py0 = oy / 2 - 2;
#pragma unroll
      for (int u = 0; u < kPatchPer; ++u) {
        const int i = tid + u * kEpiThreads;
        if (i < 3 * kLowP * kLowP) patch[i] = pf[u];
      }
      // the following tile and its patch, loading while this tile is computed
      const long long tg_next = next_tile(tg + gridDim.x);
      load_patch(tg_next, pf);
      asm volatile("bar.sync 2, %0;" ::"n"(kEpiThreads));
      // x plane (halo 3): BF16 bilinear input, channels 3..7 zero; the float input of the
      // 32 x 32 outputs is kept for the residual
      for (int p = tid; p < kGx * kGx; p += kEpiThreads) {
        const int gx = ox - 3 + p % kGx, gy = oy - 3 + p / kGx;
        float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (gx >= 0 && gx < W && gy >= 0 && gy < H) bilinear_patch(patch, px0, py0, gx, gy, v);
        // x(p) is the first half of row p and the second half of row p - 1 (32-byte
        // swizzle: the halves swap where address bit 7 is set)
        const uint4 xq = pack8(v);
        const uint32_t sw0 = ((sm0 + kOffR0 + (uint32_t)p * 32u) >> 7) & 1u;
        *reinterpret_cast<uint4*>(sm + kOffR0 + p * 32 + (sw0 << 4)) = xq;
        if (p > 0) {
          const uint32_t sw1 = ((sm0 + kOffR0 + (uint32_t)(p - 1) * 32u) >> 7) & 1u;
          *reinterpret_cast<uint4*>(sm + kOffR0 + (p - 1) * 32 + ((1u ^ sw1) << 4)) = xq;
        }
        const int i = p / kGx - 3, j = p % kGx - 3;
        if (i >= 0 && i < kT && j >= 0 && j < kT) {
          float* xr = xres + (i * kT + j) * 3;
          xr[0] = v[0];
          xr[1] = v[1];
          xr[2] = v[2];
        }
      }
      for (int layer = 1; layer <= 3 && ok; ++layer) {
        fence_async_smem();  // this warp's writes of the layer's input, to the tensor cores
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(bar_ready);
        const int nt = layer == 1 ? kMt1 : (layer == 2 ? kMt2 : kMt3);
        const int gin = layer == 1 ? kGx : (layer == 2 ? kG1 : kG2);
        const int gout = layer == 1 ? kG1 : (layer == 2 ? kG2 : kT);
        for (int mt = 0; mt < nt && ok; ++mt, ++cnt) {
          if ((int)(cnt % kEpiGroups) != group) continue;  // another group's M tile
          const uint32_t b = cnt & (kAcc - 1u);
          ok = mbar_wait(bar_full + 8u * b, (ph_full >> b) & 1u, abort);
          ph_full ^= 1u << b;
          if (!__all_sync(0xffffffffu, ok)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const int m = mt * 128 + (warp & 3) * 32 + (tid & 31);
          const int oi = m / gin, oj = m - oi * gin;
          const uint32_t taddr = tmem + lane_base + 32u * b;
          if (layer < 3) {
            float v[32];
            tmem_ld32(taddr, v);
            tc_fence_before();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(bar_empty + 8u * b);
            if (oi < gout && oj < gout) {
              const int off = layer == 1 ? 2 : 1;
              const int gx = ox - off + oj, gy = oy - off + oi;
              const bool in = gx >= 0 && gx < W && gy >= 0 && gy < H;
              const float* bb = bias + (layer == 1 ? 0 : 32);
#pragma unroll
              for (int c = 0; c < 32; ++c) v[c] = in ? fmaxf(v[c] + bb[c], 0.f) : 0.f;
              const uint32_t row = (uint32_t)(layer == 1 ? kOffR1 : kOffR0) + (uint32_t)(oi * gout + oj) * 64u;
              const uint32_t sw = ((sm0 + row) >> 7) & 3u;  // 64-byte swizzle of this row
#pragma unroll
              for (int q = 0; q < 4; ++q) *reinterpret_cast<uint4*>(sm + row + ((q ^ sw) << 4)) = pack8(v + 8 * q);
            }
          } else {  // three output channels
            float v[4];
            tmem_ld4(taddr, v);
            tc_fence_before();
            __syncwarp();
            if ((tid & 31) == 0) mbar_arrive(bar_empty + 8u * b);
            const int gx = ox + oj, gy = oy + oi;
            if (oi < kT && oj < kT && gx < W && gy < H) {
              const float* xr = xres + (oi * kT + oj) * 3;
              float* o = out + (long long)view * 3 * HW + (long long)gy * W + gx;
#pragma unroll
              for (int c = 0; c < 3; ++c) o[(long long)c * HW] = xr[c] + v[c] + bias[64 + c];
            }
          }
        }
      }
      // the next tile's patch, x plane and residual input overwrite shared memory: conv3's
      // MMAs (which read R0) have all completed, and every epilogue warp is past its reads
      asm volatile("bar.sync 1, %0;" ::"n"(kEpiThreads));
      tg = tg_next;
    }
  }
  if (!ok) atomicOr(status, kStTimeout);
  // every committed MMA has completed here: the epilogue warps awaited each one, or, when
  // the block gave up, the issuing lane did
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kEpiWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(32 * kAcc));
}

unsigned grid_for(long long n) {
  return (unsigned)std::min<long long>((n + 255) / 256, (long long)device_sm_count() * 16);
}

}  // namespace

void net_mse(const float* y, const float* t, long long n, float* loss, float* dy, double* scratch, cudaStream_t st) {
  cudaMemsetAsync(scratch, 0, sizeof(double), st);
  mse_kernel<<<grid_for(n), 256, 0, st>>>(y, t, n, scratch, dy, (float)(2.0 / (double)n));
  mse_finalize_kernel<<<1, 1, 0, st>>>(scratch, n, loss);
}

void net_periphery(const float* params, const float* low, float* out, const uint8_t* tile_class,
                   const ViewParams* views, int n_views, int tiles_per_view, int W, int H, uint32_t* status,
                   cudaStream_t st) {
  static std::atomic<int> smem_set[kMemoDevices];
  ensure_dynamic_smem(smem_set, net_periphery_kernel, kNetSmem);
  const long long n = (long long)n_views * tiles_per_view;
  const unsigned grid = (unsigned)std::min<long long>(n, (long long)device_sm_count());
  net_periphery_kernel<<<grid, kNetThreads, kNetSmem, st>>>(params, low, out, tile_class, views, n_views,
                                                            tiles_per_view, W, H, status);
}

void launch_mbar_timeout_test(uint32_t* status, cudaStream_t st) { mbar_timeout_kernel<<<1, 128, 0, st>>>(status, 1000); }

int net_smem_bytes() { return kNetSmem; }

}  // namespace vrs
