// vrs_measure_peaks: microbenchmarks of the throughputs that bound the render kernel
// (FP32 FMA, the exp2f of the pair opacity, 32-bit logic on the integer ALU pipe) and of
// the L2 and HBM read bandwidths that serve its record re-reads.  They give the measured
// denominators of the render roofline; the device properties (SM count, clock, L2 size)
// come from the runtime.
//
// Each throughput kernel keeps kChains independent dependency chains per thread, and
// a grid of 8 blocks of 256 threads per SM (64 warps, the SM's limit), so that latency
// is hidden and the pipe under test is the bound.  Each result is the best of kTrials
// timed launches after one untimed launch, timed with CUDA events on the caller's
// stream.
#include <cuda_runtime.h>

#include <cstdint>

#include "vrsplat.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;
constexpr int kThroughputThreads = 256;
constexpr int kBlocksPerSm = 8;
constexpr int kTrials = 5;

__global__ void __launch_bounds__(kThroughputThreads) fma_peak_kernel(float x, float y, int iters, float* out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1e-3f * (float)threadIdx.x + (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], x, y);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// the opacity exponent as the render kernel evaluates it: exp2f of a difference
__global__ void __launch_bounds__(kThroughputThreads) exp2_peak_kernel(float c, int iters, float* out) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 0.01f * (float)(threadIdx.x & 7) + 0.1f * (float)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = exp2f(c - a[k]);
    }
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// one three-input logic operation per step: (a & x) ^ (a | y)
__global__ void __launch_bounds__(kThroughputThreads) logic_peak_kernel(uint32_t x, uint32_t y, int iters,
                                                                       uint32_t* out) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 2654435761u + (uint32_t)k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = (a[k] & x) ^ (a[k] | y);
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// reads n4 float4 `reps` times; kL2 selects ld.global.cg (cached in L2, not L1) or
// ld.global.cs (streaming, evict first)
template <bool kL2>
__global__ void __launch_bounds__(512, 2) read_peak_kernel(const float4* __restrict__ buf, long long n4, int reps,
                                                        float* out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  for (int r = 0; r < reps; ++r) {
    for (long long i = i0; i < n4; i += 4 * stride) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const long long j = i + u * stride;
        if (j < n4) {
          v[u] = kL2 ? __ldcg(buf + j) : __ldcs(buf + j);
        } else {
          v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
    }
  }
  out[i0] = acc;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t err = cudaSuccess;
  Timer() {
    err = cudaEventCreate(&a);
    if (err == cudaSuccess) err = cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// best time (ms) of kTrials launches of `launch` after one untimed launch
template <class F>
cudaError_t best_ms(Timer& t, cudaStream_t st, F launch, float* ms) {
  launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  float best = 1e30f;
  for (int i = 0; i < kTrials; ++i) {
    cudaEventRecord(t.a, st);
    launch();
    cudaEventRecord(t.b, st);
    e = cudaEventSynchronize(t.b);
    if (e != cudaSuccess) return e;
    float m = 0.f;
    e = cudaEventElapsedTime(&m, t.a, t.b);
    if (e != cudaSuccess) return e;
    if (m < best) best = m;
  }
  *ms = best;
  return cudaGetLastError();
}

}  // namespace

extern "C" vrs_status vrs_measure_peaks(vrs_peaks* out, void* stream) {
  if (!out) return VRS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0, clk = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return VRS_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&clk, cudaDevAttrClockRate, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess)
    return VRS_ERR_CUDA;
  out->sm_count = sms;
  out->max_sm_clock_khz = clk;
  out->l2_bytes = l2;

  Timer t;
  if (t.err != cudaSuccess) return VRS_ERR_CUDA;
  const int grid = sms * kBlocksPerSm;
  const long long threads = (long long)grid * kThroughputThreads;
  // L2 working set: a quarter of the L2; HBM working set: 2 GiB, read once
  const long long l2_n4 = ((long long)l2 / 4) / 16;
  const long long dram_n4 = (2ll << 30) / 16;
  void* sink = nullptr;
  void* buf = nullptr;
  vrs_status rc = VRS_OK;
  float ms = 0.f;
  const int fma_iters = 2048, exp_iters = 512, logic_iters = 2048, l2_reps = 256;
  const int read_grid = sms * 2;  // two blocks of 512 per SM (the register limit)
  do {
    if (cudaMalloc(&sink, (size_t)(threads > (long long)read_grid * 512 ? threads : (long long)read_grid * 512) * 4) !=
            cudaSuccess ||
        cudaMalloc(&buf, (size_t)dram_n4 * 16) != cudaSuccess ||
        cudaMemsetAsync(buf, 0, (size_t)dram_n4 * 16, st) != cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    float* fs = (float*)sink;
    if (best_ms(t, st, [&] { fma_peak_kernel<<<grid, kThroughputThreads, 0, st>>>(0.999f, 1e-3f, fma_iters, fs); },
                &ms) != cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    out->fp32_tflops = 2.0 * (double)threads * fma_iters * kUnroll * kChains / (ms * 1e-3) / 1e12;
    if (best_ms(t, st, [&] { exp2_peak_kernel<<<grid, kThroughputThreads, 0, st>>>(0.f, exp_iters, fs); }, &ms) !=
        cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    out->exp2_gops = (double)threads * exp_iters * kUnroll * kChains / (ms * 1e-3) / 1e9;
    if (best_ms(t, st,
                [&] {
                  logic_peak_kernel<<<grid, kThroughputThreads, 0, st>>>(0x9e3779b9u, 0x7f4a7c15u, logic_iters,
                                                                         (uint32_t*)sink);
                },
                &ms) != cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    out->logic_gops = (double)threads * logic_iters * kUnroll * kChains / (ms * 1e-3) / 1e9;
    const float4* b4 = (const float4*)buf;
    if (best_ms(t, st, [&] { read_peak_kernel<true><<<read_grid, 512, 0, st>>>(b4, l2_n4, l2_reps, fs); }, &ms) !=
        cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    out->l2_read_gbs = (double)l2_n4 * 16 * l2_reps / (ms * 1e-3) / 1e9;
    if (best_ms(t, st, [&] { read_peak_kernel<false><<<read_grid, 512, 0, st>>>(b4, dram_n4, 1, fs); }, &ms) !=
        cudaSuccess) {
      rc = VRS_ERR_CUDA;
      break;
    }
    out->dram_read_gbs = (double)dram_n4 * 16 / (ms * 1e-3) / 1e9;
  } while (false);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  return rc;
}
