// The periphery network's parameter layout, and the device helpers its tensor-core kernels
// (inference in net.cu, training in net_train.cu) share: BF16 conversions, tcgen05
// shared-memory and instruction descriptors, the MMA and its commit, bounded mbarrier
// waits, tensor-memory loads and the fences between the generic, async and tensor-core
// proxies.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace vrs {

// parameters: one float32 buffer, OIHW: w1[32][3][3][3] b1[32] w2[32][32][3][3] b2[32]
// w3[3][32][3][3] b3[3]
constexpr int kNetCh = 32;
constexpr int kW1 = 0, kB1 = 864, kW2 = 896, kB2 = 10112, kW3 = 10144, kB3 = 11008, kNetParams = 11011;
static_assert(kB1 == kW1 + kNetCh * 3 * 9 && kW2 == kB1 + kNetCh && kB2 == kW2 + kNetCh * kNetCh * 9 &&
                  kW3 == kB2 + kNetCh && kB3 == kW3 + 3 * kNetCh * 9 && kNetParams == kB3 + 3,
              "parameter offsets (OIHW)");

namespace {

__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

__device__ __forceinline__ uint16_t bf16bits(float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  return *reinterpret_cast<const uint16_t*>(&b);
}

__device__ __forceinline__ float bits2f(uint16_t u) {
  return __uint_as_float(((uint32_t)u) << 16);
}

constexpr long long kWaitLimit = 1ll << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: no swizzle, K-core stride lbo, 8-row-group stride 128 B
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)(128u >> 4) << 32) | (1ull << 46);
}

// shared-memory matrix descriptor, K-major with a 32-byte (layout 6) or 64-byte (layout
// 4) swizzle: rows of 32 or 64 bytes, 8-row groups sbo bytes apart; the swizzle acts on
// absolute address bits (XOR of bits 7 (.. 8) into bits 4 (.. 5)), so a start shifted by
// whole rows, or by 32 bytes along K inside a 64-byte row, needs no base offset
__device__ __forceinline__ uint64_t umma_desc_sw(uint32_t addr, uint32_t sbo, uint32_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | (1ull << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46) | ((uint64_t)layout << 61);
}

// instruction descriptor: BF16 A and B (K-major), FP32 accumulator, M x N
__device__ __forceinline__ uint32_t umma_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

// waits for the phase of the given parity; false when the wait gave up or another thread
// of the block did (*abort)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, volatile uint32_t* abort,
                                          long long limit = kWaitLimit) {
  uint32_t done = 0;
  for (long long it = 0; it < limit && !done; ++it) {
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity));
    if (!done && *abort) return false;
  }
  if (!done) *abort = 1u;
  return done != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  __syncwarp();
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 32; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float v[4]) {
  uint32_t r[4];
  __syncwarp();
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 4; ++c) v[c] = __uint_as_float(r[c]);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16-byte asynchronous copy global -> shared; src_bytes 0 reads nothing and zero-fills
// (src must still be a valid address)
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// 8 BF16 values of one 16-byte plane slot
__device__ __forceinline__ uint4 pack8(const float* v) {
  uint4 q;
  q.x = (uint32_t)bf16bits(v[0]) | ((uint32_t)bf16bits(v[1]) << 16);
  q.y = (uint32_t)bf16bits(v[2]) | ((uint32_t)bf16bits(v[3]) << 16);
  q.z = (uint32_t)bf16bits(v[4]) | ((uint32_t)bf16bits(v[5]) << 16);
  q.w = (uint32_t)bf16bits(v[6]) | ((uint32_t)bf16bits(v[7]) << 16);
  return q;
}


}  // namespace
}  // namespace vrs
