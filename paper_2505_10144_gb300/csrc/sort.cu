// Device-wide exclusive scan and a onesweep LSD radix sort of (uint64 key, uint32 value)
// pairs: one pass builds the 8-bit digit histograms of every pass, then one kernel per
// digit ranks a 4096-item tile in shared memory, publishes its digit counts and finds
// its global offsets by decoupled look-back over the preceding tiles.  Tiles are taken
// in order from an atomic counter by resident CTAs, so every tile a CTA waits on is
// already held by a running CTA.  Every wait is bounded; on timeout the kernel raises
// kStTimeout in the status word and finishes without hanging.
//
// The sorted order is stable, which gives the (tile | depth, Gaussian index) order of
// Sec. 3 ("this arrangement is sorted") since instances are emitted in index order.
#include <algorithm>

#include "common.cuh"

namespace vrs {

namespace {

constexpr int kScanItems = 16;
constexpr int kScanTile = kBlock * kScanItems;  // 4096

constexpr int kSortItems = 16;
constexpr int kSortWarps = kBlock / 32;
constexpr int kSortTile = kBlock * kSortItems;  // 4096
constexpr int kMaxPasses = 8;
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPrefix = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kSpinLimit = 1 << 22;

// tiles a look-back step reads at once
constexpr int kLookWindow = 16;

__device__ __forceinline__ uint32_t load_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Decoupled look-back: the sum of digit d's counts over the tiles before `tile`, read from
// their published (flag | count) words, walking back until a tile that holds its full
// prefix.  Each step reads the words of kLookWindow preceding tiles at once (for a warp,
// one 128-byte line per tile) and consumes them nearest first.  The tiles of a CTA wave
// publish their aggregates at about the same time, and tile k of the wave would otherwise
// read one word per L2 round trip until it meets a prefix, about k / 2 steps in; with a
// window it is about k / (kLookWindow + 1) steps.  A word not yet published is polled
// again; after spin_limit such polls the wait gives up, raises kStTimeout and returns
// false (excl then holds a partial sum).  The words carry the counts themselves, so
// relaxed loads suffice.
__device__ __forceinline__ bool lookback_prefix(uint32_t* look, long long tile, int d, int spin_limit,
                                                uint32_t* status, uint32_t& excl) {
  excl = 0;
  long long j = tile - 1;  // the nearest tile not yet consumed
  int spins = 0;
  while (j >= 0) {
    uint32_t lv[kLookWindow];
#pragma unroll
    for (int q = 0; q < kLookWindow; ++q) lv[q] = j - q >= 0 ? load_relaxed(look + (j - q) * 256 + d) : kFlagPrefix;
    bool blocked = false, done = false;
    int used = 0;
#pragma unroll
    for (int q = 0; q < kLookWindow; ++q) {
      if (blocked || done) continue;
      const uint32_t flag = lv[q] & ~kCountMask;
      if (flag == 0u) {
        blocked = true;
      } else {
        excl += lv[q] & kCountMask;
        ++used;
        done = flag == kFlagPrefix;
      }
    }
    if (done) return true;
    j -= used;
    if (blocked) {
      if (++spins > spin_limit) {
        atomicOr(status, kStTimeout);
        return false;
      }
      __nanosleep(20);
    }
  }
  return true;
}

// failure-detection check: tile 1 waits on tile 0's words, which nothing publishes (the
// caller zeroes them), so every thread's wait gives up after spin_limit polls
__global__ void lookback_timeout_kernel(uint32_t* look, uint32_t* status, int spin_limit) {
  uint32_t excl;
  lookback_prefix(look, 1, (int)threadIdx.x, spin_limit, status, excl);
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < kBlock / 32 ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kBlock / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  const uint32_t wprefix = wid ? warp_sums[wid - 1] : 0u;
  if (total) *total = warp_sums[kBlock / 32 - 1];
  const uint32_t r = wprefix + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kBlock) scan_reduce_kernel(const uint32_t* __restrict__ in, long long n,
                                                             uint32_t* __restrict__ partials) {
  __shared__ uint32_t ws[32];
  const long long base = (long long)blockIdx.x * kScanTile;
  uint32_t s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + (long long)k * kBlock + threadIdx.x;
    if (i < n) s += in[i];
  }
  uint32_t total;
  block_exclusive_scan(s, ws, &total);
  if (threadIdx.x == 0) partials[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kBlock) scan_partials_kernel(uint32_t* partials, long long nb, uint32_t* d_total) {
  __shared__ uint32_t ws[32];
  uint32_t carry = 0;
  for (long long b0 = 0; b0 < nb; b0 += kBlock) {
    const long long i = b0 + threadIdx.x;
    const uint32_t v = i < nb ? partials[i] : 0u;
    uint32_t total;
    const uint32_t e = block_exclusive_scan(v, ws, &total);
    if (i < nb) partials[i] = carry + e;
    carry += total;
  }
  if (threadIdx.x == 0) *d_total = carry;
}

__global__ void __launch_bounds__(kBlock) scan_final_kernel(const uint32_t* __restrict__ in, long long n,
                                                            const uint32_t* __restrict__ partials,
                                                            uint32_t* __restrict__ out) {
  __shared__ uint32_t ws[32];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    v[k] = i < n ? in[i] : 0u;
    s += v[k];
  }
  uint32_t run = partials[blockIdx.x] + block_exclusive_scan(s, ws, nullptr);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const long long i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

// digit histograms of every pass in one read of the keys
__device__ __forceinline__ uint32_t digit_mask(int bits, int pass) {
  const int rem = bits - 8 * pass;
  return rem >= 8 ? 0xFFu : ((1u << rem) - 1u);
}

__global__ void __launch_bounds__(kBlock) histogram_kernel(const uint64_t* __restrict__ keys, const uint32_t* d_n,
                                                           int passes, int bits, uint32_t* __restrict__ hist) {
  __shared__ uint32_t h[kMaxPasses][256];
  for (int i = threadIdx.x; i < kMaxPasses * 256; i += kBlock) (&h[0][0])[i] = 0u;
  __syncthreads();
  const long long n = *d_n;
  for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock) {
    const uint64_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & digit_mask(bits, p)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += kBlock) {
    const uint32_t v = (&h[0][0])[i];
    if (v) atomicAdd(&hist[i], v);
  }
}

// The lanes of the warp whose digit equals this lane's (d < 256, or 256 for an item past
// the end): one ballot per digit bit, each keeping the lanes that agree on that bit.
// __match_any_sync gives the same mask, but it runs on a low-throughput unit: with it the
// ranking loop was the pass's bottleneck (short-scoreboard stalls, 8 of 16 cycles per
// issued instruction, on 2.47 M keys).
__device__ __forceinline__ unsigned digit_peers(int d) {
  unsigned peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool bit = (d >> b) & 1;
    const unsigned bal = __ballot_sync(0xffffffffu, bit);
    peers &= bit ? bal : ~bal;
  }
  return peers;
}

struct SortSmem {
  uint64_t keys[kSortTile];
  uint32_t vals[kSortTile];
  uint32_t warp_hist[kSortWarps][256];
  uint32_t digit_start[256];
  uint32_t digit_offset[256];  // first output position of each digit (scan of the pass's histogram)
  uint32_t global_base[256];
  uint32_t ws[32];
  uint32_t tile;
};

__global__ void __launch_bounds__(kBlock) onesweep_kernel(const uint64_t* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                          const uint32_t* d_n, int shift, uint32_t dmask,
                                                          const uint32_t* __restrict__ digit_counts,
                                                          uint32_t* __restrict__ look, uint32_t* tile_counter,
                                                          uint32_t* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SortSmem& S = *reinterpret_cast<SortSmem*>(smem_raw);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long n = *d_n;
  const uint32_t lt_mask = (1u << lane) - 1u;
  // the pass's digit offsets, scanned by every CTA from the histogram (256 values) instead
  // of by a separate one-block launch
  S.digit_offset[threadIdx.x] = block_exclusive_scan(digit_counts[threadIdx.x], S.ws, nullptr);
  for (;;) {
    if (threadIdx.x == 0) S.tile = atomicAdd(tile_counter, 1u);
    for (int i = threadIdx.x; i < kSortWarps * 256; i += kBlock) (&S.warp_hist[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t tile = S.tile;
    const long long base = (long long)tile * kSortTile;
    if (base >= n) break;
    const long long wbase = base + (long long)wid * 32 * kSortItems;
    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank[kSortItems];
    int dg[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const long long idx = wbase + it * 32 + lane;
      const bool ok = idx < n;
      k[it] = ok ? kin[idx] : 0ull;
      v[it] = ok ? vin[idx] : 0u;
      dg[it] = ok ? (int)((k[it] >> shift) & dmask) : 256;
    }
    // warp-level stable ranking: items in (it, lane) order
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const unsigned peers = digit_peers(dg[it]);
      const int leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (dg[it] < 256) before = S.warp_hist[wid][dg[it]];
      rank[it] = before + __popc(peers & lt_mask);
      __syncwarp();
      if (lane == leader && dg[it] < 256) S.warp_hist[wid][dg[it]] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // per digit: counts across warps, tile-local digit starts, look-back
    const int d = threadIdx.x;
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = S.warp_hist[w][d];
      S.warp_hist[w][d] = cnt;  // becomes the exclusive offset of warp w within digit d
      cnt += c;
    }
    uint32_t* my_look = look + (long long)tile * 256 + d;
    if (tile == 0) {
      atomicExch(my_look, kFlagPrefix | cnt);
    } else {
      atomicExch(my_look, kFlagAgg | cnt);
    }
    uint32_t excl = 0;
    if (tile > 0) {
      lookback_prefix(look, tile, d, kSpinLimit, status, excl);
      atomicExch(my_look, kFlagPrefix | (excl + cnt));
    }
    S.global_base[d] = S.digit_offset[d] + excl;
    const uint32_t start = block_exclusive_scan(cnt, S.ws, nullptr);
    S.digit_start[d] = start;
    __syncthreads();
    // stage in digit order
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      if (dg[it] < 256) {
        const uint32_t pos = S.digit_start[dg[it]] + S.warp_hist[wid][dg[it]] + rank[it];
        S.keys[pos] = k[it];
        S.vals[pos] = v[it];
      }
    }
    __syncthreads();
    const int valid = (int)min((long long)kSortTile, n - base);
    for (int i = threadIdx.x; i < valid; i += kBlock) {
      const uint64_t kk = S.keys[i];
      const int dd = (int)((kk >> shift) & dmask);
      const uint32_t o = S.global_base[dd] + (uint32_t)i - S.digit_start[dd];
      if ((long long)o < n) {  // always true unless a look-back timed out
        kout[o] = kk;
        vout[o] = S.vals[i];
      }
    }
    __syncthreads();
  }
}

__global__ void ranges_kernel(const uint64_t* __restrict__ keys, const uint32_t* d_n, uint32_t* __restrict__ ranges,
                              long long n_tiles) {
  const long long n = *d_n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(keys[i] >> 32);
    if ((long long)t >= n_tiles) continue;
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != t) ranges[2 * (long long)t] = (uint32_t)i;
    if (i == n - 1 || (uint32_t)(keys[i + 1] >> 32) != t) ranges[2 * (long long)t + 1] = (uint32_t)(i + 1);
  }
}

}  // namespace

size_t scan_partials_bytes(long long n) { return (size_t)((n + kScanTile - 1) / kScanTile + 1) * sizeof(uint32_t); }

void launch_scan_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* d_total, uint32_t* partials,
                     cudaStream_t st) {
  if (n <= 0) {
    cudaMemsetAsync(d_total, 0, sizeof(uint32_t), st);
    return;
  }
  const long long nb = (n + kScanTile - 1) / kScanTile;
  scan_reduce_kernel<<<(unsigned)nb, kBlock, 0, st>>>(in, n, partials);
  scan_partials_kernel<<<1, kBlock, 0, st>>>(partials, nb, d_total);
  scan_final_kernel<<<(unsigned)nb, kBlock, 0, st>>>(in, n, partials, out);
}

size_t sort_scratch_bytes(long long cap) {
  const long long tiles = (cap + kSortTile - 1) / kSortTile + 1;
  return (size_t)(kMaxPasses * 256 + 16) * sizeof(uint32_t) + (size_t)kMaxPasses * tiles * 256 * sizeof(uint32_t);
}

void sort_scratch_carve(void* base, long long cap, SortScratch* s) {
  uint32_t* p = reinterpret_cast<uint32_t*>(base);
  s->hist = p;
  s->counters = p + kMaxPasses * 256;
  s->look = s->counters + 16;
  s->max_tiles = (cap + kSortTile - 1) / kSortTile + 1;
}

int device_sm_count() {
  static std::atomic<int> sms[kMemoDevices];
  return per_device_memo(sms, [] {
    int n = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  });
}

int launch_radix_sort(uint64_t* keys[2], uint32_t* vals[2], const uint32_t* d_n, long long cap, int bits,
                      const SortScratch& s, uint32_t* status, cudaStream_t st) {
  const int passes = (bits + 7) / 8;
  if (cap <= 0 || passes <= 0) return 0;
  const long long tiles = (cap + kSortTile - 1) / kSortTile;
  cudaMemsetAsync(s.hist, 0, sizeof(uint32_t) * (kMaxPasses * 256 + 16), st);
  cudaMemsetAsync(s.look, 0, sizeof(uint32_t) * (size_t)passes * (size_t)(tiles + 1) * 256, st);
  const int sms = device_sm_count();
  const unsigned hgrid = (unsigned)std::min<long long>((cap + kBlock * 8 - 1) / (kBlock * 8), (long long)sms * 8);
  histogram_kernel<<<hgrid, kBlock, 0, st>>>(keys[0], d_n, passes, bits, s.hist);
  const int smem = (int)sizeof(SortSmem);
  static std::atomic<int> smem_set[kMemoDevices], occupancy[kMemoDevices];
  ensure_dynamic_smem(smem_set, onesweep_kernel, smem);
  const int per_sm = per_device_memo(occupancy, [smem] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, onesweep_kernel, kBlock, smem);
    return b > 0 ? b : 1;
  });
  const unsigned grid = (unsigned)std::min<long long>(tiles, (long long)sms * per_sm);
  int cur = 0;
  for (int p = 0; p < passes; ++p) {
    const int rem = bits - 8 * p;
    const uint32_t dmask = rem >= 8 ? 0xFFu : ((1u << rem) - 1u);
    onesweep_kernel<<<grid, kBlock, smem, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], d_n, 8 * p, dmask,
                                                s.hist + p * 256, s.look + (size_t)p * (size_t)(tiles + 1) * 256,
                                                s.counters + p, status);
    cur ^= 1;
  }
  return cur;
}

void launch_ranges(const uint64_t* keys, const uint32_t* d_n, long long cap, uint32_t* ranges, long long n_tiles,
                   cudaStream_t st) {
  if (cap <= 0) return;
  const unsigned grid = (unsigned)std::min<long long>((cap + 255) / 256, (long long)device_sm_count() * 8);
  ranges_kernel<<<grid, 256, 0, st>>>(keys, d_n, ranges, n_tiles);
}

void launch_lookback_timeout_test(uint32_t* zeroed_look, uint32_t* status, cudaStream_t st) {
  lookback_timeout_kernel<<<1, 256, 0, st>>>(zeroed_look, status, 1000);
}

}  // namespace vrs
