// vrs_sort_pairs_noalloc: the radix sort of vrs_sort_pairs without any memory
// allocation, for callers that cannot allocate GPU memory when they need to sort.
//
// Who cannot allocate: code running inside a frame callback with a hard latency budget
// (a VR compositor or engine plugin), where cudaMalloc / cudaFree can synchronise the
// device and stall the frame; applications that hand all GPU memory to their own pool
// and forbid other allocations; and code that must not fail part-way through a frame
// because an allocation hit memory pressure.  Such callers get a fixed scratch area
// that is reserved when the library is loaded.
//
// The scratch is one file-scope device array, g_noalloc_scratch, of fixed size.  Every
// GPU that loads the library holds it until the process exits.  It serves every call:
// it holds the second ping-pong buffer of keys and values, the digit histograms, the
// look-back flags, the tile counters and the item count.  Each call clears the parts
// that must start at zero (histograms, flags, counters) on its stream before it sorts.
// Calls whose work overlaps on the GPU (on different streams, or from several host
// threads) race on this one array and give undefined results: serialise them.
#include "common.cuh"

namespace vrs {

namespace {

constexpr long long kNoallocMax = VRS_SORT_NOALLOC_MAX_PAIRS;
constexpr long long kNoallocTiles = (kNoallocMax + 4095) / 4096 + 1;
// sort scratch as the sort carves it: histograms + counters, then look-back flags
constexpr size_t kSortScratchBytes = (size_t)(8 * 256 + 16) * 4 + (size_t)8 * kNoallocTiles * 256 * 4;
constexpr size_t kKeysOff = 0;
constexpr size_t kValsOff = kKeysOff + (size_t)kNoallocMax * 8;
constexpr size_t kSortOff = (kValsOff + (size_t)kNoallocMax * 4 + 255) / 256 * 256;
constexpr size_t kMiscOff = (kSortOff + kSortScratchBytes + 255) / 256 * 256;  // item count, status
constexpr size_t kNoallocBytes = kMiscOff + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

__global__ void noalloc_set_n_kernel(uint32_t* p, uint32_t v) { *p = v; }

__global__ void noalloc_status_kernel(const uint32_t* status, uint32_t* out) { *out = *status; }

// Device address of the scratch array on the current device.  In host code the array's
// name is only a stand-in, so the address comes from cudaGetSymbolAddress, with the
// device current.  The lookup is a host-side call and runs on every call: a cached
// address would go stale if the device's primary context were reset and re-created.
vrs_status scratch_for_current_device(unsigned char** out) {
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return VRS_ERR_CUDA;
  *out = static_cast<unsigned char*>(p);
  return VRS_OK;
}

}  // namespace

}  // namespace vrs

extern "C" vrs_status vrs_sort_pairs_noalloc(const uint64_t* d_keys_in, const uint32_t* d_vals_in,
                                             uint64_t* d_keys_out, uint32_t* d_vals_out, int64_t n, int bits,
                                             uint32_t* d_status, void* stream) {
  using namespace vrs;
  if (n < 0 || n > kNoallocMax || bits < 1 || bits > 64) return VRS_ERR_INVALID;
  if (n > 0 && (!d_keys_in || !d_vals_in || !d_keys_out || !d_vals_out)) return VRS_ERR_INVALID;
  if (sort_scratch_bytes(kNoallocMax) > kSortScratchBytes) return VRS_ERR_UNSUPPORTED;
  if (n == 0) return VRS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // an error left by an earlier, unrelated runtime call is not this call's: clear it so
  // that the check at the end reports only what this call launched
  (void)cudaGetLastError();
  unsigned char* base = nullptr;
  vrs_status s = scratch_for_current_device(&base);
  if (s != VRS_OK) return s;
  uint64_t* alt_keys = reinterpret_cast<uint64_t*>(base + kKeysOff);
  uint32_t* alt_vals = reinterpret_cast<uint32_t*>(base + kValsOff);
  uint32_t* misc = reinterpret_cast<uint32_t*>(base + kMiscOff);  // [0] item count, [1] status
  SortScratch ss;
  sort_scratch_carve(base + kSortOff, kNoallocMax, &ss);
  if (cudaMemsetAsync(misc, 0, 2 * sizeof(uint32_t), st) != cudaSuccess) return VRS_ERR_CUDA;
  if (d_keys_out != d_keys_in &&
      cudaMemcpyAsync(d_keys_out, d_keys_in, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return VRS_ERR_CUDA;
  if (d_vals_out != d_vals_in &&
      cudaMemcpyAsync(d_vals_out, d_vals_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return VRS_ERR_CUDA;
  noalloc_set_n_kernel<<<1, 1, 0, st>>>(misc, (uint32_t)n);
  uint64_t* kb[2] = {d_keys_out, alt_keys};
  uint32_t* vb[2] = {d_vals_out, alt_vals};
  // launch_radix_sort clears the histograms, counters and look-back flags it uses
  const int cur = launch_radix_sort(kb, vb, misc, n, bits, ss, misc + 1, st);
  // a failed launch or clear inside the sort leaves the alternate buffer stale: stop
  // before copying it out
  if (cudaGetLastError() != cudaSuccess) return VRS_ERR_CUDA;
  if (cur == 1) {
    if (cudaMemcpyAsync(d_keys_out, alt_keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(d_vals_out, alt_vals, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return VRS_ERR_CUDA;
  }
  if (d_status) noalloc_status_kernel<<<1, 1, 0, st>>>(misc + 1, d_status);
  return cudaGetLastError() == cudaSuccess ? VRS_OK : VRS_ERR_CUDA;
}
