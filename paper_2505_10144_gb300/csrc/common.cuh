// Internal declarations shared by the CUDA translation units of libvrsplat.
//
// Projected record of one Gaussian for one view (Optimal Projection, Sec. 4.2), six
// float4 = 96 bytes, all in pixel units relative to the projected mean pm = K u / u_z:
//
//   f0 = (pm_x, pm_y, h00, h01)      a = h00 dx + h01 dy         (dx, dy) = p - pm
//   f1 = (h10, h11, h20, h21)        b = h10 dx + h11 dy
//   f2 = (h22, a00, a01x2, a11)      w = h20 dx + h21 dy + h22   (a, b, w) = [E; u] K^-1 p~
//   f3 = (log2 sigma, n0, n1, n2)    tangent-plane point s = (a, b) / w
//   f4 = (m00, m01x2, m11, m02x2)    q' = s^T A' s,  A' = 0.5 log2(e) Sigma_p^-1
//   f5 = (m12x2, r, g, b)            alpha = min(0.99, 2^(log2 sigma - q'))
//
// depth of maximum response along the ray (StopThePop, Sec. 4.1):
//   t* = (n0 dx + n1 dy + n2) / (m00 dx^2 + m01x2 dx dy + m11 dy^2 + m02x2 dx + m12x2 dy + 1)
// which is the camera-space z of argmax_t G(t v), v = K^-1 p~, normalised so that
// t*(pm) = n2 = z of the mean.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/vrsplat.h"

namespace vrs {

constexpr int kRecF4 = 6;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTStop = 1e-4f;
constexpr float kLog2_255 = 7.994353436858858f;
constexpr float kHalfLog2e = 0.7213475204444817f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kDilationPx2 = 0.3f;

// device status word bits
constexpr uint32_t kStTimeout = 1u;
constexpr uint32_t kStOverflow = 2u;

constexpr int kMaxWin = 32;
constexpr int kBlock = 256;
// instances of one render (32-bit list indices in the render kernels)
constexpr long long kMaxInstances = (1ll << 31) - 1;

struct ViewParams {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, near_z;
  int W, H;
  int scene;
  int ntx, nty;     // key tiles per row / column
  long long base;   // offset of this view in the per-(view, Gaussian) arrays
  float gaze_x, gaze_y, radius, band;
  const uint8_t* visible;  // [H][W] headset visibility mask (nonzero = visible) or null
  // the layer this view renders: Gaussians whose world-space mean lies at distance d from
  // dist_ref with dist_min <= d < dist_max (stereo reuse of distant content; 0 and
  // infinity otherwise)
  float dist_ref[3];
  float dist_min, dist_max;
};

struct SceneDev {
  const float *mean, *ls, *quat, *logit, *sh;
  long long n;
  int deg;
};

struct WorkItem {
  int tile;  // view * tiles_per_view + tile index
  int code;  // kind (0 full-res 16x16 pixels, 1 half-res 16x16 groups) | sub << 4
};

enum { kKindFull = 0, kKindLow = 1 };
enum { kClassFocus = 0, kClassHybrid = 1, kClassPeriphery = 2 };
// flag or'ed into the class of a key tile with no visible pixel (visibility culling)
constexpr uint8_t kClassInvisible = 4;

// Visible key tiles per view and their summed-area table (visibility culling, Sec. 4.3):
// tvis[view * tiles_per_view + tile] is 1 when a pixel of the tile is visible; sat[view]
// holds (nty + 1) x (ntx + 1) counts, sat[y][x] = visible tiles in rows < y, columns < x.
struct Visibility {
  const uint8_t* tvis;
  const uint32_t* sat;
  int tiles_per_view;
  int sat_per_view;
};

__device__ __forceinline__ uint32_t sat_count(const Visibility& v, int view, int ntx, int tx0, int ty0, int tx1,
                                              int ty1) {
  const uint32_t* S = v.sat + (long long)view * v.sat_per_view;
  const int w = ntx + 1;
  return S[(ty1 + 1) * w + tx1 + 1] - S[ty0 * w + tx1 + 1] - S[(ty1 + 1) * w + tx0] + S[ty0 * w + tx0];
}

__host__ __device__ inline uint32_t float_order_bits(float f) {
  uint32_t b;
#ifdef __CUDA_ARCH__
  b = __float_as_uint(f);
#else
  union { float f; uint32_t u; } c;
  c.f = f;
  b = c.u;
#endif
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// ---- per-pair evaluation, shared by every render path ------------------------------

// returns true when the pair is kept (ray meets the tangent plane in front of o and
// alpha >= 1/255); q' is returned through *qn for the alpha computation.
__device__ __forceinline__ bool pair_test(const float4& f0, const float4& f1, const float4& f2, float lg2s,
                                          float px, float py, float& dx, float& dy, float& qw) {
  dx = px - f0.x;
  dy = py - f0.y;
  const float a = fmaf(f0.z, dx, f0.w * dy);
  const float b = fmaf(f1.x, dx, f1.y * dy);
  const float w = fmaf(f1.z, dx, fmaf(f1.w, dy, f2.x));
  const float qn = fmaf(a, fmaf(f2.y, a, f2.z * b), f2.w * b * b);
  const float w2 = w * w;
  qw = __fdividef(qn, w2);
  return (w > 0.f) && (qn <= (lg2s + kLog2_255) * w2);
}

__device__ __forceinline__ float pair_alpha(float lg2s, float qw) {
  return fminf(kAlphaMax, exp2f(lg2s - qw));
}

__device__ __forceinline__ float pair_depth(const float4& f3, const float4& f4, float m12x2, float dx, float dy) {
  const float num = fmaf(f3.y, dx, fmaf(f3.z, dy, f3.w));
  const float den = fmaf(dx, fmaf(f4.x, dx, fmaf(f4.y, dy, f4.w)), fmaf(dy, fmaf(f4.z, dy, m12x2), 1.0f));
  return __fdividef(num, den);
}

__device__ __forceinline__ bool tie_less(float ta, int ga, float tb, int gb) {
  return ta < tb || (ta == tb && ga < gb);
}

// ---- launchers implemented in the .cu files -----------------------------------------

void launch_visibility(const ViewParams* d_views, int n_views, int key_tile, int ntx, int nty, const Visibility& v,
                       cudaStream_t st);
// key_mode: 0 the Eq. 4 tile key; 3, 4 the global orders (view-space z, distance)
void launch_preprocess(const SceneDev& s, const ViewParams* d_views, const int* d_view_list, int n_views_scene,
                       int key_tile, int key_mode, const Visibility& vis, float4* rec, float4* bbox, uint32_t* count,
                       unsigned long long* kcache, cudaStream_t st);
constexpr int kKeyCacheSlots = 32;  // kept-tile keys the count pass stores per (view, Gaussian)
void launch_scan_u32(const uint32_t* in, uint32_t* out, long long n, uint32_t* d_total, uint32_t* partials,
                     cudaStream_t st);
size_t scan_partials_bytes(long long n);
void launch_duplicate(const ViewParams* d_views, int n_views, const float4* rec, const float4* bbox,
                      const uint32_t* count, const uint32_t* offsets, const long long* h_view_n, int key_tile,
                      int tiles_per_view, const Visibility& vis, const unsigned long long* kcache, int key_mode,
                      uint64_t* keys, uint32_t* vals, const uint32_t* d_total, long long cap, uint32_t* status,
                      cudaStream_t st);

struct SortScratch {
  uint32_t* hist;      // [8][256]
  uint32_t* look;      // [passes][max_tiles][256]
  uint32_t* counters;  // [8]
  long long max_tiles;
};
size_t sort_scratch_bytes(long long cap);
void sort_scratch_carve(void* base, long long cap, SortScratch* s);
// sorts n = *d_n (device) pairs; cap bounds n for grid sizing; returns index (0/1) of
// the buffer holding the result
int launch_radix_sort(uint64_t* keys[2], uint32_t* vals[2], const uint32_t* d_n, long long cap, int bits,
                      const SortScratch& s, uint32_t* status, cudaStream_t st);
void launch_ranges(const uint64_t* keys, const uint32_t* d_n, long long cap, uint32_t* ranges, long long n_tiles,
                   cudaStream_t st);

struct RenderArgs {
  const ViewParams* views;
  int n_views;
  const float4* rec;
  const float4* bbox;
  const uint32_t* vals;
  const uint32_t* ranges;
  const WorkItem* items;
  const uint32_t* n_items;
  uint32_t* queue;
  const uint8_t* tile_class;
  int fovea_mode;
  int key_tile;
  int tiles_per_view;
  int sort_mode;
  int k1, k2, k3;
  float bg[3];
  float* out;      // [V][3][H][W]
  float* low;      // [V][3][H/2][W/2] or null
  float4* s_full;  // saved per full-res sample (C, T) or null
  float4* s_low;   // saved per group sample or null
  unsigned long long* stats;  // [3] evaluated, kept, blended or null
  uint32_t* status;
  // backward
  const float* dL_dout;
  const float* dL_dlow;
  float* grad_rec;  // [sum N][16] per-(view, Gaussian) record gradients
  int max_ctas_per_sm;  // tuning: cap on resident render CTAs per SM (0 = occupancy limit)
  int stream_order;     // global orders: blend each tile list in its order (no per-ray resort)
};

void launch_workitems(const ViewParams* d_views, int n_views, int fovea_mode, int key_tile, int tiles_per_view,
                      const uint8_t* tvis, WorkItem* items, uint32_t* n_items, uint8_t* tile_class, cudaStream_t st);
// background into the output pixels (and half-resolution samples) of invisible tiles
void launch_invisible_fill(const ViewParams* d_views, int n_views, int key_tile, int tiles_per_view,
                           const uint8_t* tvis, const float bg[3], float* out, float* low, int W, int H,
                           cudaStream_t st);
void launch_render(const RenderArgs& a, long long max_items, cudaStream_t st);
void launch_composite(const RenderArgs& a, int W, int H, cudaStream_t st);
void launch_render_backward(const RenderArgs& a, long long max_items, cudaStream_t st);
void launch_composite_backward(const ViewParams* views, int n_views, const uint8_t* tile_class, int tiles_per_view,
                               int T, int fovea_mode, const float* dout, int W, int H, float4* dfull, float4* dhyb,
                               float4* dlow, cudaStream_t st);
void launch_preprocess_backward(const SceneDev& s, const ViewParams* d_views, const int* d_view_list,
                                int n_views_scene, const uint32_t* count, const float* grad_rec,
                                const vrs_gaussian_grads& g, cudaStream_t st);
int device_sm_count();

// Launch properties that depend on the device (SM count, occupancy, the dynamic shared
// memory attribute of a kernel) are memoised per device: a table of kMemoDevices
// entries, indexed by the current device, 0 meaning "not known yet".  Entries are
// atomics, so host threads may race to fill one; they store the same value.
constexpr int kMemoDevices = 64;
inline int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMemoDevices) return -1;
  return dev;
}
template <typename F>
int per_device_memo(std::atomic<int>* table, F compute) {
  const int dev = current_device();
  if (dev < 0) return compute();
  int v = table[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    v = compute();
    table[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}
// Raises a kernel's dynamic shared memory limit to at least `bytes` on the current
// device; `table` remembers per device the largest limit set so far.
template <typename K>
void ensure_dynamic_smem(std::atomic<int>* table, K kernel, int bytes) {
  const int dev = current_device();
  if (dev >= 0 && table[dev].load(std::memory_order_acquire) >= bytes) return;
  static std::mutex m;  // one per kernel: the attribute only ever grows
  std::lock_guard<std::mutex> lock(m);
  if (dev >= 0 && table[dev].load(std::memory_order_relaxed) >= bytes) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (dev >= 0) table[dev].store(bytes, std::memory_order_release);
}

// per-view parameters of the two-pass foveated baseline (passed by value)
constexpr int kTwoPassMaxViews = 64;
struct TwoPassViews {
  float gaze_x[kTwoPassMaxViews], gaze_y[kTwoPassMaxViews], radius[kTwoPassMaxViews], band[kTwoPassMaxViews];
  int x0[kTwoPassMaxViews], y0[kTwoPassMaxViews];  // centre square origin (full-resolution pixels)
};
void launch_lowmask(const TwoPassViews& tp, int n_views, int W, int H, uint8_t* mask, cudaStream_t st);
void launch_two_pass_composite(const TwoPassViews& tp, int n_views, int W, int H, int SW, int SH, const float* centre,
                               const float* low, float* out, cudaStream_t st);

}  // namespace vrs
