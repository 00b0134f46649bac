// vrs_probe_orders: the front-to-back blend order of single rays of the last render.
//
// For a probe (view, x, y) the ray through the image point (x, y) meets the Gaussians of
// the key tile that holds the point.  Each is evaluated with the render's own pair
// functions (plane map, conic cut, exp2 opacity, depth t* of Sec. 4.1), so a probe at a
// sample position of the render sees the pairs and values the render saw there.  The
// order is then the render's:
//   exact (sort mode 0): kept pairs by ascending (t*, Gaussian index), found by repeated
//     selection of the smallest pair above the last one over the tile list;
//   global orders (3, 4): kept pairs in tile-list order.
// Blending stops before the pair that would take the transmittance below 1e-4, as in
// the render.  One warp per probe; lanes evaluate 32 list entries at a time.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "common.cuh"

namespace vrs {

namespace {

constexpr unsigned kAll = 0xffffffffu;

struct ProbeArgs {
  const ViewParams* views;
  int n_views;
  const float4* rec;
  const uint32_t* vals;
  const uint32_t* ranges;
  int key_tile, tiles_per_view, list_order;
  const float* probes;
  int n, max_len;
  int* ids;
  float* depth;
  int* len;
};

// the pair evaluation of the render: true when the ray keeps the pair (alpha >= 1/255)
__device__ __forceinline__ bool probe_eval(const float4* r, float px, float py, float& alpha, float& t) {
  const float4 f0 = r[0], f1 = r[1], f2 = r[2], f3 = r[3];
  float dx, dy, qw;
  if (!pair_test(f0, f1, f2, f3.x, px, py, dx, dy, qw)) return false;
  alpha = pair_alpha(f3.x, qw);
  t = pair_depth(f3, r[4], r[5].x, dx, dy);
  return true;
}

__global__ void __launch_bounds__(128) probe_orders_kernel(ProbeArgs a) {
  const int lane = threadIdx.x & 31;
  const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= a.n) return;
  const float* pr = a.probes + 3 * w;
  const float fv = pr[0], x = pr[1], y = pr[2];
  int* ids = a.ids + w * a.max_len;
  float* dep = a.depth ? a.depth + w * a.max_len : nullptr;
  const int v = (int)fv;
  const bool ok_view = fv == (float)v && v >= 0 && v < a.n_views;
  const ViewParams vp = a.views[ok_view ? v : 0];
  if (!ok_view || !(x >= 0.f && x < (float)vp.W && y >= 0.f && y < (float)vp.H)) {
    if (lane == 0) a.len[w] = -1;
    return;
  }
  const int tile = v * a.tiles_per_view + (int)(y / a.key_tile) * vp.ntx + (int)(x / a.key_tile);
  const uint32_t b = a.ranges[2 * tile], e = a.ranges[2 * tile + 1];
  const float4* recv = a.rec + vp.base * kRecF4;
  float T = 1.f;
  int n = 0;
  if (!a.list_order) {
    // exact: repeated selection of the smallest kept (t*, index) above the last one
    float pt = -INFINITY;
    int pg = -1;
    for (;;) {
      float bt = INFINITY, ba = 0.f;
      int bg = INT_MAX;
      for (uint32_t i = b + lane; i < e; i += 32) {
        const int g = (int)a.vals[i];
        float al, t;
        if (!probe_eval(recv + (long long)g * kRecF4, x, y, al, t)) continue;
        if (!tie_less(pt, pg, t, g)) continue;  // not above the last blended pair
        if (tie_less(t, g, bt, bg)) {
          bt = t;
          bg = g;
          ba = al;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const float ot = __shfl_xor_sync(kAll, bt, o);
        const int og = __shfl_xor_sync(kAll, bg, o);
        const float oa = __shfl_xor_sync(kAll, ba, o);
        if (tie_less(ot, og, bt, bg)) {
          bt = ot;
          bg = og;
          ba = oa;
        }
      }
      if (bg == INT_MAX) break;
      const float test = T * (1.f - ba);
      if (test < kTStop) break;
      if (lane == 0 && n < a.max_len) {
        ids[n] = bg;
        if (dep) dep[n] = bt;
      }
      ++n;
      T = test;
      pt = bt;
      pg = bg;
    }
  } else {
    // global orders: kept pairs in list order
    bool done = false;
    for (uint32_t base = b; base < e && !done; base += 32) {
      const uint32_t i = base + lane;
      float al = 0.f, t = 0.f;
      int g = 0;
      bool kept = false;
      if (i < e) {
        g = (int)a.vals[i];
        kept = probe_eval(recv + (long long)g * kRecF4, x, y, al, t);
      }
      unsigned m = __ballot_sync(kAll, kept);
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const float sa = __shfl_sync(kAll, al, src);
        const float st = __shfl_sync(kAll, t, src);
        const int sg = __shfl_sync(kAll, g, src);
        const float test = T * (1.f - sa);
        if (test < kTStop) {
          done = true;
          break;
        }
        if (lane == 0 && n < a.max_len) {
          ids[n] = sg;
          if (dep) dep[n] = st;
        }
        ++n;
        T = test;
      }
    }
  }
  if (lane == 0) a.len[w] = n;
}

}  // namespace

void launch_probe_orders(const ViewParams* views, int n_views, const float4* rec, const uint32_t* vals,
                         const uint32_t* ranges, int key_tile, int tiles_per_view, int list_order,
                         const float* probes, int n, int max_len, int* ids, float* depth, int* len,
                         cudaStream_t st) {
  if (n <= 0) return;
  ProbeArgs a{views, n_views, rec, vals, ranges, key_tile, tiles_per_view, list_order, probes, n, max_len,
              ids, depth, len};
  const long long threads = (long long)n * 32;
  probe_orders_kernel<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(a);
}

}  // namespace vrs
