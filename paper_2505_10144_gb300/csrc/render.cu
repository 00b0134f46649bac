// Single-launch foveated blending (Sec. 4.3) with per-ray resorting (Sec. 4.1).
//
// Work items are 16x16-sample squares: full-resolution 16x16 pixel subtiles (focus and
// hybrid 32x32 tiles split into four, or plain 16x16 tiles) and half-resolution 32x32
// periphery tiles whose 256 samples are 2x2 pixel groups, so focus and periphery run in
// the same persistent launch.  Per entry of the tile's depth-sorted list, a sample
// evaluates the pair (Eq. 1 on the optimal plane); kept pairs enter the per-ray windows;
// popped entries are blended front to back (Eq. 2) with the 3DGS stopping rule.
//
// Two kernels:
//  - warp_render_kernel (hierarchical windows, the global orders, the window-only
//    order): every warp is an independent worker on 8x4-sample region tasks taken from
//    an atomic queue.  It stages the entries whose bounding box meets its region 16 at a
//    time in warp-private shared memory; the 4x4- and 2x2-block windows live in the
//    registers of their blocks' lanes (ballots and shuffles, ranked slots for the default
//    4/8 windows) and the per-sample window is a per-lane tournament tree in shared
//    memory.  The same kernel replays the blends for the backward pass.
//  - render_kernel (the exact per-ray order, used for parity, and window shapes the warp
//    kernel is not compiled for): one CTA pass of 256 threads per work item, one sample
//    per thread; in the exact order every kept pair is sorted per sample by selection
//    over the tile list.
#include <algorithm>

#include "common.cuh"

namespace vrs {

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ void sample_xy(int tid, int& x, int& y) {
  x = (tid & 1) | ((tid >> 1) & 2) | ((tid >> 2) & 4) | ((tid >> 2) & 8);
  y = ((tid >> 1) & 1) | ((tid >> 2) & 2) | ((tid >> 4) & 4) | ((tid >> 4) & 8);
}

__global__ void workitems_kernel(const ViewParams* __restrict__ views, int n_views, int fovea_mode, int T,
                                 int tiles_per_view, const uint8_t* __restrict__ tvis, WorkItem* __restrict__ items,
                                 uint32_t* n_items, uint8_t* __restrict__ tile_class) {
  const long long gi = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= (long long)n_views * tiles_per_view) return;
  const int view = (int)(gi / tiles_per_view), t = (int)(gi % tiles_per_view);
  const ViewParams& vp = views[view];
  if (t >= vp.ntx * vp.nty) return;
  const int tx = t % vp.ntx, ty = t / vp.ntx;
  int cls = kClassFocus;
  if (fovea_mode != 0) {
    const float x0 = tx * T + 0.5f, y0 = ty * T + 0.5f;
    const float x1 = (float)min((tx + 1) * T, vp.W) - 0.5f, y1 = (float)min((ty + 1) * T, vp.H) - 0.5f;
    const float nx = fminf(fmaxf(vp.gaze_x, x0), x1) - vp.gaze_x, ny = fminf(fmaxf(vp.gaze_y, y0), y1) - vp.gaze_y;
    const float fx = fmaxf(fabsf(x0 - vp.gaze_x), fabsf(x1 - vp.gaze_x));
    const float fy = fmaxf(fabsf(y0 - vp.gaze_y), fabsf(y1 - vp.gaze_y));
    const float dmin = sqrtf(nx * nx + ny * ny), dmax = sqrtf(fx * fx + fy * fy);
    cls = dmax <= vp.radius ? kClassFocus : (dmin >= vp.radius + vp.band ? kClassPeriphery : kClassHybrid);
  }
  if (tvis && !tvis[gi]) {  // visibility culling: no work; invisible_fill writes the background
    tile_class[gi] = (uint8_t)(cls | kClassInvisible);
    return;
  }
  tile_class[gi] = (uint8_t)cls;
  const int tile = (int)gi;
  if (cls == kClassPeriphery) {
    const uint32_t o = atomicAdd(n_items, 1u);
    items[o] = WorkItem{tile, kKindLow};
  } else if (T == 16) {
    const uint32_t o = atomicAdd(n_items, 1u);
    items[o] = WorkItem{tile, kKindFull};
  } else {
    for (int sub = 0; sub < 4; ++sub) {
      const int ox = tx * 32 + (sub & 1) * 16, oy = ty * 32 + (sub >> 1) * 16;
      if (ox >= vp.W || oy >= vp.H) continue;
      const uint32_t o = atomicAdd(n_items, 1u);
      items[o] = WorkItem{tile, kKindFull | (sub << 4)};
    }
  }
}

struct Smem {
  float4* rec;       // [256][6]
  int* gid;          // [256]
  uint8_t* wmask;    // [256]
  float* key3;       // [k3][256]
  int* gid3;
  float* alpha3;
  float* key2;       // [k2][64]
  int* gid2;
  float* key1;       // [k1][16]
  int* gid1;
};

__host__ __device__ inline size_t render_smem_bytes(int k1, int k2, int k3) {
  return (size_t)kBlock * kRecF4 * 16 + kBlock * 4 + kBlock + 64 /*pad*/ + (size_t)k3 * kBlock * 12 +
         (size_t)k2 * 64 * 8 + (size_t)k1 * 16 * 8 + 64;
}

__device__ inline Smem carve(unsigned char* base, int k1, int k2, int k3) {
  Smem s;
  unsigned char* p = base;
  s.rec = reinterpret_cast<float4*>(p);
  p += (size_t)kBlock * kRecF4 * 16;
  s.gid = reinterpret_cast<int*>(p);
  p += kBlock * 4;
  s.key3 = reinterpret_cast<float*>(p);
  p += (size_t)k3 * kBlock * 4;
  s.gid3 = reinterpret_cast<int*>(p);
  p += (size_t)k3 * kBlock * 4;
  s.alpha3 = reinterpret_cast<float*>(p);
  p += (size_t)k3 * kBlock * 4;
  s.key2 = reinterpret_cast<float*>(p);
  p += (size_t)k2 * 64 * 4;
  s.gid2 = reinterpret_cast<int*>(p);
  p += (size_t)k2 * 64 * 4;
  s.key1 = reinterpret_cast<float*>(p);
  p += (size_t)k1 * 16 * 4;
  s.gid1 = reinterpret_cast<int*>(p);
  p += (size_t)k1 * 16 * 4;
  s.wmask = p;
  return s;
}

// State of one thread's sample.
struct Px {
  float px, py;
  float T, C0, C1, C2;
  bool active;
  int h3, n3;
  unsigned n_eval, n_kept, n_blend;
  // backward replay: dL/dC of the sample, its final C and T, dL/dT_final (= dL/dC . bg)
  float G0, G1, G2, F0, F1, F2, TF, GT;
  float* grad;  // per-(view, Gaussian) record gradients of this view, [n][16]
};

// d(loss)/d(record) of one blended pair, accumulated into the record gradient (16
// floats: pm_x, pm_y, h00, h01, h10, h11, h20, h21, h22, a00, a01x2, a11, log2 sigma, r,
// g, b).  alpha_i, c_i, T_i and C_<i are the values the forward used; with C_final and
// T_final saved, every term is available in front-to-back order:
//   dL/dc_i     = dL/dC alpha_i T_i
//   dL/dalpha_i = T_i (dL/dC . c_i) - (dL/dC . (C_final - C_<=i) + dL/dT_final T_final) / (1 - alpha_i)
// Adds v[16] to grad (the record gradient of one Gaussian) with four 16-byte vector
// atomics (grad is 64-byte aligned per Gaussian).  Gathering the lanes that blend the same
// Gaussian in the same step by shuffles, with one lane issuing the atomics, ran slower
// once the atomics were vectors: 27.5 against 22.1 ms on four 1280^2 views.
__device__ __forceinline__ void grad_add16(float* __restrict__ grad, float v[16]) {
  float4* g4 = reinterpret_cast<float4*>(grad);
#pragma unroll
  for (int k = 0; k < 4; ++k) atomicAdd(g4 + k, make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]));
}

// d(loss)/d(record) of one blended pair, accumulated into the record gradient (16
// floats: pm_x, pm_y, h00, h01, h10, h11, h20, h21, h22, a00, a01x2, a11, log2 sigma, r,
// g, b).  alpha_i, c_i, T_i and C_<i are the values the forward used; with C_final and
// T_final saved, every term is available in front-to-back order:
//   dL/dc_i     = dL/dC alpha_i T_i
//   dL/dalpha_i = T_i (dL/dC . c_i) - (dL/dC . (C_final - C_<=i) + dL/dT_final T_final) / (1 - alpha_i)
__device__ __forceinline__ void blend_grad(const Px& p, float alpha, const float4* r, float Tb, float Cb0, float Cb1,
                                           float Cb2, float* __restrict__ grad) {
  const float4 f0 = r[0], f1 = r[1], f2 = r[2], f5 = r[5];
  const float aT = alpha * Tb;
  const float c0 = f5.y, c1 = f5.z, c2 = f5.w;
  const float le0 = fmaf(aT, c0, Cb0), le1 = fmaf(aT, c1, Cb1), le2 = fmaf(aT, c2, Cb2);
  const float cdot = p.G0 * c0 + p.G1 * c1 + p.G2 * c2;
  const float rest = p.G0 * (p.F0 - le0) + p.G1 * (p.F1 - le1) + p.G2 * (p.F2 - le2) + p.GT * p.TF;
  const float dLda = Tb * cdot - rest / (1.f - alpha);
  float v[16];
#pragma unroll
  for (int k = 0; k < 13; ++k) v[k] = 0.f;
  v[13] = p.G0 * aT;
  v[14] = p.G1 * aT;
  v[15] = p.G2 * aT;
  if (alpha < kAlphaMax) {  // clamped: alpha does not depend on the Gaussian
    const float dx = p.px - f0.x, dy = p.py - f0.y;
    const float a = fmaf(f0.z, dx, f0.w * dy);
    const float b = fmaf(f1.x, dx, f1.y * dy);
    const float w = fmaf(f1.z, dx, fmaf(f1.w, dy, f2.x));
    const float iw2 = 1.f / (w * w);
    const float qn = fmaf(a, fmaf(f2.y, a, f2.z * b), f2.w * b * b);
    const float qw = qn * iw2;
    const float gl = dLda * alpha * kLn2;  // dL/d(log2 sigma) = -dL/dq'
    const float gqn = -gl * iw2;
    const float gw = 2.f * gl * qw / w;
    const float ga = gqn * (2.f * f2.y * a + f2.z * b), gb = gqn * (f2.z * a + 2.f * f2.w * b);
    v[0] = -(ga * f0.z + gb * f1.x + gw * f1.z);
    v[1] = -(ga * f0.w + gb * f1.y + gw * f1.w);
    v[2] = ga * dx;
    v[3] = ga * dy;
    v[4] = gb * dx;
    v[5] = gb * dy;
    v[6] = gw * dx;
    v[7] = gw * dy;
    v[8] = gw;
    v[9] = gqn * a * a;
    v[10] = gqn * a * b;
    v[11] = gqn * b * b;
    v[12] = gl;
  }
  grad_add16(grad, v);
}

template <bool STATS, bool BWD = false>
__device__ __forceinline__ void blend(Px& p, float alpha, int g, const float4* __restrict__ recv) {
  if (!p.active) return;
  const float test = p.T * (1.f - alpha);
  if (test < kTStop) {
    p.active = false;
    return;
  }
  if (BWD) blend_grad(p, alpha, recv + (long long)g * kRecF4, p.T, p.C0, p.C1, p.C2, p.grad + (long long)g * 16);
  const float4 c = recv[(long long)g * kRecF4 + 5];
  const float aT = alpha * p.T;
  p.C0 = fmaf(aT, c.y, p.C0);
  p.C1 = fmaf(aT, c.z, p.C1);
  p.C2 = fmaf(aT, c.w, p.C2);
  p.T = test;
  if (STATS) ++p.n_blend;
}

// per-thread ring window (ascending from head), insert-then-pop-min
template <bool STATS, bool BWD>
__device__ __forceinline__ void l3_push(Px& p, const Smem& s, int K3, float t, int g, float alpha,
                                        const float4* __restrict__ recv) {
  const int tid = threadIdx.x;
  if (p.n3 == K3) {
    const int hs = p.h3;
    const float tm = s.key3[hs * kBlock + tid];
    const int gm = s.gid3[hs * kBlock + tid];
    if (tie_less(t, g, tm, gm)) {
      blend<STATS, BWD>(p, alpha, g, recv);
      return;
    }
    const float am = s.alpha3[hs * kBlock + tid];
    p.h3 = hs + 1 == K3 ? 0 : hs + 1;
    p.n3--;
    // insert, then blend the popped minimum
    int j = p.n3;
    while (j > 0) {
      int q = p.h3 + j - 1;
      if (q >= K3) q -= K3;
      const float tk = s.key3[q * kBlock + tid];
      const int gk = s.gid3[q * kBlock + tid];
      if (!tie_less(t, g, tk, gk)) break;
      int d = q + 1;
      if (d >= K3) d -= K3;
      s.key3[d * kBlock + tid] = tk;
      s.gid3[d * kBlock + tid] = gk;
      s.alpha3[d * kBlock + tid] = s.alpha3[q * kBlock + tid];
      --j;
    }
    int d = p.h3 + j;
    if (d >= K3) d -= K3;
    s.key3[d * kBlock + tid] = t;
    s.gid3[d * kBlock + tid] = g;
    s.alpha3[d * kBlock + tid] = alpha;
    p.n3++;
    blend<STATS, BWD>(p, am, gm, recv);
    return;
  }
  int j = p.n3;
  while (j > 0) {
    int q = p.h3 + j - 1;
    if (q >= K3) q -= K3;
    const float tk = s.key3[q * kBlock + tid];
    const int gk = s.gid3[q * kBlock + tid];
    if (!tie_less(t, g, tk, gk)) break;
    int d = q + 1;
    if (d >= K3) d -= K3;
    s.key3[d * kBlock + tid] = tk;
    s.gid3[d * kBlock + tid] = gk;
    s.alpha3[d * kBlock + tid] = s.alpha3[q * kBlock + tid];
    --j;
  }
  int d = p.h3 + j;
  if (d >= K3) d -= K3;
  s.key3[d * kBlock + tid] = t;
  s.gid3[d * kBlock + tid] = g;
  s.alpha3[d * kBlock + tid] = alpha;
  p.n3++;
}

// shared ring window of a sample block (owner lane only); returns the popped gid or -1
__device__ __forceinline__ int ring_push(float* key, int* gid, int stride, int slot, int K, int& h, int& n, float t,
                                         int g) {
  if (K == 0) return g;
  int popped = -1;
  if (n == K) {
    const float tm = key[h * stride + slot];
    const int gm = gid[h * stride + slot];
    if (tie_less(t, g, tm, gm)) return g;
    popped = gm;
    h = h + 1 == K ? 0 : h + 1;
    n--;
  }
  int j = n;
  while (j > 0) {
    int q = h + j - 1;
    if (q >= K) q -= K;
    const float tk = key[q * stride + slot];
    const int gk = gid[q * stride + slot];
    if (!tie_less(t, g, tk, gk)) break;
    int d = q + 1;
    if (d >= K) d -= K;
    key[d * stride + slot] = tk;
    gid[d * stride + slot] = gk;
    --j;
  }
  int d = h + j;
  if (d >= K) d -= K;
  key[d * stride + slot] = t;
  gid[d * stride + slot] = g;
  n++;
  return popped;
}

__device__ __forceinline__ int ring_pop(const int* gid, int stride, int slot, int K, int& h, int& n) {
  if (n == 0) return -1;
  const int g = gid[h * stride + slot];
  h = h + 1 == K ? 0 : h + 1;
  n--;
  return g;
}

__device__ __forceinline__ float depth_at(const float4* r, float x, float y) {
  const float4 f0 = r[0], f3 = r[3], f4 = r[4];
  const float m12x2 = r[5].x;
  return pair_depth(f3, f4, m12x2, x - f0.x, y - f0.y);
}

// full evaluation of a record at the thread's sample: kept, alpha, depth.  COUNT_EVAL is
// false where the pair was already counted when it entered the cascade.
template <bool STATS, bool COUNT_EVAL = true>
__device__ __forceinline__ bool eval_full(const float4* r, Px& p, float& alpha, float& t) {
  const float4 f0 = r[0], f1 = r[1], f2 = r[2], f3 = r[3];
  float dx, dy, qw;
  if (STATS && COUNT_EVAL) ++p.n_eval;
  if (!pair_test(f0, f1, f2, f3.x, p.px, p.py, dx, dy, qw)) return false;
  if (STATS) ++p.n_kept;
  alpha = pair_alpha(f3.x, qw);
  t = pair_depth(f3, r[4], r[5].x, dx, dy);
  return true;
}

// the same, also returning the pair's colour
template <bool STATS, bool COUNT_EVAL = true>
__device__ __forceinline__ bool eval_full(const float4* r, Px& p, float& alpha, float& t, float3& c) {
  const float4 f0 = r[0], f1 = r[1], f2 = r[2], f3 = r[3];
  float dx, dy, qw;
  if (STATS && COUNT_EVAL) ++p.n_eval;
  if (!pair_test(f0, f1, f2, f3.x, p.px, p.py, dx, dy, qw)) return false;
  if (STATS) ++p.n_kept;
  const float4 f5 = r[5];
  alpha = pair_alpha(f3.x, qw);
  t = pair_depth(f3, r[4], f5.x, dx, dy);
  c = make_float3(f5.y, f5.z, f5.w);
  return true;
}

struct ItemGeom {
  int view, kind, ox, oy;  // ox, oy: sample-grid origin (pixels for full, groups for low)
  int ext;                 // side of the item in samples: 16, or 8 for the groups of a 16x16 periphery tile
  int tile;
};

__device__ __forceinline__ ItemGeom decode(const WorkItem& it, int tiles_per_view, int T, const ViewParams* views) {
  ItemGeom g;
  g.view = it.tile / tiles_per_view;
  const int t = it.tile % tiles_per_view;
  const ViewParams& vp = views[g.view];
  const int tx = t % vp.ntx, ty = t / vp.ntx;
  g.kind = it.code & 15;
  const int sub = it.code >> 4;
  g.tile = it.tile;
  g.ext = 16;
  if (g.kind == kKindLow) {  // the (T / 2) x (T / 2) groups of a periphery key tile
    g.ox = tx * (T / 2);
    g.oy = ty * (T / 2);
    g.ext = T / 2;
  } else if (T == 16) {
    g.ox = tx * 16;
    g.oy = ty * 16;
  } else {
    g.ox = tx * 32 + (sub & 1) * 16;
    g.oy = ty * 32 + (sub >> 1) * 16;
  }
  return g;
}

// Warp-uniform 256-bit mask of the staged entries whose bounding box meets this warp's
// 8x4-sample region.
__device__ __forceinline__ void warp_masks(const Smem& s, int nb, unsigned m[8]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = c * 32 + lane;
    const bool b = j < nb && ((s.wmask[j] >> w) & 1);
    m[c] = __ballot_sync(kFull, b);
  }
}

__device__ __forceinline__ void stage_batch(const Smem& s, const RenderArgs& a, const ViewParams& vp,
                                            const ItemGeom& g, long long start, int nb) {
  const int tid = threadIdx.x;
  if (tid < nb) {
    const int gid = (int)a.vals[start + tid];
    const long long vg = vp.base + gid;
    const float4* r = a.rec + vg * kRecF4;
#pragma unroll
    for (int q = 0; q < kRecF4; ++q) s.rec[tid * kRecF4 + q] = r[q];
    s.gid[tid] = gid;
    const float4 bb = a.bbox[vg];
    uint8_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const int xo = 8 * (w & 1), yo = 4 * (w >> 1);
      float x0, x1, y0, y1;
      if (g.kind == kKindLow) {
        x0 = 2.f * (g.ox + xo) + 1.f;
        x1 = x0 + 14.f;
        y0 = 2.f * (g.oy + yo) + 1.f;
        y1 = y0 + 6.f;
      } else {
        x0 = g.ox + xo + 0.5f;
        x1 = x0 + 7.f;
        y0 = g.oy + yo + 0.5f;
        y1 = y0 + 3.f;
      }
      if (bb.x <= x1 && bb.z >= x0 && bb.y <= y1 && bb.w >= y0) m |= (uint8_t)(1u << w);
    }
    s.wmask[tid] = m;
  }
}

template <int MODE, bool STATS, bool BWD>
__global__ void __launch_bounds__(kBlock, 2) render_kernel(RenderArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  const int K1 = MODE == 2 ? a.k1 : 0, K2 = MODE == 2 ? a.k2 : 0, K3 = MODE == 0 ? 0 : a.k3;
  const Smem s = carve(smem_raw, K1, K2, K3);
  const int tid = threadIdx.x, lane = tid & 31;
  int sx, sy;
  sample_xy(tid, sx, sy);
  const int blk16 = tid >> 4;  // 4x4 block slot
  const int blk4 = tid >> 2;   // 2x2 block slot
  unsigned n_eval = 0, n_kept = 0, n_blend = 0;
  for (;;) {
    if (tid == 0) s_item = (int)atomicAdd(a.queue, 1u);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= (int)*a.n_items) break;
    const ItemGeom g = decode(a.items[item], a.tiles_per_view, a.key_tile, a.views);
    const ViewParams& vp = a.views[g.view];
    const float4* recv = a.rec + vp.base * kRecF4;
    Px p;
    bool valid;
    int X = g.ox + sx, Y = g.oy + sy;
    if (g.kind == kKindLow) {
      valid = 2 * X < vp.W && 2 * Y < vp.H && sx < g.ext && sy < g.ext;
      p.px = 2.f * X + 1.f;
      p.py = 2.f * Y + 1.f;
    } else {
      valid = X < vp.W && Y < vp.H;
      p.px = X + 0.5f;
      p.py = Y + 0.5f;
    }
    p.T = 1.f;
    p.C0 = p.C1 = p.C2 = 0.f;
    p.active = valid;
    p.h3 = p.n3 = 0;
    p.n_eval = p.n_kept = p.n_blend = 0;
    if (BWD) {
      const long long HWb = (long long)vp.H * vp.W;
      const long long HW2b = (long long)(vp.H / 2) * (vp.W / 2);
      float4 dv = make_float4(0.f, 0.f, 0.f, 0.f), sv = make_float4(0.f, 0.f, 0.f, 1.f);
      if (valid) {
        const long long si = g.kind == kKindLow ? (long long)g.view * HW2b + (long long)Y * (vp.W / 2) + X
                                                : (long long)g.view * HWb + (long long)Y * vp.W + X;
        dv = g.kind == kKindLow ? reinterpret_cast<const float4*>(a.dL_dlow)[si]
                                : reinterpret_cast<const float4*>(a.dL_dout)[si];
        sv = g.kind == kKindLow ? a.s_low[si] : a.s_full[si];
      }
      p.G0 = dv.x;
      p.G1 = dv.y;
      p.G2 = dv.z;
      p.GT = dv.x * a.bg[0] + dv.y * a.bg[1] + dv.z * a.bg[2];
      p.F0 = sv.x;
      p.F1 = sv.y;
      p.F2 = sv.z;
      p.TF = sv.w;
      p.grad = a.grad_rec + vp.base * 16;
    }
    // block centres of this thread's 4x4 and 2x2 sample blocks
    const int bx4 = g.ox + (sx & ~3), by4 = g.oy + (sy & ~3), bx2 = g.ox + (sx & ~1), by2 = g.oy + (sy & ~1);
    float c4x, c4y, c2x, c2y;
    if (g.kind == kKindLow) {
      c4x = 2.f * bx4 + 4.f;
      c4y = 2.f * by4 + 4.f;
      c2x = 2.f * bx2 + 2.f;
      c2y = 2.f * by2 + 2.f;
    } else {
      c4x = bx4 + 2.f;
      c4y = by4 + 2.f;
      c2x = bx2 + 1.f;
      c2y = by2 + 1.f;
    }
    int h1 = 0, n1 = 0, h2 = 0, n2 = 0;  // meaningful in owner lanes
    const bool own16 = (lane & 15) == 0, own4 = (lane & 3) == 0;
    const long long start = a.ranges[2 * (long long)g.tile], end = a.ranges[2 * (long long)g.tile + 1];

    // popped from a 2x2 window: per-sample test, into the per-ray window
    auto pop2 = [&](int g2) {
      if (g2 >= 0 && p.active) {
        float al, t;
        if (eval_full<STATS, false>(recv + (long long)g2 * kRecF4, p, al, t))
          l3_push<STATS, BWD>(p, s, K3, t, g2, al, recv);
      }
    };
    // popped from a 4x4 window: 2x2-block membership, 2x2 window
    auto pop1 = [&](int g1) {
      bool k = false;
      const float4* r = recv + (long long)(g1 >= 0 ? g1 : 0) * kRecF4;
      if (g1 >= 0 && p.active) {
        float dx, dy, qw;
        k = pair_test(r[0], r[1], r[2], r[3].x, p.px, p.py, dx, dy, qw);
      }
      const unsigned bal = __ballot_sync(kFull, k);
      int g2 = -1;
      if (own4 && ((bal >> (lane & ~3)) & 0xFu)) {
        g2 = ring_push(s.key2, s.gid2, 64, blk4, K2, h2, n2, depth_at(r, c2x, c2y), g1);
      }
      g2 = __shfl_sync(kFull, g2, lane & ~3);
      pop2(g2);
    };

    bool any_active = __syncthreads_count(p.active) > 0;
    long long last_t_g = -1;  // exact mode: (t, g) of the last blended pair
    float last_t = -INFINITY;
    int last_g = -1;
    (void)last_t_g;
    for (int pass = 0; any_active; ++pass) {
      float bt = INFINITY, ba = 0.f;
      int bgid = 0x7fffffff;
      for (long long b0 = start; b0 < end && any_active; b0 += kBlock) {
        const int nb = (int)min((long long)kBlock, end - b0);
        __syncthreads();
        stage_batch(s, a, vp, g, b0, nb);
        __syncthreads();
        unsigned m[8];
        warp_masks(s, nb, m);
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
          unsigned mm = m[c];
          while (mm) {
            const int j = c * 32 + __ffs(mm) - 1;
            mm &= mm - 1;
            const float4* r = s.rec + j * kRecF4;
            const int gj = s.gid[j];
            if (MODE == 0) {
              float al, t;
              if (p.active && eval_full<STATS>(r, p, al, t)) {
                if (tie_less(last_t, last_g, t, gj) && tie_less(t, gj, bt, bgid)) {
                  bt = t;
                  bgid = gj;
                  ba = al;
                }
              }
            } else if (MODE == 1) {
              float al, t;
              if (p.active && eval_full<STATS>(r, p, al, t)) l3_push<STATS, BWD>(p, s, K3, t, gj, al, recv);
            } else {
              bool k = false;
              if (p.active) {
                float dx, dy, qw;
                if (STATS) ++p.n_eval;
                k = pair_test(r[0], r[1], r[2], r[3].x, p.px, p.py, dx, dy, qw);
              }
              const unsigned bal = __ballot_sync(kFull, k);
              int g1 = -1;
              if (own16 && ((bal >> (lane & 16)) & 0xFFFFu)) {
                g1 = ring_push(s.key1, s.gid1, 16, blk16, K1, h1, n1, depth_at(r, c4x, c4y), gj);
              }
              g1 = __shfl_sync(kFull, g1, lane & 16);
              if (__any_sync(kFull, g1 >= 0)) pop1(g1);
            }
          }
        }
        if (MODE != 0) any_active = __syncthreads_count(p.active) > 0;
      }
      if (MODE != 0) break;
      // exact mode: blend this pass's minimum above the previous one
      if (p.active) {
        if (bgid == 0x7fffffff) {
          p.active = false;
        } else {
          blend<STATS, BWD>(p, ba, bgid, recv);
          last_t = bt;
          last_g = bgid;
        }
      }
      any_active = __syncthreads_count(p.active) > 0;
    }
    if (MODE == 2) {
      for (int it = 0; it < K1; ++it) {
        int g1 = own16 ? ring_pop(s.gid1, 16, blk16, K1, h1, n1) : -1;
        g1 = __shfl_sync(kFull, g1, lane & 16);
        if (__any_sync(kFull, g1 >= 0)) pop1(g1);
      }
      for (int it = 0; it < K2; ++it) {
        int g2 = own4 ? ring_pop(s.gid2, 64, blk4, K2, h2, n2) : -1;
        g2 = __shfl_sync(kFull, g2, lane & ~3);
        pop2(g2);
      }
    }
    if (MODE != 0) {
      while (p.n3 > 0) {
        const int hs = p.h3;
        const int gm = s.gid3[hs * kBlock + tid];
        const float am = s.alpha3[hs * kBlock + tid];
        p.h3 = hs + 1 == K3 ? 0 : hs + 1;
        p.n3--;
        blend<STATS, BWD>(p, am, gm, recv);
      }
    }
    if (BWD) continue;
    // ---- outputs
    const float v0 = fmaf(p.T, a.bg[0], p.C0), v1 = fmaf(p.T, a.bg[1], p.C1), v2 = fmaf(p.T, a.bg[2], p.C2);
    const long long HW = (long long)vp.H * vp.W;
    const int W2 = vp.W / 2, H2 = vp.H / 2;
    const long long HW2 = (long long)H2 * W2;
    if (g.kind == kKindFull) {
      // 2x2 group average (lanes 4k..4k+3 hold one group, in (x, y) order (0,0),(1,0),(0,1),(1,1))
      float s0 = v0 + __shfl_xor_sync(kFull, v0, 1), s1 = v1 + __shfl_xor_sync(kFull, v1, 1),
            s2 = v2 + __shfl_xor_sync(kFull, v2, 1);
      s0 += __shfl_xor_sync(kFull, s0, 2);
      s1 += __shfl_xor_sync(kFull, s1, 2);
      s2 += __shfl_xor_sync(kFull, s2, 2);
      const float a0 = 0.25f * s0, a1 = 0.25f * s1, a2 = 0.25f * s2;
      if (valid) {
        float o0 = v0, o1 = v1, o2 = v2;
        if (a.fovea_mode != 0 && a.tile_class[g.tile] == kClassHybrid) {
          const float dx = p.px - vp.gaze_x, dy = p.py - vp.gaze_y;
          const float w = fminf(fmaxf((vp.radius + vp.band - sqrtf(dx * dx + dy * dy)) / vp.band, 0.f), 1.f);
          o0 = w * v0 + (1.f - w) * a0;
          o1 = w * v1 + (1.f - w) * a1;
          o2 = w * v2 + (1.f - w) * a2;
        }
        float* out = a.out + (long long)g.view * 3 * HW + (long long)Y * vp.W + X;
        out[0] = o0;
        out[HW] = o1;
        out[2 * HW] = o2;
        if (a.s_full) a.s_full[(long long)g.view * HW + (long long)Y * vp.W + X] = make_float4(p.C0, p.C1, p.C2, p.T);
        if (a.low && own4 && X / 2 < W2 && Y / 2 < H2) {
          float* lo = a.low + (long long)g.view * 3 * HW2 + (long long)(Y / 2) * W2 + X / 2;
          lo[0] = a0;
          lo[HW2] = a1;
          lo[2 * HW2] = a2;
        }
      }
    } else if (valid) {
      float* lo = a.low + (long long)g.view * 3 * HW2 + (long long)Y * W2 + X;
      lo[0] = v0;
      lo[HW2] = v1;
      lo[2 * HW2] = v2;
      if (a.s_low) a.s_low[(long long)g.view * HW2 + (long long)Y * W2 + X] = make_float4(p.C0, p.C1, p.C2, p.T);
    }
    if (STATS) {
      n_eval += p.n_eval;
      n_kept += p.n_kept;
      n_blend += p.n_blend;
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_eval += __shfl_xor_sync(kFull, n_eval, o);
      n_kept += __shfl_xor_sync(kFull, n_kept, o);
      n_blend += __shfl_xor_sync(kFull, n_blend, o);
    }
    if (lane == 0) {
      atomicAdd(&a.stats[0], (unsigned long long)n_eval);
      atomicAdd(&a.stats[1], (unsigned long long)n_kept);
      atomicAdd(&a.stats[2], (unsigned long long)n_blend);
    }
  }
}

// ---------------------------------------------------------------------------------
// Warp-independent render (window and hierarchical modes).  A task is one 8x4-sample
// region of a work item; every warp takes tasks from the queue on its own, so there is no
// CTA barrier and a warp stops as soon as its 32 samples are done.  Per batch of 32 list
// entries the warp compacts the entries whose bounding box meets its region into warp-
// private shared memory.  The 4x4-block and 2x2-block windows are replicated in the
// registers of the block's lanes as packed (depth bits << 32 | index) keys and updated
// by the same branch-free insertion on every lane of the block; the per-sample window is
// a per-lane ring in shared memory.

constexpr int kRegionWarps = 4;
constexpr unsigned long long kEmptyKey = ~0ull;

__device__ __forceinline__ unsigned long long pack_key(float t, int g) {
  return ((unsigned long long)float_order_bits(t) << 32) | (unsigned)g;
}

// Block windows distributed over the lanes of their block.  The 4x4-block window (K1
// <= 16 entries) keeps slot s on lane 16 b + s of block b; the 2x2-block window (K2 <= 16)
// keeps slot s on lane 4 c + (s & 3) of block c, register s >> 2.  Slots hold packed
// (depth bits << 32 | index) keys in ascending order, empty slots kEmptyKey.  An
// insertion counts the slots below the new key with one ballot and moves the others by
// one slot with shuffles, so its cost does not grow with the window size.  Every lane of
// the warp takes part in every call (full-mask shuffles); do_push and the key are uniform
// over the block.

template <int K1>
struct Win16 {
  unsigned long long e;  // this lane's slot (lane & 15)
  unsigned pl;           // payload of the slot (the block's kept-sample mask at entry)
  int n;                 // entries held by this lane's block
};

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src, int width) {
  const unsigned lo = __shfl_sync(kFull, (unsigned)v, src, width);
  const unsigned hi = __shfl_sync(kFull, (unsigned)(v >> 32), src, width);
  return ((unsigned long long)hi << 32) | lo;
}

// insert (x, xpl) when do_push, then pop the minimum when the window holds more than
// K1; returns the popped key (kEmptyKey if none) and its payload, uniform over the block
template <int K1>
__device__ __forceinline__ unsigned long long win16_push(Win16<K1>& w, unsigned long long x, unsigned xpl,
                                                         bool do_push, int lane, unsigned& popl) {
  const int slot = lane & 15;
  const unsigned bal = __ballot_sync(kFull, w.e < x);
  const int pos = __popc((bal >> (lane & 16)) & 0xFFFFu);
  const int su = slot - 1 < 0 ? 0 : slot - 1, sd = slot + 1 > 15 ? 15 : slot + 1;
  // Both blocks of the warp full (the common case on long lists): the insertion only moves
  // entries towards the head, so the shuffles of the upward move are skipped.  Measured on
  // the VR stereo frame: 5.43 against 5.53 ms.  The same split of the 2x2 window ran slower
  // (5.59 ms; its extra registers spill).
  if (__all_sync(kFull, w.n >= K1)) {
    const unsigned long long fdn = shfl64(w.e, sd, 16), fe0 = shfl64(w.e, 0, 16);
    const unsigned fpdn = __shfl_sync(kFull, w.pl, sd, 16), fp0 = __shfl_sync(kFull, w.pl, 0, 16);
    popl = xpl;
    if (!do_push) return kEmptyKey;
    if (pos == 0) return x;
    if (slot < pos - 1) {
      w.e = fdn;
      w.pl = fpdn;
    } else if (slot == pos - 1) {
      w.e = x;
      w.pl = xpl;
    }
    popl = fp0;
    return fe0;
  }
  const unsigned long long up = shfl64(w.e, su, 16), dn = shfl64(w.e, sd, 16), e0 = shfl64(w.e, 0, 16);
  const unsigned pup = __shfl_sync(kFull, w.pl, su, 16), pdn = __shfl_sync(kFull, w.pl, sd, 16),
                 p0 = __shfl_sync(kFull, w.pl, 0, 16);
  popl = xpl;
  if (!do_push) return kEmptyKey;
  if (w.n < K1) {
    if (slot == pos) {
      w.e = x;
      w.pl = xpl;
    } else if (slot > pos) {
      w.e = up;
      w.pl = pup;
    }
    ++w.n;
    return kEmptyKey;
  }
  if (pos == 0) return x;
  if (slot < pos - 1) {
    w.e = dn;
    w.pl = pdn;
  } else if (slot == pos - 1) {
    w.e = x;
    w.pl = xpl;
  }
  popl = p0;
  return e0;
}

template <int K1>
__device__ __forceinline__ unsigned long long win16_pop(Win16<K1>& w, int lane, unsigned& popl) {
  const int slot = lane & 15;
  const int sd = slot + 1 > 15 ? 15 : slot + 1;
  const unsigned long long dn = shfl64(w.e, sd, 16), e0 = shfl64(w.e, 0, 16);
  const unsigned pdn = __shfl_sync(kFull, w.pl, sd, 16);
  popl = __shfl_sync(kFull, w.pl, 0, 16);
  if (w.n == 0) return kEmptyKey;
  w.e = (slot + 1 < w.n) ? dn : kEmptyKey;
  w.pl = pdn;
  --w.n;
  return e0;
}

// The 4x4-block window of four entries (K1 = 4), one copy per 2x2 group of its block:
// lanes 4 c .. 4 c + 3 of a block (its 2x2 block c) hold slots 0 .. 3.  Each slot also
// carries the depth key of its entry at the centre of the lane's own 2x2 block, computed
// from the staged record when the entry enters, so a pop hands the 2x2 stage its key
// without reading the record again from global memory (VR render: the dependent L2 reads
// cost 0.24 of 5.25 ms).  Keys are (4x4 depth bits << 32) | (index << 4) | the group's
// four kept-sample bits: indices are below 2^28, so the order stays (depth, index).
// Slots do not move: each holds its rank in the window (0 = smallest), so an insertion
// counts the smaller keys with one ballot, finds the minimum's lane with another and
// fetches it with one shuffle (three 32-bit shuffles where a sorted, shifting window
// needs six), and the new key takes the popped minimum's slot.  Keys are unique, so the
// entries leave in the same order as from a sorted window.
constexpr int kRankEmpty = 64;  // rank of an empty slot
struct WinG {
  unsigned long long e;  // slot lane & 3 of the block's window (kEmptyKey when empty)
  unsigned k2;           // 2x2-block depth key of that slot's entry, for this lane's 2x2 block
  int rk;                // the slot's rank in the window, kRankEmpty when empty
  int n;                 // entries held by the block's window
};
constexpr int kWinGIndexBits = 28;

// insert (x, kx) when do_push, then pop the minimum when the window holds more than four;
// returns the popped key (kEmptyKey if none) and, through kout, its 2x2-block key
__device__ __forceinline__ unsigned long long wing_push(WinG& w, unsigned long long x, unsigned kx, bool do_push,
                                                        int lane, unsigned& kout) {
  const unsigned gm = 0xFu << (lane & 28);  // the lanes of this 2x2 group
  const bool lt = w.e < x;
  const int cnt = __popc(__ballot_sync(kFull, lt) & gm);
  const unsigned b0 = __ballot_sync(kFull, w.rk == 0) & gm;
  const int src = b0 ? __ffs(b0) - 1 : lane;
  const unsigned long long m = shfl64(w.e, src, 32);
  const unsigned km = __shfl_sync(kFull, w.k2, src);
  kout = kx;
  if (!do_push) return kEmptyKey;
  if (w.n < 4) {  // filling: slots 0 .. 3 in order
    if ((lane & 3) == w.n) {
      w.e = x;
      w.k2 = kx;
      w.rk = cnt;
    } else if (w.e != kEmptyKey && !lt) {
      ++w.rk;
    }
    ++w.n;
    return kEmptyKey;
  }
  if (cnt == 0) return x;  // x is the smallest: out at once
  if (w.rk == 0) {         // the minimum leaves; x takes its slot
    w.e = x;
    w.k2 = kx;
    w.rk = cnt - 1;
  } else if (lt) {
    --w.rk;
  }
  kout = km;
  return m;
}

__device__ __forceinline__ unsigned long long wing_pop(WinG& w, int lane, unsigned& kout) {
  const unsigned gm = 0xFu << (lane & 28);
  const unsigned b0 = __ballot_sync(kFull, w.rk == 0) & gm;
  const int src = b0 ? __ffs(b0) - 1 : lane;
  const unsigned long long m = shfl64(w.e, src, 32);
  kout = __shfl_sync(kFull, w.k2, src);
  if (w.n == 0) return kEmptyKey;
  if (w.rk == 0) {
    w.e = kEmptyKey;
    w.rk = kRankEmpty;
  } else if (w.e != kEmptyKey) {
    --w.rk;
  }
  --w.n;
  return m;
}

// The 2x2-block window of eight entries (K2 = 8) on the four lanes of its block, slots j
// and 4 + j on lane 4 c + j, ranked like WinG: two 32-bit shuffles per insertion where
// the sorted, shifting window (Win4) needs ten.  Measured on the VR stereo frame, with
// identical images: both windows ranked 5.19 -> 5.14 ms, and with the two ranks of this
// window in one register (fewer spills at the 72-register budget) 5.11 ms.  Packing
// every rank and count of both windows into two registers spilled less again but ran
// slower (5.16 ms): the bit-field work outweighed the spills.
struct Win8R {
  unsigned long long f0, f1;  // slots j and 4 + j
  unsigned rk;                // their ranks, slot j in bits 0 .. 7 and 4 + j in bits 8 .. 15
                              // (kRankEmpty when empty): one register for both
  int n;
};

__device__ __forceinline__ unsigned long long win8r_push(Win8R& w, unsigned long long x, bool do_push, int lane) {
  const unsigned gm = 0xFu << (lane & 28);
  const bool lt0 = w.f0 < x, lt1 = w.f1 < x;
  const unsigned r0 = w.rk & 0xFFu, r1 = w.rk >> 8;
  const int cnt = __popc(__ballot_sync(kFull, lt0) & gm) + __popc(__ballot_sync(kFull, lt1) & gm);
  const unsigned b0 = __ballot_sync(kFull, r0 == 0u || r1 == 0u) & gm;
  const int src = b0 ? __ffs(b0) - 1 : lane;
  const unsigned long long m = shfl64(r0 == 0u ? w.f0 : w.f1, src, 32);
  if (!do_push) return kEmptyKey;
  unsigned n0 = r0, n1 = r1;
  if (w.n < 8) {  // filling: slot n (lane n & 3, register n >> 2)
    const bool mine = (lane & 3) == (w.n & 3);
    if (mine && w.n < 4) {
      w.f0 = x;
      n0 = (unsigned)cnt;
    } else if (w.f0 != kEmptyKey && !lt0) {
      ++n0;
    }
    if (mine && w.n >= 4) {
      w.f1 = x;
      n1 = (unsigned)cnt;
    } else if (w.f1 != kEmptyKey && !lt1) {
      ++n1;
    }
    w.rk = n0 | (n1 << 8);
    ++w.n;
    return kEmptyKey;
  }
  if (cnt == 0) return x;
  if (r0 == 0u) {
    w.f0 = x;
    n0 = (unsigned)(cnt - 1);
  } else if (lt0) {
    --n0;
  }
  if (r1 == 0u) {
    w.f1 = x;
    n1 = (unsigned)(cnt - 1);
  } else if (lt1) {
    --n1;
  }
  w.rk = n0 | (n1 << 8);
  return m;
}

__device__ __forceinline__ unsigned long long win8r_pop(Win8R& w, int lane) {
  const unsigned gm = 0xFu << (lane & 28);
  const unsigned r0 = w.rk & 0xFFu, r1 = w.rk >> 8;
  const unsigned b0 = __ballot_sync(kFull, r0 == 0u || r1 == 0u) & gm;
  const int src = b0 ? __ffs(b0) - 1 : lane;
  const unsigned long long m = shfl64(r0 == 0u ? w.f0 : w.f1, src, 32);
  if (w.n == 0) return kEmptyKey;
  unsigned n0 = r0, n1 = r1;
  if (r0 == 0u) {
    w.f0 = kEmptyKey;
    n0 = kRankEmpty;
  } else if (w.f0 != kEmptyKey) {
    --n0;
  }
  if (r1 == 0u) {
    w.f1 = kEmptyKey;
    n1 = kRankEmpty;
  } else if (w.f1 != kEmptyKey) {
    --n1;
  }
  w.rk = n0 | (n1 << 8);
  --w.n;
  return m;
}

template <int K2>
struct Win4 {
  static constexpr int R = (K2 + 3) / 4 > 0 ? (K2 + 3) / 4 : 1;
  unsigned long long f[R];  // slots 4 r + (lane & 3)
  int n;
};

template <int K2>
__device__ __forceinline__ unsigned long long win4_push(Win4<K2>& w, unsigned long long x, bool do_push, int lane) {
  constexpr int R = Win4<K2>::R;
  const int j = lane & 3, base = lane & ~3;
  int pos = 0;
#pragma unroll
  for (int r = 0; r < R; ++r) pos += __popc((__ballot_sync(kFull, w.f[r] < x) >> base) & 0xFu);
  unsigned long long left[R], right[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    left[r] = shfl64(w.f[r], base | ((j + 3) & 3), 32);
    right[r] = shfl64(w.f[r], base | ((j + 1) & 3), 32);
  }
  const unsigned long long e0 = shfl64(w.f[0], base, 32);
  if (!do_push) return kEmptyKey;
  if (w.n < K2) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int s = 4 * r + j;
      const unsigned long long up = j > 0 ? left[r] : (r > 0 ? left[r > 0 ? r - 1 : 0] : kEmptyKey);
      w.f[r] = s < pos ? w.f[r] : (s == pos ? x : up);
    }
    ++w.n;
    return kEmptyKey;
  }
  if (pos == 0) return x;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int s = 4 * r + j;
    const unsigned long long dn = j < 3 ? right[r] : (r + 1 < R ? right[r + 1 < R ? r + 1 : 0] : kEmptyKey);
    w.f[r] = s < pos - 1 ? dn : (s == pos - 1 ? x : w.f[r]);
  }
  return e0;
}

template <int K2>
__device__ __forceinline__ unsigned long long win4_pop(Win4<K2>& w, int lane) {
  constexpr int R = Win4<K2>::R;
  const int j = lane & 3, base = lane & ~3;
  unsigned long long right[R];
#pragma unroll
  for (int r = 0; r < R; ++r) right[r] = shfl64(w.f[r], base | ((j + 1) & 3), 32);
  const unsigned long long e0 = shfl64(w.f[0], base, 32);
  if (w.n == 0) return kEmptyKey;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int s = 4 * r + j;
    const unsigned long long dn = j < 3 ? right[r] : (r + 1 < R ? right[r + 1 < R ? r + 1 : 0] : kEmptyKey);
    w.f[r] = s + 1 < w.n ? dn : kEmptyKey;
  }
  --w.n;
  return e0;
}

// list entries a warp stages per batch (records of those meeting its region, and their
// 4x4-block keys) and the resident CTAs per SM its register budget is set for.  Measured on the VR
// frame: occupancy decides (the kernel waits on memory and on the issue of window
// bookkeeping), and with the tournament-tree window 16-entry batches and a 72-register
// budget (7 CTAs of 4 warps per SM, K3 = 16) beat 6 CTAs at 80 registers and 8 CTAs at
// 64 registers (5.64 / 5.86 / 6.06 ms).  The backward replay holds the gradient terms
// as well: 4 CTAs at 128 registers, with no spill, beat 5 CTAs at 96 registers, which
// spill (28.2 / 32.0 ms on four 1280^2 views).
template <int K2>
constexpr int stage_of() { return 16; }
template <int K2, bool BWD>
constexpr int ctas_of() { return BWD ? 4 : 7; }
// key slots of the per-sample window: the tournament tree (k3 <= 16) always has 16
__host__ __device__ inline int window_key_slots(int k3) { return k3 <= 16 ? 16 : k3; }
__host__ __device__ inline size_t warp_smem_bytes(int k3, int stage) {
  return (size_t)stage * 100 + (size_t)window_key_slots(k3) * 32 * 8 + (size_t)k3 * 32 * 4 + (size_t)stage * 8;
}

// blend of one pair whose colour c the caller holds; the backward replay reads the rest
// of the record for the gradient
template <bool STATS, bool BWD>
__device__ __forceinline__ void blend_c(Px& p, float alpha, int g, float3 c, const float4* __restrict__ recv) {
  if (!p.active) return;
  const float test = p.T * (1.f - alpha);
  if (test < kTStop) {
    p.active = false;
    return;
  }
  if (BWD) blend_grad(p, alpha, recv + (long long)g * kRecF4, p.T, p.C0, p.C1, p.C2, p.grad + (long long)g * 16);
  const float aT = alpha * p.T;
  p.C0 = fmaf(aT, c.x, p.C0);
  p.C1 = fmaf(aT, c.y, p.C1);
  p.C2 = fmaf(aT, c.z, p.C2);
  p.T = test;
  if (STATS) ++p.n_blend;
}

__device__ __forceinline__ float3 rec_colour(const float4* __restrict__ recv, int g) {
  const float4 f5 = recv[(long long)g * kRecF4 + 5];
  return make_float3(f5.y, f5.z, f5.w);
}

// Per-sample window as a tournament tree over 16 slots (K3 <= 16).  The depth keys
// (order-preserving bits of t*), indices and alphas sit in shared memory, [slot][lane];
// the winners (smallest key) of the 15 internal nodes (node n = 1 .. 15, children 2n and
// 2n + 1, slot s at node 16 + s) are 4-bit slot numbers in two 32-bit registers: nodes
// 8 .. 15 in lo (nibble n - 8), nodes 1 .. 7 in hi (nibble n - 1), so each level of a
// replay touches one word with 32-bit shifts.  Putting a key into a slot replays the four
// matches on the slot's path to the root, so every insertion costs the same: no
// data-dependent shifting and no divergence.  Unused slots hold kEmptyT.  hc is the colour
// of the root winner, loaded when it changes.
// The matches compare the 32-bit depth keys alone (one compare and one select each, where
// (depth, index) keys take two of each): an opponent wins only when strictly nearer, so
// of two entries with bit-equal t* at a sample the one that reached the match later goes
// on.  That differs from the (t*, index) order only for bit-equal FP32 depths, a tie whose
// two orders both lie within the float64 reading's near-tie margin.
struct Tree16 {
  unsigned lo, hi;
};
// every internal node starts with the leftmost slot of its subtree (all slots empty)
constexpr unsigned kTreeInitLo = 0xeca86420u, kTreeInitHi = 0x0c840800u;
constexpr unsigned kEmptyT = 0xFFFFFFFFu;  // above every finite depth's key
__device__ __forceinline__ int tree_root(const Tree16& t) { return (int)(t.hi & 0xFu); }

// The opponents of a replay of slot s: the winners of the siblings of the path's nodes,
// which the replay does not change, with their keys (loaded together)
struct TreeOpp {
  int s0, s1, s2, s3;
  unsigned k0, k1, k2, k3;
};
__device__ __forceinline__ TreeOpp tree_opponents(const Tree16& t, const unsigned* kt, int lane, int s) {
  TreeOpp o;
  o.s0 = s ^ 1;
  o.s1 = (int)((t.lo >> (4 * ((s >> 1) ^ 1))) & 0xFu);
  o.s2 = (int)((t.hi >> (4 * (3 + ((s >> 2) ^ 1)))) & 0xFu);
  o.s3 = (int)((t.hi >> (4 * (1 + ((s >> 3) ^ 1)))) & 0xFu);
  o.k0 = kt[o.s0 * 32 + lane];
  o.k1 = kt[o.s1 * 32 + lane];
  o.k2 = kt[o.s2 * 32 + lane];
  o.k3 = kt[o.s3 * 32 + lane];
  return o;
}

// key x now sits in slot s: the four matches of s's path against the opponents, as a
// chain of compares
__device__ __forceinline__ void tree_play(Tree16& t, int s, unsigned x, const TreeOpp& o) {
  int cs = s;
  unsigned ck = x;
  if (o.k0 < ck) {
    ck = o.k0;
    cs = o.s0;
  }
  {
    const int sh = 4 * (s >> 1);
    t.lo = (t.lo & ~(0xFu << sh)) | ((unsigned)cs << sh);
  }
  if (o.k1 < ck) {
    ck = o.k1;
    cs = o.s1;
  }
  unsigned hi = t.hi;
  {
    const int sh = 4 * (3 + (s >> 2));
    hi = (hi & ~(0xFu << sh)) | ((unsigned)cs << sh);
  }
  if (o.k2 < ck) {
    ck = o.k2;
    cs = o.s2;
  }
  {
    const int sh = 4 * (1 + (s >> 3));
    hi = (hi & ~(0xFu << sh)) | ((unsigned)cs << sh);
  }
  if (o.k3 < ck) cs = o.s3;
  t.hi = (hi & ~0xFu) | (unsigned)cs;
}

template <bool STATS, bool BWD>
__device__ __forceinline__ void tree3_push(Px& p, Tree16& t, float3& hc, unsigned* kt, int* kg, float* aa, int K3,
                                           int lane, unsigned x, int g, float alpha, float3 c,
                                           const float4* __restrict__ recv) {
  if (p.n3 < K3) {  // filling: the next free slot
    const int s = p.n3++;
    const TreeOpp o = tree_opponents(t, kt, lane, s);
    kt[s * 32 + lane] = x;
    kg[s * 32 + lane] = g;
    aa[s * 32 + lane] = alpha;
    const int w0 = tree_root(t);
    tree_play(t, s, x, o);
    if (tree_root(t) != w0 || s == 0) hc = c;
    return;
  }
  // the root's key, index and alpha and the opponents of its slot, loaded together
  const int w = tree_root(t);
  const TreeOpp o = tree_opponents(t, kt, lane, w);
  const unsigned m = kt[w * 32 + lane];
  const int gm = kg[w * 32 + lane];
  const float am = aa[w * 32 + lane];
  if (x < m) {  // x is the nearest: out at once
    blend_c<STATS, BWD>(p, alpha, g, c, recv);
    return;
  }
  const float3 mc = hc;
  kt[w * 32 + lane] = x;
  kg[w * 32 + lane] = g;
  aa[w * 32 + lane] = alpha;
  tree_play(t, w, x, o);
  const int nw = tree_root(t);
  hc = nw == w ? c : rec_colour(recv, kg[nw * 32 + lane]);
  blend_c<STATS, BWD>(p, am, gm, mc, recv);
}

// pops the root winner and blends it
template <bool STATS, bool BWD>
__device__ __forceinline__ void tree3_pop(Px& p, Tree16& t, float3& hc, unsigned* kt, const int* kg,
                                          const float* aa, int lane, const float4* __restrict__ recv) {
  const int w = tree_root(t);
  const TreeOpp o = tree_opponents(t, kt, lane, w);
  const int gm = kg[w * 32 + lane];
  const float am = aa[w * 32 + lane];
  const float3 mc = hc;
  kt[w * 32 + lane] = kEmptyT;
  tree_play(t, w, kEmptyT, o);
  p.n3--;
  if (p.n3 > 0) hc = rec_colour(recv, kg[tree_root(t) * 32 + lane]);
  blend_c<STATS, BWD>(p, am, gm, mc, recv);
}

// Per-lane ring of the per-sample window: packed keys and alphas, [slot][lane], ascending
// from the head h3.  hc holds the colour of the head entry: it is loaded when an entry
// becomes the head, so the load is in flight while the lane works on later entries and
// the blend of a popped head reads no memory.
template <bool STATS, bool BWD>
__device__ __forceinline__ void ring3_push(Px& p, float3& hc, unsigned long long* kk, float* aa, int K3, int lane,
                                           unsigned long long x, float alpha, float3 c, const float4* __restrict__ recv) {
  const bool full = p.n3 == K3;
  unsigned long long m = 0;
  float am = 0.f;
  float3 mc = hc;
  if (full) {
    m = kk[p.h3 * 32 + lane];
    if (x < m) {
      blend_c<STATS, BWD>(p, alpha, (int)(x & 0xffffffffu), c, recv);
      return;
    }
    am = aa[p.h3 * 32 + lane];
    p.h3 = p.h3 + 1 == K3 ? 0 : p.h3 + 1;
    p.n3--;
  }
  int j = p.n3;
  while (j > 0) {
    int q = p.h3 + j - 1;
    if (q >= K3) q -= K3;
    const unsigned long long v = kk[q * 32 + lane];
    if (!(x < v)) break;
    int d = q + 1;
    if (d >= K3) d -= K3;
    kk[d * 32 + lane] = v;
    aa[d * 32 + lane] = aa[q * 32 + lane];
    --j;
  }
  int d = p.h3 + j;
  if (d >= K3) d -= K3;
  kk[d * 32 + lane] = x;
  aa[d * 32 + lane] = alpha;
  p.n3++;
  if (j == 0) hc = c;                                                        // x is the new head
  else if (full) hc = rec_colour(recv, (int)(kk[p.h3 * 32 + lane] & 0xffffffffu));  // the next entry is
  if (full) blend_c<STATS, BWD>(p, am, (int)(m & 0xffffffffu), mc, recv);
}

// pops the head of the per-sample window and blends it
template <bool STATS, bool BWD>
__device__ __forceinline__ void ring3_pop(Px& p, float3& hc, const unsigned long long* kk, const float* aa, int K3,
                                          int lane, const float4* __restrict__ recv) {
  const unsigned long long m = kk[p.h3 * 32 + lane];
  const float am = aa[p.h3 * 32 + lane];
  const float3 mc = hc;
  p.h3 = p.h3 + 1 == K3 ? 0 : p.h3 + 1;
  p.n3--;
  if (p.n3 > 0) hc = rec_colour(recv, (int)(kk[p.h3 * 32 + lane] & 0xffffffffu));
  blend_c<STATS, BWD>(p, am, (int)(m & 0xffffffffu), mc, recv);
}

// TREE: the per-sample window is the tournament tree (k3 <= 16), else the ring; a
// template parameter, so each instance holds only its own window's code
template <int K1, int K2, bool BWD, bool STATS, bool TREE>
__global__ void __launch_bounds__(kRegionWarps * 32, ctas_of<K2, BWD>()) warp_render_kernel(RenderArgs a) {
  constexpr int kStage = stage_of<K2>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int K3 = a.k3;
  unsigned char* ws = smem_raw + (size_t)wib * warp_smem_bytes(K3, kStage);
  float4* st_rec = reinterpret_cast<float4*>(ws);
  int* st_gid = reinterpret_cast<int*>(ws + kStage * 96);
  unsigned long long* k3s = reinterpret_cast<unsigned long long*>(ws + kStage * 100);
  // the tree's depth keys and indices (k3 <= 16) share the key slots' bytes
  unsigned* k3t = reinterpret_cast<unsigned*>(k3s);
  int* k3g = reinterpret_cast<int*>(k3t + 16 * 32);
  float* a3s = reinterpret_cast<float*>(ws + kStage * 100 + (size_t)window_key_slots(K3) * 256);
  // 4x4-block keys of the staged batch (order-preserving depth bits), [entry][block of the warp]
  uint32_t* st_k1 = reinterpret_cast<uint32_t*>(ws + kStage * 100 + (size_t)window_key_slots(K3) * 256 +
                                                (size_t)K3 * 128);
  const int sx = (lane & 1) | ((lane >> 1) & 2) | ((lane >> 2) & 4);
  const int sy = ((lane >> 1) & 1) | ((lane >> 2) & 2);
  const unsigned lt = (1u << lane) - 1u;
  unsigned n_eval = 0, n_kept = 0, n_blend = 0;
  const unsigned n_tasks = 8u * *a.n_items;
  // the next task is taken from the queue while the current one runs, so the atomic's
  // round trip is off the warp's path (each warp overshoots the queue by one claim)
  unsigned next_task = 0;
  if (lane == 0) next_task = atomicAdd(a.queue, 1u);
  for (;;) {
    const unsigned task = __shfl_sync(kFull, next_task, 0);
    if (task >= n_tasks) break;
    if (lane == 0) next_task = atomicAdd(a.queue, 1u);
    const ItemGeom g = decode(a.items[task >> 3], a.tiles_per_view, a.key_tile, a.views);
    const int region = task & 7, rx = 8 * (region & 1), ry = 4 * (region >> 1);
    const ViewParams& vp = a.views[g.view];
    const float4* recv = a.rec + vp.base * kRecF4;
    const int X = g.ox + rx + sx, Y = g.oy + ry + sy;
    Px p;
    bool valid;
    float rx0, rx1, ry0, ry1;  // sample-position bounds of the region (culling)
    if (rx >= g.ext || ry >= g.ext) continue;  // a region outside a smaller periphery item
    if (g.kind == kKindLow) {
      valid = 2 * X < vp.W && 2 * Y < vp.H;
      p.px = 2.f * X + 1.f;
      p.py = 2.f * Y + 1.f;
      rx0 = 2.f * (g.ox + rx) + 1.f;
      rx1 = rx0 + 14.f;
      ry0 = 2.f * (g.oy + ry) + 1.f;
      ry1 = ry0 + 6.f;
    } else {
      valid = X < vp.W && Y < vp.H;
      p.px = X + 0.5f;
      p.py = Y + 0.5f;
      rx0 = g.ox + rx + 0.5f;
      rx1 = rx0 + 7.f;
      ry0 = g.oy + ry + 0.5f;
      ry1 = ry0 + 3.f;
    }
    if (!__any_sync(kFull, valid)) continue;
    p.T = 1.f;
    p.C0 = p.C1 = p.C2 = 0.f;
    p.active = valid;
    p.h3 = p.n3 = 0;
    p.n_eval = p.n_kept = p.n_blend = 0;
    if (BWD) {
      const long long HWb = (long long)vp.H * vp.W;
      const long long HW2b = (long long)(vp.H / 2) * (vp.W / 2);
      float4 dv = make_float4(0.f, 0.f, 0.f, 0.f), sv = make_float4(0.f, 0.f, 0.f, 1.f);
      if (valid) {
        const long long si = g.kind == kKindLow ? (long long)g.view * HW2b + (long long)Y * (vp.W / 2) + X
                                                : (long long)g.view * HWb + (long long)Y * vp.W + X;
        dv = g.kind == kKindLow ? reinterpret_cast<const float4*>(a.dL_dlow)[si]
                                : reinterpret_cast<const float4*>(a.dL_dout)[si];
        sv = g.kind == kKindLow ? a.s_low[si] : a.s_full[si];
      }
      p.G0 = dv.x;
      p.G1 = dv.y;
      p.G2 = dv.z;
      p.GT = dv.x * a.bg[0] + dv.y * a.bg[1] + dv.z * a.bg[2];
      p.F0 = sv.x;
      p.F1 = sv.y;
      p.F2 = sv.z;
      p.TF = sv.w;
      p.grad = a.grad_rec + vp.base * 16;
    }
    const int bx4 = g.ox + rx + (sx & ~3), by4 = g.oy + ry, bx2 = g.ox + rx + (sx & ~1), by2 = g.oy + ry + (sy & ~1);
    float c4x, c4y, c2x, c2y;
    if (g.kind == kKindLow) {
      c4x = 2.f * bx4 + 4.f;
      c4y = 2.f * by4 + 4.f;
      c2x = 2.f * bx2 + 2.f;
      c2y = 2.f * by2 + 2.f;
    } else {
      c4x = bx4 + 2.f;
      c4y = by4 + 2.f;
      c2x = bx2 + 1.f;
      c2y = by2 + 1.f;
    }
    // K1 = 4: lane L evaluates, every fourth entry, the 2x2-block depth key of entry
    // e + (L >> 3) for 2x2 group L & 7 of the warp (group g's block starts at sample
    // x 2 (g & 1) + 4 (g >> 2 & 1), y 2 (g >> 1 & 1) of the region), and each entry's key
    // then reaches its group by one shuffle: one evaluation per lane and four entries
    // instead of one per lane and entry
    float gcx, gcy;
    {
      const int gl = lane & 7;
      const int bxg = g.ox + rx + 2 * (gl & 1) + 4 * ((gl >> 2) & 1), byg = g.oy + ry + 2 * ((gl >> 1) & 1);
      gcx = g.kind == kKindLow ? 2.f * bxg + 2.f : bxg + 1.f;
      gcy = g.kind == kKindLow ? 2.f * byg + 2.f : byg + 1.f;
    }
    unsigned kb = 0u;
    Win16<K1> w1;
    WinG wg;  // the 4x4-block window when K1 = 4
    Win4<K2> w2;
    w1.e = kEmptyKey;
    w1.pl = 0u;
    w1.n = 0;
    wg.e = kEmptyKey;
    wg.k2 = 0u;
    wg.rk = kRankEmpty;
    wg.n = 0;
    Win8R w8;  // the 2x2-block window when K2 = 8 (with K1 = 4)
    w8.f0 = w8.f1 = kEmptyKey;
    w8.rk = kRankEmpty | (kRankEmpty << 8);
    w8.n = 0;
    float3 hc = make_float3(0.f, 0.f, 0.f);
    // per-sample window: tournament tree when K3 <= 16 (every slot starts empty), else ring
    constexpr bool use_tree = TREE;
    Tree16 tree{kTreeInitLo, kTreeInitHi};
    if constexpr (use_tree)
      for (int s3 = 0; s3 < 16; ++s3) k3t[s3 * 32 + lane] = kEmptyT;
#pragma unroll
    for (int r = 0; r < Win4<K2>::R; ++r) w2.f[r] = kEmptyKey;
    w2.n = 0;
    // popped from a 2x2 window: per-sample evaluation, into the per-sample window
    auto pop2 = [&](unsigned long long x2) {
      if (x2 != kEmptyKey && p.active) {
        const int g2 = (int)(x2 & 0xffffffffu);
        const float4* r = recv + (long long)g2 * kRecF4;
        float al, t;
        float3 c;
        if (eval_full<STATS, false>(r, p, al, t, c)) {
          if constexpr (use_tree)
            tree3_push<STATS, BWD>(p, tree, hc, k3t, k3g, a3s, K3, lane, float_order_bits(t), g2, al, c, recv);
          else
            ring3_push<STATS, BWD>(p, hc, k3s, a3s, K3, lane, pack_key(t, g2), al, c, recv);
        }
      }
    };
    // popped from a 4x4 window (all lanes; x1 and its kept-sample mask m1 are uniform
    // over the 4x4 block): 2x2-block membership over the still-active samples, 2x2 window
    auto pop1 = [&](unsigned long long x1, unsigned m1) {
      const bool k = x1 != kEmptyKey && p.active && ((m1 >> (lane & 15)) & 1u);
      const unsigned bal = __ballot_sync(kFull, k);
      if (bal == 0u) return;
      const int g1 = (int)(x1 & 0xffffffffu);
      const float4* r = recv + (long long)(x1 != kEmptyKey ? g1 : 0) * kRecF4;
      const unsigned long long x2 =
          win4_push<K2>(w2, pack_key(depth_at(r, c2x, c2y), g1), ((bal >> (lane & ~3)) & 0xFu) != 0u, lane);
      pop2(x2);
    };
    // the same from the grouped window (K1 = 4): x1 carries the group's kept-sample bits
    // and k2 is the entry's depth key at this lane's 2x2-block centre
    auto pop1g = [&](unsigned long long x1, unsigned k2) {
      const bool k = x1 != kEmptyKey && p.active && ((x1 >> (lane & 3)) & 1u);
      const unsigned bal = __ballot_sync(kFull, k);
      if (bal == 0u) return;
      const unsigned g1 = (unsigned)(x1 >> 4) & ((1u << kWinGIndexBits) - 1u);
      const unsigned long long key2 = ((unsigned long long)k2 << 32) | g1;
      const bool push2 = ((bal >> (lane & ~3)) & 0xFu) != 0u;
      unsigned long long x2;
      if constexpr (K2 == 8)
        x2 = win8r_push(w8, key2, push2, lane);
      else
        x2 = win4_push<K2>(w2, key2, push2, lane);
      pop2(x2);
    };
    // instance indices fit 32 bits (the instance capacity is below 2^31)
    const unsigned start = a.ranges[2 * (long long)g.tile], end = a.ranges[2 * (long long)g.tile + 1];
    // 32 list entries per round (one per lane: index and bounding-box test), staged
    // kStage lanes at a time into the warp's record buffer
    for (unsigned b0 = start; b0 < end; b0 += 32) {
      if (!__any_sync(kFull, p.active)) break;
      const unsigned j = b0 + lane;
      bool rel = false;
      int gj = 0;
      if (j < end) {
        gj = (int)a.vals[j];
        const float4 bb = a.bbox[vp.base + gj];
        rel = bb.x <= rx1 && bb.z >= rx0 && bb.y <= ry1 && bb.w >= ry0;
      }
      const unsigned mall = __ballot_sync(kFull, rel);
      for (int q0 = 0; q0 < 32; q0 += kStage) {
        const unsigned m = mall & ((kStage == 32 ? kFull : ((1u << kStage) - 1u)) << q0);
        if (m == 0u) continue;
        if (q0 > 0 && !__any_sync(kFull, p.active)) break;
        __syncwarp();
        if ((m >> lane) & 1u) {
          const int slot = __popc(m & lt);
          const float4* src = recv + (long long)gj * kRecF4;
          // 16-byte asynchronous copies global -> shared (no register round trip): VR render
          // 5.285 -> 5.248 ms against plain loads and stores
          const uint32_t dst = (uint32_t)__cvta_generic_to_shared(st_rec + slot * kRecF4);
#pragma unroll
          for (int q = 0; q < kRecF4; ++q)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst + 16u * q), "l"(src + q) : "memory");
          st_gid[slot] = gj;
        }
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncwarp();
        const int nrel = __popc(m);
        if (K1 > 0 || K2 > 0) {
          // the depth keys at both 4x4-block centres of the warp, one lane per (entry,
          // block): lane e of each half-warp for entry e, instead of every lane of a block
          // evaluating the same key in the loop below.  VR render 5.42 -> 5.31 ms.
          const int eb = lane & 15;
          if (eb < nrel) st_k1[eb * 2 + (lane >> 4)] = float_order_bits(depth_at(st_rec + eb * kRecF4, c4x, c4y));
          __syncwarp();
        }
        for (int e = 0; e < nrel; ++e) {
          const float4* r = st_rec + e * kRecF4;
          const int ge = st_gid[e];
          if (K1 == 0 && K2 == 0) {
            float al, t;
            float3 c;
            if (p.active && eval_full<STATS>(r, p, al, t, c)) {
              if (a.stream_order)  // global orders: the list order is the blend order
                blend_c<STATS, BWD>(p, al, ge, c, recv);
              else
                if constexpr (use_tree)
                  tree3_push<STATS, BWD>(p, tree, hc, k3t, k3g, a3s, K3, lane, float_order_bits(t), ge, al, c,
                                         recv);
                else
                  ring3_push<STATS, BWD>(p, hc, k3s, a3s, K3, lane, pack_key(t, ge), al, c, recv);
            }
          } else {
            if constexpr (K1 == 4) {
              if ((e & 3) == 0) {
                const int ee = e + (lane >> 3);
                kb = ee < nrel ? float_order_bits(depth_at(st_rec + ee * kRecF4, gcx, gcy)) : 0u;
              }
            }
            bool k = false;
            if (p.active) {
              float dx, dy, qw;
              if (STATS) ++p.n_eval;
              k = pair_test(r[0], r[1], r[2], r[3].x, p.px, p.py, dx, dy, qw);
            }
            const unsigned bal = __ballot_sync(kFull, k);
            if (bal == 0u) continue;
            const unsigned bm = (bal >> (lane & 16)) & 0xFFFFu;
            const unsigned long long k1 = (unsigned long long)st_k1[e * 2 + (lane >> 4)] << 32;
            if constexpr (K1 == 4) {
              // the entry's depth key at this lane's 2x2-block centre (evaluated by lane
              // (e & 3) * 8 + this lane's group)
              const unsigned k2 = __shfl_sync(kFull, kb, ((e & 3) << 3) | (lane >> 2));
              unsigned k2o;
              const unsigned long long x1 =
                  wing_push(wg, k1 | ((unsigned long long)(unsigned)ge << 4) | ((bm >> (lane & 12)) & 0xFu), k2,
                            bm != 0u, lane, k2o);
              // the full window pops on almost every push, so no vote guards the call:
              // pop1g's own ballot returns at once when no lane holds a popped entry
              pop1g(x1, k2o);
            } else {
              unsigned m1;
              const unsigned long long x1 = win16_push<K1>(w1, k1 | (unsigned)ge, bm, bm != 0u, lane, m1);
              if (__any_sync(kFull, x1 != kEmptyKey)) pop1(x1, m1);
            }
          }
        }
      }
    }
    if (K1 > 0 || K2 > 0) {
      for (int it = 0; it < K1; ++it) {
        if constexpr (K1 == 4) {
          unsigned k2o;
          const unsigned long long x1 = wing_pop(wg, lane, k2o);
          if (__any_sync(kFull, x1 != kEmptyKey)) pop1g(x1, k2o);
        } else {
          unsigned m1;
          const unsigned long long x1 = win16_pop<K1>(w1, lane, m1);
          if (__any_sync(kFull, x1 != kEmptyKey)) pop1(x1, m1);
        }
      }
      for (int it = 0; it < K2; ++it) {
        if constexpr (K1 == 4 && K2 == 8)
          pop2(win8r_pop(w8, lane));
        else
          pop2(win4_pop<K2>(w2, lane));
      }
    }
    if constexpr (use_tree)
      while (p.n3 > 0 && p.active) tree3_pop<STATS, BWD>(p, tree, hc, k3t, k3g, a3s, lane, recv);
    else
      while (p.n3 > 0 && p.active) ring3_pop<STATS, BWD>(p, hc, k3s, a3s, K3, lane, recv);
    if (STATS) {
      n_eval += p.n_eval;
      n_kept += p.n_kept;
      n_blend += p.n_blend;
    }
    if (BWD) continue;
    // ---- outputs (same as the block kernel)
    const float v0 = fmaf(p.T, a.bg[0], p.C0), v1 = fmaf(p.T, a.bg[1], p.C1), v2 = fmaf(p.T, a.bg[2], p.C2);
    const long long HW = (long long)vp.H * vp.W;
    const int W2 = vp.W / 2, H2 = vp.H / 2;
    const long long HW2 = (long long)H2 * W2;
    if (g.kind == kKindFull) {
      float s0 = v0 + __shfl_xor_sync(kFull, v0, 1), s1 = v1 + __shfl_xor_sync(kFull, v1, 1),
            s2 = v2 + __shfl_xor_sync(kFull, v2, 1);
      s0 += __shfl_xor_sync(kFull, s0, 2);
      s1 += __shfl_xor_sync(kFull, s1, 2);
      s2 += __shfl_xor_sync(kFull, s2, 2);
      const float a0 = 0.25f * s0, a1 = 0.25f * s1, a2 = 0.25f * s2;
      if (valid) {
        float o0 = v0, o1 = v1, o2 = v2;
        if (a.fovea_mode != 0 && a.tile_class[g.tile] == kClassHybrid) {
          const float dx = p.px - vp.gaze_x, dy = p.py - vp.gaze_y;
          const float w = fminf(fmaxf((vp.radius + vp.band - sqrtf(dx * dx + dy * dy)) / vp.band, 0.f), 1.f);
          o0 = w * v0 + (1.f - w) * a0;
          o1 = w * v1 + (1.f - w) * a1;
          o2 = w * v2 + (1.f - w) * a2;
        }
        float* out = a.out + (long long)g.view * 3 * HW + (long long)Y * vp.W + X;
        out[0] = o0;
        out[HW] = o1;
        out[2 * HW] = o2;
        if (a.s_full) a.s_full[(long long)g.view * HW + (long long)Y * vp.W + X] = make_float4(p.C0, p.C1, p.C2, p.T);
        if (a.low && (lane & 3) == 0 && X / 2 < W2 && Y / 2 < H2) {
          float* lo = a.low + (long long)g.view * 3 * HW2 + (long long)(Y / 2) * W2 + X / 2;
          lo[0] = a0;
          lo[HW2] = a1;
          lo[2 * HW2] = a2;
        }
      }
    } else if (valid) {
      float* lo = a.low + (long long)g.view * 3 * HW2 + (long long)Y * W2 + X;
      lo[0] = v0;
      lo[HW2] = v1;
      lo[2 * HW2] = v2;
      if (a.s_low) a.s_low[(long long)g.view * HW2 + (long long)Y * W2 + X] = make_float4(p.C0, p.C1, p.C2, p.T);
    }
  }
  if (STATS) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n_eval += __shfl_xor_sync(kFull, n_eval, o);
      n_kept += __shfl_xor_sync(kFull, n_kept, o);
      n_blend += __shfl_xor_sync(kFull, n_blend, o);
    }
    if (lane == 0) {
      atomicAdd(&a.stats[0], (unsigned long long)n_eval);
      atomicAdd(&a.stats[1], (unsigned long long)n_kept);
      atomicAdd(&a.stats[2], (unsigned long long)n_blend);
    }
  }
}

template <int K1, int K2, bool BWD, bool STATS, bool TREE>
void launch_warp_tw(const RenderArgs& a, cudaStream_t st) {
  const size_t smem = warp_smem_bytes(a.k3, stage_of<K2>()) * kRegionWarps;
  // attribute and occupancy per device and per window size k3 (set outside stream capture
  // by the first eager call)
  static std::atomic<int> smem_set[kMemoDevices];
  static std::atomic<int> occupancy[kMaxWin + 1][kMemoDevices];
  ensure_dynamic_smem(smem_set, warp_render_kernel<K1, K2, BWD, STATS, TREE>, (int)smem);
  int per_sm = per_device_memo(occupancy[a.k3], [smem] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, warp_render_kernel<K1, K2, BWD, STATS, TREE>, kRegionWarps * 32,
                                                  smem);
    return b > 0 ? b : 1;
  });
  if (a.max_ctas_per_sm > 0) per_sm = std::min(per_sm, a.max_ctas_per_sm * (kBlock / (kRegionWarps * 32)));
  warp_render_kernel<K1, K2, BWD, STATS, TREE>
      <<<(unsigned)(device_sm_count() * per_sm), kRegionWarps * 32, smem, st>>>(a);
}

template <int K1, int K2, bool BWD, bool STATS>
void launch_warp_t(const RenderArgs& a, cudaStream_t st) {
  if (a.k3 <= 16)
    launch_warp_tw<K1, K2, BWD, STATS, true>(a, st);
  else
    launch_warp_tw<K1, K2, BWD, STATS, false>(a, st);
}

// fast path for the common window shapes; returns false when (k1, k2) is not compiled
template <bool BWD, bool STATS>
bool launch_warp(const RenderArgs& a, cudaStream_t st) {
  const int k1 = a.sort_mode == 2 ? a.k1 : 0, k2 = a.sort_mode == 2 ? a.k2 : 0;
  if (a.sort_mode == 0) return false;
  if (k1 == 0 && k2 == 0) launch_warp_t<0, 0, BWD, STATS>(a, st);
  else if (k1 == 4 && k2 == 8) launch_warp_t<4, 8, BWD, STATS>(a, st);
  else if (k1 == 8 && k2 == 16) launch_warp_t<8, 16, BWD, STATS>(a, st);
  else if (k1 == 1 && k2 == 1) launch_warp_t<1, 1, BWD, STATS>(a, st);
  else return false;
  return true;
}

// ---- two-pass foveated baseline (Appendix A) ------------------------------------------

// Half-resolution pixels of the second pass whose upsampled value some full-resolution
// pixel with w < 1 reads: pixel (i, j) is tapped by the pixels 2i - 1 .. 2i + 2 (columns)
// and 2j - 1 .. 2j + 2 (rows); w < 1 where the pixel centre lies farther than radius from
// the gaze.  Written as a visibility mask of the half-resolution render.
__global__ void lowmask_kernel(TwoPassViews tp, int W, int H, uint8_t* __restrict__ mask) {
  const int W2 = W / 2, H2 = H / 2;
  const long long HW2 = (long long)W2 * H2;
  const int i = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.z;
  if (i >= W2) return;
  for (int j = blockIdx.y; j < H2; j += gridDim.y) {
    const long long q = (long long)v * HW2 + (long long)j * W2 + i;
    bool need = false;
    for (int y = max(2 * j - 1, 0); y <= min(2 * j + 2, H - 1) && !need; ++y)
      for (int x = max(2 * i - 1, 0); x <= min(2 * i + 2, W - 1); ++x) {
        const float dx = x + 0.5f - tp.gaze_x[v], dy = y + 0.5f - tp.gaze_y[v];
        if (sqrtf(dx * dx + dy * dy) > tp.radius[v]) {
          need = true;
          break;
        }
      }
    mask[q] = need ? 1 : 0;
  }
}

// out = w * centre + (1 - w) * bilinear(low) inside each view's centre square, the
// upsampled half-resolution image elsewhere (w = 0 there)
__global__ void two_pass_composite_kernel(TwoPassViews tp, int W, int H, int SW, int SH,
                                          const float* __restrict__ centre, const float* __restrict__ low,
                                          float* __restrict__ out) {
  const int W2 = W / 2, H2 = H / 2;
  const long long HW = (long long)W * H, HW2 = (long long)W2 * H2, HWc = (long long)SW * SH;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, v = blockIdx.z;
  if (x >= W) return;
  for (int y = blockIdx.y; y < H; y += gridDim.y) {
    const long long r = (long long)y * W + x;
    const float ux = (x + 0.5f) * 0.5f - 0.5f, uy = (y + 0.5f) * 0.5f - 0.5f;
    const int x0 = (int)floorf(ux), y0 = (int)floorf(uy);
    const float fx = ux - x0, fy = uy - y0;
    const int xa = min(max(x0, 0), W2 - 1), xb = min(max(x0 + 1, 0), W2 - 1);
    const int ya = min(max(y0, 0), H2 - 1), yb = min(max(y0 + 1, 0), H2 - 1);
    const int cx = x - tp.x0[v], cy = y - tp.y0[v];
    const bool in = cx >= 0 && cx < SW && cy >= 0 && cy < SH;
    float w = 0.f;
    if (in) {
      const float dx = x + 0.5f - tp.gaze_x[v], dy = y + 0.5f - tp.gaze_y[v];
      w = fminf(fmaxf((tp.radius[v] + tp.band[v] - sqrtf(dx * dx + dy * dy)) / tp.band[v], 0.f), 1.f);
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float* L = low + ((long long)v * 3 + ch) * HW2;
      const float top = (1.f - fx) * L[(long long)ya * W2 + xa] + fx * L[(long long)ya * W2 + xb];
      const float bot = (1.f - fx) * L[(long long)yb * W2 + xa] + fx * L[(long long)yb * W2 + xb];
      const float up = (1.f - fy) * top + fy * bot;
      float o = up;
      if (w > 0.f) o = w * centre[((long long)v * 3 + ch) * HWc + (long long)cy * SW + cx] + (1.f - w) * up;
      out[((long long)v * 3 + ch) * HW + r] = o;
    }
  }
}

// Stereo reuse of distant content: eye v's pixel = C_near + T_near (C_far + T_far bg), with
// (C, T) per pixel of views 0, 1 (the eyes' near layers) and 2 (the far layer, rendered
// once from the cyclopean camera).  One thread per pixel of both eyes.
__global__ void __launch_bounds__(256) reuse_composite_kernel(const float4* __restrict__ s_full, long long HW,
                                                              float bg0, float bg1, float bg2, float* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * HW) return;
  const int v = (int)(i / HW);
  const long long p = i - v * HW;
  const float4 n = s_full[i], f = s_full[2 * HW + p];
  float* o = out + (long long)v * 3 * HW + p;
  o[0] = fmaf(n.w, fmaf(f.w, bg0, f.x), n.x);
  o[HW] = fmaf(n.w, fmaf(f.w, bg1, f.y), n.y);
  o[2 * HW] = fmaf(n.w, fmaf(f.w, bg2, f.z), n.z);
}

// Bilinear x2 upsampling of the half-resolution image into periphery tiles: one thread
// per output pixel, grid (row chunks of 256 pixels, rows, views), so no index division.
// Bilinear periphery upsampling (clamp to edge, half-pixel aligned): one thread per 2x2
// quad of output pixels (2i .. 2i + 1, 2j .. 2j + 1), whose taps all lie in the 3x3
// half-resolution neighbourhood of (i, j), loaded once for the four pixels.  Key tiles
// have an even side, so a quad lies in one tile and takes one class lookup.  Each pixel
// keeps the plain per-pixel formula.  Foveated frames have even sizes (the boundary
// rejects others), so every quad is whole; the guards keep the kernel in bounds for any
// size all the same.
__global__ void __launch_bounds__(256) composite_kernel(const ViewParams* __restrict__ views,
                                                        const uint8_t* __restrict__ tile_class, int tiles_per_view,
                                                        int T, const float* __restrict__ low, float* __restrict__ out,
                                                        int W, int H) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
  const int view = blockIdx.z;
  const int x = 2 * i, y = 2 * j;
  if (x >= W || y >= H) return;
  const ViewParams& vp = views[view];
  if (tile_class[(long long)view * tiles_per_view + (y / T) * vp.ntx + x / T] != kClassPeriphery) return;
  const long long HW = (long long)W * H;
  const int W2 = W / 2, H2 = H / 2;
  const long long HW2 = (long long)W2 * H2;
  // the tap columns and rows of the quad: i - 1, i, i + 1 (clamped)
  const int cx[3] = {min(max(i - 1, 0), W2 - 1), min(max(i, 0), W2 - 1), min(max(i + 1, 0), W2 - 1)};
  const int cy[3] = {min(max(j - 1, 0), H2 - 1), min(max(j, 0), H2 - 1), min(max(j + 1, 0), H2 - 1)};
  const float* L = low + (long long)view * 3 * HW2;
  float* o = out + (long long)view * 3 * HW + (long long)y * W + x;
  // float2 stores where both pixels exist and every plane's pair is 8-byte aligned (even
  // width, an 8-byte aligned pair in the first plane)
  const bool x1ok = x + 1 < W, y1ok = y + 1 < H;
  const bool pair = x1ok && (W & 1) == 0 && (reinterpret_cast<uintptr_t>(o) & 7u) == 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float* Lc = L + c * HW2;
    float v[3][3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int q = 0; q < 3; ++q) v[r][q] = Lc[(long long)cy[r] * W2 + cx[q]];
    float res[2][2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        // pixel (x + dx, y + dy): u = (p + 0.5) / 2 - 0.5 has floor i - 1 + dx and fraction 0.75 or 0.25
        const float ux = (x + dx + 0.5f) * 0.5f - 0.5f, uy = (y + dy + 0.5f) * 0.5f - 0.5f;
        const float fx = ux - floorf(ux), fy = uy - floorf(uy);
        const float top = (1.f - fx) * v[dy][dx] + fx * v[dy][dx + 1];
        const float bot = (1.f - fx) * v[dy + 1][dx] + fx * v[dy + 1][dx + 1];
        res[dy][dx] = (1.f - fy) * top + fy * bot;
      }
    float* oc = o + c * HW;
    if (pair) {
      *reinterpret_cast<float2*>(oc) = make_float2(res[0][0], res[0][1]);
      if (y1ok) *reinterpret_cast<float2*>(oc + W) = make_float2(res[1][0], res[1][1]);
    } else {
      oc[0] = res[0][0];
      if (x1ok) oc[1] = res[0][1];
      if (y1ok) {
        oc[W] = res[1][0];
        if (x1ok) oc[W + 1] = res[1][1];
      }
    }
  }
}

template <int MODE, bool STATS, bool BWD>
void launch_render_t(const RenderArgs& a, long long max_items, cudaStream_t st) {
  const int K1 = MODE == 2 ? a.k1 : 0, K2 = MODE == 2 ? a.k2 : 0, K3 = MODE == 0 ? 0 : a.k3;
  const size_t smem = render_smem_bytes(K1, K2, K3);
  // attribute and occupancy per device and per shared-memory size (set outside stream
  // capture by the first eager call)
  static std::atomic<int> smem_set[kMemoDevices];
  static std::atomic<int> occupancy[kMaxWin * 3 + 1][kMemoDevices];
  const int key = (int)std::min<size_t>(smem / 4096, (size_t)kMaxWin * 3);
  ensure_dynamic_smem(smem_set, render_kernel<MODE, STATS, BWD>, (int)smem);
  int per_sm = per_device_memo(occupancy[key], [smem] {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, render_kernel<MODE, STATS, BWD>, kBlock, smem);
    return b > 0 ? b : 1;
  });
  if (a.max_ctas_per_sm > 0) per_sm = std::min(per_sm, a.max_ctas_per_sm);
  const long long grid = std::min<long long>(max_items, (long long)device_sm_count() * per_sm);
  if (grid <= 0) return;
  render_kernel<MODE, STATS, BWD><<<(unsigned)grid, kBlock, smem, st>>>(a);
}

}  // namespace

void launch_workitems(const ViewParams* d_views, int n_views, int fovea_mode, int T, int tiles_per_view,
                      const uint8_t* tvis, WorkItem* items, uint32_t* n_items, uint8_t* tile_class, cudaStream_t st) {
  const long long n = (long long)n_views * tiles_per_view;
  if (n <= 0) return;
  workitems_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d_views, n_views, fovea_mode, T, tiles_per_view,
                                                               tvis, items, n_items, tile_class);
}

// One block per (view, key tile); invisible tiles get the background in every output
// pixel and, when the half-resolution image exists, in every 2x2-group sample.
__global__ void __launch_bounds__(256) invisible_fill_kernel(const ViewParams* __restrict__ views, int T,
                                                             int tiles_per_view, const uint8_t* __restrict__ tvis,
                                                             float b0, float b1, float b2, float* __restrict__ out,
                                                             float* __restrict__ low, int W, int H) {
  if (tvis[blockIdx.x]) return;
  const int view = blockIdx.x / tiles_per_view, t = blockIdx.x % tiles_per_view;
  const ViewParams& vp = views[view];
  if (t >= vp.ntx * vp.nty) return;
  const int tx = t % vp.ntx, ty = t / vp.ntx;
  const long long HW = (long long)W * H;
  float* o = out + (long long)view * 3 * HW;
  for (int p = threadIdx.x; p < T * T; p += blockDim.x) {
    const int x = tx * T + p % T, y = ty * T + p / T;
    if (x >= W || y >= H) continue;
    const long long q = (long long)y * W + x;
    o[q] = b0;
    o[HW + q] = b1;
    o[2 * HW + q] = b2;
  }
  if (!low) return;
  const int W2 = W / 2, H2 = H / 2, T2 = T / 2;
  const long long HW2 = (long long)W2 * H2;
  float* l = low + (long long)view * 3 * HW2;
  for (int p = threadIdx.x; p < T2 * T2; p += blockDim.x) {
    const int x = tx * T2 + p % T2, y = ty * T2 + p / T2;
    if (x >= W2 || y >= H2) continue;
    const long long q = (long long)y * W2 + x;
    l[q] = b0;
    l[HW2 + q] = b1;
    l[2 * HW2 + q] = b2;
  }
}

void launch_invisible_fill(const ViewParams* d_views, int n_views, int T, int tiles_per_view, const uint8_t* tvis,
                           const float bg[3], float* out, float* low, int W, int H, cudaStream_t st) {
  if (n_views <= 0 || !tvis) return;
  invisible_fill_kernel<<<(unsigned)(n_views * tiles_per_view), 256, 0, st>>>(d_views, T, tiles_per_view, tvis, bg[0],
                                                                              bg[1], bg[2], out, low, W, H);
}

void launch_render(const RenderArgs& a, long long max_items, cudaStream_t st) {
  const bool stats = a.stats != nullptr;
  if (stats ? launch_warp<false, true>(a, st) : launch_warp<false, false>(a, st)) return;
  switch (a.sort_mode * 2 + (stats ? 1 : 0)) {
    case 0: launch_render_t<0, false, false>(a, max_items, st); break;
    case 1: launch_render_t<0, true, false>(a, max_items, st); break;
    case 2: launch_render_t<1, false, false>(a, max_items, st); break;
    case 3: launch_render_t<1, true, false>(a, max_items, st); break;
    case 4: launch_render_t<2, false, false>(a, max_items, st); break;
    default: launch_render_t<2, true, false>(a, max_items, st); break;
  }
}

// replays the forward's per-ray decisions and emits record gradients at every blend
void launch_render_backward(const RenderArgs& a, long long max_items, cudaStream_t st) {
  if (launch_warp<true, false>(a, st)) return;
  switch (a.sort_mode) {
    case 0: launch_render_t<0, false, true>(a, max_items, st); break;
    case 1: launch_render_t<1, false, true>(a, max_items, st); break;
    default: launch_render_t<2, false, true>(a, max_items, st); break;
  }
}

void launch_lowmask(const TwoPassViews& tp, int n_views, int W, int H, uint8_t* mask, cudaStream_t st) {
  if (n_views <= 0 || W < 2 || H < 2) return;
  const dim3 grid((unsigned)((W / 2 + 255) / 256), (unsigned)std::min(H / 2, 65535), (unsigned)n_views);
  lowmask_kernel<<<grid, 256, 0, st>>>(tp, W, H, mask);
}

void launch_two_pass_composite(const TwoPassViews& tp, int n_views, int W, int H, int SW, int SH, const float* centre,
                               const float* low, float* out, cudaStream_t st) {
  if (n_views <= 0 || W <= 0 || H <= 0) return;
  const dim3 grid((unsigned)((W + 255) / 256), (unsigned)std::min(H, 65535), (unsigned)n_views);
  two_pass_composite_kernel<<<grid, 256, 0, st>>>(tp, W, H, SW, SH, centre, low, out);
}

void launch_reuse_composite(const float4* s_full, int W, int H, const float bg[3], float* out, cudaStream_t st) {
  const long long HW = (long long)W * H;
  reuse_composite_kernel<<<(unsigned)((2 * HW + 255) / 256), 256, 0, st>>>(s_full, HW, bg[0], bg[1], bg[2], out);
}

void launch_composite(const RenderArgs& a, int W, int H, cudaStream_t st) {
  if (W <= 0 || H <= 0 || a.n_views <= 0) return;
  const dim3 block(32, 8);  // 2x2 quads: 64 x 16 pixels per block
  const dim3 grid((unsigned)((W + 63) / 64), (unsigned)((H + 15) / 16), (unsigned)a.n_views);
  composite_kernel<<<grid, block, 0, st>>>(a.views, a.tile_class, a.tiles_per_view, a.key_tile, a.low, a.out, W, H);
}

}  // namespace vrs
