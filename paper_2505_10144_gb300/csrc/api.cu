// The C ABI (include/vrsplat.h): argument checking, workspace ownership and the order of
// the stages of one render: foveation map, Optimal-Projection preprocess, scan,
// duplicate, radix sort, tile ranges, single-launch render, composite.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "common.cuh"

using namespace vrs;

namespace vrs {
void launch_project_only(const SceneDev& s, const ViewParams* d_vp, int T, float* out, float* bbox, uint32_t* count,
                         cudaStream_t st);
size_t net_train_pack_bytes();
bool net_forward_train(const float* params, const float* x, int B, int H, int W, float* y, uint16_t* acts,
                       uint16_t* a12, uint16_t* wpack, uint32_t* status, cudaStream_t st);
bool net_backward_train(const float* params, const float* x, const uint16_t* acts, const float* dy, int B, int H,
                        int W, float* dparams, uint16_t* dz2, uint16_t* dz1, uint16_t* wpack, uint32_t* status,
                        cudaStream_t st);
void net_mse(const float* y, const float* t, long long n, float* loss, float* dy, double* scratch, cudaStream_t st);
void net_periphery(const float* params, const float* low, float* out, const uint8_t* tile_class,
                   const ViewParams* views, int n_views, int tiles_per_view, int W, int H, uint32_t* status,
                   cudaStream_t st);
vrs_status loss_l1_ssim_impl(const float* img, const float* tgt, int n, int H, int W, float* loss, float* grad,
                             void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t loss_scratch_bytes(int n, int H, int W);
void launch_lookback_timeout_test(uint32_t* zeroed_look, uint32_t* status, cudaStream_t st);
void launch_mbar_timeout_test(uint32_t* status, cudaStream_t st);
void launch_reuse_composite(const float4* s_full, int W, int H, const float bg[3], float* out, cudaStream_t st);
void launch_probe_orders(const ViewParams* views, int n_views, const float4* rec, const uint32_t* vals,
                         const uint32_t* ranges, int key_tile, int tiles_per_view, int list_order,
                         const float* probes, int n, int max_len, int* ids, float* depth, int* len,
                         cudaStream_t st);
}  // namespace vrs

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Saved {
  bool valid = false;
  int n_views = 0, W = 0, H = 0, key_tile = 0, fovea_mode = 0, sort_mode = 0, tiles_per_view = 0;
  int k[3] = {0, 0, 0};
  bool has_mask = false;
  long long total_nv = 0;
  int sorted_buf = 0;
};

}  // namespace

struct vrs_ctx {
  std::string err;
  DevBuf views, view_list, rec, bbox, count, offsets, partials, keys[2], vals[2], sort_scratch, ranges, tile_class,
      items, counters, low, s_full, s_low, stats, grad_rec, dsamp_full, dsamp_low, loss_scratch, misc, net_tmp,
      tvis, sat, tp_centre, tp_low, tp_mask, kcache;
  ViewParams* h_views = nullptr;  // pinned staging
  int* h_view_list = nullptr;
  uint32_t* h_small = nullptr;    // pinned: [0] total instances, [1] status, [2] items
  int staging_cap = 0;
  cudaEvent_t staging_done = nullptr;
  long long key_cap = 0;
  long long max_needed = 0;
  long long last_instances = 0;
  int last_passes = 0;
  int last_launches = 0;
  int max_ctas_per_sm = 0;
  // stereo reuse of distant content: while set, the next plan assigns views 0 and 1 the
  // near layer [0, layer_d) and view 2 the far layer [layer_d, inf) around layer_ref
  bool layer_on = false;
  float layer_ref[3] = {0.f, 0.f, 0.f};
  float layer_d = 0.f;
  DevBuf reuse_out;
  Saved saved;
  // stage profiling: 8 events per recorded call
  std::vector<cudaEvent_t> prof_ev;
  int prof_cap = 0, prof_used = 0;
  bool prof_on = false;
};

namespace {

// record the stage boundary `k` (0..7) of the current profiled call, if any
void prof_mark(vrs_ctx* c, int k, cudaStream_t st) {
  if (!c->prof_on || c->prof_used >= c->prof_cap) return;
  cudaEventRecord(c->prof_ev[(size_t)c->prof_used * 8 + k], st);
}

enum { kCtrNItems = 0, kCtrQueue = 1, kCtrTotal = 2, kCtrStatus = 3, kCtrSortN = 4, kCtrCount = 8 };

vrs_status fail(vrs_ctx* c, vrs_status s, const char* msg) {
  if (c) c->err = msg;
  return s;
}

vrs_status cuda_fail(vrs_ctx* c, cudaError_t e, const char* where) {
  if (c) c->err = std::string(where) + ": " + cudaGetErrorString(e);
  return VRS_ERR_CUDA;
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs != cudaStreamCaptureStatusNone;
}

// grow a device buffer (never during capture); returns false on failure
bool ensure(vrs_ctx* c, DevBuf& b, size_t bytes, bool cap_mode, vrs_status* st) {
  if (bytes <= b.bytes) return true;
  if (cap_mode) {
    *st = fail(c, VRS_ERR_CAPACITY, "workspace too small during stream capture; call vrs_reserve first");
    return false;
  }
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  size_t want = bytes + bytes / 8 + 256;
  cudaError_t e = cudaMalloc(&b.p, want);
  if (e != cudaSuccess) {
    *st = cuda_fail(c, e, "cudaMalloc");
    return false;
  }
  b.bytes = want;
  return true;
}

template <class T>
T* P(DevBuf& b) {
  return reinterpret_cast<T*>(b.p);
}

__global__ void clamp_n_kernel(const uint32_t* total, uint32_t* n, long long cap, uint32_t* status) {
  uint32_t t = *total;
  if ((long long)t > cap) {
    atomicOr(status, kStOverflow);
    t = (uint32_t)cap;
  }
  *n = t;
}

__global__ void set_u32_kernel(uint32_t* p, uint32_t v) { *p = v; }

int bits_for(long long n) {
  int b = 0;
  while ((1ll << b) < n) ++b;
  return b;
}

vrs_status check_scene(vrs_ctx* c, const vrs_gaussians& s) {
  // Gaussian indices travel in 28-bit fields of the render's window keys
  if (s.n < 0 || s.n > (1ll << 28) - 1) return fail(c, VRS_ERR_INVALID, "scene size out of range");
  if (s.sh_degree < 0 || s.sh_degree > 3) return fail(c, VRS_ERR_INVALID, "sh_degree must be 0..3");
  if (s.n > 0 && (!s.mean || !s.log_scale || !s.quat || !s.opacity_logit || !s.sh))
    return fail(c, VRS_ERR_INVALID, "null scene pointer");
  return VRS_OK;
}

SceneDev to_dev(const vrs_gaussians& s) {
  SceneDev d;
  d.mean = s.mean;
  d.ls = s.log_scale;
  d.quat = s.quat;
  d.logit = s.opacity_logit;
  d.sh = s.sh;
  d.n = s.n;
  d.deg = s.sh_degree;
  return d;
}

bool finite_cam(const vrs_camera& c) {
  for (int i = 0; i < 12; ++i)
    if (!std::isfinite(c.world_to_cam[i])) return false;
  return std::isfinite(c.fx) && std::isfinite(c.fy) && std::isfinite(c.cx) && std::isfinite(c.cy) &&
         std::isfinite(c.near_z) && c.fx > 0 && c.fy > 0 && c.near_z > 0;
}

void fill_view(ViewParams& vp, const vrs_camera& c, const vrs_fovea* f, int T) {
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) vp.R[3 * r + k] = c.world_to_cam[4 * r + k];
    vp.t[r] = c.world_to_cam[4 * r + 3];
  }
  vp.fx = c.fx;
  vp.fy = c.fy;
  vp.cx = c.cx;
  vp.cy = c.cy;
  vp.near_z = c.near_z;
  vp.W = c.width;
  vp.H = c.height;
  vp.ntx = (c.width + T - 1) / T;
  vp.nty = (c.height + T - 1) / T;
  vp.gaze_x = f ? f->gaze_x : 0.f;
  vp.gaze_y = f ? f->gaze_y : 0.f;
  vp.radius = f ? f->radius_px : 0.f;
  vp.band = f ? f->band_px : 1.f;
  vp.visible = f ? f->visible : nullptr;
  vp.dist_ref[0] = vp.dist_ref[1] = vp.dist_ref[2] = 0.f;
  vp.dist_min = 0.f;
  vp.dist_max = INFINITY;
}

bool any_mask(const vrs_fovea* fov, int n_views) {
  if (!fov) return false;
  for (int v = 0; v < n_views; ++v)
    if (fov[v].visible) return true;
  return false;
}

vrs_status stage_views(vrs_ctx* c, int n_views, cudaStream_t st, bool cap_mode) {
  vrs_status s = VRS_OK;
  if (!ensure(c, c->views, sizeof(ViewParams) * n_views, cap_mode, &s)) return s;
  if (!ensure(c, c->view_list, sizeof(int) * n_views, cap_mode, &s)) return s;
  cudaError_t e = cudaMemcpyAsync(c->views.p, c->h_views, sizeof(ViewParams) * n_views, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->view_list.p, c->h_view_list, sizeof(int) * n_views, cudaMemcpyHostToDevice, st);
  // in a captured graph the copy reads the staging at every replay; the external record
  // lets vrs_update_views wait for the last replay's copy before it rewrites the staging
  if (e == cudaSuccess)
    e = cap_mode ? cudaEventRecordWithFlags(c->staging_done, st, cudaEventRecordExternal)
                 : cudaEventRecord(c->staging_done, st);
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "staging copy");
}

vrs_status reserve_staging(vrs_ctx* c, int n_views, bool cap_mode = false) {
  if (c->staging_done && !cap_mode) cudaEventSynchronize(c->staging_done);
  if (n_views <= c->staging_cap) return VRS_OK;
  if (cap_mode) return fail(c, VRS_ERR_CAPACITY, "view staging too small during stream capture");
  if (c->h_views) cudaFreeHost(c->h_views);
  if (c->h_view_list) cudaFreeHost(c->h_view_list);
  c->h_views = nullptr;
  c->h_view_list = nullptr;
  int cap = std::max(n_views, 64);
  cudaError_t e = cudaMallocHost(&c->h_views, sizeof(ViewParams) * cap);
  if (e == cudaSuccess) e = cudaMallocHost(&c->h_view_list, sizeof(int) * cap);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaMallocHost");
  c->staging_cap = cap;
  return VRS_OK;
}

struct Plan {
  int n_views, W, H, T, tiles_per_view, fovea_mode;
  int key_mode = 0;  // 3, 4: global orders
  bool has_mask = false;
  long long total_nv;
  std::vector<long long> view_n;
  std::vector<int> scene_first, scene_count;  // into the view list grouped by scene
};

vrs_status plan_render(vrs_ctx* c, const vrs_gaussians* scenes, int n_scenes, const int* view_scene,
                       const vrs_camera* cams, const vrs_fovea* fov, int n_views, const vrs_render_opts* o,
                       Plan& pl, bool cap_mode = false) {
  if (!scenes || n_scenes <= 0 || !view_scene || !cams || n_views <= 0 || !o)
    return fail(c, VRS_ERR_INVALID, "null or empty argument");
  for (int s = 0; s < n_scenes; ++s) {
    vrs_status st = check_scene(c, scenes[s]);
    if (st) return st;
  }
  if (o->sort_mode < 0 || o->sort_mode > 4) return fail(c, VRS_ERR_INVALID, "sort_mode must be 0 .. 4");
  if ((o->sort_mode == 1 || o->sort_mode == 2) && (o->win[2] < 1 || o->win[2] > kMaxWin))
    return fail(c, VRS_ERR_INVALID, "per-sample window must be 1..32");
  if (o->sort_mode == 2 && (o->win[0] < 0 || o->win[0] > kMaxWin || o->win[1] < 0 || o->win[1] > kMaxWin))
    return fail(c, VRS_ERR_INVALID, "block windows must be 0..32");
  const int W = cams[0].width, H = cams[0].height;
  if (W <= 0 || H <= 0 || (long long)W * H > (1ll << 31)) return fail(c, VRS_ERR_INVALID, "bad image size");
  const int fm = fov ? fov[0].mode : 0;
  if (fm < 0 || fm > 2) return fail(c, VRS_ERR_INVALID, "fovea mode must be 0, 1 or 2");
  int T = o->key_tile;
  if (T != 16 && T != 32) return fail(c, VRS_ERR_INVALID, "key_tile must be 16 or 32");
  if (fm != 0) {
    // the fovea classes are per key tile: 32x32 (Sec. 4.3), or 16x16 with the bilinear
    // periphery (a tuning option); the network's fused kernel works on 32x32 tiles
    if (fm == 2 && T != 32) return fail(c, VRS_ERR_INVALID, "the network periphery uses 32x32 key tiles");
    if ((W & 1) || (H & 1)) return fail(c, VRS_ERR_INVALID, "foveated rendering needs even width and height");
  }
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width != W || cams[v].height != H) return fail(c, VRS_ERR_INVALID, "views must share the image size");
    if (!finite_cam(cams[v])) return fail(c, VRS_ERR_INVALID, "non-finite or non-positive camera values");
    if (view_scene[v] < 0 || view_scene[v] >= n_scenes) return fail(c, VRS_ERR_INVALID, "view_scene out of range");
    if (fov) {
      if (fov[v].mode != fm) return fail(c, VRS_ERR_INVALID, "views must share the fovea mode");
      if (fm != 0 && !(std::isfinite(fov[v].gaze_x) && std::isfinite(fov[v].gaze_y) && fov[v].radius_px >= 0 &&
                       fov[v].band_px > 0))
        return fail(c, VRS_ERR_INVALID, "bad fovea parameters");
    }
  }
  pl.n_views = n_views;
  pl.W = W;
  pl.H = H;
  pl.T = T;
  pl.fovea_mode = fm;
  pl.key_mode = o->sort_mode >= 3 ? o->sort_mode : 0;
  pl.has_mask = any_mask(fov, n_views);
  pl.tiles_per_view = ((W + T - 1) / T) * ((H + T - 1) / T);
  if ((long long)pl.tiles_per_view * n_views >= (1ll << 31)) return fail(c, VRS_ERR_INVALID, "too many tiles");
  vrs_status st = reserve_staging(c, n_views, cap_mode);
  if (st) return st;
  pl.view_n.resize(n_views);
  long long base = 0;
  for (int v = 0; v < n_views; ++v) {
    ViewParams& vp = c->h_views[v];
    fill_view(vp, cams[v], fov ? &fov[v] : nullptr, T);
    if (c->layer_on) {
      for (int k = 0; k < 3; ++k) vp.dist_ref[k] = c->layer_ref[k];
      vp.dist_min = v < 2 ? 0.f : c->layer_d;
      vp.dist_max = v < 2 ? c->layer_d : INFINITY;
    }
    vp.scene = view_scene[v];
    vp.base = base;
    pl.view_n[v] = scenes[view_scene[v]].n;
    base += pl.view_n[v];
  }
  pl.total_nv = base;
  if (base >= (1ll << 32)) return fail(c, VRS_ERR_INVALID, "too many (view, Gaussian) pairs");
  pl.scene_first.assign(n_scenes, 0);
  pl.scene_count.assign(n_scenes, 0);
  int k = 0;
  for (int s = 0; s < n_scenes; ++s) {
    pl.scene_first[s] = k;
    for (int v = 0; v < n_views; ++v)
      if (view_scene[v] == s) c->h_view_list[k++] = v;
    pl.scene_count[s] = k - pl.scene_first[s];
  }
  return VRS_OK;
}

// everything up to (and including) the sorted, ranged instance list
vrs_status build_instances(vrs_ctx* c, const vrs_gaussians* scenes, int n_scenes, const Plan& pl, cudaStream_t st,
                           bool cap_mode) {
  vrs_status s = VRS_OK;
  const long long NV = std::max(pl.total_nv, 1ll);
  const long long VT = (long long)pl.n_views * pl.tiles_per_view;
  if (!ensure(c, c->rec, sizeof(float4) * kRecF4 * NV, cap_mode, &s) ||
      !ensure(c, c->bbox, sizeof(float4) * NV, cap_mode, &s) || !ensure(c, c->count, sizeof(uint32_t) * NV, cap_mode, &s) ||
      !ensure(c, c->kcache, sizeof(unsigned long long) * kKeyCacheSlots * NV, cap_mode, &s) ||
      !ensure(c, c->offsets, sizeof(uint32_t) * NV, cap_mode, &s) ||
      !ensure(c, c->partials, scan_partials_bytes(NV), cap_mode, &s) ||
      !ensure(c, c->ranges, sizeof(uint32_t) * 2 * VT, cap_mode, &s) ||
      !ensure(c, c->tile_class, VT, cap_mode, &s) || !ensure(c, c->items, sizeof(WorkItem) * 4 * VT, cap_mode, &s) ||
      !ensure(c, c->counters, sizeof(uint32_t) * kCtrCount, cap_mode, &s))
    return s;
  Visibility vis{nullptr, nullptr, pl.tiles_per_view, 0};
  const int ntx = (pl.W + pl.T - 1) / pl.T, nty = (pl.H + pl.T - 1) / pl.T;
  if (pl.has_mask) {
    vis.sat_per_view = (ntx + 1) * (nty + 1);
    if (!ensure(c, c->tvis, VT, cap_mode, &s) ||
        !ensure(c, c->sat, sizeof(uint32_t) * (size_t)vis.sat_per_view * pl.n_views, cap_mode, &s))
      return s;
    vis.tvis = P<uint8_t>(c->tvis);
    vis.sat = P<uint32_t>(c->sat);
  }
  if ((s = stage_views(c, pl.n_views, st, cap_mode))) return s;
  uint32_t* ctr = P<uint32_t>(c->counters);
  cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * kCtrStatus, st);  // n_items, queue, total (status is sticky)
  cudaMemsetAsync(c->ranges.p, 0, sizeof(uint32_t) * 2 * VT, st);
  prof_mark(c, 0, st);
  int launches = 0;
  if (pl.has_mask) {
    launch_visibility(P<ViewParams>(c->views), pl.n_views, pl.T, ntx, nty, vis, st);
    launches += 2;
  }
  for (int sc = 0; sc < n_scenes; ++sc) {
    if (!pl.scene_count[sc]) continue;
    ++launches;
    launch_preprocess(to_dev(scenes[sc]), P<ViewParams>(c->views), P<int>(c->view_list) + pl.scene_first[sc],
                      pl.scene_count[sc], pl.T, pl.key_mode, vis, P<float4>(c->rec), P<float4>(c->bbox), P<uint32_t>(c->count),
                      P<unsigned long long>(c->kcache), st);
  }
  prof_mark(c, 1, st);
  launch_scan_u32(P<uint32_t>(c->count), P<uint32_t>(c->offsets), pl.total_nv, ctr + kCtrTotal,
                  P<uint32_t>(c->partials), st);
  launches += pl.total_nv > 0 ? 3 : 0;
  long long need = c->key_cap;
  if (!cap_mode) {
    cudaMemcpyAsync(c->h_small, ctr + kCtrTotal, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(c, e, "instance count");
    need = c->h_small[0];
    c->last_instances = need;
    c->max_needed = std::max(c->max_needed, need);
    if (need > c->key_cap || c->key_cap == 0) {
      const long long cap = std::min(need + need / 4 + 4096, kMaxInstances);
      if (need > kMaxInstances) return fail(c, VRS_ERR_CAPACITY, "more than 2^31 - 1 instances");
      for (int b = 0; b < 2; ++b)
        if (!ensure(c, c->keys[b], sizeof(uint64_t) * cap, false, &s) || !ensure(c, c->vals[b], sizeof(uint32_t) * cap, false, &s))
          return s;
      if (!ensure(c, c->sort_scratch, sort_scratch_bytes(cap), false, &s)) return s;
      c->key_cap = cap;
    }
  }
  if (c->key_cap <= 0) return fail(c, VRS_ERR_CAPACITY, "no instance capacity reserved");
  prof_mark(c, 2, st);
  for (int v = 0; v < pl.n_views; ++v)
    if (pl.view_n[v] > 0) {
      ++launches;  // one duplicate_kernel launch for every view
      break;
    }
  launch_duplicate(P<ViewParams>(c->views), pl.n_views, P<float4>(c->rec), P<float4>(c->bbox), P<uint32_t>(c->count),
                   P<uint32_t>(c->offsets), pl.view_n.data(), pl.T, pl.tiles_per_view, vis,
                   P<unsigned long long>(c->kcache), pl.key_mode, P<uint64_t>(c->keys[0]),
                   P<uint32_t>(c->vals[0]), ctr + kCtrTotal, c->key_cap, ctr + kCtrStatus, st);
  clamp_n_kernel<<<1, 1, 0, st>>>(ctr + kCtrTotal, ctr + kCtrSortN, c->key_cap, ctr + kCtrStatus);
  prof_mark(c, 3, st);
  SortScratch ss;
  sort_scratch_carve(c->sort_scratch.p, c->key_cap, &ss);
  uint64_t* kb[2] = {P<uint64_t>(c->keys[0]), P<uint64_t>(c->keys[1])};
  uint32_t* vb[2] = {P<uint32_t>(c->vals[0]), P<uint32_t>(c->vals[1])};
  const int bits = 32 + std::max(1, bits_for(VT));
  c->last_passes = (bits + 7) / 8;
  const long long sort_n = cap_mode ? c->key_cap : std::max(need, 1ll);
  const int cur = launch_radix_sort(kb, vb, ctr + kCtrSortN, sort_n, bits, ss, ctr + kCtrStatus, st);
  c->saved.sorted_buf = cur;
  launches += 1 + 1 + c->last_passes;  // clamp_n_kernel, histogram_kernel, one onesweep pass per digit
  prof_mark(c, 4, st);
  launch_ranges(kb[cur], ctr + kCtrSortN, sort_n, P<uint32_t>(c->ranges), VT, st);
  launch_workitems(P<ViewParams>(c->views), pl.n_views, pl.fovea_mode, pl.T, pl.tiles_per_view, vis.tvis,
                   P<WorkItem>(c->items), ctr + kCtrNItems, P<uint8_t>(c->tile_class), st);
  c->last_launches = launches + 2;
  return VRS_OK;
}

RenderArgs make_args(vrs_ctx* c, const Plan& pl, const vrs_render_opts* o) {
  RenderArgs a;
  memset(&a, 0, sizeof a);
  uint32_t* ctr = P<uint32_t>(c->counters);
  a.views = P<ViewParams>(c->views);
  a.n_views = pl.n_views;
  a.rec = P<float4>(c->rec);
  a.bbox = P<float4>(c->bbox);
  a.vals = P<uint32_t>(c->vals[c->saved.sorted_buf]);
  a.ranges = P<uint32_t>(c->ranges);
  a.items = P<WorkItem>(c->items);
  a.n_items = ctr + kCtrNItems;
  a.queue = ctr + kCtrQueue;
  a.tile_class = P<uint8_t>(c->tile_class);
  a.fovea_mode = pl.fovea_mode;
  a.key_tile = pl.T;
  a.tiles_per_view = pl.tiles_per_view;
  a.sort_mode = o->sort_mode;
  a.k1 = o->win[0];
  a.k2 = o->win[1];
  a.k3 = o->sort_mode >= 3 ? 0 : o->win[2];
  a.stream_order = o->sort_mode >= 3 ? 1 : 0;
  for (int k = 0; k < 3; ++k) a.bg[k] = o->bg[k];
  a.status = ctr + kCtrStatus;
  return a;
}

}  // namespace

extern "C" {

vrs_status vrs_create(vrs_ctx** ctx, size_t workspace_bytes_hint) {
  if (!ctx) return VRS_ERR_INVALID;
  *ctx = nullptr;
  vrs_ctx* c = new (std::nothrow) vrs_ctx();
  if (!c) return VRS_ERR_CUDA;
  cudaError_t e = cudaMallocHost(&c->h_small, 16 * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->staging_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    delete c;
    return VRS_ERR_CUDA;
  }
  memset(c->h_small, 0, 16 * sizeof(uint32_t));
  vrs_status s = VRS_OK;
  if (!ensure(c, c->counters, sizeof(uint32_t) * kCtrCount, false, &s)) {
    delete c;
    return s;
  }
  cudaMemset(c->counters.p, 0, sizeof(uint32_t) * kCtrCount);
  if (workspace_bytes_hint > 0) {
    const long long cap = (long long)(workspace_bytes_hint / 24);
    for (int b = 0; b < 2; ++b)
      if (!ensure(c, c->keys[b], sizeof(uint64_t) * cap, false, &s) || !ensure(c, c->vals[b], sizeof(uint32_t) * cap, false, &s)) {
        vrs_destroy(c);
        return s;
      }
    if (!ensure(c, c->sort_scratch, sort_scratch_bytes(cap), false, &s)) {
      vrs_destroy(c);
      return s;
    }
    c->key_cap = cap;
  }
  *ctx = c;
  return VRS_OK;
}

vrs_status vrs_destroy(vrs_ctx* c) {
  if (!c) return VRS_ERR_INVALID;
  DevBuf* all[] = {&c->views, &c->view_list, &c->rec, &c->bbox, &c->count, &c->offsets, &c->partials, &c->keys[0],
                   &c->keys[1], &c->vals[0], &c->vals[1], &c->sort_scratch, &c->ranges, &c->tile_class, &c->items,
                   &c->counters, &c->low, &c->s_full, &c->s_low, &c->stats, &c->grad_rec, &c->dsamp_full,
                   &c->dsamp_low, &c->loss_scratch, &c->misc, &c->net_tmp, &c->tvis, &c->sat, &c->tp_centre,
                   &c->tp_low, &c->tp_mask, &c->kcache};
  for (DevBuf* b : all)
    if (b->p) cudaFree(b->p);
  if (c->h_views) cudaFreeHost(c->h_views);
  if (c->h_view_list) cudaFreeHost(c->h_view_list);
  if (c->h_small) cudaFreeHost(c->h_small);
  if (c->staging_done) cudaEventDestroy(c->staging_done);
  for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
  delete c;
  return VRS_OK;
}

vrs_status vrs_reserve(vrs_ctx* c, int n_views, int width, int height, int64_t total_gaussians, int64_t max_instances) {
  if (!c || n_views <= 0 || width <= 0 || height <= 0 || total_gaussians < 0 || max_instances <= 0 ||
      max_instances > kMaxInstances)
    return fail(c, VRS_ERR_INVALID, "bad reserve arguments");
  vrs_status s = VRS_OK;
  const long long VT = (long long)n_views * ((width + 15) / 16) * ((height + 15) / 16);
  const long long NV = std::max<long long>(total_gaussians, 1);
  if (reserve_staging(c, n_views)) return VRS_ERR_CUDA;
  if (!ensure(c, c->views, sizeof(ViewParams) * n_views, false, &s) || !ensure(c, c->view_list, sizeof(int) * n_views, false, &s) ||
      !ensure(c, c->rec, sizeof(float4) * kRecF4 * NV, false, &s) || !ensure(c, c->bbox, sizeof(float4) * NV, false, &s) ||
      !ensure(c, c->count, sizeof(uint32_t) * NV, false, &s) || !ensure(c, c->offsets, sizeof(uint32_t) * NV, false, &s) ||
      !ensure(c, c->kcache, sizeof(unsigned long long) * kKeyCacheSlots * NV, false, &s) ||
      !ensure(c, c->partials, scan_partials_bytes(NV), false, &s) ||
      !ensure(c, c->ranges, sizeof(uint32_t) * 2 * VT, false, &s) || !ensure(c, c->tile_class, VT, false, &s) ||
      !ensure(c, c->items, sizeof(WorkItem) * 4 * VT, false, &s) ||
      !ensure(c, c->low, sizeof(float) * 3 * (size_t)n_views * (width / 2) * (height / 2) + 16, false, &s) ||
      !ensure(c, c->tvis, VT, false, &s) ||
      !ensure(c, c->sat, sizeof(uint32_t) * (size_t)n_views * ((width + 15) / 16 + 1) * ((height + 15) / 16 + 1),
              false, &s))
    return s;
  for (int b = 0; b < 2; ++b)
    if (!ensure(c, c->keys[b], sizeof(uint64_t) * max_instances, false, &s) ||
        !ensure(c, c->vals[b], sizeof(uint32_t) * max_instances, false, &s))
      return s;
  if (!ensure(c, c->sort_scratch, sort_scratch_bytes(max_instances), false, &s)) return s;
  c->key_cap = std::max<long long>(c->key_cap, max_instances);
  return VRS_OK;
}

vrs_status vrs_render(vrs_ctx* c, const vrs_gaussians* scenes, int n_scenes, const int* view_scene,
                      const vrs_camera* cams, const vrs_fovea* fov, int n_views, const vrs_render_opts* o,
                      float* d_out_rgb, float* d_low_rgb, int save_for_backward, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_out_rgb) return fail(c, VRS_ERR_INVALID, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  const bool cap_mode = capturing(st);
  Plan pl;
  vrs_status s = plan_render(c, scenes, n_scenes, view_scene, cams, fov, n_views, o, pl, cap_mode);
  if (s) return s;
  if (pl.fovea_mode == 2 && !d_low_rgb) return fail(c, VRS_ERR_INVALID, "fovea mode 2 needs d_low_rgb");
  if ((s = build_instances(c, scenes, n_scenes, pl, st, cap_mode))) return s;
  RenderArgs a = make_args(c, pl, o);
  a.max_ctas_per_sm = c->max_ctas_per_sm;
  a.out = d_out_rgb;
  const size_t low_bytes = sizeof(float) * 3 * (size_t)n_views * (pl.W / 2) * (pl.H / 2);
  if (pl.fovea_mode != 0) {
    if (d_low_rgb) {
      a.low = d_low_rgb;
    } else {
      if (!ensure(c, c->low, low_bytes + 16, cap_mode, &s)) return s;
      a.low = P<float>(c->low);
    }
  } else {
    a.low = d_low_rgb;
  }
  const long long HW = (long long)pl.W * pl.H;
  if (save_for_backward) {
    if (!ensure(c, c->s_full, sizeof(float4) * HW * n_views, cap_mode, &s)) return s;
    a.s_full = P<float4>(c->s_full);
    if (pl.fovea_mode != 0) {
      if (!ensure(c, c->s_low, sizeof(float4) * (HW / 4 + 1) * n_views, cap_mode, &s)) return s;
      a.s_low = P<float4>(c->s_low);
    }
  }
  if (o->stats) {
    if (!ensure(c, c->stats, sizeof(unsigned long long) * 4, cap_mode, &s)) return s;
    cudaMemsetAsync(c->stats.p, 0, sizeof(unsigned long long) * 4, st);
    a.stats = P<unsigned long long>(c->stats);
  }
  const long long max_items = 4ll * n_views * pl.tiles_per_view;
  if (pl.has_mask) {
    launch_invisible_fill(P<ViewParams>(c->views), n_views, pl.T, pl.tiles_per_view, P<uint8_t>(c->tvis), o->bg,
                          d_out_rgb, a.low, pl.W, pl.H, st);
    c->last_launches += 1;
  }
  prof_mark(c, 5, st);
  launch_render(a, max_items, st);
  prof_mark(c, 6, st);
  if (pl.fovea_mode == 1) launch_composite(a, pl.W, pl.H, st);
  prof_mark(c, 7, st);
  if (c->prof_on && c->prof_used < c->prof_cap) c->prof_used++;
  c->last_launches += 1 + (pl.fovea_mode == 1 ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(c, e, "render launch");
  Saved& sv = c->saved;
  sv.valid = save_for_backward != 0;
  sv.n_views = n_views;
  sv.W = pl.W;
  sv.H = pl.H;
  sv.key_tile = pl.T;
  sv.fovea_mode = pl.fovea_mode;
  sv.sort_mode = o->sort_mode;
  sv.tiles_per_view = pl.tiles_per_view;
  sv.total_nv = pl.total_nv;
  sv.has_mask = pl.has_mask;
  for (int k = 0; k < 3; ++k) sv.k[k] = o->win[k];
  return VRS_OK;
}

vrs_status vrs_render_stereo_reuse(vrs_ctx* c, const vrs_gaussians* scene, const vrs_camera* cams,
                                   const vrs_render_opts* o, float far_distance, float* d_out_rgb, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!scene || !cams || !o || !d_out_rgb) return fail(c, VRS_ERR_INVALID, "null argument");
  if (!(far_distance > 0.f) || !std::isfinite(far_distance)) return fail(c, VRS_ERR_INVALID, "bad far distance");
  if (o->sort_mode >= 3) return fail(c, VRS_ERR_INVALID, "stereo reuse takes the per-ray orders (sort modes 0 .. 2)");
  for (int e = 0; e < 2; ++e)
    if (!finite_cam(cams[e])) return fail(c, VRS_ERR_INVALID, "non-finite or non-positive camera values");
  if (cams[1].width != cams[0].width || cams[1].height != cams[0].height || cams[1].fx != cams[0].fx ||
      cams[1].fy != cams[0].fy || cams[1].cx != cams[0].cx || cams[1].cy != cams[0].cy)
    return fail(c, VRS_ERR_INVALID, "the eyes must share image size and intrinsics");
  // both eyes share one rotation; the cyclopean camera sits at the midpoint of the centres
  double ctr[2][3];
  for (int e = 0; e < 2; ++e)
    for (int k = 0; k < 3; ++k) {
      double v = 0;
      for (int r = 0; r < 3; ++r) v -= (double)cams[e].world_to_cam[4 * r + k] * cams[e].world_to_cam[4 * r + 3];
      ctr[e][k] = v;
    }
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k)
      if (std::fabs(cams[0].world_to_cam[4 * r + k] - cams[1].world_to_cam[4 * r + k]) > 1e-6f)
        return fail(c, VRS_ERR_INVALID, "the eyes must share the head rotation");
  vrs_camera cam3[3] = {cams[0], cams[1], cams[0]};
  for (int r = 0; r < 3; ++r) {
    double t = 0;
    for (int k = 0; k < 3; ++k) t -= (double)cams[0].world_to_cam[4 * r + k] * 0.5 * (ctr[0][k] + ctr[1][k]);
    cam3[2].world_to_cam[4 * r + 3] = (float)t;
  }
  vrs_render_opts o3 = *o;
  o3.bg[0] = o3.bg[1] = o3.bg[2] = 0.f;  // the layers keep (C, T); the background goes in at the end
  const int vs[3] = {0, 0, 0};
  const int W = cams[0].width, H = cams[0].height;
  cudaStream_t st = (cudaStream_t)stream;
  vrs_status s = VRS_OK;
  if (!ensure(c, c->reuse_out, sizeof(float) * 9 * (size_t)W * H, capturing(st), &s)) return s;
  c->layer_on = true;
  for (int k = 0; k < 3; ++k) c->layer_ref[k] = (float)(0.5 * (ctr[0][k] + ctr[1][k]));
  c->layer_d = far_distance;
  s = vrs_render(c, scene, 1, vs, cam3, nullptr, 3, &o3, P<float>(c->reuse_out), nullptr, 1, stream);
  c->layer_on = false;
  if (s) return s;
  c->saved.valid = false;  // the layered render has no backward
  launch_reuse_composite(P<float4>(c->s_full), W, H, o->bg, d_out_rgb, st);
  c->last_launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "reuse composite launch");
}

vrs_status vrs_render_two_pass(vrs_ctx* c, const vrs_gaussians* scenes, int n_scenes, const int* view_scene,
                               const vrs_camera* cams, const vrs_fovea* fov, int n_views, const vrs_render_opts* o,
                               float* d_out_rgb, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_out_rgb || !cams || !fov || !o || n_views <= 0) return fail(c, VRS_ERR_INVALID, "null or empty argument");
  if (n_views > kTwoPassMaxViews) return fail(c, VRS_ERR_INVALID, "two-pass rendering takes at most 64 views");
  const int W = cams[0].width, H = cams[0].height;
  if (W <= 0 || H <= 0 || (W & 1) || (H & 1)) return fail(c, VRS_ERR_INVALID, "two-pass rendering needs even sizes");
  int half = 0;
  for (int v = 0; v < n_views; ++v) {
    if (cams[v].width != W || cams[v].height != H) return fail(c, VRS_ERR_INVALID, "views must share the image size");
    if (fov[v].mode != 1 || !std::isfinite(fov[v].gaze_x) || !std::isfinite(fov[v].gaze_y) ||
        !(fov[v].radius_px >= 0) || !(fov[v].band_px > 0) || !std::isfinite(fov[v].radius_px + fov[v].band_px))
      return fail(c, VRS_ERR_INVALID, "two-pass rendering needs fovea mode 1 and valid fovea parameters");
    half = std::max(half, (int)std::ceil(fov[v].radius_px + fov[v].band_px) + 1);
  }
  // centre squares: the focus disc and band of every view (w = 0 outside), integer offsets
  const int SW = std::min(2 * half, W), SH = std::min(2 * half, H);
  TwoPassViews tp;
  memset(&tp, 0, sizeof tp);
  std::vector<vrs_camera> cc(cams, cams + n_views), lc(cams, cams + n_views);
  std::vector<vrs_fovea> lf(n_views);
  for (int v = 0; v < n_views; ++v) {
    tp.gaze_x[v] = fov[v].gaze_x;
    tp.gaze_y[v] = fov[v].gaze_y;
    tp.radius[v] = fov[v].radius_px;
    tp.band[v] = fov[v].band_px;
    tp.x0[v] = std::min(std::max((int)std::floor(fov[v].gaze_x) - half, 0), W - SW);
    tp.y0[v] = std::min(std::max((int)std::floor(fov[v].gaze_y) - half, 0), H - SH);
    cc[v].cx -= tp.x0[v];
    cc[v].cy -= tp.y0[v];
    cc[v].width = SW;
    cc[v].height = SH;
    lc[v].fx *= 0.5f;
    lc[v].fy *= 0.5f;
    lc[v].cx *= 0.5f;
    lc[v].cy *= 0.5f;
    lc[v].width = W / 2;
    lc[v].height = H / 2;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool cap_mode = capturing(st);
  // both passes stage their views through the same pinned buffer, which a replay of a
  // captured graph would read after the second pass rewrote it
  if (cap_mode) return fail(c, VRS_ERR_UNSUPPORTED, "two-pass rendering cannot be captured in a graph");
  vrs_status s = VRS_OK;
  const size_t HW2 = (size_t)(W / 2) * (H / 2);
  if (!ensure(c, c->tp_centre, sizeof(float) * 3 * (size_t)n_views * SW * SH, cap_mode, &s) ||
      !ensure(c, c->tp_low, sizeof(float) * 3 * (size_t)n_views * HW2, cap_mode, &s) ||
      !ensure(c, c->tp_mask, (size_t)n_views * HW2, cap_mode, &s))
    return s;
  for (int v = 0; v < n_views; ++v) {
    lf[v] = vrs_fovea{0.f, 0.f, 0.f, 1.f, 0, 16, P<uint8_t>(c->tp_mask) + (size_t)v * HW2};
  }
  vrs_render_opts po = *o;
  po.key_tile = 16;
  // pass 1: the centre squares at full resolution (a tight frustum: the cropped camera)
  if ((s = vrs_render(c, scenes, n_scenes, view_scene, cc.data(), nullptr, n_views, &po, P<float>(c->tp_centre),
                      nullptr, 0, stream)))
    return s;
  const int launches1 = c->last_launches;
  // pass 2: half resolution, only where some full-resolution pixel with w < 1 reads it
  launch_lowmask(tp, n_views, W, H, P<uint8_t>(c->tp_mask), st);
  if ((s = vrs_render(c, scenes, n_scenes, view_scene, lc.data(), lf.data(), n_views, &po, P<float>(c->tp_low),
                      nullptr, 0, stream)))
    return s;
  launch_two_pass_composite(tp, n_views, W, H, SW, SH, P<float>(c->tp_centre), P<float>(c->tp_low), d_out_rgb, st);
  c->last_launches += launches1 + 2;
  c->saved.valid = false;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "two-pass composite");
}

vrs_status vrs_render_backward(vrs_ctx* c, const vrs_gaussians* scenes, int n_scenes, const int* view_scene,
                               const vrs_camera* cams, const vrs_fovea* fov, int n_views, const vrs_render_opts* o,
                               const float* d_dL_drgb, const vrs_gaussian_grads* grads, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_dL_drgb || !grads) return fail(c, VRS_ERR_INVALID, "null gradient argument");
  cudaStream_t st = (cudaStream_t)stream;
  const bool cap_mode = capturing(st);
  Saved& sv = c->saved;
  if (!sv.valid) return fail(c, VRS_ERR_INVALID, "no forward saved: call vrs_render with save_for_backward = 1");
  if (!o || !scenes || !view_scene || n_scenes <= 0) return fail(c, VRS_ERR_INVALID, "null argument");
  for (int sc = 0; sc < n_scenes; ++sc) {
    if (scenes[sc].n > 0 && (!grads[sc].mean || !grads[sc].log_scale || !grads[sc].quat ||
                             !grads[sc].opacity_logit || !grads[sc].sh))
      return fail(c, VRS_ERR_INVALID, "null gradient pointer");
  }
  const int fm = fov ? fov[0].mode : 0;
  if (n_views != sv.n_views || !cams || cams[0].width != sv.W || cams[0].height != sv.H || o->key_tile != sv.key_tile ||
      fm != sv.fovea_mode || o->sort_mode != sv.sort_mode || o->win[0] != sv.k[0] || o->win[1] != sv.k[1] ||
      o->win[2] != sv.k[2])
    return fail(c, VRS_ERR_INVALID, "backward arguments differ from the saved forward");
  // per-scene view lists (host staging still holds this call's views from the forward)
  std::vector<int> first(n_scenes, 0), cnt(n_scenes, 0);
  long long total = 0;
  {
    int k = 0;
    for (int s2 = 0; s2 < n_scenes; ++s2) {
      first[s2] = k;
      for (int v = 0; v < n_views; ++v)
        if (view_scene[v] == s2) ++k;
      cnt[s2] = k - first[s2];
    }
    for (int v = 0; v < n_views; ++v) {
      if (view_scene[v] < 0 || view_scene[v] >= n_scenes) return fail(c, VRS_ERR_INVALID, "view_scene out of range");
      total += scenes[view_scene[v]].n;
    }
  }
  if (total != sv.total_nv) return fail(c, VRS_ERR_INVALID, "scene sizes differ from the saved forward");
  const long long HW = (long long)sv.W * sv.H;
  vrs_status s = VRS_OK;
  if (!ensure(c, c->grad_rec, sizeof(float) * 16 * (size_t)std::max(total, 1ll), cap_mode, &s) ||
      !ensure(c, c->dsamp_full, sizeof(float4) * (size_t)HW * n_views * (sv.fovea_mode ? 2 : 1), cap_mode, &s) ||
      !ensure(c, c->dsamp_low, sizeof(float4) * (size_t)(HW / 4 + 1) * n_views, cap_mode, &s))
    return s;
  float4* dfull = P<float4>(c->dsamp_full);
  float4* dhyb = dfull + HW * n_views;
  float4* dlow = P<float4>(c->dsamp_low);
  cudaMemsetAsync(c->grad_rec.p, 0, sizeof(float) * 16 * (size_t)std::max(total, 1ll), st);
  launch_composite_backward(P<ViewParams>(c->views), n_views, P<uint8_t>(c->tile_class), sv.tiles_per_view, sv.key_tile,
                            sv.fovea_mode, d_dL_drgb, sv.W, sv.H, dfull, dhyb, dlow, st);
  Plan pl;
  pl.n_views = n_views;
  pl.W = sv.W;
  pl.H = sv.H;
  pl.T = sv.key_tile;
  pl.fovea_mode = sv.fovea_mode;
  pl.tiles_per_view = sv.tiles_per_view;
  pl.total_nv = sv.total_nv;
  RenderArgs a = make_args(c, pl, o);
  a.s_full = P<float4>(c->s_full);
  a.s_low = sv.fovea_mode ? P<float4>(c->s_low) : nullptr;
  a.dL_dout = reinterpret_cast<const float*>(dfull);
  a.dL_dlow = reinterpret_cast<const float*>(dlow);
  a.grad_rec = P<float>(c->grad_rec);
  uint32_t* ctr = P<uint32_t>(c->counters);
  cudaMemsetAsync(ctr + kCtrQueue, 0, sizeof(uint32_t), st);
  launch_render_backward(a, 4ll * n_views * sv.tiles_per_view, st);
  for (int sc = 0; sc < n_scenes; ++sc) {
    if (!cnt[sc] || scenes[sc].n <= 0) continue;
    launch_preprocess_backward(to_dev(scenes[sc]), P<ViewParams>(c->views), P<int>(c->view_list) + first[sc], cnt[sc],
                               P<uint32_t>(c->count), P<float>(c->grad_rec), grads[sc], st);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "backward launch");
}

vrs_status vrs_check_status(vrs_ctx* c, void* stream, int64_t* required_instances) {
  if (!c) return VRS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  uint32_t* ctr = P<uint32_t>(c->counters);
  uint32_t h[3];
  e = cudaMemcpy(h, ctr + kCtrStatus - 1, sizeof(uint32_t) * 2, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(c, e, "status read");
  const uint32_t total = h[0], status = h[1];
  c->max_needed = std::max<long long>(c->max_needed, total);
  if (required_instances) *required_instances = c->max_needed;
  cudaMemset(ctr + kCtrStatus, 0, sizeof(uint32_t));
  if (status & kStTimeout) return fail(c, VRS_ERR_TIMEOUT, "a bounded device wait gave up");
  if (status & kStOverflow) return fail(c, VRS_ERR_CAPACITY, "instance buffer overflow");
  return VRS_OK;
}

vrs_status vrs_get_stats(vrs_ctx* c, void* stream, int64_t* out) {
  if (!c || !out) return VRS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  uint32_t ctr[kCtrCount];
  cudaMemcpy(ctr, c->counters.p, sizeof ctr, cudaMemcpyDeviceToHost);
  unsigned long long st3[4] = {0, 0, 0, 0};
  if (c->stats.p) cudaMemcpy(st3, c->stats.p, sizeof st3, cudaMemcpyDeviceToHost);
  out[0] = ctr[kCtrTotal];
  out[1] = ctr[kCtrNItems];
  out[2] = (int64_t)st3[0];
  out[3] = (int64_t)st3[1];
  out[4] = (int64_t)st3[2];
  out[5] = c->saved.n_views;
  out[6] = c->last_passes;
  out[7] = c->last_launches;
  return VRS_OK;
}

vrs_status vrs_copy_instances(vrs_ctx* c, uint64_t* d_keys, uint32_t* d_vals, uint32_t* d_ranges, int64_t cap,
                              int64_t* n, void* stream) {
  if (!c || !n) return VRS_ERR_INVALID;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  uint32_t total = 0;
  cudaMemcpy(&total, P<uint32_t>(c->counters) + kCtrSortN, sizeof total, cudaMemcpyDeviceToHost);
  *n = total;
  if (total > cap) return fail(c, VRS_ERR_CAPACITY, "caller buffer too small");
  const int b = c->saved.sorted_buf;
  if (d_keys && total) cudaMemcpyAsync(d_keys, c->keys[b].p, sizeof(uint64_t) * total, cudaMemcpyDeviceToDevice, st);
  if (d_vals && total) cudaMemcpyAsync(d_vals, c->vals[b].p, sizeof(uint32_t) * total, cudaMemcpyDeviceToDevice, st);
  if (d_ranges)
    cudaMemcpyAsync(d_ranges, c->ranges.p, sizeof(uint32_t) * 2 * (size_t)c->saved.n_views * c->saved.tiles_per_view,
                    cudaMemcpyDeviceToDevice, st);
  e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "copy instances");
}

vrs_status vrs_test_bounded_wait(vrs_ctx* c, int which, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (which != 0 && which != 1) return fail(c, VRS_ERR_INVALID, "which: 0 look-back, 1 mbarrier");
  cudaStream_t st = (cudaStream_t)stream;
  if (capturing(st)) return fail(c, VRS_ERR_INVALID, "not during stream capture");
  vrs_status s = VRS_OK;
  if (!ensure(c, c->misc, 2048, false, &s)) return s;
  uint32_t* status = P<uint32_t>(c->counters) + kCtrStatus;
  if (which == 0) {
    uint32_t* look = reinterpret_cast<uint32_t*>(P<char>(c->misc) + 1024);  // 256 words nothing publishes
    cudaMemsetAsync(look, 0, 1024, st);
    launch_lookback_timeout_test(look, status, st);
  } else {
    launch_mbar_timeout_test(status, st);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "bounded-wait check");
}

vrs_status vrs_probe_orders(vrs_ctx* c, const float* d_probes, int n_probes, int max_len, int32_t* d_ids,
                            float* d_depth, int32_t* d_len, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (n_probes < 0 || max_len < 0 || (n_probes > 0 && (!d_probes || !d_ids || !d_len)))
    return fail(c, VRS_ERR_INVALID, "bad probe arguments");
  const Saved& sv = c->saved;
  if (sv.n_views <= 0 || !c->rec.p || !c->ranges.p) return fail(c, VRS_ERR_INVALID, "no render to probe");
  if (sv.sort_mode != 0 && sv.sort_mode != 3 && sv.sort_mode != 4)
    return fail(c, VRS_ERR_UNSUPPORTED, "probes follow the exact and global orders only");
  if (n_probes == 0) return VRS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  launch_probe_orders(P<ViewParams>(c->views), sv.n_views, P<float4>(c->rec), P<uint32_t>(c->vals[sv.sorted_buf]),
                      P<uint32_t>(c->ranges), sv.key_tile, sv.tiles_per_view, sv.sort_mode >= 3 ? 1 : 0, d_probes,
                      n_probes, max_len, d_ids, d_depth, d_len, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "probe launch");
}

vrs_status vrs_project(vrs_ctx* c, const vrs_gaussians* scene, const vrs_camera* cam, int key_tile, float* d_out,
                       float* d_bbox, uint32_t* d_count, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!scene || !cam || !d_out || !d_bbox || !d_count) return fail(c, VRS_ERR_INVALID, "null argument");
  vrs_status s = check_scene(c, *scene);
  if (s) return s;
  if (key_tile != 16 && key_tile != 32) return fail(c, VRS_ERR_INVALID, "key_tile must be 16 or 32");
  if (!finite_cam(*cam) || cam->width <= 0 || cam->height <= 0) return fail(c, VRS_ERR_INVALID, "bad camera");
  cudaStream_t st = (cudaStream_t)stream;
  if ((s = reserve_staging(c, 1))) return s;
  fill_view(c->h_views[0], *cam, nullptr, key_tile);
  c->h_views[0].base = 0;
  c->h_view_list[0] = 0;
  if ((s = stage_views(c, 1, st, capturing(st)))) return s;
  launch_project_only(to_dev(*scene), P<ViewParams>(c->views), key_tile, d_out, d_bbox, d_count, st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "project launch");
}

vrs_status vrs_sort_pairs(vrs_ctx* c, const uint64_t* d_keys_in, const uint32_t* d_vals_in, uint64_t* d_keys_out,
                          uint32_t* d_vals_out, int64_t n, int bits, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (n < 0 || n >= (1ll << 32) || bits < 1 || bits > 64) return fail(c, VRS_ERR_INVALID, "bad sort arguments");
  if (n > 0 && (!d_keys_in || !d_vals_in || !d_keys_out || !d_vals_out)) return fail(c, VRS_ERR_INVALID, "null pointer");
  if (n == 0) return VRS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const bool cap_mode = capturing(st);
  vrs_status s = VRS_OK;
  if (!ensure(c, c->keys[1], sizeof(uint64_t) * n, cap_mode, &s) || !ensure(c, c->vals[1], sizeof(uint32_t) * n, cap_mode, &s) ||
      !ensure(c, c->sort_scratch, sort_scratch_bytes(n), cap_mode, &s) ||
      !ensure(c, c->misc, 16, cap_mode, &s))
    return s;
  cudaMemcpyAsync(d_keys_out, d_keys_in, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(d_vals_out, d_vals_in, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  set_u32_kernel<<<1, 1, 0, st>>>(P<uint32_t>(c->misc), (uint32_t)n);
  SortScratch ss;
  sort_scratch_carve(c->sort_scratch.p, n, &ss);
  uint64_t* kb[2] = {d_keys_out, P<uint64_t>(c->keys[1])};
  uint32_t* vb[2] = {d_vals_out, P<uint32_t>(c->vals[1])};
  const int cur = launch_radix_sort(kb, vb, P<uint32_t>(c->misc), n, bits, ss, P<uint32_t>(c->counters) + kCtrStatus, st);
  if (cur == 1) {
    cudaMemcpyAsync(d_keys_out, kb[1], sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(d_vals_out, vb[1], sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, st);
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "sort launch");
}

vrs_status vrs_loss_l1_ssim(vrs_ctx* c, const float* d_img, const float* d_target, int n_images, int height, int width,
                            float* d_loss, float* d_grad, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_img || !d_target || !d_loss || n_images <= 0 || height <= 0 || width <= 0)
    return fail(c, VRS_ERR_INVALID, "bad loss arguments");
  cudaStream_t st = (cudaStream_t)stream;
  vrs_status s = VRS_OK;
  if (!ensure(c, c->loss_scratch, loss_scratch_bytes(n_images, height, width), capturing(st), &s)) return s;
  return loss_l1_ssim_impl(d_img, d_target, n_images, height, width, d_loss, d_grad, c->loss_scratch.p,
                           c->loss_scratch.bytes, st);
}

vrs_status vrs_net_forward(vrs_ctx* c, const float* d_params, const float* d_x, int n, int H, int W, float* d_y,
                           uint16_t* d_acts, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_params || !d_x || !d_y || n <= 0 || H <= 0 || W <= 0) return fail(c, VRS_ERR_INVALID, "bad net arguments");
  cudaStream_t st = (cudaStream_t)stream;
  vrs_status s = VRS_OK;
  // the packed weights, and the hidden activations when d_acts is NULL
  const size_t act_bytes = d_acts ? 0 : sizeof(uint16_t) * 64 * (size_t)n * H * W;
  if (!ensure(c, c->net_tmp, act_bytes + net_train_pack_bytes(), capturing(st), &s)) return s;
  uint16_t* wpack = P<uint16_t>(c->net_tmp);
  uint16_t* a12 = d_acts ? nullptr : wpack + net_train_pack_bytes() / 2;
  if (!net_forward_train(d_params, d_x, n, H, W, d_y, d_acts, a12, wpack, P<uint32_t>(c->counters) + kCtrStatus, st))
    return fail(c, VRS_ERR_UNSUPPORTED, "more training CTAs per SM than tensor memory holds");
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "net forward");
}

vrs_status vrs_net_backward(vrs_ctx* c, const float* d_params, const float* d_x, const uint16_t* d_acts,
                            const float* d_dy, int n, int H, int W, float* d_dparams, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_params || !d_x || !d_acts || !d_dy || !d_dparams || n <= 0 || H <= 0 || W <= 0)
    return fail(c, VRS_ERR_INVALID, "bad net arguments");
  cudaStream_t st = (cudaStream_t)stream;
  vrs_status s = VRS_OK;
  // the packed weights and the hidden-layer gradients dz2, dz1 (BF16, pixel-major)
  if (!ensure(c, c->net_tmp, net_train_pack_bytes() + sizeof(uint16_t) * 64 * (size_t)n * H * W, capturing(st), &s))
    return s;
  uint16_t* wpack = P<uint16_t>(c->net_tmp);
  uint16_t* dz2 = wpack + net_train_pack_bytes() / 2;
  uint16_t* dz1 = dz2 + (size_t)32 * n * H * W;
  if (!net_backward_train(d_params, d_x, d_acts, d_dy, n, H, W, d_dparams, dz2, dz1, wpack,
                          P<uint32_t>(c->counters) + kCtrStatus, st))
    return fail(c, VRS_ERR_UNSUPPORTED, "more training CTAs per SM than tensor memory holds");
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "net backward");
}

vrs_status vrs_net_periphery(vrs_ctx* c, const float* d_params, const float* d_low, float* d_out, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_params || !d_low || !d_out) return fail(c, VRS_ERR_INVALID, "null net argument");
  const Saved& sv = c->saved;
  if (sv.n_views <= 0 || sv.fovea_mode == 0 || sv.key_tile != 32)
    return fail(c, VRS_ERR_INVALID, "vrs_net_periphery follows a foveated vrs_render");
  net_periphery(d_params, d_low, d_out, P<uint8_t>(c->tile_class), P<ViewParams>(c->views), sv.n_views,
                sv.tiles_per_view, sv.W, sv.H, P<uint32_t>(c->counters) + kCtrStatus, (cudaStream_t)stream);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "net periphery");
}

vrs_status vrs_mse(vrs_ctx* c, const float* d_y, const float* d_t, int64_t n, float* d_loss, float* d_dy, void* stream) {
  if (!c) return VRS_ERR_INVALID;
  if (!d_y || !d_t || !d_loss || n <= 0) return fail(c, VRS_ERR_INVALID, "bad mse arguments");
  cudaStream_t st = (cudaStream_t)stream;
  vrs_status s = VRS_OK;
  if (!ensure(c, c->misc, 64, capturing(st), &s)) return s;
  net_mse(d_y, d_t, n, d_loss, d_dy, reinterpret_cast<double*>(P<char>(c->misc) + 16), st);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? VRS_OK : cuda_fail(c, e, "mse");
}

vrs_status vrs_profile_begin(vrs_ctx* c, int max_calls) {
  if (!c || max_calls <= 0 || max_calls > (1 << 20)) return fail(c, VRS_ERR_INVALID, "bad profile size");
  if (max_calls > c->prof_cap) {
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    c->prof_ev.assign((size_t)max_calls * 8, nullptr);
    for (auto& e : c->prof_ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(c, VRS_ERR_CUDA, "cudaEventCreate");
    c->prof_cap = max_calls;
  }
  c->prof_used = 0;
  c->prof_on = true;
  return VRS_OK;
}

vrs_status vrs_profile_end(vrs_ctx* c, void* stream, double* ms, int64_t* n_calls) {
  if (!c || !ms) return VRS_ERR_INVALID;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "synchronize");
  for (int k = 0; k < 8; ++k) ms[k] = 0.0;
  for (int i = 0; i < c->prof_used; ++i) {
    cudaEvent_t* ev = &c->prof_ev[(size_t)i * 8];
    for (int k = 0; k < 7; ++k) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[k], ev[k + 1]) == cudaSuccess) ms[k] += t;
    }
    float t = 0.f;
    if (cudaEventElapsedTime(&t, ev[0], ev[7]) == cudaSuccess) ms[7] += t;
  }
  if (n_calls) *n_calls = c->prof_used;
  c->prof_on = false;
  c->prof_used = 0;
  return VRS_OK;
}

vrs_status vrs_update_views(vrs_ctx* c, const vrs_camera* cams, const vrs_fovea* fov, int n_views) {
  if (!c) return VRS_ERR_INVALID;
  if (!cams || n_views <= 0 || n_views > c->staging_cap || n_views != c->saved.n_views)
    return fail(c, VRS_ERR_INVALID, "update_views needs the view count of the last render");
  for (int v = 0; v < n_views; ++v) {
    if (!finite_cam(cams[v])) return fail(c, VRS_ERR_INVALID, "non-finite or non-positive camera values");
    if (cams[v].width != c->saved.W || cams[v].height != c->saved.H)
      return fail(c, VRS_ERR_INVALID, "update_views cannot change the image size");
  }
  if (any_mask(fov, n_views) != c->saved.has_mask)
    return fail(c, VRS_ERR_INVALID, "update_views cannot add or remove visibility masks");
  if (c->staging_done) cudaEventSynchronize(c->staging_done);  // the last copy of the staging has run
  for (int v = 0; v < n_views; ++v) {
    ViewParams& vp = c->h_views[v];
    const int scene = vp.scene;
    const long long base = vp.base;
    fill_view(vp, cams[v], fov ? &fov[v] : nullptr, c->saved.key_tile);
    vp.scene = scene;
    vp.base = base;
  }
  return VRS_OK;
}

vrs_status vrs_set_tuning(vrs_ctx* c, int max_render_ctas_per_sm) {
  if (!c || max_render_ctas_per_sm < 0 || max_render_ctas_per_sm > 32) return fail(c, VRS_ERR_INVALID, "bad tuning value");
  c->max_ctas_per_sm = max_render_ctas_per_sm;
  return VRS_OK;
}

const char* vrs_last_error(vrs_ctx* c) { return c ? c->err.c_str() : "null context"; }

}  // extern "C"
