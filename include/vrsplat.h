/*
 * vrsplat.h - C ABI of the GB300 (sm_103a) foveated, popping-free Gaussian-splat
 * rasterizer: the data-parallel hot path of VRSplat (Tu et al., arXiv 2505.10144).
 *
 * The problem each call solves is the paper's rendering problem: Gaussians of Eq. 1,
 * blended front to back by Eq. 2, projected with Optimal Projection (Sec. 4.2), ordered
 * per ray by the depth of maximum response (StopThePop, Sec. 4.1), tile-culled on the
 * optimal plane (Sec. 4.2, Eq. 4), with focus and periphery rendered in one launch
 * (Sec. 4.3, "Single-Pass Foveated Rendering"), and its backward pass for the
 * fine-tuning of Sec. 4.1 / Sec. 5.
 *
 * Conventions shared by every entry point:
 *   - All pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers owned by the caller.  The library never frees caller memory.
 *   - Every call is asynchronous on the given CUDA stream (cudaStream_t passed as void*,
 *     NULL = legacy default stream) unless it says otherwise.  No C++ exception crosses
 *     the ABI; every entry point returns a vrs_status.
 *   - One vrs_ctx per host thread.  A context owns its workspace (device memory for
 *     projected records, instances, sort buffers and saved forward state).
 *   - Errors: VRS_ERR_INVALID for bad arguments (nothing is launched), VRS_ERR_CAPACITY
 *     when the workspace cannot hold the Gaussian/tile instances and may not grow
 *     (during stream capture), VRS_ERR_CUDA for a CUDA runtime error, VRS_ERR_TIMEOUT
 *     when a device-side bounded wait gave up (the kernel returns early; results of
 *     that call are invalid but the context stays usable).  vrs_last_error() gives a
 *     one-line description.
 *   - Camera model (OpenCV): camera x right, y down, z forward; world_to_cam is the
 *     row-major 3x4 [R|t]; pixel (x, y) has its centre at (x + 0.5, y + 0.5).
 */
#ifndef VRSPLAT_H
#define VRSPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VRS_OK = 0,
  VRS_ERR_INVALID = 1,
  VRS_ERR_CAPACITY = 2,
  VRS_ERR_CUDA = 3,
  VRS_ERR_TIMEOUT = 4,
  VRS_ERR_UNSUPPORTED = 5
} vrs_status;

typedef struct vrs_ctx vrs_ctx;

/* One scene of N Gaussians (Eq. 1), device SoA float32, caller-owned:
 *   mean[3][N], log_scale[3][N], quat[4][N] (w, x, y, z; need not be normalised),
 *   opacity_logit[N] (opacity = sigmoid), sh[K][3][N] with K = (sh_degree + 1)^2,
 *   sh_degree in 0..3, 0 <= N <= 2^28 - 1 (VRS_ERR_INVALID otherwise).  Non-finite
 *   parameters cull the Gaussian. */
typedef struct {
  const float* mean;
  const float* log_scale;
  const float* quat;
  const float* opacity_logit;
  const float* sh;
  int64_t n;
  int sh_degree;
} vrs_gaussians;

/* Gradients of a scene, same layout as vrs_gaussians; accumulated into (+=). */
typedef struct {
  float* mean;
  float* log_scale;
  float* quat;
  float* opacity_logit;
  float* sh;
} vrs_gaussian_grads;

/* Pinhole camera; near_z culls Gaussians whose camera-space mean has z < near_z. */
typedef struct {
  float world_to_cam[12];
  float fx, fy, cx, cy;
  int width, height;
  float near_z;
} vrs_camera;

/* Per-view foveation (Sec. 4.3).  The blend weight is
 * w(p) = clamp((radius + band - |p - gaze|) / band, 0, 1); a 32x32 tile is focus if
 * w = 1 on all its pixel centres, periphery if w = 0 on all, else hybrid.
 *   mode 0: plain, every pixel rendered at full resolution (gaze ignored)
 *   mode 1: single-pass foveated, periphery upsampled bilinearly (clamp to edge)
 *   mode 2: single-pass foveated, periphery pixels left to the periphery network:
 *           only the half-resolution image (d_low_rgb) is written for them
 * focus_tile (8 or 16) only changes how focus tiles are split into work, never the
 * image.  Foveated modes need even width and height.
 * visible (visibility culling, Sec. 4.3): NULL, or a device [height][width] byte mask of
 * the headset's visible area (nonzero = visible), caller-owned and read during the
 * render.  A key tile with no visible pixel gets no Gaussian/tile instances and no
 * render work; its pixels (and half-resolution samples) are set to bg.  It applies in
 * every mode, and the backward pass gives those pixels no gradient. */
typedef struct {
  float gaze_x, gaze_y, radius_px, band_px;
  int mode;
  int focus_tile;
  const uint8_t* visible;
} vrs_fovea;

/* Per-ray ordering (Sec. 4.1):
 *   sort_mode 0 exact: every kept pair of a sample sorted by (depth, Gaussian index)
 *   sort_mode 1 window: one per-sample min-window of win[2] entries over the tile's
 *               depth-sorted stream
 *   sort_mode 2 hierarchical: min-windows of win[0] (4x4-sample block), win[1]
 *               (2x2-sample block) and win[2] (per sample) entries in cascade
 *   sort_mode 3 global by view-space z of the mean (the order of 3DGS, Sec. 3) and
 *   sort_mode 4 global by distance of the mean from the camera centre (Mini-Splatting):
 *               every tile list is blended in its order, no per-ray resort (these
 *               orders pop; they are the paper's cheaper comparison orders)
 * win[*] <= 32 (unused by modes 0, 3 and 4).  key_tile: 16 or 32, the tile size of the global sort (foveated modes
 * use 32).  bg: background colour.  stats: 1 to collect device counters. */
typedef struct {
  int sort_mode;
  int win[3];
  int key_tile;
  float bg[3];
  int stats;
} vrs_render_opts;

/* Create a context; workspace_bytes_hint pre-sizes the instance buffers (0 = grow on
 * demand).  *ctx receives a handle to free with vrs_destroy. */
vrs_status vrs_create(vrs_ctx** ctx, size_t workspace_bytes_hint);
vrs_status vrs_destroy(vrs_ctx* ctx);

/* Pre-size the workspace for up to n_views views of width x height, total_gaussians
 * summed over the rendered views' scenes, and max_instances Gaussian/tile pairs (at
 * most 2^31 - 1 per render; a render needing more returns VRS_ERR_CAPACITY).  Must be
 * called outside stream capture before capturing vrs_render into a CUDA graph. */
vrs_status vrs_reserve(vrs_ctx* ctx, int n_views, int width, int height, int64_t total_gaussians,
                       int64_t max_instances);

/* Render n_views views (Eq. 1-2, Sec. 4).  scenes[n_scenes] (host array of device
 * SoA descriptions); h_view_scene[n_views] maps each view to its scene; h_cams and
 * h_fovea are host arrays [n_views] (all views share width, height and fovea mode).
 * d_out_rgb: device float [n_views][3][height][width], fully written.  d_low_rgb:
 * optional device float [n_views][3][height/2][width/2] half-resolution image (required
 * for fovea mode 2).  save_for_backward = 1 keeps what vrs_render_backward needs in
 * the context until the next vrs_render.  Outside stream capture the call reads the
 * instance count back (one host synchronisation) and grows the workspace as needed;
 * inside capture it uses the reserved capacity and reports overflow through the
 * status read by vrs_check_status. */
vrs_status vrs_render(vrs_ctx* ctx, const vrs_gaussians* scenes, int n_scenes, const int* h_view_scene,
                      const vrs_camera* h_cams, const vrs_fovea* h_fovea, int n_views,
                      const vrs_render_opts* opts, float* d_out_rgb, float* d_low_rgb,
                      int save_for_backward, void* stream);

/* Two-pass foveated rendering, the paper's comparison baseline (Appendix A).  Pass 1
 * renders, per view, a full-resolution square around the gaze through a tight frustum
 * (the camera cropped to side 2 * (ceil(max(radius + band)) + 1), clamped to the image,
 * placed at integer offsets inside the image).  Pass 2 renders the view at half
 * resolution: half focal length, principal point and size.  It skips, by a visibility
 * mask, the half-resolution pixels that no full-resolution pixel with w < 1 reads.  The
 * output is w * centre + (1 - w) * bilinear(half) inside the square and the bilinear
 * upsample elsewhere (w of vrs_fovea; w = 0 outside the square).
 *   h_fovea: mode 1 for every view.  opts: sort mode and windows of both passes (their
 *   key tiles are 16).  d_out_rgb: device float [n_views][3][height][width].
 * Both passes use the context's workspace (its last render is the second pass).  Not
 * capturable in a CUDA graph (VRS_ERR_UNSUPPORTED); at most 64 views; even width and
 * height. */
vrs_status vrs_render_two_pass(vrs_ctx* ctx, const vrs_gaussians* scenes, int n_scenes, const int* h_view_scene,
                               const vrs_camera* h_cams, const vrs_fovea* h_fovea, int n_views,
                               const vrs_render_opts* opts, float* d_out_rgb, void* stream);

/* Stereo reuse of distant content (named as future work in Sec. 7: monocular rendering
 * and stereoscopic reuse of distant content), on a plain (unfoveated) stereo pair.
 * The Gaussians whose world-space mean lies at distance >= far_distance from the
 * cyclopean eye (the midpoint of the two eye centres) form the far layer, rendered once,
 * from the cyclopean camera (the eyes' rotation and intrinsics, centre at the midpoint);
 * each eye renders the others, its near layer.  Each eye's pixel is C_near + T_near
 * (C_far + T_far bg): the far layer seen through the near layer's transmittance (Eq. 2).
 * For a far Gaussian at distance d the eye and cyclopean rays through a pixel differ by
 * f (IPD / 2) / d pixels (0.25 px at d = 92 m, f = 722.6, IPD = 64 mm).
 *   scene: one scene.  h_cams: the two eyes, sharing image size, intrinsics and rotation.
 *   opts: a per-ray order (sort mode 0, 1 or 2), windows and bg as for vrs_render.
 *   d_out_rgb: device float [2][3][height][width].
 * One call runs the pipeline once over three views (the two near layers and the far
 * layer), keeps each pixel's colour and transmittance, and composites them.  The context
 * keeps no state for vrs_render_backward afterwards.  VRS_ERR_INVALID for eyes that do not
 * share rotation or intrinsics, a non-positive or non-finite far_distance, or a global
 * sort mode. */
vrs_status vrs_render_stereo_reuse(vrs_ctx* ctx, const vrs_gaussians* scene, const vrs_camera* h_cams,
                                   const vrs_render_opts* opts, float far_distance, float* d_out_rgb, void* stream);

/* Backward of the last vrs_render called with save_for_backward = 1, with identical
 * scenes, cameras, foveas and options: accumulates d<d_dL_drgb, rgb>/d(params) into
 * grads[n_scenes] (device, caller-owned, same layouts).  d_dL_drgb: device float
 * [n_views][3][H][W].  Sorting, culling and windowing are treated as constant (their
 * derivative is zero almost everywhere); the per-ray order replayed is the forward's. */
vrs_status vrs_render_backward(vrs_ctx* ctx, const vrs_gaussians* scenes, int n_scenes,
                               const int* h_view_scene, const vrs_camera* h_cams,
                               const vrs_fovea* h_fovea, int n_views, const vrs_render_opts* opts,
                               const float* d_dL_drgb, const vrs_gaussian_grads* grads, void* stream);

/* Synchronise the stream and return the device status of the calls issued so far
 * (VRS_OK, VRS_ERR_CAPACITY or VRS_ERR_TIMEOUT); clears it.  required_instances, when
 * not NULL, receives the largest instance count a render needed. */
vrs_status vrs_check_status(vrs_ctx* ctx, void* stream, int64_t* required_instances);

/* Counters of the last render (host int64[8]): 0 instances, 1 work items, 2 evaluated
 * pairs, 3 kept pairs, 4 blended pairs, 5 views, 6 sort passes, 7 kernels launched.
 * Counters 2-4 are filled only when opts.stats was 1: evaluated counts each (sample,
 * Gaussian) pair tested once, kept the pairs that entered the per-sample window with
 * alpha >= 1/255, blended the pairs composited before the transmittance stop.
 * Synchronises the stream. */
vrs_status vrs_get_stats(vrs_ctx* ctx, void* stream, int64_t* h_out8);

/* Copy the sorted instances of the last render into caller buffers:
 * d_keys[cap] (uint64: (view * tiles_per_view + tile) << 32 | ordered float bits of the
 * tile depth), d_vals[cap] (uint32 Gaussian index within its scene) and d_ranges
 * [n_views * tiles_per_view][2] (uint32 start, end).  *n receives the instance count
 * (synchronises the stream).  Returns VRS_ERR_CAPACITY when cap is too small. */
vrs_status vrs_copy_instances(vrs_ctx* ctx, uint64_t* d_keys, uint32_t* d_vals, uint32_t* d_ranges,
                              int64_t cap, int64_t* n, void* stream);

/* Per-Gaussian Optimal-Projection records of one view (Sec. 4.2) for inspection:
 * d_out[N][24] float, six groups of four relative to the projected mean pm (pixels):
 * (pm.x, pm.y, H00, H01), (H10, H11, H20, H21), (H22, a00, 2 a01, a11),
 * (log2 opacity, n0, n1, n2), (m00, 2 m01, m11, 2 m02), (2 m12, r, g, b), where
 * H = [E; u] K^-1 maps a pixel offset d from pm (homogeneous (d, 1)) to the tangent
 * plane (s1, s2, w) with plane point s / w, a = 0.5 log2(e) A is the scaled conic,
 * n and m the linear and quadratic forms of t* (numerator n.(d,1), denominator
 * (d,1)^T M (d,1)), normalised so that t* at pm is the view depth of the mean;
 * d_bbox[N][4] float (xmin, ymin, xmax, ymax;
 * all zero when culled), d_count[N] uint32 tiles kept after Eq. 4 culling with
 * key_tile-sized tiles. */
vrs_status vrs_project(vrs_ctx* ctx, const vrs_gaussians* scene, const vrs_camera* h_cam, int key_tile,
                       float* d_out, float* d_bbox, uint32_t* d_count, void* stream);

/* Stable LSD radix sort of n (key, value) pairs by the low `bits` bits of the key
 * (onesweep: one histogram pass, then one decoupled-look-back pass per 8-bit digit).
 * d_keys_in/d_vals_in are not modified; results go to d_keys_out/d_vals_out.  Scratch
 * comes from the context.  bits in 1..64. */
vrs_status vrs_sort_pairs(vrs_ctx* ctx, const uint64_t* d_keys_in, const uint32_t* d_vals_in,
                          uint64_t* d_keys_out, uint32_t* d_vals_out, int64_t n, int bits, void* stream);

/* Graph replays (batched persistent launch, Sec. 4.3's single launch over all views):
 * rewrites the cameras and gaze of the views of the last vrs_render (same count, same
 * image size, same scenes) in the context's pinned staging, which a CUDA graph captured
 * around vrs_render copies to the device at every replay.  Waits for the previous
 * replay's copy of the staging before writing; launches nothing.  h_fovea may be NULL
 * (gaze unchanged). */
vrs_status vrs_update_views(vrs_ctx* ctx, const vrs_camera* h_cams, const vrs_fovea* h_fovea, int n_views);

/* Tuning knob read by vrs_render: cap on resident render CTAs per SM (0 = the
 * occupancy limit).  Changes scheduling only, never the image. */
vrs_status vrs_set_tuning(vrs_ctx* ctx, int max_render_ctas_per_sm);

/* Learned periphery network (the workload's replacement for the periphery upsampling of
 * Sec. 4.3): y = x + conv3(relu(conv2(relu(conv1(bf16(x)))))), 3 -> 32 -> 32 -> 3
 * channels, 3x3 kernels, zero padding 1, BF16 weights and activations, FP32
 * accumulation, x the bilinear x2 upsampling of the half-resolution image.  Parameters:
 * one device float buffer of VRS_NET_PARAMS values, OIHW:
 * w1[32][3][3][3] b1[32] w2[32][32][3][3] b2[32] w3[3][32][3][3] b3[3] (float master
 * copy; the kernels round weights to BF16). */
#define VRS_NET_PARAMS 11011

/* Training forward on whole images: d_x, d_y device float [n][3][H][W]; d_acts (device
 * uint16 BF16 bits [n][2][H][W][32], pixel-major, may be NULL) receives the two hidden
 * activations for vrs_net_backward.  Every convolution runs on the tensor cores
 * (tcgen05.mma).  Scratch from ctx (128 bytes per pixel when d_acts is NULL).  A
 * bounded wait that gives up raises bit 1 of the device status word (vrs_check_status);
 * VRS_ERR_UNSUPPORTED when more of the training kernels' CTAs fit on an SM than its
 * tensor memory holds. */
vrs_status vrs_net_forward(vrs_ctx* ctx, const float* d_params, const float* d_x, int n_images, int height, int width,
                           float* d_y, uint16_t* d_acts, void* stream);

/* d_dparams += d<d_dy, y>/d(params) for the forward that wrote d_acts (BF16 rounding
 * of the forward treated as identity, ReLU masks from the saved activations).  Mixed
 * precision, like the forward: the data and weight gradients are contractions on the
 * tensor cores with BF16 operands and FP32 accumulation, so d_dy and the hidden-layer
 * gradients are rounded to BF16 (nearest even) where they enter one.  Scratch from ctx
 * (128 bytes per pixel); status and errors as vrs_net_forward. */
vrs_status vrs_net_backward(vrs_ctx* ctx, const float* d_params, const float* d_x, const uint16_t* d_acts,
                            const float* d_dy, int n_images, int height, int width, float* d_dparams, void* stream);

/* After a vrs_render with fovea mode 2: writes every periphery pixel of d_out_rgb with the
 * network applied to the bilinear upsampling of d_low_rgb (the same buffers that render
 * call used), one fused tensor-core kernel over the periphery tiles of all views. */
vrs_status vrs_net_periphery(vrs_ctx* ctx, const float* d_params, const float* d_low_rgb, float* d_out_rgb,
                             void* stream);

/* Mean squared error over n values and its gradient 2 (y - t) / n (d_dy may be NULL). */
vrs_status vrs_mse(vrs_ctx* ctx, const float* d_y, const float* d_t, int64_t n, float* d_loss, float* d_dy,
                   void* stream);

/* Largest n that vrs_sort_pairs_noalloc accepts. */
#define VRS_SORT_NOALLOC_MAX_PAIRS (1 << 20)

/* vrs_sort_pairs without any allocation.  The paper has no counterpart: this entry point
 * serves callers that cannot allocate GPU memory when they sort, such as a frame
 * callback with a hard latency budget (cudaMalloc and cudaFree can synchronise the
 * device), an application whose own pool owns all GPU memory, or code that must not
 * fail mid-frame on memory pressure.  Same result as vrs_sort_pairs (stable sort of n
 * (key, value) pairs by the low `bits` bits of the key into d_keys_out / d_vals_out;
 * inputs are not modified; in and out may be the same buffers) and no context.  The
 * scratch is a fixed device array of about 14 MiB built into the library; every GPU
 * that loads the library holds it until the process exits.  n above
 * VRS_SORT_NOALLOC_MAX_PAIRS returns VRS_ERR_INVALID and launches nothing.  Each call
 * looks up the array's device address on the current device (a host-side call, made on
 * every call so that no address outlives a reset context); the first call on a device
 * also loads the module there, so make it before any stream capture.  A runtime error
 * left by an earlier unrelated call is cleared on entry; VRS_ERR_CUDA then means that
 * one of this call's own copies or launches failed.  All calls
 * share the one array and each clears what must start at zero, so calls that overlap on
 * the GPU (other streams, other host threads) race and must be serialised by the
 * caller.  d_status (device uint32, may be NULL) receives the sort's device status bits
 * (1 = a bounded look-back wait gave up and the output is not valid). */
vrs_status vrs_sort_pairs_noalloc(const uint64_t* d_keys_in, const uint32_t* d_vals_in, uint64_t* d_keys_out,
                                  uint32_t* d_vals_out, int64_t n, int bits, uint32_t* d_status, void* stream);

/* Fine-tuning loss of Sec. 5 (0.8 L1 + 0.2 (1 - SSIM), SSIM of Wang et al. with an
 * 11x11 Gaussian window, sigma 1.5, zero padding) over n_images images [3][H][W]:
 * d_loss (device float[1]) receives the mean loss over images, d_grad (device
 * [n_images][3][H][W], may be NULL) dLoss/dimage. */
vrs_status vrs_loss_l1_ssim(vrs_ctx* ctx, const float* d_img, const float* d_target, int n_images, int height,
                            int width, float* d_loss, float* d_grad, void* stream);

/* One Adam step on n float parameters: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).  All device pointers. */
vrs_status vrs_adam_step(float* d_param, const float* d_grad, float* d_m, float* d_v, int64_t n, float lr,
                         float beta1, float beta2, float eps, int step, void* stream);

/* Stage timing with CUDA events (tracing).  vrs_profile_begin arms event recording at
 * the stage boundaries of the next max_calls vrs_render calls (no host
 * synchronisation is added).  vrs_profile_end synchronises the stream and returns, per
 * stage, the summed device time in milliseconds over the recorded calls:
 * h_stage_ms[8] = {preprocess, scan (+ instance-count read-back), duplicate, sort,
 * ranges + work items, render, composite, whole call}; *n_calls the number recorded. */
vrs_status vrs_profile_begin(vrs_ctx* ctx, int max_calls);
vrs_status vrs_profile_end(vrs_ctx* ctx, void* stream, double* h_stage_ms, int64_t* n_calls);

/* Failure-detection check of the library's bounded device waits.  Runs one of them
 * against a flag that nothing sets, with a short limit (1000 polls): which = 0 the radix
 * sort's decoupled look-back wait, which = 1 the mbarrier wait of the periphery-network
 * kernel.  The wait gives up, the kernel raises the timeout status and returns, so the
 * next vrs_check_status on this stream reports VRS_ERR_TIMEOUT (and clears it); the
 * context stays usable.  Nothing faults, traps or hangs.  Not allowed during stream
 * capture; VRS_ERR_INVALID for another `which`. */
vrs_status vrs_test_bounded_wait(vrs_ctx* ctx, int which, void* stream);

/* Blend order of single rays of the last vrs_render of this context (its views, sort
 * mode, records and tile lists must be unchanged since).  d_probes is a device array
 * [n_probes][3] of (view, x, y) floats: the ray through image point (x, y) of that view,
 * in pixels (pixel (i, j) has its centre at (i + 0.5, j + 0.5); a half-resolution
 * periphery sample of the foveated render sits at (2i + 1, 2j + 1)).  For each probe
 * the Gaussians the ray blends, front to back, are written to d_ids[probe][max_len]
 * (indices into the view's scene) and their depths t* (Sec. 4.1) to
 * d_depth[probe][max_len] (d_depth may be NULL); d_len[probe] receives the number of
 * blended pairs (entries past max_len are counted but not written) or -1 for a probe
 * outside its view.  The pairs and their values are the render's own (same evaluation);
 * the order is the render's sort mode: 0 exact (ascending depth, then index) or 3 / 4
 * (global orders: tile-list order).  Blending stops before the pair that would take the
 * transmittance below 1e-4.  Sort modes 1 and 2 return VRS_ERR_UNSUPPORTED: their
 * windows order a ray by the pairs of its neighbours too.  Asynchronous on `stream`;
 * all arrays are caller-owned device memory. */
vrs_status vrs_probe_orders(vrs_ctx* ctx, const float* d_probes, int n_probes, int max_len, int32_t* d_ids,
                            float* d_depth, int32_t* d_len, void* stream);

/* Measured throughput peaks of the current device, the denominators of the render
 * kernel's roofline (the render is bound by instruction issue on plain FP32, integer and
 * special-function work, and reads its records from L2).  Runs microbenchmarks of a few
 * milliseconds each on `stream` and synchronises it; allocates and frees about 2 GiB of
 * scratch; needs no context.  Every rate is the best of five timed launches after one
 * untimed launch, with 64 warps per SM and eight independent chains per thread:
 *   fp32_tflops   FFMA throughput, 2 flop per FMA (1e12 flop/s)
 *   exp2_gops     exp2f(c - x) throughput, the pair-opacity exponent (1e9 per s)
 *   logic_gops    32-bit three-input logic throughput (1e9 operations per s)
 *   l2_read_gbs   read bandwidth of a buffer of a quarter of the L2, read 256 times
 *                 with L2-only loads (1e9 B/s)
 *   dram_read_gbs read bandwidth of 2 GiB streamed once from HBM (1e9 B/s)
 * sm_count, max_sm_clock_khz and l2_bytes are the runtime's device attributes.
 * Returns VRS_ERR_INVALID for a NULL `out`, VRS_ERR_CUDA on any runtime error. */
typedef struct {
  int sm_count;
  int max_sm_clock_khz;
  int64_t l2_bytes;
  double fp32_tflops;
  double exp2_gops;
  double logic_gops;
  double l2_read_gbs;
  double dram_read_gbs;
} vrs_peaks;
vrs_status vrs_measure_peaks(vrs_peaks* out, void* stream);

const char* vrs_last_error(vrs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* VRSPLAT_H */
