"""Python binding of libvrsplat (include/vrsplat.h).

Argument marshalling only: every step of the render, its backward, the loss and the
optimiser runs in the library's CUDA kernels; PyTorch supplies device memory and the
stream.  There is no CPU or PyTorch fallback: without the built library every call
raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib
from ._lib import VrsError

SORT_MODES = {"exact": 0, "window": 1, "hier": 2, "global_z": 3, "global_dist": 4}
FOVEA_MODES = {"plain": 0, "bilinear": 1, "net": 2}


def _ptr(t: torch.Tensor | None):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


@dataclass
class DeviceScene:
    """Gaussian parameters resident on the GPU (float32 SoA, see synth.Scene)."""
    mean: torch.Tensor
    log_scale: torch.Tensor
    quat: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @staticmethod
    def from_host(scene, device="cuda") -> "DeviceScene":
        f = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).to(device)
        return DeviceScene(f(scene.mean), f(scene.log_scale), f(scene.quat), f(scene.opacity_logit), f(scene.sh),
                           scene.sh_degree)

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    def tensors(self):
        return [self.mean, self.log_scale, self.quat, self.opacity_logit, self.sh]

    def c(self) -> _lib.Gaussians:
        for t in self.tensors():
            assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        return _lib.Gaussians(*[_ptr(t) for t in self.tensors()], self.n, self.sh_degree)

    def zeros_like(self) -> "DeviceScene":
        return DeviceScene(*[torch.zeros_like(t) for t in self.tensors()], self.sh_degree)

    def flat_zeros_like(self) -> tuple["DeviceScene", torch.Tensor]:
        """Zeroed buffers shaped like these parameters, as views of one flat float32
        buffer (each part starts on a 64-float boundary), and that buffer: gradients laid
        out this way are cleared with one fill and reduced with one collective."""
        sizes = [t.numel() for t in self.tensors()]
        offs, o = [], 0
        for n in sizes:
            offs.append(o)
            o += (n + 63) // 64 * 64
        flat = torch.zeros(o, dtype=torch.float32, device=self.mean.device)
        parts = [flat[a:a + n].view(t.shape) for a, n, t in zip(offs, sizes, self.tensors())]
        return DeviceScene(*parts, self.sh_degree), flat


def camera_c(cam) -> _lib.Camera:
    c = _lib.Camera()
    w = np.asarray(cam.world_to_cam, dtype=np.float32).ravel()
    for k in range(12):
        c.world_to_cam[k] = float(w[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height, c.near_z = int(cam.width), int(cam.height), float(cam.near_z)
    return c


def fovea_c(fov, mode: int, focus_tile: int = 16, visible=None) -> _lib.Fovea:
    f = _lib.Fovea()
    if fov is not None:
        f.gaze_x, f.gaze_y, f.radius_px, f.band_px = (float(fov.gaze_x), float(fov.gaze_y), float(fov.radius_px),
                                                      float(fov.band_px))
    else:
        f.band_px = 1.0
    f.mode, f.focus_tile = int(mode), int(focus_tile)
    f.visible = _ptr(visible)
    return f


def _check_masks(visible, cams):
    """visible: None, or one entry per view: None or a contiguous CUDA uint8 [H, W] mask."""
    if visible is None:
        return [None] * len(cams)
    if len(visible) != len(cams):
        raise ValueError("one visibility mask (or None) per view")
    for m, c in zip(visible, cams):
        if m is None:
            continue
        if m.dtype != torch.uint8 or not m.is_cuda or not m.is_contiguous() or tuple(m.shape) != (int(c.height), int(c.width)):
            raise ValueError("a visibility mask is a contiguous CUDA uint8 tensor [height, width]")
    return list(visible)


@dataclass
class RenderConfig:
    sort_mode: str = "hier"
    windows: tuple = (4, 8, 16)
    key_tile: int = 16
    fovea_mode: str = "plain"
    focus_tile: int = 16
    bg: tuple = (0.0, 0.0, 0.0)
    stats: bool = False

    def opts(self) -> _lib.RenderOpts:
        o = _lib.RenderOpts()
        o.sort_mode = SORT_MODES[self.sort_mode]
        for k in range(3):
            o.win[k] = int(self.windows[k])
            o.bg[k] = float(self.bg[k])
        o.key_tile = int(self.key_tile)
        o.stats = int(self.stats)
        return o


class Renderer:
    """One library context (workspace owner).  Not thread-safe: one per thread."""

    def __init__(self, workspace_bytes: int = 0):
        self.lib = _lib.load()
        self.ctx = C.c_void_p()
        st = self.lib.vrs_create(C.byref(self.ctx), C.c_size_t(workspace_bytes))
        if st != 0:
            raise VrsError(st, "vrs_create failed")
        self._keep = None
        # incremented by every call that overwrites the context's lists and saved state
        # (render, two-pass render, graph replay); a differentiable render checks it
        # before its backward replays that state
        self.generation = 0

    def close(self):
        if self.ctx:
            self.lib.vrs_destroy(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st: int):
        if st != 0:
            raise VrsError(st, self.lib.vrs_last_error(self.ctx).decode())

    def _marshal(self, scenes, view_scene, cams, foveas, cfg: RenderConfig, visible=None):
        n_views = len(cams)
        masks = _check_masks(visible, cams)
        sc = (_lib.Gaussians * len(scenes))(*[s.c() for s in scenes])
        vs = (C.c_int * n_views)(*[int(v) for v in view_scene])
        cm = (_lib.Camera * n_views)(*[camera_c(c) for c in cams])
        mode = FOVEA_MODES[cfg.fovea_mode]
        fv = (_lib.Fovea * n_views)(*[fovea_c(foveas[k] if foveas else None, mode, cfg.focus_tile, masks[k])
                                      for k in range(n_views)])
        o = cfg.opts()
        self._keep = (sc, vs, cm, fv, o)
        return sc, vs, cm, fv, o

    def reserve(self, n_views, width, height, total_gaussians, max_instances):
        self._check(self.lib.vrs_reserve(self.ctx, n_views, width, height, int(total_gaussians), int(max_instances)))

    def render(self, scenes, view_scene, cams, foveas=None, cfg: RenderConfig | None = None, out=None, low=None,
               save: bool = False, stream=None, visible=None) -> torch.Tensor:
        """visible: None, or per view None or a CUDA uint8 [H, W] headset visibility mask
        (visibility culling: tiles without a visible pixel are not rendered and hold bg)."""
        cfg = cfg or RenderConfig()
        n_views = len(cams)
        W, H = int(cams[0].width), int(cams[0].height)
        if out is None:
            out = torch.empty((n_views, 3, H, W), device="cuda", dtype=torch.float32)
        sc, vs, cm, fv, o = self._marshal(scenes, view_scene, cams, foveas, cfg, visible)
        self.generation += 1
        self._check(self.lib.vrs_render(self.ctx, sc, len(scenes), vs, cm, fv, n_views, C.byref(o), _ptr(out),
                                        _ptr(low), int(save), _stream(stream)))
        return out

    def render_two_pass(self, scenes, view_scene, cams, foveas, cfg: RenderConfig | None = None, out=None,
                        stream=None) -> torch.Tensor:
        """The two-pass foveated baseline (full-resolution centre square + half-resolution
        view, blended), for comparison with the single-pass render."""
        cfg = cfg or RenderConfig(fovea_mode="bilinear")
        n_views = len(cams)
        W, H = int(cams[0].width), int(cams[0].height)
        if out is None:
            out = torch.empty((n_views, 3, H, W), device="cuda", dtype=torch.float32)
        sc, vs, cm, fv, o = self._marshal(scenes, view_scene, cams, foveas, cfg)
        self.generation += 1
        self._check(self.lib.vrs_render_two_pass(self.ctx, sc, len(scenes), vs, cm, fv, n_views, C.byref(o), _ptr(out),
                                                 _stream(stream)))
        return out

    def render_stereo_reuse(self, scene, cams, far_distance: float, cfg: RenderConfig | None = None, out=None,
                            stream=None) -> torch.Tensor:
        """Stereo pair with distant content rendered once (vrs_render_stereo_reuse): the
        Gaussians at distance >= far_distance from the cyclopean eye form a far layer
        rendered from the cyclopean camera, composited behind each eye's near layer."""
        cfg = cfg or RenderConfig()
        W, H = int(cams[0].width), int(cams[0].height)
        if out is None:
            out = torch.empty((2, 3, H, W), device="cuda", dtype=torch.float32)
        sc = scene.c()
        cm = (_lib.Camera * 2)(*[camera_c(c) for c in cams])
        o = cfg.opts()
        self.generation += 1
        self._check(self.lib.vrs_render_stereo_reuse(self.ctx, C.byref(sc), cm, C.byref(o), float(far_distance),
                                                     _ptr(out), _stream(stream)))
        return out

    def backward(self, scenes, view_scene, cams, foveas, cfg: RenderConfig, dL_dout: torch.Tensor, grads,
                 stream=None, visible=None):
        sc, vs, cm, fv, o = self._marshal(scenes, view_scene, cams, foveas, cfg, visible)
        gr = (_lib.GaussianGrads * len(grads))(*[_lib.GaussianGrads(*[_ptr(t) for t in g.tensors()]) for g in grads])
        self._check(self.lib.vrs_render_backward(self.ctx, sc, len(scenes), vs, cm, fv, len(cams), C.byref(o),
                                                 _ptr(dL_dout.contiguous()), gr, _stream(stream)))

    def check(self, stream=None) -> int:
        need = C.c_int64()
        self._check(self.lib.vrs_check_status(self.ctx, _stream(stream), C.byref(need)))
        return int(need.value)

    def stats(self, stream=None) -> dict:
        out = (C.c_int64 * 8)()
        self._check(self.lib.vrs_get_stats(self.ctx, _stream(stream), out))
        return dict(zip(["instances", "work_items", "evaluated", "kept", "blended", "views", "sort_passes",
                         "kernels"], [int(v) for v in out[:8]]))

    def instances(self, n_views: int, tiles_per_view: int, stream=None):
        n = C.c_int64()
        cap = max(self.stats(stream)["instances"], 1)
        keys = torch.empty(cap, dtype=torch.int64, device="cuda")
        vals = torch.empty(cap, dtype=torch.int32, device="cuda")
        ranges = torch.empty((n_views * tiles_per_view, 2), dtype=torch.int32, device="cuda")
        self._check(self.lib.vrs_copy_instances(self.ctx, _ptr(keys), _ptr(vals), _ptr(ranges), cap, C.byref(n),
                                                _stream(stream)))
        m = int(n.value)
        return keys[:m], vals[:m], ranges

    def test_bounded_wait(self, which: int, stream=None):
        """Runs a bounded device wait (0: sort look-back, 1: network mbarrier) against a
        flag nothing sets; the next check() raises the timeout status."""
        self._check(self.lib.vrs_test_bounded_wait(self.ctx, int(which), _stream(stream)))

    def probe_orders(self, probes: torch.Tensor, max_len: int = 256, stream=None):
        """Blend order of single rays of the last render (exact or global sort modes):
        probes [n, 3] float32 (view, x, y) on the device -> (ids [n, max_len] int32,
        depth [n, max_len] float32, length [n] int32; -1 for a probe outside its view)."""
        probes = probes.to(torch.float32).contiguous()
        n = probes.shape[0]
        ids = torch.full((n, max_len), -1, dtype=torch.int32, device=probes.device)
        depth = torch.zeros((n, max_len), dtype=torch.float32, device=probes.device)
        length = torch.zeros(n, dtype=torch.int32, device=probes.device)
        self._check(self.lib.vrs_probe_orders(self.ctx, _ptr(probes), n, max_len, _ptr(ids), _ptr(depth),
                                              _ptr(length), _stream(stream)))
        return ids, depth, length

    def update_views(self, cams, foveas=None, cfg: RenderConfig | None = None, visible=None):
        """New cameras / gaze for the next replay of a captured render (same view count;
        visibility masks present exactly where the captured render had them)."""
        cfg = cfg or RenderConfig()
        n = len(cams)
        masks = _check_masks(visible, cams)
        cm = (_lib.Camera * n)(*[camera_c(c) for c in cams])
        mode = FOVEA_MODES[cfg.fovea_mode]
        fv = None
        if foveas or visible is not None:
            fv = (_lib.Fovea * n)(*[fovea_c(foveas[k] if foveas else None, mode, cfg.focus_tile, masks[k])
                                    for k in range(n)])
        self._check(self.lib.vrs_update_views(self.ctx, cm, fv, n))

    def set_tuning(self, max_render_ctas_per_sm: int = 0):
        self._check(self.lib.vrs_set_tuning(self.ctx, int(max_render_ctas_per_sm)))

    STAGES = ["preprocess", "scan", "duplicate", "sort", "ranges_workitems", "render", "composite", "total"]

    def profile_begin(self, max_calls: int):
        self._check(self.lib.vrs_profile_begin(self.ctx, int(max_calls)))

    def profile_end(self, stream=None) -> tuple[dict, int]:
        ms = (C.c_double * 8)()
        n = C.c_int64()
        self._check(self.lib.vrs_profile_end(self.ctx, _stream(stream), ms, C.byref(n)))
        return dict(zip(self.STAGES, [float(v) for v in ms])), int(n.value)

    def project(self, scene: DeviceScene, cam, key_tile: int = 16, stream=None):
        out = torch.empty((scene.n, 24), device="cuda", dtype=torch.float32)
        bbox = torch.empty((scene.n, 4), device="cuda", dtype=torch.float32)
        cnt = torch.empty(scene.n, device="cuda", dtype=torch.int32)
        g = scene.c()
        cm = camera_c(cam)
        self._check(self.lib.vrs_project(self.ctx, C.byref(g), C.byref(cm), key_tile, _ptr(out), _ptr(bbox), _ptr(cnt),
                                         _stream(stream)))
        return out, bbox, cnt

    def sort_pairs(self, keys: torch.Tensor, vals: torch.Tensor, bits: int, stream=None):
        n = keys.numel()
        ko = torch.empty_like(keys)
        vo = torch.empty_like(vals)
        self._check(self.lib.vrs_sort_pairs(self.ctx, _ptr(keys.contiguous()), _ptr(vals.contiguous()), _ptr(ko),
                                            _ptr(vo), n, bits, _stream(stream)))
        return ko, vo

    def loss(self, img: torch.Tensor, target: torch.Tensor, want_grad: bool = True, stream=None):
        img, target = img.contiguous(), target.contiguous()
        n, _, H, W = img.shape
        loss = torch.empty(1, device="cuda", dtype=torch.float32)
        grad = torch.empty_like(img) if want_grad else None
        self._check(self.lib.vrs_loss_l1_ssim(self.ctx, _ptr(img), _ptr(target), n, H, W, _ptr(loss), _ptr(grad),
                                              _stream(stream)))
        return loss, grad


def adam_step(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, lr: float, step: int,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15, stream=None):
    lib = _lib.load()
    st = lib.vrs_adam_step(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), lr, beta1, beta2, eps, step,
                           _stream(stream))
    if st != 0:
        raise VrsError(st, "vrs_adam_step failed")


def measure_peaks(stream=None) -> dict:
    """Measured FP32 FMA, exp2f and logic throughputs and L2 / HBM read bandwidths of the
    current device (vrs_measure_peaks), with its SM count, maximum SM clock and L2 size."""
    lib = _lib.load()
    p = _lib.Peaks()
    st = lib.vrs_measure_peaks(C.byref(p), _stream(stream))
    if st != 0:
        raise VrsError(st, "vrs_measure_peaks failed")
    return {name: getattr(p, name) for name, _ in p._fields_}


class RenderFunction(torch.autograd.Function):
    """Differentiable render of one scene (fine-tuning through the rasterizer).

    Forward calls vrs_render with save_for_backward; backward calls vrs_render_backward
    on the same Renderer, which replays the lists and samples the context saved.  So the
    backward must run before that renderer renders again (the usual forward -> loss ->
    backward order); a backward after another render on the same Renderer raises instead
    of returning the gradients of the other render.  Use one Renderer per differentiable
    render that must stay live (e.g. several loss terms before one backward)."""

    @staticmethod
    def forward(ctx, renderer, cfg, cams, foveas, sh_degree, mean, log_scale, quat, opacity_logit, sh):
        ds = DeviceScene(mean.detach().contiguous(), log_scale.detach().contiguous(), quat.detach().contiguous(),
                         opacity_logit.detach().contiguous(), sh.detach().contiguous(), sh_degree)
        out = renderer.render([ds], [0] * len(cams), cams, foveas, cfg, save=True)
        ctx.renderer, ctx.cfg, ctx.cams, ctx.foveas, ctx.ds = renderer, cfg, cams, foveas, ds
        ctx.generation = renderer.generation
        return out

    @staticmethod
    def backward(ctx, gout):
        if ctx.renderer.generation != ctx.generation:
            raise RuntimeError("the Renderer rendered again after this differentiable render: its saved lists and "
                               "samples now belong to another frame (use one Renderer per live render)")
        g = ctx.ds.zeros_like()
        ctx.renderer.backward([ctx.ds], [0] * len(ctx.cams), ctx.cams, ctx.foveas, ctx.cfg, gout.contiguous(), [g])
        return (None, None, None, None, None, *g.tensors())


def render_differentiable(renderer: Renderer, params: dict, sh_degree: int, cams, foveas=None,
                          cfg: RenderConfig | None = None) -> torch.Tensor:
    """params: dict of CUDA float32 tensors mean, log_scale, quat, opacity_logit, sh."""
    return RenderFunction.apply(renderer, cfg or RenderConfig(), cams, foveas, sh_degree, params["mean"],
                                params["log_scale"], params["quat"], params["opacity_logit"], params["sh"])


class LossFunction(torch.autograd.Function):
    """0.8 L1 + 0.2 (1 - SSIM) computed (with its gradient) by vrs_loss_l1_ssim."""

    @staticmethod
    def forward(ctx, renderer, img, target):
        loss, grad = renderer.loss(img.detach(), target.detach(), want_grad=True)
        ctx.save_for_backward(grad)
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return None, grad * g, None


def l1_ssim_loss(renderer: Renderer, img: torch.Tensor, target: torch.Tensor) -> torch.Tensor:
    return LossFunction.apply(renderer, img, target)


def average_gradients(flat: torch.Tensor, dist) -> None:
    """Data-parallel fine-tuning over views: every rank renders its own views of the same
    scene, and the mean of the ranks' gradients (one all-reduce of the flat gradient
    buffer, then a scale by 1 / world size) is the gradient of the loss averaged over all
    the views, so every rank's Adam step stays identical.  No-op without a group."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return
    dist.all_reduce(flat, op=dist.ReduceOp.SUM)
    flat.mul_(1.0 / dist.get_world_size())


class Adam:
    """Adam on CUDA float32 tensors, stepped by vrs_adam_step (one kernel per tensor)."""

    def __init__(self, params: dict, lrs: dict, beta1=0.9, beta2=0.999, eps=1e-15):
        self.params, self.lrs = params, lrs
        self.m = {k: torch.zeros_like(v) for k, v in params.items()}
        self.v = {k: torch.zeros_like(v) for k, v in params.items()}
        self.t = 0
        self.b1, self.b2, self.eps = beta1, beta2, eps

    def step(self, grads: dict):
        self.t += 1
        for k, p in self.params.items():
            g = grads[k]
            if g is None:
                continue
            adam_step(p, g.contiguous(), self.m[k], self.v[k], self.lrs.get(k, 0.0), self.t, self.b1, self.b2, self.eps)


class GraphedRender:
    """One vrs_render over many scenes and views (a single persistent render launch)
    captured in a CUDA graph; replay() re-renders with new cameras and gaze.

    The workspace is sized by an eager render first (instance count x headroom); a replay
    whose instances exceed it raises VRS_ERR_CAPACITY at the next check()."""

    def __init__(self, renderer: Renderer, scenes, view_scene, cams, foveas, cfg: RenderConfig,
                 headroom: float = 1.3, instances: int | None = None, visible=None):
        """instances: instance capacity to reserve (e.g. the largest count over a known
        camera path); default: the count of this first render x headroom."""
        self.R, self.scenes, self.view_scene, self.cfg = renderer, scenes, list(view_scene), cfg
        self.visible = visible  # fixed per eye: every replay reads the same masks
        n_views = len(cams)
        W, H = int(cams[0].width), int(cams[0].height)
        self.out = torch.empty((n_views, 3, H, W), device="cuda", dtype=torch.float32)
        renderer.render(scenes, self.view_scene, cams, foveas, cfg, out=self.out, visible=visible)
        renderer.check()
        need = renderer.stats()["instances"]
        total = sum(scenes[v].n for v in self.view_scene)
        cap = int(instances) if instances is not None else int(need * headroom) + (1 << 16)
        renderer.reserve(n_views, W, H, total, max(cap, need))
        renderer.render(scenes, self.view_scene, cams, foveas, cfg, out=self.out, visible=visible)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        self.stream = torch.cuda.Stream()
        with torch.cuda.graph(self.graph, stream=self.stream):
            renderer.render(scenes, self.view_scene, cams, foveas, cfg, out=self.out, stream=self.stream,
                            visible=visible)

    def replay(self, cams=None, foveas=None) -> torch.Tensor:
        if cams is not None:
            self.R.update_views(cams, foveas, self.cfg, visible=self.visible)
        self.R.generation += 1
        self.graph.replay()
        return self.out
