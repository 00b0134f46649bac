"""Learned periphery: training and evaluation of the BF16 periphery network.

Everything numeric runs in libvrsplat kernels (rendering of the training pairs, the
network's forward and backward, the MSE loss, Adam, and the fused tensor-core inference
over a frame's periphery tiles); this module orders the calls.

Pairs: for a seeded head pose and a 32-aligned crop of the 2064x2208 eye image (a crop is
the same camera with its principal point shifted, so every pixel keeps its ray), the
input is the foveated render with every tile in the periphery (its half-resolution image
upsampled bilinearly, i.e. the network's input x) and the target the plain full-
resolution render.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib, api, synth

NET_PARAMS = 11011
OFF = {"w1": (0, (32, 3, 3, 3)), "b1": (864, (32,)), "w2": (896, (32, 32, 3, 3)), "b2": (10112, (32,)),
       "w3": (10144, (3, 32, 3, 3)), "b3": (11008, (3,))}


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _s():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class PeripheryNet:
    """Parameters (float master copy, CUDA) of the 3 -> 32 -> 32 -> 3 residual network."""

    def __init__(self, renderer: api.Renderer, seed: int = 0, zero_last: bool = False, last_scale: float = 0.1):
        self.R = renderer
        rng = np.random.default_rng(seed)
        p = np.zeros(NET_PARAMS, np.float32)
        for name, (o, shape) in OFF.items():
            if name.startswith("w"):
                fan_in = shape[1] * 9
                w = rng.normal(0.0, math.sqrt(2.0 / fan_in), size=shape)
                if name == "w3":
                    w *= 0.0 if zero_last else last_scale
                p[o:o + w.size] = w.ravel()
        self.params = torch.tensor(p, device="cuda")
        self.grad = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0

    def numpy_weights(self) -> dict:
        p = self.params.cpu().numpy().astype(np.float64)
        return {k: p[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in OFF.items()}

    def forward(self, x: torch.Tensor, save: bool = True):
        x = x.contiguous()
        B, _, H, W = x.shape
        y = torch.empty_like(x)
        acts = torch.empty((B, 2, H, W, 32), dtype=torch.int16, device="cuda") if save else None
        self.R._check(self.R.lib.vrs_net_forward(self.R.ctx, _p(self.params), _p(x), B, H, W, _p(y), _p(acts), _s()))
        return y, acts

    def backward(self, x: torch.Tensor, acts: torch.Tensor, dy: torch.Tensor):
        B, _, H, W = x.shape
        self.R._check(self.R.lib.vrs_net_backward(self.R.ctx, _p(self.params), _p(x.contiguous()), _p(acts),
                                                  _p(dy.contiguous()), B, H, W, _p(self.grad), _s()))

    def mse(self, y: torch.Tensor, t: torch.Tensor, want_grad: bool = True):
        loss = torch.empty(1, device="cuda")
        dy = torch.empty_like(y) if want_grad else None
        self.R._check(self.R.lib.vrs_mse(self.R.ctx, _p(y.contiguous()), _p(t.contiguous()), y.numel(), _p(loss),
                                         _p(dy), _s()))
        return loss, dy

    def step(self, lr: float):
        self.t += 1
        api.adam_step(self.params, self.grad, self.m, self.v, lr, self.t, 0.9, 0.999, 1e-8)
        self.grad.zero_()

    def apply_periphery(self, low: torch.Tensor, out: torch.Tensor):
        """After Renderer.render(..., fovea_mode='net', low=low, out=out)."""
        self.R._check(self.R.lib.vrs_net_periphery(self.R.ctx, _p(self.params), _p(low), _p(out), _s()))
        return out


def crop_camera(cam, x0, y0, w, h):
    return synth.Camera(cam.world_to_cam, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.near_z)


def random_pose_camera(rng, width=2064, height=2208, hfov=110.0):
    yaw = rng.uniform(-math.pi, math.pi)
    pitch = rng.uniform(-0.3, 0.3)
    pos = rng.normal(0.0, 0.1, 3)
    f = synth.focal_for_hfov(width, hfov)
    return synth.camera_from_pose(synth.head_rotation(yaw, pitch), pos, width, height, f)


ALL_PERIPHERY = synth.Fovea(-1e6, -1e6, 1.0, 1.0)


def make_pairs(renderer: api.Renderer, scene: api.DeviceScene, n_pairs: int, rng, crop: int = 256,
               width: int = 2064, height: int = 2208, windows=(4, 8, 16), sort_mode: str = "exact"):
    """-> (x, target) float32 CUDA tensors [n_pairs, 3, crop, crop].  Training pairs use
    the exact per-ray order by default, so that the target differs from the input only by
    what upsampling loses (the hierarchical approximation's order differs between 32x32
    periphery and 16x16 plain tiles and would add noise the network cannot predict)."""
    xs = torch.empty((n_pairs, 3, crop, crop), device="cuda")
    ts = torch.empty_like(xs)
    fov_cfg = api.RenderConfig(sort_mode=sort_mode, windows=windows, key_tile=32, fovea_mode="bilinear")
    plain_cfg = api.RenderConfig(sort_mode=sort_mode, windows=windows, key_tile=16, fovea_mode="plain")
    for i in range(n_pairs):
        cam = random_pose_camera(rng, width, height)
        x0 = int(rng.integers(0, (width - crop) // 32 + 1)) * 32
        y0 = int(rng.integers(0, (height - crop) // 32 + 1)) * 32
        c = crop_camera(cam, x0, y0, crop, crop)
        renderer.render([scene], [0], [c], [ALL_PERIPHERY], fov_cfg, out=xs[i:i + 1])
        renderer.render([scene], [0], [c], None, plain_cfg, out=ts[i:i + 1])
    renderer.check()
    return xs, ts


def train(net: PeripheryNet, xs: torch.Tensor, ts: torch.Tensor, steps: int, batch: int = 8, lr: float = 1e-3,
          seed: int = 0):
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = xs.shape[0]
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).cuda()
        x, t = xs[idx].contiguous(), ts[idx].contiguous()
        y, acts = net.forward(x)
        loss, dy = net.mse(y, t)
        net.backward(x, acts, dy)
        warm = min(1.0, (s + 1) / max(1, steps // 10))
        net.step(lr * warm * (0.5 * (1 + math.cos(math.pi * s / steps))))
        losses.append(loss)
    return torch.cat(losses).cpu().numpy()


def psnr(mse: float) -> float:
    return float("inf") if mse <= 0 else 10.0 * math.log10(1.0 / mse)


def evaluate_frames(renderer: api.Renderer, net: PeripheryNet, scene: api.DeviceScene, frames, windows=(4, 8, 16),
                    sort_mode: str = "hier"):
    """Per-frame PSNR / max abs error of the learned and the bilinear periphery against
    the plain full-resolution render, on periphery pixels and on the whole frame.  With
    sort_mode "exact" the three renders share the exact per-ray order, so the periphery's
    error is what reconstruction from the half-resolution samples loses; with "hier" the
    foveated frame (32x32 key tiles, 4x4 blocks of half-resolution groups) and the plain
    render (16x16 key tiles, 4x4 blocks of pixels) also differ by their hierarchical
    windows' approximation."""
    fov_cfg = api.RenderConfig(sort_mode=sort_mode, windows=windows, key_tile=32, fovea_mode="bilinear")
    net_cfg = api.RenderConfig(sort_mode=sort_mode, windows=windows, key_tile=32, fovea_mode="net")
    plain_cfg = api.RenderConfig(sort_mode=sort_mode, windows=windows, key_tile=16, fovea_mode="plain")
    acc = {k: [] for k in ["net_periph_mse", "bil_periph_mse", "net_frame_mse", "bil_frame_mse", "net_periph_max",
                           "bil_periph_max"]}
    for fr in frames:
        W, H = fr.cameras[0].width, fr.cameras[0].height
        plain = renderer.render([scene], [0, 0], fr.cameras, None, plain_cfg).clone()
        bil = renderer.render([scene], [0, 0], fr.cameras, fr.foveas, fov_cfg).clone()
        low = torch.empty((2, 3, H // 2, W // 2), device="cuda")
        out = renderer.render([scene], [0, 0], fr.cameras, fr.foveas, net_cfg, low=low)
        net.apply_periphery(low, out)
        # periphery mask from the tile classes the render used (recomputed here from the
        # bilinear / net difference would be circular): pixels whose 32x32 tile lies
        # entirely outside radius + band
        mask = periphery_mask(fr, W, H).cuda()
        for name, img in (("net", out), ("bil", bil)):
            d = img - plain
            acc[f"{name}_frame_mse"].append(float((d ** 2).mean()))
            dm = d.abs().amax(dim=1)[mask]
            acc[f"{name}_periph_mse"].append(float((d ** 2).permute(1, 0, 2, 3)[:, mask].mean()))
            acc[f"{name}_periph_max"].append(float(dm.max()))
    res = {k: float(np.mean(v)) if "mse" in k else float(np.max(v)) for k, v in acc.items()}
    for k in ["net_periph", "bil_periph", "net_frame", "bil_frame"]:
        res[k + "_psnr_db"] = psnr(res[k + "_mse"])
    return res


def periphery_mask(frame, W, H) -> torch.Tensor:
    """[2, H, W] bool: pixels of 32x32 tiles whose pixel centres are all at distance >=
    radius + band from the gaze point (the periphery class)."""
    masks = []
    for fv in frame.foveas:
        ty, tx = np.mgrid[0:(H + 31) // 32, 0:(W + 31) // 32]
        x0, y0 = tx * 32 + 0.5, ty * 32 + 0.5
        x1, y1 = np.minimum((tx + 1) * 32, W) - 0.5, np.minimum((ty + 1) * 32, H) - 0.5
        nx = np.clip(np.float32(fv.gaze_x), x0, x1) - np.float32(fv.gaze_x)
        ny = np.clip(np.float32(fv.gaze_y), y0, y1) - np.float32(fv.gaze_y)
        per = np.sqrt(nx * nx + ny * ny) >= np.float32(fv.radius_px) + np.float32(fv.band_px)
        m = np.repeat(np.repeat(per, 32, 0), 32, 1)[:H, :W]
        masks.append(m)
    return torch.tensor(np.stack(masks))
