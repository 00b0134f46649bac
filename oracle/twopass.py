"""Two-pass foveated rendering, the paper's comparison baseline (Appendix A), as a
composition of plain oracle renders.  TEST INFRASTRUCTURE ONLY.

Pass 1 renders the centre at full resolution through a tight frustum: the camera cropped
to the square around the gaze that holds the focus disc and its transition band.  Pass 2
renders the whole view at half resolution: half focal length, half principal point,
half size, so that its pixel (i, j) looks along the ray of the full-resolution point
(2i + 1, 2j + 1), the group centre of the single-pass method.  The half-resolution image
is upsampled bilinearly (half-pixel aligned, clamped to the edge) and the two are
blended with the continuous mask w of Sec. 4.3: w * centre + (1 - w) * upsampled.

Readings: the centre square's side is 2 * ceil(radius + band) + 2 pixels (at most the
image size), placed at integer offsets and moved inside the image; outside it w = 0.
Samples of the half-resolution pass whose upsampled value is never used (all four
full-resolution pixels that tap them have w = 1) may be skipped: they do not change the
image.  The half-resolution pass is a render of its own: its 0.3-pixel dilation is in
half-resolution pixels (four times the area of the single-pass group samples'), so its
samples differ slightly from the single-pass periphery samples on the same rays.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import native as on
from .grad import bilinear_up2


def centre_rect(width: int, height: int, fovea) -> tuple[int, int, int, int]:
    """(x0, y0, side_w, side_h) of the full-resolution centre pass."""
    half = math.ceil(float(np.float32(fovea.radius_px)) + float(np.float32(fovea.band_px))) + 1
    sw, sh = min(2 * half, width), min(2 * half, height)
    gx, gy = float(np.float32(fovea.gaze_x)), float(np.float32(fovea.gaze_y))
    x0 = min(max(int(math.floor(gx)) - half, 0), width - sw)
    y0 = min(max(int(math.floor(gy)) - half, 0), height - sh)
    return x0, y0, sw, sh


def crop_camera(cam, x0, y0, w, h):
    c = type(cam)(cam.world_to_cam, cam.fx, cam.fy, cam.cx - x0, cam.cy - y0, w, h, cam.near_z)
    return c


def half_camera(cam):
    return type(cam)(cam.world_to_cam, 0.5 * float(np.float32(cam.fx)), 0.5 * float(np.float32(cam.fy)),
                     0.5 * float(np.float32(cam.cx)), 0.5 * float(np.float32(cam.cy)), cam.width // 2,
                     cam.height // 2, cam.near_z)


def fovea_weight_image(width: int, height: int, fovea) -> np.ndarray:
    ys, xs = np.mgrid[0:height, 0:width]
    gx, gy = float(np.float32(fovea.gaze_x)), float(np.float32(fovea.gaze_y))
    r, b = float(np.float32(fovea.radius_px)), float(np.float32(fovea.band_px))
    d = np.hypot(xs + 0.5 - gx, ys + 0.5 - gy)
    return np.clip((r + b - d) / b, 0.0, 1.0)


def render(scene, cam, fovea, mode: str = "hier", windows=(4, 8, 16), bg=(0.0, 0.0, 0.0)) -> dict:
    """-> dict(image [3, H, W], centre, low, rect, marginal [H, W])."""
    W, H = int(cam.width), int(cam.height)
    x0, y0, sw, sh = centre_rect(W, H, fovea)
    c = on.render(scene, crop_camera(cam, x0, y0, sw, sh), mode, windows=windows, key_tile=16, bg=bg)
    lo = on.render(scene, half_camera(cam), mode, windows=windows, key_tile=16, bg=bg)
    up = bilinear_up2(torch.tensor(lo["image"])).numpy()
    w = fovea_weight_image(W, H, fovea)
    img = up.copy()
    wc = w[y0:y0 + sh, x0:x0 + sw]
    img[:, y0:y0 + sh, x0:x0 + sw] = wc[None] * c["image"] + (1.0 - wc[None]) * up[:, y0:y0 + sh, x0:x0 + sw]
    assert not w[:, :x0].any() and not w[:, x0 + sw:].any() and not w[:y0].any() and not w[y0 + sh:].any()
    # marginal: a marginal centre pixel, or a marginal low sample under a bilinear tap
    lm = lo["marginal"]
    ux = np.floor((np.arange(W) + 0.5) / 2 - 0.5).astype(int)
    uy = np.floor((np.arange(H) + 0.5) / 2 - 0.5).astype(int)
    xa, xb = np.clip(ux, 0, W // 2 - 1), np.clip(ux + 1, 0, W // 2 - 1)
    ya, yb = np.clip(uy, 0, H // 2 - 1), np.clip(uy + 1, 0, H // 2 - 1)
    marg = lm[ya][:, xa] | lm[ya][:, xb] | lm[yb][:, xa] | lm[yb][:, xb]
    marg = marg & (w < 1.0)
    marg[y0:y0 + sh, x0:x0 + sw] |= c["marginal"] & (wc > 0.0)
    return dict(image=img, centre=c["image"], low=lo["image"], rect=(x0, y0, sw, sh), marginal=marg)
