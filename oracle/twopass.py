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


def _alts(ref, k):
    """The values of pixel k of a plain render: its own, then its alternatives."""
    off, vals = ref["alt"]
    H, W = ref["image"].shape[1:]
    y, x = divmod(k, W)
    return [ref["image"][:, y, x]] + [vals[j] for j in range(off[k], off[k + 1])]


def render(scene, cam, fovea, mode: str = "hier", windows=(4, 8, 16), bg=(0.0, 0.0, 0.0),
           outcomes: bool = False) -> dict:
    """-> dict(image [3, H, W], centre, low, rect, marginal [H, W]); with outcomes, also
    the outcome sets of the composed image ("alt", "unchecked", as native.render): every
    combination of the valid values of the centre pixel and of the four half-resolution
    pixels it reads, through the same blend."""
    W, H = int(cam.width), int(cam.height)
    x0, y0, sw, sh = centre_rect(W, H, fovea)
    c = on.render(scene, crop_camera(cam, x0, y0, sw, sh), mode, windows=windows, key_tile=16, bg=bg,
                  outcomes=outcomes)
    lo = on.render(scene, half_camera(cam), mode, windows=windows, key_tile=16, bg=bg, outcomes=outcomes)
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
    out = dict(image=img, centre=c["image"], low=lo["image"], rect=(x0, y0, sw, sh), marginal=marg)
    if outcomes:
        W2 = W // 2
        ncen = np.diff(c["alt"][0]).reshape(sh, sw)
        nlow = np.diff(lo["alt"][0]).reshape(H // 2, W2)
        unchecked = np.zeros((H, W), bool)
        alt_lists = {}
        for y in range(H):
            for x in range(W):
                wv = w[y, x]
                inside = x0 <= x < x0 + sw and y0 <= y < y0 + sh
                taps = [(ya[y], xa[x]), (ya[y], xb[x]), (yb[y], xa[x]), (yb[y], xb[x])]
                fx = (x + 0.5) / 2 - 0.5 - ux[x]
                fy = (y + 0.5) / 2 - 0.5 - uy[y]
                bw = [(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy]
                need_c = inside and wv > 0 and ncen[y - y0, x - x0] > 0
                need_l = wv < 1 and any(nlow[t] > 0 for t in taps)
                if not (need_c or need_l):
                    continue
                if (inside and wv > 0 and c["unchecked"][y - y0, x - x0]) or \
                        (wv < 1 and any(lo["unchecked"][t] for t in taps)):
                    unchecked[y, x] = True
                    continue
                cs = _alts(c, (y - y0) * sw + (x - x0)) if inside and wv > 0 else [np.zeros(3)]
                ls = [_alts(lo, t[0] * W2 + t[1]) if wv < 1 else [np.zeros(3)] for t in taps]
                if len(cs) * np.prod([len(l) for l in ls]) > 4096:
                    unchecked[y, x] = True
                    continue
                vals = []
                for cv in cs:
                    for l0 in ls[0]:
                        for l1 in ls[1]:
                            for l2 in ls[2]:
                                for l3 in ls[3]:
                                    upv = bw[0] * l0 + bw[1] * l1 + bw[2] * l2 + bw[3] * l3
                                    v = wv * cv + (1.0 - wv) * upv if inside else upv
                                    if np.abs(v - img[:, y, x]).max() > 0:
                                        vals.append(v)
                alt_lists[y * W + x] = vals
        off = np.zeros(W * H + 1, np.int64)
        for k, v in alt_lists.items():
            off[k + 1] = len(v)
        off = np.cumsum(off)
        vals = [v for k in sorted(alt_lists) for v in alt_lists[k]]
        out["alt"] = (off, np.array(vals).reshape(-1, 3))
        out["unchecked"] = unchecked
    return out
