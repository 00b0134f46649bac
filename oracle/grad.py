"""Gradient oracle: the forward definition restated in float64 PyTorch, differentiated by
autograd.  TEST INFRASTRUCTURE ONLY.

The paper fine-tunes positions, rotations, scales, opacities and SH coefficients through
the StopThePop + Optimal-Projection renderer (Sec. 4.1, 4.2; Sec. 5 "fine-tuned for 5K
iterations").  Sorting, culling and windowing are piecewise constant, so the gradient of
an image is the gradient of Eq. 2 with the blend order of every sample held fixed.  The
C oracle supplies those orders; this module recomputes every per-pair alpha and colour
from the parameters with the same formulas and lets autograd differentiate them.
"""
from __future__ import annotations

import math

import numpy as np
import torch

ALPHA_MAX = 0.99
DILATION_PX2 = 0.3


def params_from_scene(scene, requires_grad: bool = True) -> dict:
    p = {k: torch.tensor(np.asarray(v, dtype=np.float64), requires_grad=requires_grad)
         for k, v in zip(["mean", "log_scale", "quat", "opacity_logit", "sh"], scene.arrays())}
    return p


def sh_basis(degree: int, d: torch.Tensor) -> torch.Tensor:
    """Real SH basis in the 3DGS sign convention; d is [3, M] unit vectors -> [K, M]."""
    x, y, z = d[0], d[1], d[2]
    s = 1.0 / math.sqrt(math.pi)
    out = [0.5 * s * torch.ones_like(x)]
    if degree >= 1:
        c1 = 0.5 * math.sqrt(3.0) * s
        out += [-c1 * y, c1 * z, -c1 * x]
    if degree >= 2:
        out += [0.5 * math.sqrt(15.0) * s * x * y, -0.5 * math.sqrt(15.0) * s * y * z,
                0.25 * math.sqrt(5.0) * s * (2 * z * z - x * x - y * y),
                -0.5 * math.sqrt(15.0) * s * x * z, 0.25 * math.sqrt(15.0) * s * (x * x - y * y)]
    if degree >= 3:
        out += [-0.25 * math.sqrt(35.0 / 2.0) * s * y * (3 * x * x - y * y),
                0.5 * math.sqrt(105.0) * s * x * y * z,
                -0.25 * math.sqrt(21.0 / 2.0) * s * y * (4 * z * z - x * x - y * y),
                0.25 * math.sqrt(7.0) * s * z * (2 * z * z - 3 * x * x - 3 * y * y),
                -0.25 * math.sqrt(21.0 / 2.0) * s * x * (4 * z * z - x * x - y * y),
                0.25 * math.sqrt(105.0) * s * z * (x * x - y * y),
                -0.25 * math.sqrt(35.0 / 2.0) * s * x * (x * x - 3 * y * y)]
    return torch.stack(out)


def _cam_numbers(cam):
    w2c = torch.tensor(np.asarray(cam.world_to_cam, dtype=np.float32).astype(np.float64))
    f = lambda v: float(np.float32(v))
    return w2c[:, :3], w2c[:, 3], f(cam.fx), f(cam.fy), f(cam.cx), f(cam.cy)


def project(p: dict, sh_degree: int, cam, idx: torch.Tensor) -> dict:
    """Optimal-Projection quantities of the Gaussians idx (all assumed valid)."""
    Rw, t, fx, fy, cx, cy = _cam_numbers(cam)
    m = p["mean"][:, idx]
    ls = p["log_scale"][:, idx]
    q = p["quat"][:, idx]
    q = q / torch.linalg.norm(q, dim=0, keepdim=True)
    w, x, y, z = q[0], q[1], q[2], q[3]
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)]),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)]),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]),
    ])  # [3, 3, M]
    R = R.permute(2, 0, 1)  # [M, 3, 3]
    Rc = torch.einsum("ab,mbc->mac", Rw, R)
    S2 = torch.exp(2 * ls).T  # [M, 3]
    Si2 = torch.exp(-2 * ls).T
    Sc = torch.einsum("mak,mk,mbk->mab", Rc, S2, Rc)
    Sci = torch.einsum("mak,mk,mbk->mab", Rc, Si2, Rc)
    mu = (Rw @ m).T + t  # [M, 3]
    d = torch.linalg.norm(mu, dim=1)
    u = mu / d[:, None]
    rho = torch.sqrt(u[:, 0] ** 2 + u[:, 2] ** 2)
    e1 = torch.stack([u[:, 2] / rho, torch.zeros_like(rho), -u[:, 0] / rho], dim=1)
    e2 = torch.linalg.cross(u, e1, dim=1)
    E = torch.stack([e1, e2], dim=1)  # [M, 2, 3]
    Sp = torch.einsum("mak,mkl,mbl->mab", E, Sc, E) / (d * d)[:, None, None]
    Sp = Sp + (DILATION_PX2 / (fx * fy)) * torch.eye(2, dtype=Sp.dtype)
    det = Sp[:, 0, 0] * Sp[:, 1, 1] - Sp[:, 0, 1] * Sp[:, 1, 0]
    A = torch.stack([torch.stack([Sp[:, 1, 1], -Sp[:, 0, 1]], 1),
                     torch.stack([-Sp[:, 1, 0], Sp[:, 0, 0]], 1)], 1) / det[:, None, None]
    sigma = torch.sigmoid(p["opacity_logit"][idx])
    dirw = (Rw.T @ u.T)  # [3, M]
    Y = sh_basis(sh_degree, dirw)  # [K, M]
    K = (sh_degree + 1) ** 2
    sh = p["sh"][:K][:, :, idx]  # [K, 3, M]
    rgb = torch.clamp_min(torch.einsum("km,kcm->cm", Y, sh) + 0.5, 0.0).T  # [M, 3]
    return dict(mu=mu, u=u, E=E, A=A, sigma=sigma, rgb=rgb, Sci=Sci,
                fx=fx, fy=fy, cx=cx, cy=cy)


def alpha_at(pr: dict, j: torch.Tensor, px: torch.Tensor, py: torch.Tensor) -> torch.Tensor:
    """alpha = min(0.99, sigma exp(-1/2 s^T A s)) of projected Gaussian rows j at samples."""
    v = torch.stack([(px - pr["cx"]) / pr["fx"], (py - pr["cy"]) / pr["fy"], torch.ones_like(px)], 1)
    u, E, A = pr["u"][j], pr["E"][j], pr["A"][j]
    w = (u * v).sum(1)
    s = torch.einsum("mak,mk->ma", E, v) / w[:, None]
    q = torch.einsum("ma,mab,mb->m", s, A, s)
    return torch.clamp_max(pr["sigma"][j] * torch.exp(-0.5 * q), ALPHA_MAX)


def sample_positions(W: int, H: int):
    """Continuous positions of every sample index: full-res pixels, then 2x2 groups."""
    ys, xs = np.mgrid[0:H, 0:W]
    W2, H2 = W // 2, H // 2
    gy, gx = np.mgrid[0:H2, 0:W2]
    px = np.concatenate([xs.ravel() + 0.5, 2.0 * gx.ravel() + 1.0])
    py = np.concatenate([ys.ravel() + 0.5, 2.0 * gy.ravel() + 1.0])
    return px, py


def blend_samples(p: dict, sh_degree: int, cam, orders, bg=(0.0, 0.0, 0.0)):
    """Eq. 2 at every sample with the fixed blend orders -> (C [S, 3], T [S])."""
    order, off = orders
    W, H = int(cam.width), int(cam.height)
    nsamp = len(off) - 1
    lens = np.diff(off)
    L = int(lens.max()) if nsamp else 0
    gids = np.unique(order)
    row = np.full(int(p["mean"].shape[1]), -1, np.int64)
    row[gids] = np.arange(len(gids))
    pr = project(p, sh_degree, cam, torch.tensor(gids))
    px, py = sample_positions(W, H)
    sidx = np.repeat(np.arange(nsamp), lens)
    kpos = np.arange(len(order)) - np.repeat(off[:-1], lens)
    j = torch.tensor(row[order])
    a = alpha_at(pr, j, torch.tensor(px[sidx]), torch.tensor(py[sidx]))
    one_minus = torch.ones(nsamp, max(L, 1), dtype=torch.float64)
    one_minus = one_minus.index_put((torch.tensor(sidx), torch.tensor(kpos)), 1.0 - a)
    Tincl = torch.cumprod(one_minus, dim=1)
    Texcl = torch.cat([torch.ones(nsamp, 1, dtype=torch.float64), Tincl[:, :-1]], 1)
    Tj = Texcl[torch.tensor(sidx), torch.tensor(kpos)]
    contrib = (a * Tj)[:, None] * pr["rgb"][j]
    C = torch.zeros(nsamp, 3, dtype=torch.float64).index_add(0, torch.tensor(sidx), contrib)
    T = Tincl[:, -1]
    return C, T


def fovea_weight(px, py, fovea):
    d = torch.sqrt((px - float(np.float32(fovea.gaze_x))) ** 2 + (py - float(np.float32(fovea.gaze_y))) ** 2)
    R, b = float(np.float32(fovea.radius_px)), float(np.float32(fovea.band_px))
    return torch.clamp((R + b - d) / b, 0.0, 1.0)


def image_from_samples(C, T, cam, tile_class=None, fovea=None, bg=(0.0, 0.0, 0.0), key_tile=32):
    """Compose the output image from sample colours (plain, or single-pass foveated).
    A tile class with 4 added marks a tile without visible pixels (visibility culling,
    Sec. 4.3): its samples render nothing and its pixels are the background constant."""
    W, H = int(cam.width), int(cam.height)
    bgt = torch.tensor([float(np.float32(b)) for b in bg], dtype=torch.float64)
    val = C + T[:, None] * bgt  # [S, 3]
    full = val[: W * H].T.reshape(3, H, W)
    if fovea is None:  # samples of invisible tiles have empty orders: C = 0, T = 1, i.e. bg
        return full
    W2, H2 = W // 2, H // 2
    grp = val[W * H:].T.reshape(3, H2, W2)
    cls_all = np.repeat(np.repeat(np.asarray(tile_class), key_tile, 0), key_tile, 1)[:H, :W]
    invisible = (cls_all & 4) != 0
    cls = cls_all & 3
    cls_g = cls[0::2, 0::2]
    avg = full.reshape(3, H2, 2, W2, 2).mean(dim=(2, 4))
    lowimg = torch.where(torch.tensor(cls_g == 2)[None], grp, avg)
    ys, xs = np.mgrid[0:H, 0:W]
    w = fovea_weight(torch.tensor(xs + 0.5), torch.tensor(ys + 0.5), fovea)
    up_avg = lowimg.repeat_interleave(2, 1).repeat_interleave(2, 2)
    hybrid = w[None] * full + (1 - w[None]) * up_avg
    up = bilinear_up2(lowimg)
    c = torch.tensor(cls)[None]
    img = torch.where(c == 0, full, torch.where(c == 1, hybrid, up))
    return torch.where(torch.tensor(invisible)[None], bgt[:, None, None].expand(3, H, W), img)


def bilinear_up2(L: torch.Tensor) -> torch.Tensor:
    """x2 bilinear upsampling, half-pixel aligned, clamp to edge: [C, h, w] -> [C, 2h, 2w]."""
    Cc, h, w = L.shape

    def axis(n):
        u = (np.arange(2 * n) + 0.5) / 2 - 0.5
        i0 = np.floor(u).astype(np.int64)
        f = u - i0
        return np.clip(i0, 0, n - 1), np.clip(i0 + 1, 0, n - 1), f

    ya, yb, fy = axis(h)
    xa, xb, fx = axis(w)
    fx = torch.tensor(fx)[None, None, :]
    fy = torch.tensor(fy)[None, :, None]
    top = (1 - fx) * L[:, ya][:, :, xa] + fx * L[:, ya][:, :, xb]
    bot = (1 - fx) * L[:, yb][:, :, xa] + fx * L[:, yb][:, :, xb]
    return (1 - fy) * top + fy * bot


def render_image(p: dict, sh_degree: int, cam, orders, tile_class=None, fovea=None,
                 bg=(0.0, 0.0, 0.0)):
    C, T = blend_samples(p, sh_degree, cam, orders, bg)
    return image_from_samples(C, T, cam, tile_class, fovea, bg)


def image_grad(scene, cam, orders, dL_dimg: np.ndarray, tile_class=None, fovea=None,
               bg=(0.0, 0.0, 0.0)) -> dict:
    """d<dL_dimg, image>/d(params) with the orders fixed, float64."""
    p = params_from_scene(scene)
    img = render_image(p, scene.sh_degree, cam, orders, tile_class, fovea, bg)
    (img * torch.tensor(dL_dimg, dtype=torch.float64)).sum().backward()
    return {k: v.grad.numpy().copy() if v.grad is not None else np.zeros(v.shape) for k, v in p.items()}
