"""Fine-tuning loss oracle: 0.8 L1 + 0.2 (1 - SSIM), float64.  TEST INFRASTRUCTURE ONLY.

SSIM follows Wang et al. 2004 (the loss 3DGS-style fine-tuning uses, Sec. 5): 11x11
Gaussian window with sigma 1.5, C1 = 0.01^2, C2 = 0.03^2, computed per channel on
windows centred at every pixel with zero padding outside the image, averaged over
pixels and channels.  The zero padding is a reading; the paper does not spell it out.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

C1 = 0.01 ** 2
C2 = 0.03 ** 2
WIN = 11
SIGMA = 1.5
LAMBDA_SSIM = 0.2


def gaussian_1d(size: int = WIN, sigma: float = SIGMA) -> torch.Tensor:
    x = torch.arange(size, dtype=torch.float64) - (size - 1) / 2
    g = torch.exp(-x * x / (2 * sigma * sigma))
    return g / g.sum()


def _filt(x: torch.Tensor) -> torch.Tensor:
    """2D Gaussian window sums per channel, zero padded, same size.  x: [C, H, W]."""
    g = gaussian_1d()
    k = torch.outer(g, g)[None, None].expand(x.shape[0], 1, WIN, WIN)
    return F.conv2d(x[None], k, padding=WIN // 2, groups=x.shape[0])[0]


def ssim_map(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    mx, my = _filt(x), _filt(y)
    sxx = _filt(x * x) - mx * mx
    syy = _filt(y * y) - my * my
    sxy = _filt(x * y) - mx * my
    return ((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2))


def ssim(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    return ssim_map(x, y).mean()


def loss(x: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    return (1 - LAMBDA_SSIM) * (x - y).abs().mean() + LAMBDA_SSIM * (1 - ssim(x, y))


def loss_and_grad(x: np.ndarray, y: np.ndarray):
    """-> (loss, dloss/dx) for images [C, H, W] (or [V, C, H, W], averaged over views)."""
    xt = torch.tensor(np.asarray(x, dtype=np.float64), requires_grad=True)
    yt = torch.tensor(np.asarray(y, dtype=np.float64))
    if xt.dim() == 4:
        L = sum(loss(xt[v], yt[v]) for v in range(xt.shape[0])) / xt.shape[0]
    else:
        L = loss(xt, yt)
    L.backward()
    return float(L.detach()), xt.grad.numpy().copy()


def ssim_brute(x: np.ndarray, y: np.ndarray) -> float:
    """Window-by-window SSIM with explicit loops (small images only)."""
    C_, H, W = x.shape
    g = gaussian_1d().numpy()
    w2 = np.outer(g, g)
    r = WIN // 2
    tot = 0.0
    for c in range(C_):
        xp = np.pad(x[c], r)
        yp = np.pad(y[c], r)
        for i in range(H):
            for j in range(W):
                a = xp[i:i + WIN, j:j + WIN]
                b = yp[i:i + WIN, j:j + WIN]
                mx, my = (w2 * a).sum(), (w2 * b).sum()
                vx = (w2 * a * a).sum() - mx * mx
                vy = (w2 * b * b).sum() - my * my
                cxy = (w2 * a * b).sum() - mx * my
                tot += ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
    return tot / (C_ * H * W)
