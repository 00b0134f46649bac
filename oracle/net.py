"""Periphery network oracle, float64.  TEST INFRASTRUCTURE ONLY.

The network is not in the paper (which reconstructs the periphery by nearest-neighbour
upsampling and a 3x3 blur, Sec. 4.3); it is the learned replacement the workload asks
for: y = up + conv3(relu(conv2(relu(conv1(up))))), 3 -> 32 -> 32 -> 3 channels, 3x3
kernels, zero padding 1, where up is the x2 bilinear upsampling of the half-resolution
periphery.  Weights, the network input and the two hidden activations are BF16 values;
accumulation is exact here (float64) and FP32 on the GPU.  Rounding to BF16 happens at
the same three places on both sides: the input, and each hidden activation after bias
and ReLU.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

CH = 32


def bf16(x: torch.Tensor) -> torch.Tensor:
    """Round to the nearest BF16 value (ties to even), returned in float64."""
    return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)


def init_weights(rng: np.random.Generator, zero_last: bool = False) -> dict:
    """He-initialised weights (OIHW) and zero biases, BF16-representable."""
    def he(o, i):
        return rng.normal(0, np.sqrt(2.0 / (i * 9)), size=(o, i, 3, 3))
    w = {"w1": he(CH, 3), "b1": np.zeros(CH), "w2": he(CH, CH), "b2": np.zeros(CH),
         "w3": he(3, CH) * (0.0 if zero_last else 0.1), "b3": np.zeros(3)}
    return {k: bf16(torch.tensor(v)).numpy() if k.startswith("w") else v.astype(np.float32).astype(np.float64)
            for k, v in w.items()}


def forward(x: torch.Tensor, w: dict, round_acts: bool = True):
    """x: [B, 3, H, W] float64 network input (already upsampled).  -> (y, (a1, a2)).
    Weights are used as BF16 values (biases as given)."""
    t = {k: (v if torch.is_tensor(v) else torch.tensor(v, dtype=torch.float64)) for k, v in w.items()}
    r = bf16 if round_acts else (lambda z: z)
    if round_acts:
        t = {k: bf16(v) if k.startswith("w") else v for k, v in t.items()}
    xin = r(x)
    a1 = r(F.relu(F.conv2d(xin, t["w1"], t["b1"], padding=1)))
    a2 = r(F.relu(F.conv2d(a1, t["w2"], t["b2"], padding=1)))
    y = x + F.conv2d(a2, t["w3"], t["b3"], padding=1)
    return y, (xin, a1, a2)


def _gamma(n: int, u: float) -> float:
    """Relative error bound of an n-term sum accumulated in floating point with unit
    roundoff u (Higham's gamma_n = n u / (1 - n u))."""
    return n * u / (1.0 - n * u)


def _flip(z: torch.Tensor, D: torch.Tensor) -> torch.Tensor:
    """Largest |bf16(relu(z')) - bf16(relu(z))| over |z' - z| <= D: ReLU and rounding are
    monotone, so the ends of the interval give it."""
    a = bf16(F.relu(z))
    return torch.maximum((bf16(F.relu(z + D)) - a).abs(), (bf16(F.relu(z - D)) - a).abs())


def forward_bound(x: torch.Tensor, w: dict, x_err: float = 0.0, u: float = 2.0 ** -22, moves: bool = False):
    """The float64 forward and, per output, a bound on how far an evaluation that
    accumulates in lower precision (unit roundoff u) and rounds to BF16 at the same three
    places can land from it.

    Layer by layer: a sum of n products carries at most gamma_n (sum |w a| + |b|) of
    accumulation error; a hidden value then rounds to the same BF16 value unless its
    pre-rounding value lies within that distance (plus what changed activations of the
    layer before move it) of a rounding boundary, and the rounded value then moves by at
    most _flip.  The bound of an output adds its accumulation error and |w3| times the
    moves of the activations it reads.  x_err bounds the difference of the other side's
    input (e.g. an FP32 bilinear upsample) from x.  u = 2^-22 leaves two bits for
    accumulation orders (tensor-core trees) coarser than a sequential FP32 sum.
    -> (y, bound), both [B, 3, H, W] float64; with moves, also ((a1, da1), (a2, da2)):
    the hidden activations and their largest moves."""
    t = {k: (v if torch.is_tensor(v) else torch.tensor(v, dtype=torch.float64)) for k, v in w.items()}
    t = {k: bf16(v) if k.startswith("w") else v for k, v in t.items()}
    aw = {k: t[k].abs() for k in ("w1", "w2", "w3")}
    ab = {k: t[k].abs() for k in ("b1", "b2", "b3")}
    xin = bf16(x)
    dxin = torch.maximum((bf16(x + x_err) - xin).abs(), (bf16(x - x_err) - xin).abs())
    z1 = F.conv2d(xin, t["w1"], t["b1"], padding=1)
    D1 = _gamma(28, u) * F.conv2d(xin.abs(), aw["w1"], ab["b1"], padding=1) + F.conv2d(dxin, aw["w1"], padding=1)
    a1 = bf16(F.relu(z1))
    da1 = _flip(z1, D1)
    z2 = F.conv2d(a1, t["w2"], t["b2"], padding=1)
    D2 = _gamma(289, u) * F.conv2d(a1 + da1, aw["w2"], ab["b2"], padding=1) + F.conv2d(da1, aw["w2"], padding=1)
    a2 = bf16(F.relu(z2))
    da2 = _flip(z2, D2)
    y = x + F.conv2d(a2, t["w3"], t["b3"], padding=1)
    bound = (_gamma(290, u) * (F.conv2d(a2 + da2, aw["w3"], ab["b3"], padding=1) + x.abs())
             + F.conv2d(da2, aw["w3"], padding=1) + x_err)
    if moves:
        return y, bound, ((a1, da1), (a2, da2))
    return y, bound


def conv_direct(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """3x3, pad 1 convolution by explicit sums (pins the library convolution)."""
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    xp = np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))
    y = np.zeros((B, Co, H, W))
    for o in range(Co):
        acc = np.full((B, H, W), b[o], dtype=np.float64)
        for i in range(Ci):
            for ky in range(3):
                for kx in range(3):
                    acc += w[o, i, ky, kx] * xp[:, i, ky:ky + H, kx:kx + W]
        y[:, o] = acc
    return y


def grads(x: np.ndarray, w: dict, dy: np.ndarray) -> dict:
    """d<dy, y>/d(weights, biases) with BF16 rounding treated as identity (the
    straight-through rule the GPU backward also uses)."""
    wm = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in w.items()}
    # BF16 weights in the forward, gradients straight through to the float master copy
    wt = {k: (v + (bf16(v) - v).detach()) if k.startswith("w") else v for k, v in wm.items()}
    xt = torch.tensor(x, dtype=torch.float64)
    xin = bf16(xt)
    with torch.no_grad():
        a1r = bf16(F.relu(F.conv2d(xin, wt["w1"], wt["b1"], padding=1)))
        a2r = bf16(F.relu(F.conv2d(a1r, wt["w2"], wt["b2"], padding=1)))
    # straight-through: forward values are the rounded ones, gradients pass unchanged
    z1 = F.conv2d(xin, wt["w1"], wt["b1"], padding=1)
    a1 = F.relu(z1) + (a1r - F.relu(z1)).detach()
    z2 = F.conv2d(a1, wt["w2"], wt["b2"], padding=1)
    a2 = F.relu(z2) + (a2r - F.relu(z2)).detach()
    y = xt + F.conv2d(a2, wt["w3"], wt["b3"], padding=1)
    (y * torch.tensor(dy, dtype=torch.float64)).sum().backward()
    return {k: v.grad.numpy().copy() for k, v in wm.items()}


def _corr(a: torch.Tensor, g: torch.Tensor, cout: int) -> torch.Tensor:
    """sum over images and pixels p of a[c](p + tap) g[o](p): the weight gradient of a 3x3,
    pad-1 convolution with input a and output gradient g, [cout, cin, 3, 3]."""
    return torch.nn.grad.conv2d_weight(a, (cout, a.shape[1], 3, 3), g, padding=1)


def _conv_t(g: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """Data gradient of a 3x3, pad-1 convolution with weights w (OIHW): [B, cin, H, W]."""
    return F.conv_transpose2d(g, w, padding=1)


def _rflip(v: torch.Tensor, D: torch.Tensor) -> torch.Tensor:
    """Largest |bf16(v') - bf16(v)| over |v' - v| <= D (rounding is monotone)."""
    r = bf16(v)
    return torch.maximum((bf16(v + D) - r).abs(), (bf16(v - D) - r).abs())


def grads_mixed(x: np.ndarray, w: dict, dy: np.ndarray, bound: bool = False, u: float = 2.0 ** -22,
                round_grads: bool = True):
    """The parameter gradients of the mixed-precision backward, in float64: BF16 rounding
    of the forward treated as identity (as in grads), and dy and the hidden gradients
    dz2 = [a2 > 0] conv_T(dy, w3), dz1 = [a1 > 0] conv_T(dz2, w2) rounded to BF16 where
    they enter a contraction, the same places the tensor-core backward rounds them.
    With round_grads=False this is grads.  With bound, also per parameter a bound on how
    far a backward can land that accumulates with unit roundoff u, rounds at those places
    and runs on the forward's low-precision activations (within forward_bound's moves,
    with the ReLU masks they imply): a hidden gradient rounds to the same BF16 value
    unless its pre-rounding value lies within its accumulation error (plus what the
    previous gradient's moves add) of a rounding boundary (_rflip), or where the mask may
    differ (the activation within its move of zero: at most |both values|); a weight
    gradient sum_p a g then moves by corr(da, |g| + dg) + corr(|a|, dg) plus
    gamma_n corr(|a| + da, |g| + dg), a bias gradient by sum dg + gamma_n sum(|g| + dg).
    -> grads dict, or (grads, bound) dicts, float64 numpy."""
    r = bf16 if round_grads else (lambda z: z)
    t = {k: bf16(torch.tensor(v, dtype=torch.float64)) if k.startswith("w") else torch.tensor(v, dtype=torch.float64)
         for k, v in w.items()}
    xt = torch.tensor(x, dtype=torch.float64)
    _, _, ((a1, da1), (a2, da2)) = forward_bound(xt, w, u=u, moves=True)
    xin = bf16(xt)
    m1, m2 = (a1 > 0).double(), (a2 > 0).double()
    g3 = r(torch.tensor(dy, dtype=torch.float64))
    z2 = _conv_t(g3, t["w3"])
    dz2 = r(m2 * z2)
    z1 = _conv_t(dz2, t["w2"])
    dz1 = r(m1 * z1)
    out = {"w3": _corr(a2, g3, 3), "b3": g3.sum(dim=(0, 2, 3)), "w2": _corr(a1, dz2, 32), "b2": dz2.sum(dim=(0, 2, 3)),
           "w1": _corr(xin, dz1, 32), "b1": dz1.sum(dim=(0, 2, 3))}
    out = {k: v.numpy() for k, v in out.items()}
    if not bound:
        return out
    aw = {k: t[k].abs() for k in ("w2", "w3")}
    flip1 = (da1 > 0) & (a1 <= da1)
    flip2 = (da2 > 0) & (a2 <= da2)
    # dz2: K = 3 channels x 9 taps of the same rounded dy on both sides
    D2 = _gamma(27, u) * _conv_t(g3.abs(), aw["w3"])
    e2 = torch.where(flip2, 2.02 * (z2.abs() + D2), _rflip(m2 * z2, m2 * D2))
    # dz1: K = 32 channels x 9 taps of dz2, which may differ by e2
    D1 = _conv_t(e2, aw["w2"]) + _gamma(288, u) * _conv_t(dz2.abs() + e2, aw["w2"])
    e1 = torch.where(flip1, 2.02 * (z1.abs() + D1), _rflip(m1 * z1, m1 * D1))
    gn = _gamma(x.shape[0] * x.shape[2] * x.shape[3], u)
    bnd = {}
    for wk, bk, a, da, g, eg, cout in (("w3", "b3", a2, da2, g3, torch.zeros_like(g3), 3),
                                       ("w2", "b2", a1, da1, dz2, e2, 32),
                                       ("w1", "b1", xin, torch.zeros_like(xin), dz1, e1, 32)):
        ga = g.abs() + eg
        bnd[wk] = (_corr(da, ga, cout) + _corr(a.abs(), eg, cout) + gn * _corr(a.abs() + da, ga, cout)).numpy()
        bnd[bk] = (eg.sum(dim=(0, 2, 3)) + gn * ga.sum(dim=(0, 2, 3))).numpy()
    return out, bnd
