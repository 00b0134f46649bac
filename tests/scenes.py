"""Hand-built scenes for the pins (test helpers; no rasterizer arithmetic)."""
import math

import numpy as np

from paper_2505_10144_gb300 import synth

# half-range of a uniform degree-0 SH draw, see synth
SQRT_PI = math.sqrt(math.pi)


def make_scene(means, log_scales=None, quats=None, logits=None, dc=None, sh_degree=0, rng=None):
    means = np.asarray(means, dtype=np.float64).reshape(-1, 3).T
    n = means.shape[1]
    rng = np.random.default_rng(0) if rng is None else rng
    ls = np.full((3, n), -3.0) if log_scales is None else np.asarray(log_scales, dtype=np.float64).reshape(n, 3).T
    q = np.tile([[1.0], [0], [0], [0]], (1, n)) if quats is None else np.asarray(quats, dtype=np.float64).reshape(n, 4).T
    lg = np.zeros(n) if logits is None else np.asarray(logits, dtype=np.float64).reshape(n)
    K = (sh_degree + 1) ** 2
    sh = np.zeros((K, 3, n))
    sh[0] = 0.0 if dc is None else np.asarray(dc, dtype=np.float64).reshape(n, 3).T
    if K > 1:
        sh[1:] = rng.normal(0, 0.2, size=(K - 1, 3, n))
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return synth.Scene(f(means), f(ls), f(q), f(lg), f(sh), sh_degree)


def random_scene(n, rng, sh_degree=0, z=(2.0, 4.0), xy=1.0, ls_mu=-3.0, ls_sd=0.4):
    means = np.stack([rng.uniform(-xy, xy, n), rng.uniform(-xy, xy, n), rng.uniform(z[0], z[1], n)], 1)
    ls = rng.normal(ls_mu, ls_sd, size=(n, 3))
    q = rng.normal(size=(n, 4))
    lg = rng.normal(0.5, 1.0, size=n)
    dc = rng.uniform(-SQRT_PI, SQRT_PI, size=(n, 3))
    return make_scene(means, ls, q, lg, dc, sh_degree, rng)
