"""Planted mistakes in the oracles, on the CPU: the float64 gradient oracle
(``oracle/grad.py``), the C forward oracle and its outcome sets.

The gradient oracle is pinned by central differences of the C forward oracle, which
re-sorts and re-culls at every evaluation and shares no code with it.  These tests show
that this pin is sharp enough: each plausible slip below (a sign in the real SH basis,
the 1/2 in the Gaussian's exponent, the direction of the focus/periphery blend
weight of Sec. 4.3, the bilinear weights of the upsampled periphery) makes the
autograd gradient disagree with the differences.  The mistakes are planted by patching
the oracle module inside the test only.
"""
import numpy as np
import pytest
import torch

from oracle import grad as og
from oracle import native as on
from paper_2505_10144_gb300 import synth
from scenes import random_scene

TOL = 1e-6  # the central-difference pin's bound, relative to max(1, |gradient|)


@pytest.fixture(scope="module")
def case():
    """A 96x96 foveated view in 32-pixel tiles: the centre tile holds the focus circle's
    blend band (hybrid), the eight others are periphery; 12 Gaussians at SH degree 3."""
    rng = np.random.default_rng(404)
    sc = random_scene(12, rng, sh_degree=3, z=(1.5, 2.5), xy=0.9, ls_mu=-1.6, ls_sd=0.3)
    sc = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in sc.arrays()], sc.sh_degree)
    c = synth.camera_from_pose(np.eye(3), (0, 0, 0), 96, 96, 84.0)
    fov = synth.Fovea(48.0, 48.0, 10.0, 5.0)
    base = on.render(sc, c, "exact", key_tile=32, fovea=fov, want_orders=True)
    cls = np.asarray(base["tile_class"]) & 3
    assert (cls == 1).any() and (cls == 2).any()
    w = rng.normal(size=base["image"].shape)
    fd = {}
    for name in ["mean", "log_scale", "quat", "opacity_logit", "sh"]:
        flat = getattr(sc, name).reshape(-1)
        for j in rng.choice(flat.size, size=min(16, flat.size), replace=False):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            vals, same = [], True
            for s in (+1, -1):
                flat[j] = x0 + s * h
                r = on.render(sc, c, "exact", key_tile=32, fovea=fov, want_orders=True)
                same &= all(np.array_equal(r["orders"][k], base["orders"][k]) for k in (0, 1))
                vals.append((r["image"] * w).sum())
            flat[j] = x0
            if same:  # otherwise a sort, cull or stop decision moved: not differentiable there
                fd[(name, int(j))] = (vals[0] - vals[1]) / (2 * h)
    assert len(fd) > 50
    return sc, c, fov, base, w, fd


def _worst(case):
    """Largest disagreement of the oracle's autograd gradient with the differences."""
    sc, c, fov, base, w, fd = case
    g = og.image_grad(sc, c, base["orders"], w, base["tile_class"], fov)
    return max(abs(v - g[n].reshape(-1)[j]) / max(1.0, abs(g[n].reshape(-1)[j])) for (n, j), v in fd.items())


def test_unmodified_gradient_oracle_meets_the_pin(case):
    assert _worst(case) <= TOL


def _sh_sign_slip(degree, d):
    b = _sh_basis(degree, d).clone()
    b[1] = -b[1]  # the l=1, m=-1 term with the wrong sign
    return b


def _blend_weight_reversed(px, py, fovea):
    return 1.0 - _fovea_weight(px, py, fovea)


def _bilinear_weights_swapped(L):
    """x2 bilinear upsampling with the two neighbours' fractions exchanged."""
    Cc, h, wd = L.shape

    def axis(n):
        u = (np.arange(2 * n) + 0.5) / 2 - 0.5
        i0 = np.floor(u).astype(np.int64)
        return np.clip(i0, 0, n - 1), np.clip(i0 + 1, 0, n - 1), 1.0 - (u - i0)

    ya, yb, fy = axis(h)
    xa, xb, fx = axis(wd)
    fx = torch.tensor(fx)[None, None, :]
    fy = torch.tensor(fy)[None, :, None]
    top = (1 - fx) * L[:, ya][:, :, xa] + fx * L[:, ya][:, :, xb]
    bot = (1 - fx) * L[:, yb][:, :, xa] + fx * L[:, yb][:, :, xb]
    return (1 - fy) * top + fy * bot


_sh_basis = og.sh_basis
_fovea_weight = og.fovea_weight


def _alpha_exponent_without_half(pr, j, px, py):
    v = torch.stack([(px - pr["cx"]) / pr["fx"], (py - pr["cy"]) / pr["fy"], torch.ones_like(px)], 1)
    u, E, A = pr["u"][j], pr["E"][j], pr["A"][j]
    s = torch.einsum("mak,mk->ma", E, v) / (u * v).sum(1)[:, None]
    q = torch.einsum("ma,mab,mb->m", s, A, s)
    return torch.clamp_max(pr["sigma"][j] * torch.exp(-q), og.ALPHA_MAX)


@pytest.mark.parametrize("target, mutant", [
    ("sh_basis", _sh_sign_slip),
    ("alpha_at", _alpha_exponent_without_half),
    ("fovea_weight", _blend_weight_reversed),
    ("bilinear_up2", _bilinear_weights_swapped),
], ids=["sh-sign", "exponent-half", "blend-weight", "bilinear-weights"])
def test_planted_mistake_fails_the_pin(case, monkeypatch, target, mutant):
    monkeypatch.setattr(og, target, mutant)
    assert _worst(case) > 100 * TOL, target


# ---------------------------------------------------------------- the C forward oracle

_C_SLIPS = {
    # the l=1, m=-1 harmonic with the wrong sign
    "sh-sign": ("Y[1] = -c1 * y;", "Y[1] = c1 * y;"),
    # the 1/2 dropped from the plane Gaussian's exponent
    "exponent-half": ("*sg = p->sigma * exp(-0.5 * q);", "*sg = p->sigma * exp(-1.0 * q);"),
    # front-to-back blending (Eq. 2) without the transmittance factor
    "blend-transmittance": ("s->C[c] += alpha * s->T * rgb[c];", "s->C[c] += alpha * rgb[c];"),
    # the inverse 2x2 covariance with the off-diagonal sign lost
    "conic-sign": ("p->A[0][1] = p->A[1][0] = -p->Sp[0][1] / det;", "p->A[0][1] = p->A[1][0] = p->Sp[0][1] / det;"),
    # the focus/periphery blend weight (Sec. 4.3) without the band's offset
    "fovea-weight": ("double w = (o->radius + o->band - sqrt(dx * dx + dy * dy)) / o->band;",
                     "double w = (o->radius - sqrt(dx * dx + dy * dy)) / o->band;"),
    # the per-sample window of the hierarchical resort holding one entry fewer than k
    "window-capacity": ("if (B->L3[i].n > B->k3) blend_at(B, i, win_pop(&B->L3[i]).gid);",
                        "if (B->L3[i].n >= B->k3) blend_at(B, i, win_pop(&B->L3[i]).gid);"),
    # the hybrid blend (Sec. 4.3) with its two weights exchanged
    "hybrid-weights": ("v[ch] = w * (S[k].C[ch] + S[k].T * bg[ch]) + (1 - w) * lowimg[ch * W2 * H2 + g];",
                       "v[ch] = (1 - w) * (S[k].C[ch] + S[k].T * bg[ch]) + w * lowimg[ch * W2 * H2 + g];"),
    # the hybrid pixel's 2x2 average taken over the wrong group (the next one to the right)
    "hybrid-group": ("int64_t g = (int64_t)(y / 2) * W2 + x / 2;\n        for (int ch = 0; ch < 3; ++ch)\n          v[ch] = w",
                     "int64_t g = (int64_t)(y / 2) * W2 + (x / 2 + 1 < W2 ? x / 2 + 1 : x / 2);\n        for (int ch = 0; ch < 3; ++ch)\n          v[ch] = w"),
}


@pytest.mark.parametrize("slip", sorted(_C_SLIPS))
def test_planted_mistake_in_the_c_oracle_fails_a_pin(slip, tmp_path):
    """A copy of the C oracle with one slip, built beside the test, fails the pins."""
    import os
    import subprocess
    import sys
    from pathlib import Path

    root = Path(__file__).resolve().parent.parent
    src = (root / "oracle" / "vrs_oracle.c").read_text()
    old, new = _C_SLIPS[slip]
    assert src.count(old) == 1
    (tmp_path / "mutant.c").write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                           str(tmp_path / "mutant.c"), "-lm"])
    env = dict(os.environ, VRS_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", str(root / "tests" / "test_oracle_pins.py"), "-x", "-q",
                        "-p", "no:cacheprovider"], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, r.stdout[-2000:]


# ---------------------------------------------------------------- the outcome sets

_OUTCOME_SLIPS = {
    # near-tied depths or keys blended in one order only
    "tie-orders": ("  const int np = permutations(g, perms);", "  const int np = permutations(g, perms) > 0;"),
    # a keep decision within the alpha margin taken one way only (exact and global orders)
    "keep-branch": ("    if (!c->amb && keep != c->kept) continue;", "    if (keep != c->kept) continue;"),
    # a transmittance test within the stop margin taken one way only
    "stop-branch": ("    int amb_stop = fabs(test - OG_T_STOP) < g_margin_stop * OG_T_STOP;", "    int amb_stop = 0;"),
    # hierarchical windows: a forced tie flip that does not flip
    "window-tie-flip": ("    less = !less;", "    less = less;"),
    # hierarchical blocks: forced keep / stop flips that do not flip
    "block-keep-flip": ("(dec){OG_DEC_KEEP, i, g, 0})) k = !k;", "(dec){OG_DEC_KEEP, i, g, 0})) k = k;"),
    "block-stop-flip": ("(dec){OG_DEC_STOP, i, g, 0})) stop = !stop;", "(dec){OG_DEC_STOP, i, g, 0})) stop = stop;"),
    # opacities within the margin below 1/255 culled at projection
    "projection-cull": ("const double sigma_min = o->outcomes ? OG_ALPHA_MIN * (1.0 - o->margin_alpha) : OG_ALPHA_MIN;",
                        "const double sigma_min = OG_ALPHA_MIN;"),
    # tile lists without the pairs whose largest alpha over the tile is just below the cut
    "relaxed-lists": ("double relax = o->outcomes ? -2.0 * log1p(-o->margin_alpha) : 0.0;", "double relax = 0.0;"),
}


@pytest.mark.parametrize("slip", sorted(_OUTCOME_SLIPS))
def test_planted_mistake_in_the_outcome_sets_fails_a_pin(slip, tmp_path):
    """A copy of the C oracle whose outcome enumeration skips one kind of decision fails
    the outcome-set pins (renders of nearby scenes fall outside the sets)."""
    import os
    import subprocess
    import sys
    from pathlib import Path

    root = Path(__file__).resolve().parent.parent
    src = (root / "oracle" / "vrs_oracle.c").read_text()
    old, new = _OUTCOME_SLIPS[slip]
    assert src.count(old) == 1, slip
    (tmp_path / "mutant.c").write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                           str(tmp_path / "mutant.c"), "-lm"])
    env = dict(os.environ, VRS_ORACLE_LIB=str(lib), OMP_NUM_THREADS="4")
    r = subprocess.run([sys.executable, "-m", "pytest", str(root / "tests" / "test_outcome_pins.py"), "-q",
                        "-p", "no:cacheprovider"], cwd=root, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and " failed" in r.stdout, r.stdout[-2000:]
