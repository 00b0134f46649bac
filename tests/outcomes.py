"""GPU images against the FP64 oracle's outcome sets (a test helper, no test here).

The rule: 2e-4 per FP32 channel, the workload's bound for the exact order, applied to
every order.  A pixel passes when it lies within the bound of the oracle's value or of
one of its alternative values: the composited results of the decisions that lie within
the comparison margins (alpha against 1/255, transmittance against 1e-4, near-equal
depths or keys, hierarchical window and stream ties, Sec. 4.1-4.3) taken the other way.
``oracle.native.render(outcomes=True)`` enumerates them.  A pixel whose set is too large
to enumerate is "unchecked"; every check bounds, asserts and prints that fraction:
0.1% for the exact and global orders, 1% for the window and hierarchical orders.
"""
from __future__ import annotations

import numpy as np

from oracle import native as on

TOL = 2e-4
MAX_UNCHECKED = {"exact": 0.001, "global_z": 0.001, "global_dist": 0.001, "window": 0.01, "hier": 0.01}


def reference(scene, cam, mode, **kw) -> dict:
    """The oracle's render of one view with its outcome sets."""
    return on.render(scene, cam, mode, outcomes=True, **kw)


def sub(ref: dict, y0: int, x0: int, h: int, w: int) -> dict:
    """The window [y0, y0 + h) x [x0, x0 + w) of a reference render, outcome sets included."""
    H, W = ref["image"].shape[1:]
    off, vals = ref["alt"]
    rows = []
    counts = []
    for y in range(y0, y0 + h):
        a, b = off[y * W + x0], off[y * W + x0 + w]
        rows.append(vals[a:b])
        counts.append(np.diff(off[y * W + x0:y * W + x0 + w + 1]))
    cnt = np.concatenate(counts) if counts else np.zeros(0, np.int64)
    noff = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
    nvals = np.concatenate(rows) if rows else np.zeros((0, 3))
    return dict(image=ref["image"][:, y0:y0 + h, x0:x0 + w], unchecked=ref["unchecked"][y0:y0 + h, x0:x0 + w],
                alt=(noff, nvals), marginal=ref["marginal"][y0:y0 + h, x0:x0 + w])


def crop_reference(scene, cam, x0: int, y0: int, w: int, h: int, mode: str, fovea=None, margin: int = 32,
                   **kw) -> dict:
    """The oracle over the window [x0, x0 + w) x [y0, y0 + h) of a full view, rendered
    through a crop camera widened by `margin` pixels on each side (within the view), so
    that the window's pixels read the same samples (bilinear taps across the window's
    edge included) as in the full view.  x0, y0 and margin are multiples of 32: key tiles,
    hierarchical blocks and the half-resolution grid stay aligned with the full view."""
    from paper_2505_10144_gb300 import synth
    assert x0 % 32 == 0 and y0 % 32 == 0 and margin % 32 == 0
    W, H = int(cam.width), int(cam.height)
    ex0, ey0 = max(x0 - margin, 0), max(y0 - margin, 0)
    ex1, ey1 = min(x0 + w + margin, W), min(y0 + h + margin, H)
    c2 = synth.Camera(cam.world_to_cam, cam.fx, cam.fy, cam.cx - ex0, cam.cy - ey0, ex1 - ex0, ey1 - ey0, cam.near_z)
    f2 = None
    if fovea is not None:
        f2 = synth.Fovea(fovea.gaze_x - ex0, fovea.gaze_y - ey0, fovea.radius_px, fovea.band_px)
    ref = reference(scene, c2, mode, fovea=f2, **kw)
    out = sub(ref, y0 - ey0, x0 - ex0, h, w)
    out["tile_class"] = ref["tile_class"]
    return out


def check(gpu, ref: dict, mode: str, tol: float = TOL, max_unchecked: float | None = None, label: str = "") -> dict:
    """Asserts that every enumerated pixel of gpu [3, H, W] matches the oracle's value or
    an alternative within tol, and that the unchecked fraction is within its bound.
    Returns the figures it printed."""
    gpu = np.asarray(gpu, dtype=np.float64)
    d = np.abs(gpu - ref["image"]).max(axis=0)
    unchecked = np.asarray(ref["unchecked"], dtype=bool)
    ok = d <= tol
    off, vals = ref["alt"]
    W = d.shape[1]
    by_alt = 0
    for k in np.nonzero(~ok.ravel() & ~unchecked.ravel())[0]:
        a, b = off[k], off[k + 1]
        if b > a:
            y, x = divmod(int(k), W)
            if np.abs(vals[a:b] - gpu[:, y, x][None, :]).max(axis=1).min() <= tol:
                ok.flat[k] = True
                by_alt += 1
    bad = ~ok & ~unchecked
    n = d.size
    frac_unchecked = float(unchecked.mean()) if n else 0.0
    worst = float(d[ok & ~unchecked].max()) if (ok & ~unchecked).any() else 0.0
    has_alt = float((np.diff(off) > 0).mean()) if n else 0.0
    stats = dict(pixels=int(n), unchecked=frac_unchecked, with_alternatives=has_alt, matched_by_alternative=by_alt,
                 worst_nominal=float(d[(d <= tol) & ~unchecked].max()) if ((d <= tol) & ~unchecked).any() else 0.0)
    print(f"[parity {label}] {n} px, unchecked {frac_unchecked:.4%}, with alternatives {has_alt:.3%}, "
          f"matched by an alternative {by_alt}, worst matched |d| {worst:.3g}")
    bound = MAX_UNCHECKED[mode] if max_unchecked is None else max_unchecked
    assert not bad.any(), (f"{label}: {int(bad.sum())} pixels match no valid outcome within {tol} "
                           f"(largest |d| {float(d[bad].max()):.3g})")
    assert frac_unchecked <= bound, f"{label}: {frac_unchecked:.4%} unchecked > {bound:.2%}"
    return stats
