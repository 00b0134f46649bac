"""Stereo reuse of distant content (named as future work in Sec. 7: monocular rendering
and stereoscopic reuse of distant content), as a composition of plain oracle renders.
TEST INFRASTRUCTURE ONLY.

Reading: a Gaussian belongs to the far layer when its mean lies at world-space distance
d >= D from the cyclopean eye (the midpoint of the two eye centres), to the near layer
otherwise.  Each eye renders its near layer (per-ray order, background black) and keeps
each pixel's colour C_near and transmittance T_near; the far layer is rendered once, from
the cyclopean camera (the left eye's rotation and intrinsics, centre at the midpoint),
with the background.  Each eye's pixel is C_near + T_near * far(pixel): the far layer is
seen through the near layer's transmittance, front to back as in Eq. 2.

For a far Gaussian at distance d, an eye's ray and the cyclopean ray through the same
pixel meet it (IPD / 2) / d apart, f (IPD / 2) / d pixels: 0.25 px at D = 92 m, f = 722.6,
IPD = 64 mm.  The method is exact (up to the stop rule across the two layers) when the
eyes coincide.
"""
from __future__ import annotations

import numpy as np

from . import native as on


def render(scene, cams, far_distance: float, mode: str = "hier", windows=(4, 8, 16), key_tile: int = 16,
           bg=(0.0, 0.0, 0.0), outcomes: bool = False, cyclopean=None) -> dict:
    """-> dict(images [2, 3, H, W], far, near [(C, T) per eye]); with outcomes, also
    per eye the outcome sets ("alt", "unchecked" as native.render): every combination of
    the valid (C, T) of the eye's near sample and of the far sample of the pixel.
    cyclopean: the far layer's camera (by default the camera between the two eyes)."""
    from paper_2505_10144_gb300 import synth
    cyc = cyclopean if cyclopean is not None else synth.cyclopean_camera(cams[0], cams[1])
    ref = np.asarray(cyc.center(), dtype=np.float64)
    bg = np.asarray([float(np.float32(b)) for b in bg])
    far = on.render(scene, cyc, mode, windows=windows, key_tile=key_tile, bg=tuple(bg), outcomes=outcomes,
                    distance=(ref, far_distance, np.inf), want_samples=True)
    H, W = far["image"].shape[1:]
    Cf, Tf = far["full"][:3], far["full"][3]
    out = {"images": np.zeros((2, 3, H, W)), "far": far, "near": [], "alt": [], "unchecked": []}
    for e in range(2):
        near = on.render(scene, cams[e], mode, windows=windows, key_tile=key_tile, bg=(0.0, 0.0, 0.0),
                         outcomes=outcomes, distance=(ref, 0.0, far_distance), want_samples=True)
        Cn, Tn = near["full"][:3], near["full"][3]
        out["images"][e] = Cn + Tn[None] * (Cf + Tf[None] * bg[:, None, None])
        out["near"].append((Cn, Tn))
        if outcomes:
            noff, n4 = near["alt"][0], near["alt4"]
            foff, f4 = far["alt"][0], far["alt4"]
            unchecked = near["unchecked"] | far["unchecked"]
            offs, vals = [0], []
            for k in range(W * H):
                y, x = divmod(k, W)
                ns = [np.concatenate([Cn[:, y, x], [Tn[y, x]]])] + [n4[j] for j in range(noff[k], noff[k + 1])]
                fs = [np.concatenate([Cf[:, y, x], [Tf[y, x]]])] + [f4[j] for j in range(foff[k], foff[k + 1])]
                if (len(ns) > 1 or len(fs) > 1) and not unchecked[y, x]:
                    for a in ns:
                        for b in fs:
                            v = a[:3] + a[3] * (b[:3] + b[3] * bg)
                            if np.abs(v - out["images"][e][:, y, x]).max() > 0:
                                vals.append(v)
                offs.append(len(vals))
            out["alt"].append((np.asarray(offs, np.int64), np.asarray(vals).reshape(-1, 3)))
            out["unchecked"].append(unchecked)
    return out
