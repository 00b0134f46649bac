"""Pins of the oracle's outcome sets, on the CPU.

The FP32-vs-FP64 comparison checks every pixel against the set of values that the
decisions within the rule's margins allow: a pair's alpha against the 1/255 cut
(Sec. 4.2), the transmittance test against the 1e-4 stop, the order of near-equal depths
of maximum response (Sec. 4.1) or of near-equal list keys, and the hierarchical windows'
and the tile stream's near-ties.  The oracle enumerates that set (``outcomes=True``).

What pins it without any GPU: the same scene with its parameters moved by FP32-sized
amounts (relative 1e-7 on the means, 1e-7 on the log-scales, 3e-6 on the opacity logits,
inside every margin) is rendered by the plain FP64 definition, which then takes some of
those decisions the other way.  Every pixel of such a render must lie within 2e-5 of a
value of the unperturbed render's outcome set.  The scenes are built so that many
decisions sit at their thresholds: near-duplicate Gaussian pairs (depth ties in every
pixel they cover), Gaussians whose alpha at a sample is within 2e-6 of 1/255, and
opaque stacks whose transmittance test at a sample lands within 5e-6 of 1e-4.  The
planted mistakes in ``test_oracle_mutants.py`` (an enumeration that skips one kind of
decision) each fail these pins.
"""
import math

import numpy as np
import pytest

from oracle import native as on
from paper_2505_10144_gb300 import synth

COVER_TOL = 2e-5
MODES = [("exact", (0, 0, 0)), ("hier", (4, 8, 16)), ("window", (0, 0, 4)), ("global_z", (0, 0, 0))]


def _logit(p):
    return math.log(p / (1.0 - p))


def stress_scene(rng, cam, sample_points, n_pairs=80, corners=()):
    """Float64 scene whose decisions sit at their thresholds (see the module docstring).
    sample_points: continuous pixel positions of samples (pixel or group centres) that
    the alpha-cut Gaussians and the stop stacks are centred on.  corners: sample
    positions at the top-left corner of a key tile; a Gaussian centred 2.5 pixels up and
    left of each has its largest alpha over that tile (Eq. 4) at the corner sample, 1e-6
    below 1/255, so the FP64 tile test drops the pair and an FP32 one may keep it."""
    K = np.array([[cam.fx, 0, cam.cx], [0, cam.fy, cam.cy], [0, 0, 1.0]])
    Ki = np.linalg.inv(K)
    means, ls, quats, logits, dcs = [], [], [], [], []

    def add(m, s, q, lg, dc):
        means.append(m), ls.append(s), quats.append(q), logits.append(lg), dcs.append(dc)

    # near-duplicate pairs: depths tie wherever both are kept
    for _ in range(n_pairs):
        z = rng.uniform(1.5, 3.0)
        p = np.array([rng.uniform(0, cam.width), rng.uniform(0, cam.height), 1.0])
        m = z * (Ki @ p)
        s = rng.normal(-3.2, 0.3, 3)
        q = rng.normal(size=4)
        lg = rng.normal(0.5, 1.0)
        add(m, s, q, lg, rng.uniform(-1.7, 1.7, 3))
        add(m * (1 + 1e-9 * rng.uniform(-1, 1)), s, q, lg, rng.uniform(-1.7, 1.7, 3))
    pts = list(sample_points)
    rng.shuffle(pts)
    # alpha at the cut: the mean on a sample's ray, so G = 1 there and sigma G = sigma
    for px, py in pts[:40]:
        m = rng.uniform(1.5, 3.0) * (Ki @ np.array([px, py, 1.0]))
        sig = (1.0 / 255.0) * (1.0 + 2e-6 * rng.uniform(-1, 1))
        add(m, np.full(3, -3.5), rng.normal(size=4), _logit(sig), rng.uniform(-1.7, 1.7, 3))
    # transmittance at the stop: alphas 0.9, 0.99 (clamped) and 0.9 (1 + 5e-7 u) on one
    # sample's ray leave T (1 - alpha_3) = 1e-4 (1 - 4.5e-6 u)
    for px, py in pts[40:70]:
        v = Ki @ np.array([px, py, 1.0])
        z0 = rng.uniform(0.9, 1.1)
        for z, sig in ((z0, 0.9), (z0 + 0.3, 0.995), (z0 + 0.6, 0.9 * (1.0 + 5e-7 * rng.uniform(-1, 1)))):
            add(z * v, np.full(3, -3.3), np.array([1.0, 0, 0, 0]), _logit(sig), rng.uniform(-1.7, 1.7, 3))
    for cx, cy in corners:
        m = rng.uniform(1.5, 3.0) * (Ki @ np.array([cx - 2.5, cy - 2.5, 1.0]))
        s_ = np.full(3, -2.5)
        q = np.array([1.0, 0, 0, 0])
        # G at the corner for this shape, from the plain definition (sigma = 1/2)
        one = synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64)[..., None] for a in (m, s_, q)],
                          np.zeros(1), np.zeros((1, 3, 1)), 0)
        G = on.eval_one(one, 0, cam, cx, cy)[3] / 0.5
        add(m, s_, q, _logit((1.0 / 255.0) * (1.0 - 1e-6) / G), rng.uniform(-1.7, 1.7, 3))
    n = len(means)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    sh = np.zeros((1, 3, n))
    sh[0] = np.array(dcs).T
    return synth.Scene(f(np.array(means).T), f(np.array(ls).T), f(np.array(quats).T), f(np.array(logits)), f(sh), 0)


def perturbed(scene, rng):
    s = scene.copy()
    s.mean = s.mean * (1 + 1e-7 * rng.standard_normal(s.mean.shape))
    s.log_scale = s.log_scale + 1e-7 * rng.standard_normal(s.log_scale.shape)
    s.opacity_logit = s.opacity_logit + 3e-6 * rng.standard_normal(s.opacity_logit.shape)
    return s


def covered(img, ref, tol=COVER_TOL):
    """-> (pixels within tol of the nominal value or of an alternative, |img - nominal|)."""
    d = np.abs(img - ref["image"]).max(axis=0)
    ok = d <= tol
    off, vals = ref["alt"]
    W = d.shape[1]
    for k in np.nonzero(~ok.ravel())[0]:
        a, b = off[k], off[k + 1]
        if b > a:
            y, x = divmod(int(k), W)
            ok.flat[k] = np.abs(vals[a:b] - img[:, y, x][None, :]).max(axis=1).min() <= tol
    return ok, d


@pytest.fixture(scope="module")
def plain_case():
    cam = synth.identity_camera(64, 64, 90.0)
    pts = [(x + 0.5, y + 0.5) for y in range(4, 60) for x in range(4, 60)]
    corners = [(16 * tx + 0.5, 16 * ty + 0.5) for ty in range(1, 4) for tx in range(1, 4)]
    return stress_scene(np.random.default_rng(2024), cam, pts, corners=corners), cam


@pytest.fixture(scope="module")
def foveated_case():
    cam = synth.identity_camera(96, 96, 90.0)
    fov = synth.Fovea(48.0, 48.0, 14.0, 6.0)
    # group centres of periphery tiles and pixel centres of the focus and hybrid tile
    pts = [(2 * gx + 1.0, 2 * gy + 1.0) for gy in range(2, 46) for gx in range(2, 46)
           if not (16 <= gx < 32 and 16 <= gy < 32)]
    pts += [(x + 0.5, y + 0.5) for y in range(34, 62) for x in range(34, 62)]
    return stress_scene(np.random.default_rng(2025), cam, pts), cam, fov


def _check(scene, cam, mode, win, key_tile, fov=None, seeds=3):
    """-> (flipped, uncovered) pixels over renders of perturbed copies, among the pixels
    whose outcome set the oracle enumerates (a few of these dense scenes' pixels have
    more valid values than the enumeration's limits)."""
    ref = on.render(scene, cam, mode, windows=win, key_tile=key_tile, fovea=fov, outcomes=True)
    unchecked = ref["unchecked"]
    assert unchecked.mean() < 0.05, f"{unchecked.mean():.2%} of the pixels unchecked"
    flipped = uncovered = 0
    for seed in range(seeds):
        img = on.render(perturbed(scene, np.random.default_rng(seed)), cam, mode, windows=win, key_tile=key_tile,
                        fovea=fov)["image"]
        ok, d = covered(img, ref)
        flipped += int(((d > COVER_TOL) & ~unchecked).sum())
        uncovered += int((~ok & ~unchecked).sum())
    return flipped, uncovered


@pytest.mark.parametrize("mode,win", MODES)
def test_outcome_sets_cover_renders_of_nearby_scenes(plain_case, mode, win):
    scene, cam = plain_case
    flipped, uncovered = _check(scene, cam, mode, win, 16)
    assert uncovered == 0, f"{uncovered} of {flipped} flipped pixels outside the outcome set"
    assert flipped >= 20, f"only {flipped} pixels flipped: the pin has lost its power"


@pytest.mark.parametrize("mode,win", MODES[:3])
def test_outcome_sets_cover_foveated_renders_of_nearby_scenes(foveated_case, mode, win):
    scene, cam, fov = foveated_case
    flipped, uncovered = _check(scene, cam, mode, win, 32, fov)
    assert uncovered == 0, f"{uncovered} of {flipped} flipped pixels outside the outcome set"
    assert flipped >= 20, f"only {flipped} pixels flipped: the pin has lost its power"


def test_outcome_sets_hold_the_nominal_value_and_no_more_than_needed(plain_case):
    """Without any decision within the margins a pixel has no alternative; a pixel's
    alternatives differ from its value; the same render with margins of zero has none."""
    scene, cam = plain_case
    for mode, win in MODES:
        ref = on.render(scene, cam, mode, windows=win, key_tile=16, outcomes=True)
        off, vals = ref["alt"]
        n = np.diff(off).reshape(ref["image"].shape[1:])
        assert not (n > 0)[~ref["marginal"]].any(), mode
        for k in np.nonzero(n.ravel() > 0)[0][:200]:
            y, x = divmod(int(k), n.shape[1])
            assert np.abs(vals[off[k]:off[k + 1]] - ref["image"][:, y, x]).max() > 0
        z = on.render(scene, cam, mode, windows=win, key_tile=16, outcomes=True, margins=(0.0, 0.0, 0.0))
        assert z["alt"][1].shape[0] == 0 and np.array_equal(z["image"], ref["image"])
