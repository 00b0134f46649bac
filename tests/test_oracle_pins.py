"""Pins of the FP64 oracle to facts fixed by the paper and by mathematics, independent of
the oracle's own code: closed forms, textbook special cases, brute force, invariants."""
import json
import math
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F
from scipy.optimize import minimize_scalar
from scipy.spatial.transform import Rotation

from oracle import grad as og
from oracle import loss as ol
from oracle import native as on
from oracle import net as onet
from paper_2505_10144_gb300 import synth
from scenes import SQRT_PI, make_scene, random_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cam(W, H, f, cx=None, cy=None, pose=np.eye(3), pos=(0, 0, 0)):
    return synth.camera_from_pose(pose, pos, W, H, f, cx=cx, cy=cy)


def covariance(scene, i):
    """Sigma = R S^2 R^T built with scipy's rotation, independent of the oracle."""
    w, x, y, z = scene.quat[:, i].astype(np.float64)
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    S2 = np.diag(np.exp(2 * scene.log_scale[:, i].astype(np.float64)))
    return R @ S2 @ R.T


# ---------------------------------------------------------------- spherical harmonics

def test_sh_basis_orthonormal():
    """The degree-0..3 real SH basis is orthonormal on the sphere (pins every constant)."""
    ct, wt = np.polynomial.legendre.leggauss(40)
    phi = (np.arange(80) + 0.5) * 2 * np.pi / 80
    G = np.zeros((16, 16))
    for c, w in zip(ct, wt):
        st = math.sqrt(1 - c * c)
        for p in phi:
            Y = on.sh_basis(3, [st * math.cos(p), st * math.sin(p), c])
            G += np.outer(Y, Y) * w * (2 * np.pi / 80)
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_basis_signs_match_scipy_complex_harmonics():
    """The 3DGS sign convention, pinned against scipy's complex harmonics (Condon-Shortley
    phase included): Y_l0 = Y_l^0, Y_lm = sqrt(2) Re Y_l^m and Y_l,-m = sqrt(2) Im Y_l^m
    for m > 0.  Orthonormality alone leaves every sign free."""
    from scipy.special import sph_harm_y
    rng = np.random.default_rng(5)
    for _ in range(16):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        th, ph = math.acos(d[2]), math.atan2(d[1], d[0])
        ref = []
        for l in range(4):
            for m in range(-l, l + 1):
                y = sph_harm_y(l, abs(m), th, ph)
                ref.append(y.real if m == 0 else math.sqrt(2) * (y.real if m > 0 else y.imag))
        assert np.abs(on.sh_basis(3, d) - np.array(ref)).max() < 1e-13


def test_sh_degree_truncation():
    d = np.array([0.3, -0.5, 0.8]) / np.linalg.norm([0.3, -0.5, 0.8])
    Y3 = on.sh_basis(3, d)
    for deg in range(3):
        Yd = on.sh_basis(deg, d)
        K = (deg + 1) ** 2
        assert np.array_equal(Yd[:K], Y3[:K]) and not Yd[K:].any()


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("logit", [-1.0, 0.5, 6.0])
def test_single_gaussian_peak_closed_form(logit):
    """A Gaussian whose mean lies on a pixel's ray renders min(0.99, sigma) * rgb there."""
    W, H, f = 64, 48, 50.0
    c = cam(W, H, f)
    px, py = 20, 37
    v = np.array([(px + 0.5 - W / 2) / f, (py + 0.5 - H / 2) / f, 1.0])
    mu = 3.1 * v
    dc = np.array([0.7, -1.1, 0.2])
    sc = make_scene([mu], [[-2.7, -3.3, -3.0]], [[0.3, 0.5, -0.2, 0.7]], [logit], [dc])
    # make the mean exactly representable so the ray passes through it
    r = on.render(sc, c, "exact", key_tile=16)
    sigma = 1 / (1 + math.exp(-np.float32(logit)))
    rgb = 0.5 + sc.sh[0, :, 0].astype(np.float64) / (2 * SQRT_PI)
    expect = min(0.99, sigma) * rgb
    got = r["image"][:, py, px]
    # the float32 mean is within 1 ulp of the ray, so G = 1 - O(1e-12)
    assert np.allclose(got, expect, rtol=0, atol=1e-9), (got, expect)


def test_ewa_limit_on_axis_exact():
    """On the optical axis the tangent plane is parallel to the image plane, so Optimal
    Projection and the local-affine (EWA) projection of Eq. 3 coincide exactly."""
    W, H, f = 64, 64, 40.0
    c = cam(W, H, f)
    sc = make_scene([[0, 0, 2.5]], [[-2.2, -2.9, -2.5]], [[0.9, 0.2, -0.3, 0.1]], [1.0], [[0.4, 0.0, -0.4]])
    pr = on.project_one(sc, 0, c)
    m2, S2 = on.ewa_one(sc, 0, c)
    dil = 0.3 / float(np.float32(f)) ** 2
    Sp = pr["Sp"] - dil * np.eye(2)
    assert np.allclose(np.float32(f) ** 2 * Sp, S2 - 0.3 * np.eye(2), rtol=1e-12, atol=1e-14)
    # EWA image of the single Gaussian, built here from its mean and covariance
    ys, xs = np.mgrid[0:H, 0:W]
    D = np.stack([xs + 0.5 - m2[0], ys + 0.5 - m2[1]], -1)
    Si = np.linalg.inv(S2)
    q = np.einsum("...a,ab,...b->...", D, Si, D)
    a = pr["sigma"] * np.exp(-0.5 * q)
    a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
    ewa = a[None] * pr["rgb"][:, None, None]
    r = on.render(sc, c, "exact", key_tile=16)
    assert np.abs(r["image"] - ewa).max() < 1e-12


def test_op_matches_ewa_to_first_order_everywhere():
    """At the projected mean the two projections share the same 2D covariance (chain rule
    through the ray direction), for any position in the field of view."""
    W, H, f = 96, 80, 40.0
    c = cam(W, H, f)
    rng = np.random.default_rng(3)
    for _ in range(10):
        mu = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), rng.uniform(1, 3)])
        sc = make_scene([mu], rng.normal(-2.5, 0.4, (1, 3)), rng.normal(size=(1, 4)), [0.0], [[0, 0, 0]])
        pr = on.project_one(sc, 0, c)
        _, S2 = on.ewa_one(sc, 0, c)
        u, E = pr["u"], pr["E"]
        fxy = float(np.float32(f))
        J = np.zeros((2, 2))
        for k in range(2):
            for a in range(2):
                J[a, k] = fxy * (E[k, a] * u[2] - u[a] * E[k, 2]) / u[2] ** 2
        Sp = pr["Sp"] - 0.3 / fxy ** 2 * np.eye(2)
        assert np.allclose(J @ Sp @ J.T, S2 - 0.3 * np.eye(2), rtol=1e-9, atol=1e-12)


def test_op_ewa_image_difference_vanishes_on_axis():
    W, H, f = 128, 128, 60.0
    c = cam(W, H, f)
    diffs = []
    for ang in [0.6, 0.3, 0.15, 0.0]:
        mu = 2.0 * np.array([math.sin(ang), 0.0, math.cos(ang)])
        sc = make_scene([mu], [[-1.9, -2.6, -2.2]], [[0.8, 0.1, 0.4, -0.3]], [2.0], [[0.5, 0.5, 0.5]])
        pr = on.project_one(sc, 0, c)
        m2, S2 = on.ewa_one(sc, 0, c)
        ys, xs = np.mgrid[0:H, 0:W]
        D = np.stack([xs + 0.5 - m2[0], ys + 0.5 - m2[1]], -1)
        q = np.einsum("...a,ab,...b->...", D, np.linalg.inv(S2), D)
        a = pr["sigma"] * np.exp(-0.5 * q)
        a = np.where(a >= 1 / 255, np.minimum(a, 0.99), 0.0)
        op = on.render(sc, c, "exact", key_tile=16)["image"][0] / pr["rgb"][0]
        diffs.append(np.abs(op - a).max())
    assert diffs[0] > diffs[1] > diffs[2] > 0 and diffs[3] < 1e-12, diffs


def test_tstar_is_argmax_along_ray():
    """t* equals the brute-force maximiser of the 3D Gaussian (Eq. 1) along the ray."""
    rng = np.random.default_rng(7)
    W, H, f = 64, 64, 50.0
    pose = synth.head_rotation(0.3, -0.2)
    c = cam(W, H, f, pose=pose, pos=(0.1, -0.2, 0.05))
    R = c.world_to_cam[:, :3].astype(np.float64)
    t = c.world_to_cam[:, 3].astype(np.float64)
    checked = 0
    for _ in range(40):
        fwd = pose[:, 2]
        mu_w = np.array([0.1, -0.2, 0.05]) + 2.5 * fwd + rng.normal(0, 0.3, 3)
        sc = make_scene([mu_w], rng.normal(-2.0, 0.5, (1, 3)), rng.normal(size=(1, 4)), [1.0], [[0, 0, 0]])
        Sw = covariance(sc, 0)
        Sc = R @ Sw @ R.T
        Sci = np.linalg.inv(Sc)
        mu_c = R @ sc.mean[:, 0].astype(np.float64) + t
        fz = float(np.float32(f))
        px = fz * mu_c[0] / mu_c[2] + W / 2 + rng.uniform(-3, 3)
        py = fz * mu_c[1] / mu_c[2] + H / 2 + rng.uniform(-3, 3)
        v = np.array([(px - W / 2) / fz, (py - H / 2) / fz, 1.0])
        kept, a, tstar, sg = on.eval_one(sc, 0, c, px, py)
        if not kept:
            continue
        res = minimize_scalar(lambda s: (s * v - mu_c) @ Sci @ (s * v - mu_c),
                              bracket=(0.0, 10.0), tol=1e-12)
        assert abs(res.x - tstar) < 1e-6 * abs(tstar), (res.x, tstar)
        checked += 1
    assert checked > 5


def test_op_second_order_agrees_with_exact_ray_maximum():
    """Around the centre ray, the tangent-plane exponent and the exact maximum-along-ray
    exponent r^T S^-1 r - (v^T S^-1 r)^2 / v^T S^-1 v agree in value and Hessian (both
    reduce to the Schur complement of Sigma^-1 on u-perp)."""
    rng = np.random.default_rng(11)
    c = cam(64, 64, 1e7)  # dilation 0.3/f^2 becomes negligible
    for _ in range(8):
        mu = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(1.5, 3)])
        sc = make_scene([mu], rng.normal(-1.5, 0.4, (1, 3)), rng.normal(size=(1, 4)), [1.0], [[0, 0, 0]])
        pr = on.project_one(sc, 0, c)
        Sc = covariance(sc, 0)  # identity camera: camera frame == world frame
        Sci = np.linalg.inv(Sc)
        r = sc.mean[:, 0].astype(np.float64)
        u, E = pr["u"], pr["E"]

        def q_ray(s):
            v = u + E.T @ s
            return r @ Sci @ r - (v @ Sci @ r) ** 2 / (v @ Sci @ v)

        assert abs(q_ray(np.zeros(2))) < 1e-9
        h = 1e-4
        Hs = np.zeros((2, 2))
        for a in range(2):
            for b in range(2):
                ea, eb = np.eye(2)[a] * h, np.eye(2)[b] * h
                Hs[a, b] = (q_ray(ea + eb) - q_ray(ea - eb) - q_ray(-ea + eb) + q_ray(-ea - eb)) / (4 * h * h)
        assert np.allclose(Hs, 2 * pr["A"], rtol=1e-5), (Hs, 2 * pr["A"])


# ---------------------------------------------------------------- Eq. 4 and culling

def test_edge_maximum_eq4_matches_dense_sampling():
    rng = np.random.default_rng(5)
    for _ in range(200):
        M = rng.normal(size=(2, 2))
        A = M @ M.T + 0.1 * np.eye(2)
        P, D = rng.normal(size=2), rng.normal(size=2)
        t, q = on.edge_max(A, P, D)
        ts = np.linspace(0, 1, 200001)
        X = P[None] + ts[:, None] * D[None]
        qs = np.einsum("na,ab,nb->n", X, A, X)
        assert qs.min() >= q - 1e-12 and qs.min() - q < 1e-8
        assert abs(ts[qs.argmin()] - t) < 1e-4


def _q_at(pr, c, px, py):
    v = np.array([(px - np.float32(c.cx)) / np.float32(c.fx), (py - np.float32(c.cy)) / np.float32(c.fy), 1.0])
    w = pr["u"] @ v
    s = pr["E"] @ v / w
    return s @ pr["A"] @ s, w


def test_tile_culling_bound_is_tight_and_conservative():
    """Eq. 4 on the optimal plane: the tile minimum of the exponent is at the projected
    mean when it is inside the tile, otherwise on the boundary; dense sampling of the
    tile never goes below it, and gets arbitrarily close."""
    rng = np.random.default_rng(9)
    W, H, f = 256, 256, 90.0
    c = cam(W, H, f)
    inside = 0
    for _ in range(60):
        mu = np.array([rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5), rng.uniform(1, 3)])
        sc = make_scene([mu], rng.normal(-2.0, 0.5, (1, 3)), rng.normal(size=(1, 4)), [2.0], [[0, 0, 0]])
        pr = on.project_one(sc, 0, c)
        tx, ty = rng.integers(0, 8, 2)
        mpx, mpy = 90.0 * mu[0] / mu[2] + 128, 90.0 * mu[1] / mu[2] + 128
        if _ % 3 == 0 and 0 < mpx < 256 and 0 < mpy < 256:
            tx, ty = int(mpx // 32), int(mpy // 32)  # the tile holding the projected mean
        x0, y0, x1, y1 = tx * 32 + 0.5, ty * 32 + 0.5, tx * 32 + 31.5, ty * 32 + 31.5
        keep, key, qmin = on.tile_one(sc, 0, c, x0, y0, x1, y1)
        if min(_q_at(pr, c, x, y)[1] for x in (x0, x1) for y in (y0, y1)) <= 0:
            assert keep  # quad unbounded on the plane: kept, conservatively
            continue
        g = np.linspace(0, 1, 257)
        qs = [_q_at(pr, c, x0 + a * (x1 - x0), y0 + b * (y1 - y0))[0] for a in g for b in g]
        qs = np.array(qs)
        assert qs.min() >= qmin - 1e-9
        assert qs.min() - qmin < 1e-3 * max(1.0, qmin)
        assert keep == (qmin <= pr["r2"])
        if qmin == 0.0:
            inside += 1
            assert key == pr["mu"][2]
    assert inside > 0


# ---------------------------------------------------------------- whole-render pins

def _wide_scene(rng, n=60):
    """Gaussians all around a wide camera, including large, near and off-screen ones."""
    sc = random_scene(n, rng, sh_degree=2, z=(0.25, 3.0), xy=3.0, ls_mu=-2.2, ls_sd=0.8)
    return sc


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_equals_tiled(seed):
    """All-pairs rendering with no tiles, rectangles or culling equals the tiled render:
    the bounding conic and Eq. 4 culling only drop pairs with alpha < 1/255."""
    rng = np.random.default_rng(seed)
    sc = _wide_scene(rng)
    c = cam(40, 32, 14.0)
    brute = on.render(sc, c, "exact", brute=True)["image"]
    for kt in (16, 32):
        for cull in (True, False):
            tiled = on.render(sc, c, "exact", key_tile=kt, tile_cull=cull)["image"]
            assert np.array_equal(tiled, brute)


def test_large_fov_crop_invariance():
    """Sec. 5.2 / Appendix 'Large FOV': focal length / 3 at resolution x 3 (same focal in
    pixels) must give a centre crop that exactly matches the original render."""
    rng = np.random.default_rng(4)
    sc = random_scene(300, rng, sh_degree=3, z=(0.5, 4.0), xy=4.0, ls_mu=-2.0, ls_sd=0.6)
    W, H, f = 48, 40, 36.0
    small = on.render(sc, cam(W, H, f), "exact", key_tile=16)["image"]
    big = on.render(sc, cam(3 * W, 3 * H, f), "exact", key_tile=16)["image"]
    assert np.array_equal(big[:, H:2 * H, W:2 * W], small)
    assert np.abs(small).max() > 0.05


def test_transmittance_and_colour_bounds():
    rng = np.random.default_rng(12)
    sc = random_scene(400, rng, sh_degree=1)
    c = cam(64, 64, 40.0)
    r = on.render(sc, c, "exact", key_tile=16, want_samples=True)
    C, T = r["full"][:3], r["full"][3]
    assert (T > 0).all() and (T <= 1).all()
    assert (C >= 0).all()
    # colour is a convex combination of clamped SH colours
    rgbmax = max(on.project_one(sc, i, c)["rgb"].max() for i in range(sc.n))
    assert (C <= rgbmax * (1 - T) + 1e-12).all()


def test_adding_a_gaussian_never_raises_transmittance():
    rng = np.random.default_rng(13)
    base = random_scene(50, rng)
    base.opacity_logit[:] = -3.0  # keeps T far above the stop threshold
    c = cam(48, 48, 30.0)
    T0 = on.render(base, c, "exact", want_samples=True)["full"][3]
    extra = random_scene(1, rng)
    both = synth.Scene(*[np.concatenate([a, b], axis=-1) for a, b in zip(base.arrays(), extra.arrays())], 0)
    T1 = on.render(both, c, "exact", want_samples=True)["full"][3]
    assert (T1 <= T0 + 1e-15).all() and (T1 < T0).any()


def test_two_identical_gaussians():
    """Two copies of one Gaussian blend to c (1 - (1 - alpha)^2) (Eq. 2)."""
    one = make_scene([[0.1, -0.05, 2.0]], [[-2.0, -2.3, -2.1]], [[1, 0.2, 0, 0.1]], [0.3], [[0.5, -0.2, 0.1]])
    two = synth.Scene(*[np.concatenate([a, a], axis=-1) for a in one.arrays()], 0)
    c = cam(48, 48, 40.0)
    i1 = on.render(one, c, "exact")["image"]
    i2 = on.render(two, c, "exact")["image"]
    rgb = on.project_one(one, 0, c)["rgb"]
    a = i1[0] / rgb[0]
    assert np.allclose(i2, rgb[:, None, None] * (1 - (1 - a) ** 2)[None], atol=1e-14)


def test_window_cascade_with_unbounded_windows_is_exact():
    rng = np.random.default_rng(14)
    sc = random_scene(800, rng, sh_degree=1)
    c = cam(64, 48, 40.0)
    ex = on.render(sc, c, "exact", key_tile=16)["image"]
    big = 1 << 20
    assert np.array_equal(on.render(sc, c, "hier", windows=(big, big, big), key_tile=16)["image"], ex)
    assert np.array_equal(on.render(sc, c, "window", windows=(0, 0, big), key_tile=16)["image"], ex)
    fov = synth.Fovea(30.0, 20.0, 12.0, 4.0)
    exf = on.render(sc, c, "exact", key_tile=32, fovea=fov)["image"]
    assert np.array_equal(on.render(sc, c, "hier", windows=(big, big, big), key_tile=32, fovea=fov)["image"], exf)


def _sample_streams(sc, c, T):
    """Per pixel: the Gaussians of its key tile's list (oracle tile lists, sorted by
    (key, index)) that are kept at the pixel centre, with their depth t*, in list order."""
    counts, gids, keys = on.tile_lists(sc, c, T)
    off = np.concatenate([[0], np.cumsum(counts.ravel())])
    ntx = counts.shape[1]
    streams = {}
    for y in range(c.height):
        for x in range(c.width):
            t = (y // T) * ntx + x // T
            st = []
            for g in gids[off[t]:off[t + 1]]:
                kept, a, ts, _ = on.eval_one(sc, int(g), c, x + 0.5, y + 0.5)
                if kept:
                    st.append((ts, int(g), a))
            streams[(y, x)] = st
    return streams


def _blend_order(seq):
    """Gaussians blended front to back from a sequence of (t, id, alpha), with the
    transmittance stop at 1e-4 (Eq. 2 and the stop rule)."""
    T, out = 1.0, []
    for _, g, a in seq:
        if T * (1.0 - a) < 1e-4:
            break
        T *= 1.0 - a
        out.append(g)
    return out


def _orders(r, W, H):
    order, off = r["orders"]
    return {(y, x): order[off[y * W + x]:off[y * W + x + 1]].tolist() for y in range(H) for x in range(W)}


@pytest.fixture(scope="module")
def stream_case():
    rng = np.random.default_rng(17)
    sc = random_scene(300, rng, sh_degree=0, ls_mu=-2.6)
    c = cam(40, 32, 60.0)
    return sc, c, _sample_streams(sc, c, 16)


def test_cascade_with_zero_windows_blends_in_tile_list_order(stream_case):
    """Reading of the hierarchical resort (Sec. 4.1): windows of size zero pass every
    entry straight through, so each pixel blends its kept pairs in the order of its key
    tile's sorted list (the tile keys of Eq. 4's maximum point, ties by index)."""
    sc, c, streams = stream_case
    r = on.render(sc, c, "hier", windows=(0, 0, 0), key_tile=16, want_orders=True)
    got = _orders(r, c.width, c.height)
    assert sum(len(v) for v in streams.values()) > 2000
    for k, st in streams.items():
        assert got[k] == _blend_order(st), k


@pytest.mark.parametrize("k", [1, 3, 8])
def test_per_sample_window_is_a_size_k_min_heap_over_the_kept_stream(stream_case, k):
    """With the block windows off, the per-sample window of size k is the textbook
    bounded priority queue: push each kept pair of the stream, pop the smallest (t*, id)
    once more than k are held, drain in order at the end (heapq as the reference)."""
    import heapq
    sc, c, streams = stream_case
    r = on.render(sc, c, "window", windows=(0, 0, k), key_tile=16, want_orders=True)
    got = _orders(r, c.width, c.height)
    differs = 0
    for key, st in streams.items():
        h, out = [], []
        for e in st:
            heapq.heappush(h, e)
            if len(h) > k:
                out.append(heapq.heappop(h))
        while h:
            out.append(heapq.heappop(h))
        assert got[key] == _blend_order(out), key
        differs += _blend_order(out) != _blend_order(sorted(st))
    assert differs > 0  # the window does reorder against the exact order somewhere


def test_cascade_equals_exact_order_for_separated_layers():
    """Layers of Gaussians far apart in depth, each layer's Gaussians side by side: every
    ray meets the layers in the same order and no layer's pairs overtake another's in any
    window, so the hierarchical cascade blends the exact order."""
    rng = np.random.default_rng(18)
    means, ls = [], []
    for z in (1.5, 2.5, 3.5, 4.5):
        for _ in range(40):
            means.append([rng.uniform(-0.8, 0.8) * z / 2, rng.uniform(-0.6, 0.6) * z / 2, z + rng.normal(0, 0.002)])
            ls.append([-2.5, -2.5, -5.0])
    sc = make_scene(means, log_scales=ls, logits=np.full(len(means), -1.0),
                    dc=rng.uniform(-SQRT_PI, SQRT_PI, size=(len(means), 3)))
    c = cam(64, 48, 60.0)
    ex = on.render(sc, c, "exact", key_tile=16)
    for win in [(4, 8, 16), (1, 1, 1)]:
        h = on.render(sc, c, "hier", windows=win, key_tile=16)
        assert np.abs(h["image"] - ex["image"]).max() < 1e-12, win


@pytest.mark.parametrize("T", [32, 16])
def test_foveated_focus_pixels_equal_plain_render(T):
    rng = np.random.default_rng(15)
    sc = random_scene(600, rng, sh_degree=2)
    c = cam(192, 128, 80.0)
    fov = synth.Fovea(80.0, 60.0, 34.0, 6.0)
    plain = on.render(sc, c, "exact", key_tile=16)["image"]
    r = on.render(sc, c, "exact", key_tile=T, fovea=fov)
    cls = np.repeat(np.repeat(r["tile_class"], T, 0), T, 1)[:128, :192]
    assert (cls == 0).any() and (cls == 1).any() and (cls == 2).any()
    assert np.array_equal(r["image"][:, cls == 0], plain[:, cls == 0])


@pytest.mark.parametrize("T", [32, 16])
def test_hybrid_blend_follows_the_focus_circle_and_its_band(T):
    """Sec. 4.3: hybrid tiles blend the full-resolution render with its 2x2-group
    average by a continuous mask that is 1 on the focus circle and falls to 0 across the
    band.  Against the plain render of the same rays (exact order, so per-pixel results
    do not depend on the tiling): a hybrid pixel within the circle equals the plain
    pixel; one beyond radius + band equals the mean of its plain 2x2 group; in between
    it lies on the segment between the two, at the parameter 1 - (d - R) / b."""
    rng = np.random.default_rng(16)
    sc = random_scene(600, rng, sh_degree=2)
    H, W = 128, 192
    c = cam(W, H, 80.0)
    R, b = 30.0, 10.0
    fov = synth.Fovea(80.3, 60.7, R, b)
    plain = on.render(sc, c, "exact", key_tile=16)["image"]
    r = on.render(sc, c, "exact", key_tile=T, fovea=fov)
    cls = np.repeat(np.repeat(r["tile_class"], T, 0), T, 1)[:H, :W]
    grp = plain.reshape(3, H // 2, 2, W // 2, 2).mean(axis=(2, 4))
    A = np.repeat(np.repeat(grp, 2, 1), 2, 2)
    ys, xs = np.mgrid[0:H, 0:W]
    d = np.hypot(xs + 0.5 - np.float32(fov.gaze_x), ys + 0.5 - np.float32(fov.gaze_y))
    hyb = cls == 1
    inner, outer = hyb & (d <= R - 1e-6), hyb & (d >= R + b + 1e-6)
    band = hyb & (d > R + 0.5) & (d < R + b - 0.5) & (np.abs(plain - A).max(axis=0) > 1e-3)
    assert inner.sum() > 50 and outer.sum() > 50 and band.sum() > 50
    assert np.abs(r["image"][:, inner] - plain[:, inner]).max() < 1e-12
    assert np.abs(r["image"][:, outer] - A[:, outer]).max() < 1e-12
    ch = np.abs(plain - A).argmax(axis=0)  # the channel where the two differ most
    V, C0, A0 = (np.take_along_axis(x, ch[None], 0)[0] for x in (r["image"], plain, A))
    t = (V[band] - A0[band]) / (C0[band] - A0[band])
    assert np.abs(t - (1.0 - (d[band] - R) / b)).max() < 1e-9
    # between the circle and R + b the mask is continuous: no jump at either edge
    assert t.min() > 0.0 and t.max() < 1.0


def test_foveated_constant_scene_stays_constant():
    """Every composite of Sec. 4.3 (hybrid blend, bilinear periphery) is an average of
    samples with weights that sum to one: a scene whose every sample has the same colour
    (one Gaussian far larger than the view, alpha clamped at 0.99 everywhere) renders the
    same constant in focus, hybrid and periphery tiles."""
    sc = make_scene([[0.0, 0.0, 3.0]], log_scales=[[5.0, 5.0, 5.0]], logits=[10.0], dc=[[0.4, -0.3, 0.9]])
    c = cam(160, 128, 80.0)
    fov = synth.Fovea(70.0, 60.0, 50.0, 10.0)
    r = on.render(sc, c, "exact", key_tile=32, fovea=fov, bg=(0.2, 0.1, 0.3))
    assert set(np.unique(r["tile_class"])) >= {0, 1, 2}
    ref = on.render(sc, c, "exact", key_tile=16, bg=(0.2, 0.1, 0.3))["image"]
    v = ref[:, 0, 0]
    assert np.abs(ref - v[:, None, None]).max() < 1e-12
    assert np.abs(r["image"] - v[:, None, None]).max() < 1e-12


def _gap_scene(rng, n_near=300, n_far=300):
    """Near Gaussians 1.5-3 m ahead, far ones 120-200 m ahead, nothing in between."""
    near = [[rng.uniform(-1, 1), rng.uniform(-0.8, 0.8), rng.uniform(1.5, 3.0)] for _ in range(n_near)]
    far = [[rng.uniform(-80, 80), rng.uniform(-60, 60), rng.uniform(120.0, 200.0)] for _ in range(n_far)]
    ls = [[-2.8] * 3] * n_near + [[np.log(0.02 * 160)] * 3] * n_far
    return make_scene(near + far, log_scales=ls, logits=rng.normal(0.5, 1.0, n_near + n_far),
                      dc=rng.uniform(-SQRT_PI, SQRT_PI, size=(n_near + n_far, 3)), rng=rng)


def test_stereo_reuse_without_far_layer_is_the_plain_render():
    """Sec. 7 (stereo reuse of distant content), reading: near layer per eye, far layer
    once from the cyclopean eye, C_near + T_near far.  With no Gaussian in the far layer
    the far image is the background and each eye is its plain render, bit for bit."""
    from oracle import reuse
    rng = np.random.default_rng(19)
    sc = _gap_scene(rng)
    cams = synth.stereo_cameras((0.0, 0.0, 0.0), 0.1, 64, 48, 80.0)
    bg = (0.2, 0.4, 0.1)
    r = reuse.render(sc, cams, 1e9, "exact", bg=bg)
    for e in range(2):
        plain = on.render(sc, cams[e], "exact", key_tile=16, bg=bg)["image"]
        assert np.array_equal(r["images"][e], plain)


@pytest.mark.parametrize("mode", ["exact", "hier"])
def test_stereo_reuse_with_coinciding_eyes_is_the_plain_render_up_to_the_stop(mode):
    """With both eyes at the cyclopean point and the split in a gap of the scene, every ray
    meets the near layer first, and the layered blend equals the one-pass blend of Eq. 2
    except after the transmittance stop, which the far layer applies to its own T: there
    the one-pass render stops once T_near T_far (1 - alpha) < 1e-4, so the two differ by
    at most the light left at that point, T < 1e-4 / (1 - alpha_max) = 1e-2."""
    from oracle import reuse
    rng = np.random.default_rng(20)
    sc = _gap_scene(rng)
    c = synth.identity_camera(64, 48, 80.0)
    r = reuse.render(sc, [c, c], 60.0, mode, bg=(0.3, 0.3, 0.3))
    plain = on.render(sc, c, mode, key_tile=16, bg=(0.3, 0.3, 0.3))["image"]
    d = np.abs(r["images"][0] - plain).max(axis=0)
    near = on.render(sc, c, mode, key_tile=16, distance=(np.zeros(3), 0.0, 60.0), want_samples=True)["full"][3]
    assert d.max() <= 1e-2 and (d > 1e-12).mean() < 0.05
    # where the near layer leaves T >= 0.5, the stop cannot move by more than 2e-4 of light
    assert d[near >= 0.5].max() <= 2e-4
    assert (near < 0.99).mean() > 0.3 and (near >= 0.5).mean() > 0.3  # both layers are visible


def _partial_mask(H, W):
    """Visible everywhere except the left 40 columns and the bottom-right corner, with one
    tile kept by a single visible pixel (tile-level culling keeps it whole)."""
    m = np.ones((H, W), np.uint8)
    m[:, :40] = 0
    m[H - 40:, W - 56:] = 0
    m[5, 3] = 1
    return m


def test_visibility_all_visible_is_no_mask():
    """Visibility culling with every pixel visible changes nothing (bitwise)."""
    rng = np.random.default_rng(21)
    sc = random_scene(500, rng, sh_degree=1)
    c = cam(160, 128, 70.0)
    ones = np.ones((128, 160), np.uint8)
    fov = synth.Fovea(70.0, 60.0, 30.0, 6.0)
    for kw in (dict(key_tile=16), dict(key_tile=32, fovea=fov)):
        for mode in ("exact", "hier"):
            a = on.render(sc, c, mode, **kw)
            b = on.render(sc, c, mode, visible=ones, **kw)
            assert np.array_equal(a["image"], b["image"]) and a["stats"] == b["stats"]


def test_visibility_culls_exactly_the_invisible_tiles():
    """Sec. 4.3 visibility culling: a tile with no visible pixel loses its instances and
    outputs the background; every other tile keeps the same sorted list, and (plain
    method: a pixel depends on its own tile only) the same pixels."""
    rng = np.random.default_rng(22)
    sc = random_scene(700, rng, sh_degree=1)
    W, H, T = 160, 128, 16
    c = cam(W, H, 70.0)
    m = _partial_mask(H, W)
    ty, tx = np.mgrid[0:H // T, 0:W // T]
    tvis = m.reshape(H // T, T, W // T, T).any(axis=(1, 3))
    assert (~tvis).sum() >= 10 and tvis[0, 0]  # the single-pixel tile stays
    c0, g0, k0 = on.tile_lists(sc, c, key_tile=T)
    c1, g1, k1 = on.tile_lists(sc, c, key_tile=T, visible=m)
    assert c1[~tvis].sum() == 0 and np.array_equal(c1[tvis], c0[tvis])
    off0 = np.concatenate([[0], np.cumsum(c0.ravel())])
    off1 = np.concatenate([[0], np.cumsum(c1.ravel())])
    for t in np.flatnonzero(tvis.ravel()):
        assert np.array_equal(g0[off0[t]:off0[t + 1]], g1[off1[t]:off1[t + 1]])
        assert np.array_equal(k0[off0[t]:off0[t + 1]], k1[off1[t]:off1[t + 1]])
    bg = (0.2, 0.4, 0.6)
    a = on.render(sc, c, "exact", key_tile=T, bg=bg)["image"]
    b = on.render(sc, c, "exact", key_tile=T, bg=bg, visible=m)["image"]
    pix_vis = np.repeat(np.repeat(tvis, T, 0), T, 1)
    assert np.array_equal(b[:, pix_vis], a[:, pix_vis])
    for ch in range(3):
        assert np.all(b[ch][~pix_vis] == np.float32(bg[ch]))


def test_visibility_foveated_periphery_reads_background():
    """Foveated: invisible tiles output the background, and visible periphery pixels
    whose bilinear taps stay in visible tiles are unchanged."""
    rng = np.random.default_rng(23)
    sc = random_scene(700, rng, sh_degree=1)
    W, H, T = 192, 128, 32
    c = cam(W, H, 80.0)
    fov = synth.Fovea(140.0, 70.0, 26.0, 5.0)
    m = np.ones((H, W), np.uint8)
    m[:, :32] = 0  # the first tile column
    bg = (0.1, 0.3, 0.5)
    a = on.render(sc, c, "hier", key_tile=T, fovea=fov, bg=bg)
    b = on.render(sc, c, "hier", key_tile=T, fovea=fov, bg=bg, visible=m)
    assert (a["tile_class"][:, 0] == 2).all()
    for ch in range(3):
        assert np.all(b["image"][ch][:, :32] == np.float32(bg[ch]))
    # bilinear taps of pixel x reach low-res column floor((x + 0.5) / 2 - 0.5) ... + 1,
    # i.e. full-res columns >= 32 only for x >= 34
    assert np.array_equal(b["image"][:, :, 34:], a["image"][:, :, 34:])


def test_tile_census_from_paper():
    g = json.load(open(os.path.join(GOLDEN, "tile_census.json")))
    empty = make_scene(np.zeros((0, 3)))
    for W, H, n in [(g["width"], g["height"], g["tiles"]), (2064, 2208, 65 * 69)]:
        c = synth.identity_camera(W, H, 110.0)
        fov = synth.fovea_for(W, (W / 2, H / 2))
        r = on.render(empty, c, "exact", key_tile=g["tile"], fovea=fov)
        cls = r["tile_class"]
        assert cls.size == n
        counts = np.bincount(cls.ravel(), minlength=3)
        assert counts.sum() == n and counts.min() > 0


def test_two_pass_baseline_composition():
    """Appendix A two-pass baseline: the centre pass is the plain render cropped (same
    rays); outside the band the image is the half-resolution render upsampled (checked
    against torch's half-pixel bilinear resize); in the band it is the w-blend of the
    two; where w = 1 it is the full-resolution pixel."""
    import torch.nn.functional as F
    from oracle import twopass as otp
    rng = np.random.default_rng(25)
    sc = random_scene(800, rng, sh_degree=2)
    W, H = 192, 128
    c = cam(W, H, 80.0)
    fov = synth.Fovea(84.0, 60.0, 22.0, 5.0)
    tp = otp.render(sc, c, fov, "exact")
    x0, y0, sw, sh = tp["rect"]
    assert sw == sh == 2 * (27 + 1) and 0 <= x0 <= W - sw and 0 <= y0 <= H - sh
    plain = on.render(sc, c, "exact", key_tile=16)["image"]
    assert np.allclose(tp["centre"], plain[:, y0:y0 + sh, x0:x0 + sw], rtol=0, atol=1e-12)
    low = on.render(sc, otp.half_camera(c), "exact", key_tile=16)["image"]
    assert np.array_equal(low, tp["low"])
    up = F.interpolate(torch.tensor(low)[None], scale_factor=2, mode="bilinear", align_corners=False)[0].numpy()
    w = otp.fovea_weight_image(W, H, fov)
    assert (w == 0).mean() > 0.5 and (w == 1).any() and ((w > 0) & (w < 1)).any()
    z = w == 0
    assert np.allclose(tp["image"][:, z], up[:, z], rtol=0, atol=1e-12)
    o = w == 1
    assert np.allclose(tp["image"][:, o], plain[:, o], rtol=0, atol=1e-12)
    b = (w > 0) & (w < 1)
    blend = w[None] * plain + (1 - w[None]) * up
    assert np.allclose(tp["image"][:, b], blend[:, b], rtol=0, atol=1e-12)


def test_global_sort_orders_two_gaussians_closed_form():
    """Global orders (Sec. 3: 3DGS sorts by view-space z, Mini-Splatting by distance):
    B is nearer in z, A nearer in distance; where both cover a pixel the blend is
    alpha_1 c_1 + (1 - alpha_1) alpha_2 c_2 in the respective order."""
    W, H, f = 96, 64, 40.0
    c = cam(W, H, f)
    A = [0.0, 0.0, 2.0]
    B = [1.5, 0.0, 1.9]
    sc = make_scene([A, B], [[-1.2] * 3, [-1.2] * 3], [[1, 0, 0, 0], [1, 0, 0, 0]], [1.0, 1.0],
                    [[1.5, -1.0, -1.0], [-1.0, -1.0, 1.5]])
    gz = on.render(sc, c, "global_z", key_tile=16)["image"]
    gd = on.render(sc, c, "global_dist", key_tile=16)["image"]
    rgb = [0.5 + sc.sh[0, :, i].astype(np.float64) / (2 * SQRT_PI) for i in range(2)]
    checked = 0
    for py in range(H):
        for px in range(W):
            ka, aa, _, _ = on.eval_one(sc, 0, c, px + 0.5, py + 0.5)
            kb, ab, _, _ = on.eval_one(sc, 1, c, px + 0.5, py + 0.5)
            if not (ka and kb):
                continue
            z_first = ab * rgb[1] + (1 - ab) * aa * rgb[0]
            d_first = aa * rgb[0] + (1 - aa) * ab * rgb[1]
            assert np.allclose(gz[:, py, px], z_first, atol=1e-12)
            assert np.allclose(gd[:, py, px], d_first, atol=1e-12)
            checked += 1
    assert checked > 20


def test_global_sort_equals_exact_when_layers_are_separated():
    """Isotropic Gaussians on fronto-parallel layers far apart in depth: the per-ray
    order of maximum response, the z order and the distance order coincide."""
    rng = np.random.default_rng(26)
    pts = []
    for z in (2.0, 3.0, 4.0):  # a grid per layer, spaced wider than a footprint, shifted per layer
        off = rng.uniform(0, 0.3, 2)
        for i in range(6):
            for j in range(5):
                pts.append([((i - 2.5) * 0.3 + off[0]) * z * 0.5, ((j - 2.0) * 0.3 + off[1]) * z * 0.5, z])
    n = len(pts)
    sc = make_scene(np.array(pts), np.full((n, 3), -3.0), np.tile([1.0, 0, 0, 0], (n, 1)),
                    rng.normal(0, 1, n), rng.normal(0, 1, (n, 3)))
    c = cam(80, 64, 40.0)
    ex = on.render(sc, c, "exact", key_tile=16, want_orders=True)
    order, off = ex["orders"]
    assert (np.diff(off[:80 * 64]) >= 2).sum() > 200  # pixels where two layers blend
    for mode in ("global_z", "global_dist"):
        g = on.render(sc, c, mode, key_tile=16)
        ok = ~(ex["marginal"] | g["marginal"])
        assert ok.mean() > 0.9
        assert np.allclose(g["image"][:, ok], ex["image"][:, ok], rtol=0, atol=1e-12)


# ---------------------------------------------------------------- gradients

def _fd_scene(rng):
    sc = random_scene(6, rng, sh_degree=3, z=(1.5, 2.5), xy=0.4, ls_mu=-2.0, ls_sd=0.3)
    return synth.Scene(*[np.ascontiguousarray(a, dtype=np.float64) for a in sc.arrays()], sc.sh_degree)


@pytest.mark.parametrize("fovea", [False, True])
def test_gradient_matches_central_differences(fovea):
    """Autograd of the fixed-order restatement vs central differences of the full C
    oracle (which re-sorts and re-culls at every step), float64."""
    rng = np.random.default_rng(21 + fovea)
    sc = _fd_scene(rng)
    c = cam(32, 32, 28.0)
    fov = synth.Fovea(16.0, 16.0, 10.0, 6.0) if fovea else None
    kt = 32 if fovea else 16
    base = on.render(sc, c, "exact", key_tile=kt, fovea=fov, want_orders=True)
    w = rng.normal(size=base["image"].shape)
    g = og.image_grad(sc, c, base["orders"], w, base["tile_class"], fov)
    checked = 0
    for name in ["mean", "log_scale", "quat", "opacity_logit", "sh"]:
        arr = getattr(sc, name)
        flat = arr.reshape(-1)
        for j in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            vals = []
            same = True
            for s in (+1, -1):
                flat[j] = x0 + s * h
                r = on.render(sc, c, "exact", key_tile=kt, fovea=fov, want_orders=True)
                same &= np.array_equal(r["orders"][0], base["orders"][0]) and np.array_equal(r["orders"][1], base["orders"][1])
                vals.append((r["image"] * w).sum())
            flat[j] = x0
            if not same:
                continue  # a sort, cull or stop decision moved: not differentiable here
            fd = (vals[0] - vals[1]) / (2 * h)
            an = g[name].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, j, fd, an)
            checked += 1
    assert checked > 30


def test_gradient_with_visibility_mask_matches_central_differences():
    """Foveated render under a visibility mask (three 32x32 tiles: hybrid, periphery,
    invisible): autograd of the restatement, whose invisible pixels are the constant
    background and whose periphery reads background samples from the invisible tile, vs
    central differences of the C oracle."""
    rng = np.random.default_rng(24)
    sc = _fd_scene(rng)
    c = cam(96, 32, 40.0)
    fov = synth.Fovea(14.0, 16.0, 8.0, 4.0)
    vis = np.ones((32, 96), np.uint8)
    vis[:, 64:] = 0
    bg = (0.3, 0.2, 0.1)
    base = on.render(sc, c, "exact", key_tile=32, fovea=fov, want_orders=True, visible=vis, bg=bg)
    assert list(base["tile_class"][0]) == [1, 2, 6]
    w = rng.normal(size=base["image"].shape)
    g = og.image_grad(sc, c, base["orders"], w, base["tile_class"], fov, bg)
    checked = 0
    for name in ["mean", "log_scale", "opacity_logit", "sh"]:
        flat = getattr(sc, name).reshape(-1)
        for j in rng.choice(flat.size, size=min(10, flat.size), replace=False):
            x0 = flat[j]
            h = 1e-6 * max(1.0, abs(x0))
            vals, same = [], True
            for s in (+1, -1):
                flat[j] = x0 + s * h
                r = on.render(sc, c, "exact", key_tile=32, fovea=fov, want_orders=True, visible=vis, bg=bg)
                same &= all(np.array_equal(a, b) for a, b in zip(r["orders"], base["orders"]))
                vals.append((r["image"] * w).sum())
            flat[j] = x0
            if not same:
                continue
            fd = (vals[0] - vals[1]) / (2 * h)
            an = g[name].reshape(-1)[j]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (name, j, fd, an)
            checked += 1
    assert checked > 20


# ---------------------------------------------------------------- loss and network

def test_ssim_identity_and_brute_force():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(3, 13, 17))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    assert abs(float(ol.ssim(torch.tensor(x), torch.tensor(x))) - 1.0) < 1e-14
    L, g = ol.loss_and_grad(x, x)
    assert abs(L) < 1e-14 and np.abs(g[np.abs(g) > 0]).max() <= 0.8 / x.size + 1e-15
    assert abs(float(ol.ssim(torch.tensor(x), torch.tensor(y))) - ol.ssim_brute(x, y)) < 1e-12


def test_ssim_gradient_fd():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 9, 8))
    y = rng.uniform(size=(3, 9, 8))
    L, g = ol.loss_and_grad(x, y)
    for _ in range(10):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (ol.loss_and_grad(xp, y)[0] - ol.loss_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-8


def test_net_conv_matches_direct_sum_and_zero_last_layer_is_identity():
    rng = np.random.default_rng(2)
    w = onet.init_weights(rng)
    x = rng.uniform(size=(2, 3, 7, 9))
    y, _ = onet.forward(torch.tensor(x), w, round_acts=False)
    a1 = np.maximum(onet.conv_direct(x, w["w1"], w["b1"]), 0)
    a2 = np.maximum(onet.conv_direct(a1, w["w2"], w["b2"]), 0)
    assert np.abs(y.numpy() - (x + onet.conv_direct(a2, w["w3"], w["b3"]))).max() < 1e-12
    w0 = onet.init_weights(rng, zero_last=True)
    y0, _ = onet.forward(torch.tensor(x), w0)
    assert np.array_equal(y0.numpy(), x)


def _net_case(seed, signed, shape=(2, 3, 11, 13)):
    """Weights (BF16 values), input and output gradient: random signs, or all >= 0 (no
    cancellation anywhere, so the mixed-precision bound is tight)."""
    rng = np.random.default_rng(seed)
    w = onet.init_weights(rng)
    if not signed:
        w = {k: np.abs(v) if k.startswith("w") else np.abs(rng.normal(0, 0.1, size=v.shape)) for k, v in w.items()}
    w["w3"] = w["w3"] * 10.0
    w = {k: onet.bf16(torch.tensor(v)).numpy() if k.startswith("w") else v for k, v in w.items()}
    x = rng.uniform(0, 1, size=shape)
    dy = (rng.normal(size=shape) if signed else rng.uniform(0, 1, size=shape)).astype(np.float32).astype(np.float64)
    return w, x, dy


def test_net_grads_match_direct_sums():
    """The straight-through gradients against the backward written out as sums: dz2 =
    [a2 > 0] sum_{o, tap} w3[o][c][tap] dy[o](p - tap + 1), dz1 likewise through w2, and
    each weight gradient sum_p a[c](p + tap - 1) dz[o](p)."""
    w, x, dy = _net_case(5, True, shape=(1, 3, 5, 6))
    g = onet.grads(x, w, dy)
    _, (xin, a1, a2) = onet.forward(torch.tensor(x), w)
    xin, a1, a2 = xin.numpy(), a1.numpy(), a2.numpy()
    H, W = x.shape[2:]

    def data_grad(gz, wk, mask):
        cin = w[wk].shape[1]
        out = np.zeros((1, cin, H, W))
        for c in range(cin):
            for py in range(H):
                for px in range(W):
                    s = 0.0
                    for o in range(w[wk].shape[0]):
                        for ky in range(3):
                            for kx in range(3):
                                qy, qx = py - ky + 1, px - kx + 1
                                if 0 <= qy < H and 0 <= qx < W:
                                    s += w[wk][o, c, ky, kx] * gz[0, o, qy, qx]
                    out[0, c, py, px] = s if mask[0, c, py, px] > 0 else 0.0
        return out

    def weight_grad(a, gz):
        cin, cout = a.shape[1], gz.shape[1]
        ap = np.pad(a, ((0, 0), (0, 0), (1, 1), (1, 1)))
        return np.array([[[[np.sum(ap[0, c, ky:ky + H, kx:kx + W] * gz[0, o]) for kx in range(3)] for ky in range(3)]
                          for c in range(cin)] for o in range(cout)])

    dz2 = data_grad(dy, "w3", a2)
    dz1 = data_grad(dz2, "w2", a1)
    ref = {"w3": weight_grad(a2, dy), "b3": dy.sum(axis=(0, 2, 3)), "w2": weight_grad(a1, dz2),
           "b2": dz2.sum(axis=(0, 2, 3)), "w1": weight_grad(xin, dz1), "b1": dz1.sum(axis=(0, 2, 3))}
    for k in ref:
        assert np.abs(g[k] - ref[k]).max() <= 1e-10 * max(1.0, np.abs(ref[k]).max()), k


def test_net_mixed_gradients_without_rounding_are_the_straight_through_ones():
    w, x, dy = _net_case(6, True)
    g, g0 = onet.grads(x, w, dy), onet.grads_mixed(x, w, dy, round_grads=False)
    for k in g:
        assert np.abs(g[k] - g0[k]).max() <= 1e-12 * np.abs(g[k]).max(), k


def _emulate_backward_fp32(x, w, dy, flip_taps=True, round_dz2=True):
    """The tensor-core backward's arithmetic emulated with float32 library convolutions
    (sequential-order GEMMs: the oneDNN path, which may use Winograd, is off): BF16
    weights, activations and gradient operands, float32 accumulation."""
    f = torch.float32

    def bfr(z):
        return z.to(torch.bfloat16).to(f)

    wt = {k: bfr(torch.tensor(v, dtype=f)) if k.startswith("w") else torch.tensor(v, dtype=f) for k, v in w.items()}
    with torch.backends.mkldnn.flags(enabled=False):
        xin = bfr(torch.tensor(x, dtype=f))
        a1 = bfr(torch.relu(F.conv2d(xin, wt["w1"], wt["b1"], padding=1)))
        a2 = bfr(torch.relu(F.conv2d(a1, wt["w2"], wt["b2"], padding=1)))
        g3 = bfr(torch.tensor(dy, dtype=f))

        def ct(g, wk):
            return F.conv_transpose2d(g, wt[wk] if flip_taps else wt[wk].flip(2, 3), padding=1)

        dz2 = (a2 > 0) * ct(g3, "w3")
        dz2 = bfr(dz2) if round_dz2 else dz2
        dz1 = bfr((a1 > 0) * ct(dz2, "w2"))

        def cw(a, g, co):
            return torch.nn.grad.conv2d_weight(a, (co, a.shape[1], 3, 3), g, padding=1)

        out = {"w3": cw(a2, g3, 3), "b3": g3.sum((0, 2, 3)), "w2": cw(a1, dz2, 32), "b2": dz2.sum((0, 2, 3)),
               "w1": cw(xin, dz1, 32), "b1": dz1.sum((0, 2, 3))}
    return {k: v.double().numpy() for k, v in out.items()}


@pytest.mark.parametrize("signed", [False, True])
def test_net_mixed_gradient_bound_holds_for_an_fp32_evaluation_and_catches_mistakes(signed):
    w, x, dy = _net_case(7, signed)
    g, b = onet.grads_mixed(x, w, dy, bound=True)
    emu = _emulate_backward_fp32(x, w, dy)
    worst = max(float((np.abs(emu[k] - g[k]) / np.maximum(b[k], 1e-300)).max()) for k in g)
    assert worst <= 1.0, worst
    if not signed:  # no cancellation: the bound is tight (under 0.1% of each gradient)
        assert all((b[k] <= 1e-3 * np.abs(g[k])).all() for k in g)
        for bad in (dict(flip_taps=False), dict(round_dz2=False)):
            emu = _emulate_backward_fp32(x, w, dy, **bad)
            assert any((np.abs(emu[k] - g[k]) > b[k]).any() for k in g), bad


def test_bilinear_upsampling_pins():
    L = torch.full((3, 5, 6), 0.37, dtype=torch.float64)
    assert torch.allclose(og.bilinear_up2(L), torch.full((3, 10, 12), 0.37, dtype=torch.float64))
    # a linear ramp sampled at low-res centres is reproduced at interior high-res centres
    gy, gx = np.mgrid[0:5, 0:6]
    ramp = torch.tensor(0.1 * (2 * gx + 1) + 0.03 * (2 * gy + 1), dtype=torch.float64)[None]
    up = og.bilinear_up2(ramp)[0].numpy()
    ys, xs = np.mgrid[0:10, 0:12]
    ref = 0.1 * (xs + 0.5) + 0.03 * (ys + 0.5)
    assert np.abs(up[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() < 1e-14
