"""ctypes binding of the FP64 C oracle (``oracle/vrs_oracle.c``).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The product path never imports this package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "vrs_oracle.c"
# VRS_ORACLE_LIB names a prebuilt variant of the library to load instead: the tests that
# plant a mistake in a copy of the C source and check that a pin fails use it.
_VARIANT = os.environ.get("VRS_ORACLE_LIB")
_LIB = Path(_VARIANT) if _VARIANT else _HERE / "lib" / "libvrs_oracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile the oracle with the host compiler (portable C, OpenMP)."""
    if _VARIANT:
        return _LIB
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        _LIB.parent.mkdir(parents=True, exist_ok=True)
        tmp = _LIB.with_suffix(f".tmp{os.getpid()}.so")
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", str(tmp), str(_SRC), "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Scene(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64),
                ("sh_degree", C.c_int)]


class _Camera(C.Structure):
    _fields_ = [("w2c", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("width", C.c_int),
                ("height", C.c_int), ("near_z", C.c_double)]


class _Opts(C.Structure):
    _fields_ = [("mode", C.c_int), ("k1", C.c_int), ("k2", C.c_int), ("k3", C.c_int),
                ("key_tile", C.c_int), ("foveated", C.c_int), ("tile_cull", C.c_int),
                ("brute", C.c_int), ("gaze_x", C.c_double), ("gaze_y", C.c_double),
                ("radius", C.c_double), ("band", C.c_double), ("bg", C.c_double * 3),
                ("margin_alpha", C.c_double), ("margin_stop", C.c_double), ("margin_tie", C.c_double),
                ("visible", C.c_void_p), ("outcomes", C.c_int), ("dist_cull", C.c_int),
                ("dist_ref", C.c_double * 3), ("dist_min", C.c_double), ("dist_max", C.c_double)]


class _Out(C.Structure):
    _fields_ = [("image", C.c_void_p), ("full", C.c_void_p), ("low", C.c_void_p),
                ("lowimg", C.c_void_p), ("marginal", C.c_void_p), ("tile_class", C.c_void_p),
                ("order", C.c_void_p), ("order_off", C.c_void_p), ("max_order", C.c_int64),
                ("n_order", C.c_int64), ("stats", C.c_int64 * 8), ("unchecked", C.c_void_p),
                ("alt_off", C.POINTER(C.c_int64)), ("alt", C.POINTER(C.c_double)), ("alt4", C.POINTER(C.c_double)),
                ("n_alt", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = C.CDLL(str(_LIB))
        dp = C.POINTER(C.c_double)
        _lib.og_render.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), C.POINTER(_Opts), C.POINTER(_Out)]
        _lib.og_render.restype = C.c_int
        _lib.og_project_one.argtypes = [C.POINTER(_Scene), C.c_int64, C.POINTER(_Camera), dp]
        _lib.og_eval_one.argtypes = [C.POINTER(_Scene), C.c_int64, C.POINTER(_Camera), C.c_double, C.c_double, dp]
        _lib.og_tile_one.argtypes = [C.POINTER(_Scene), C.c_int64, C.POINTER(_Camera)] + [C.c_double] * 4 + [dp]
        _lib.og_ewa_one.argtypes = [C.POINTER(_Scene), C.c_int64, C.POINTER(_Camera), dp]
        _lib.og_edge_max.argtypes = [dp, dp, dp, dp]
        _lib.og_sh_basis.argtypes = [C.c_int, dp, dp]
        _lib.og_tile_lists.argtypes = [C.POINTER(_Scene), C.POINTER(_Camera), C.c_int, C.c_int,
                                       C.c_void_p, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_int64]
        _lib.og_free.argtypes = [C.c_void_p]
        _lib.og_tile_lists.restype = C.c_int64
        _lib.og_num_threads.restype = C.c_int
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _SceneRef:
    """Keeps float64 copies of the parameters alive while the C side reads them."""

    def __init__(self, scene):
        self.arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in scene.arrays()]
        self.s = _Scene(*[_ptr(a) for a in self.arrs], scene.n, scene.sh_degree)


def _cam(cam) -> _Camera:
    c = _Camera()
    w = np.asarray(cam.world_to_cam, dtype=np.float32).astype(np.float64).ravel()
    for k in range(12):
        c.w2c[k] = w[k]
    # the product receives float32 camera numbers; the oracle uses the same values
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(np.float32(cam.near_z))
    return c


PROJ_FIELDS = [("valid", 1), ("mu", 3), ("d", 1), ("u", 3), ("E", 6), ("Sc", 9), ("Sci", 9),
               ("Sp", 4), ("A", 4), ("sigma", 1), ("r2", 1), ("rgb", 3), ("bbox", 4), ("bounded", 1)]


def project_one(scene, i: int, cam) -> dict:
    sr = _SceneRef(scene)
    out = np.zeros(52)
    lib().og_project_one(C.byref(sr.s), i, C.byref(_cam(cam)), _dptr(out))
    res, k = {}, 0
    for name, n in PROJ_FIELDS:
        res[name] = out[k:k + n].copy() if n > 1 else float(out[k])
        k += n
    res["E"] = res["E"].reshape(2, 3)
    for m in ("Sc", "Sci"):
        res[m] = res[m].reshape(3, 3)
    for m in ("Sp", "A"):
        res[m] = res[m].reshape(2, 2)
    return res


def eval_one(scene, i: int, cam, px: float, py: float):
    """-> (kept, alpha, tstar, sigma*G) of Gaussian i at continuous pixel (px, py)."""
    sr = _SceneRef(scene)
    out = np.zeros(4)
    lib().og_eval_one(C.byref(sr.s), i, C.byref(_cam(cam)), px, py, _dptr(out))
    return bool(out[0]), out[1], out[2], out[3]


def tile_one(scene, i: int, cam, x0, y0, x1, y1):
    """-> (keep, key, qmin) of Gaussian i against the sample quad [x0,x1]x[y0,y1]."""
    sr = _SceneRef(scene)
    out = np.zeros(3)
    lib().og_tile_one(C.byref(sr.s), i, C.byref(_cam(cam)), x0, y0, x1, y1, _dptr(out))
    return bool(out[0]), out[1], out[2]


def ewa_one(scene, i: int, cam):
    sr = _SceneRef(scene)
    out = np.zeros(5)
    ok = lib().og_ewa_one(C.byref(sr.s), i, C.byref(_cam(cam)), _dptr(out))
    return (out[:2].copy(), np.array([[out[2], out[3]], [out[3], out[4]]])) if ok else None


def edge_max(A, P, D):
    """Eq. 4 on one segment: -> (t, q) for the plane conic A (2x2)."""
    A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).ravel())
    P = np.ascontiguousarray(np.asarray(P, dtype=np.float64))
    D = np.ascontiguousarray(np.asarray(D, dtype=np.float64))
    out = np.zeros(2)
    lib().og_edge_max(_dptr(A), _dptr(P), _dptr(D), _dptr(out))
    return out[0], out[1]


def sh_basis(degree: int, direction) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(direction, dtype=np.float64))
    Y = np.zeros(16)
    lib().og_sh_basis(degree, _dptr(d), _dptr(Y))
    return Y


MODES = {"exact": 0, "window": 1, "hier": 2, "global_z": 3, "global_dist": 4}
# relative margins of the FP32-vs-FP64 comparison rule: sigma G against 1/255, the
# transmittance test against 1e-4, and near-equal depths or keys
MARGINS = (5e-5, 1e-5, 3e-7)


def render(scene, cam, mode: str = "exact", windows=(4, 8, 16), key_tile: int = 16, fovea=None,
           bg=(0.0, 0.0, 0.0), tile_cull: bool = True, brute: bool = False,
           want_orders: bool = False, want_samples: bool = False, margins=MARGINS,
           visible=None, outcomes: bool = False, distance=None) -> dict:
    """Render one view.  fovea: None for the plain method, else an object with gaze_x,
    gaze_y, radius_px, band_px (single-pass foveation, 32x32 key tiles).  visible: None,
    or an [H, W] array, nonzero where the pixel is visible (visibility culling).

    outcomes: also enumerate, per pixel, every composited value that the decisions of
    its samples within the margins allow (keep against 1/255, stop against 1e-4, order
    of near-tied depths or keys, hierarchical window and stream ties): the result gets
    "alt" = (offsets [H*W + 1], values [n, 3]) of the values other than "image" and
    "unchecked" [H, W], true where there are too many to enumerate (and, for plain renders,
    "alt4": the (C rgb, T) of each alternative).  distance: None, or (ref_xyz, d_min,
    d_max): render only the Gaussians whose world-space mean is at distance d_min <= d <
    d_max from the point ref_xyz."""
    W, H = int(cam.width), int(cam.height)
    o = _Opts()
    vis = None
    if visible is not None:
        vis = np.ascontiguousarray(np.asarray(visible) != 0, dtype=np.uint8)
        if vis.shape != (H, W):
            raise ValueError("visible must be [H, W]")
        o.visible = vis.ctypes.data
    o.mode = MODES[mode]
    o.k1, o.k2, o.k3 = (int(k) for k in windows)
    o.key_tile = int(key_tile)
    o.foveated = 0 if fovea is None else 1
    o.tile_cull = int(tile_cull)
    o.brute = int(brute)
    if fovea is not None:
        o.gaze_x, o.gaze_y = float(np.float32(fovea.gaze_x)), float(np.float32(fovea.gaze_y))
        o.radius, o.band = float(np.float32(fovea.radius_px)), float(np.float32(fovea.band_px))
    for k in range(3):
        o.bg[k] = float(np.float32(bg[k]))
    o.margin_alpha, o.margin_stop, o.margin_tie = (float(m) for m in margins)
    o.outcomes = int(outcomes)
    if distance is not None:
        ref, dmin, dmax = distance
        o.dist_cull = 1
        for k in range(3):
            o.dist_ref[k] = float(ref[k])
        o.dist_min, o.dist_max = float(dmin), float(dmax)
    T = int(key_tile)
    ntx, nty = (W + T - 1) // T, (H + T - 1) // T
    W2, H2 = W // 2, H // 2
    nsamp = W * H + W2 * H2
    image = np.zeros((3, H, W))
    marginal = np.zeros((H, W), np.uint8)
    tcls = np.zeros((nty, ntx), np.uint8)
    full = np.zeros((4, H, W)) if want_samples else None
    low = np.zeros((4, max(H2, 1), max(W2, 1))) if want_samples else None
    lowimg = np.zeros((3, max(H2, 1), max(W2, 1)))
    off = np.zeros(nsamp + 1, np.int64)
    out = _Out()
    out.image, out.full, out.low, out.lowimg = _ptr(image), _ptr(full), _ptr(low), _ptr(lowimg)
    out.marginal, out.tile_class, out.order_off = _ptr(marginal), _ptr(tcls), _ptr(off)
    unchecked = np.zeros((H, W), np.uint8) if outcomes else None
    out.unchecked = _ptr(unchecked)
    sr = _SceneRef(scene)
    camc = _cam(cam)
    rc = lib().og_render(C.byref(sr.s), C.byref(camc), C.byref(o), C.byref(out))
    if rc != 0:
        raise ValueError("oracle render rejected its arguments")
    alt = None
    if outcomes:
        n_alt = int(out.n_alt)
        aoff = np.ctypeslib.as_array(out.alt_off, shape=(W * H + 1,)).copy()
        vals = np.ctypeslib.as_array(out.alt, shape=(n_alt * 3,)).reshape(n_alt, 3).copy() if n_alt else np.zeros((0, 3))
        alt4 = None
        if fovea is None:
            alt4 = np.ctypeslib.as_array(out.alt4, shape=(n_alt * 4,)).reshape(n_alt, 4).copy() if n_alt \
                else np.zeros((0, 4))
            lib().og_free(C.cast(out.alt4, C.c_void_p))
        lib().og_free(C.cast(out.alt_off, C.c_void_p))
        lib().og_free(C.cast(out.alt, C.c_void_p))
        alt = (aoff, vals)
    orders = None
    if want_orders:
        order = np.zeros(max(int(out.n_order), 1), np.int32)
        out.order, out.max_order = _ptr(order), len(order)
        o.outcomes = 0
        rc = lib().og_render(C.byref(sr.s), C.byref(camc), C.byref(o), C.byref(out))
        orders = (order[:int(out.n_order)], off.copy())
    stats = dict(zip(["valid", "instances", "evaluated", "kept", "blended", "marginal_px", "samples",
                      "unchecked_px"], [int(v) for v in out.stats[:8]]))
    return dict(image=image, marginal=marginal.astype(bool), tile_class=tcls, full=full, low=low,
                lowimg=lowimg if fovea is not None else None, orders=orders, stats=stats,
                alt=alt, unchecked=None if unchecked is None else unchecked.astype(bool),
                alt4=alt4 if outcomes else None)


def tile_lists(scene, cam, key_tile: int = 16, tile_cull: bool = True, visible=None, relax: float = 0.0,
               want_slack: bool = False):
    """-> (counts[nty, ntx], gids, keys) of the oracle's sorted per-tile instance lists,
    plus slack (qmin - r2 of each entry's Eq. 4 test) when want_slack.  relax > 0 adds the
    entries with 0 < qmin - r2 <= relax."""
    W, H, T = int(cam.width), int(cam.height), int(key_tile)
    vis = None if visible is None else np.ascontiguousarray(np.asarray(visible) != 0, dtype=np.uint8)
    vp = None if vis is None else C.c_void_p(vis.ctypes.data)
    ntx, nty = (W + T - 1) // T, (H + T - 1) // T
    counts = np.zeros(ntx * nty, np.int64)
    sr = _SceneRef(scene)
    camc = _cam(cam)
    tot = lib().og_tile_lists(C.byref(sr.s), C.byref(camc), T, int(tile_cull), vp, float(relax), _ptr(counts), None,
                              None, None, 0)
    gids = np.zeros(max(tot, 1), np.int32)
    keys = np.zeros(max(tot, 1))
    slack = np.zeros(max(tot, 1))
    lib().og_tile_lists(C.byref(sr.s), C.byref(camc), T, int(tile_cull), vp, float(relax), _ptr(counts), _ptr(gids),
                        _ptr(keys), _ptr(slack), len(gids))
    if want_slack:
        return counts.reshape(nty, ntx), gids[:tot], keys[:tot], slack[:tot]
    return counts.reshape(nty, ntx), gids[:tot], keys[:tot]


def alpha_relax(margin_alpha: float = None) -> float:
    """Eq. 4 exponent slack of the alpha margin: sigma G > (1 - m) / 255 <=> q < r2 - 2 ln(1 - m)."""
    m = MARGINS[0] if margin_alpha is None else margin_alpha
    return -2.0 * float(np.log1p(-m))


def num_threads() -> int:
    return int(lib().og_num_threads())
