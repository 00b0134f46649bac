"""Seeded synthetic inputs: Gaussian scenes, pinhole cameras, head trajectories, gaze.

This module only draws random numbers and builds camera poses.  It holds none of the
rasterizer's arithmetic (no projection, no spherical-harmonics evaluation, no blending),
so both the CUDA path and the CPU oracle may take their inputs from it.

Conventions (OpenCV): camera x right, y down, z forward; a camera is a world-to-camera
rigid transform [R|t] (row-major 3x4) plus pinhole intrinsics fx, fy, cx, cy, with pixel
(x, y) centred at (x + 0.5, y + 0.5).  The world frame uses the same axes as a camera
with identity pose, so "up" is -y and a head yaw turns about the world y axis.

The paper's scenes (Mip-NeRF 360, Tanks & Temples, Deep Blending; Sec. 5) are not
available; these generators stand in for them, with Gaussian counts in the range the
paper reports for its Mini-Splatting models (0.19M-1.0M, Table "performance per scene").
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 20250515

# sqrt(pi): half-width of the uniform draw of a degree-0 SH coefficient that makes the
# degree-0 colour uniform in [0, 1] (the degree-0 basis function is 1 / (2 sqrt(pi))).
_DC_HALF_RANGE = math.sqrt(math.pi)


def rng_for(config_index: int, salt: int = 0) -> np.random.Generator:
    """Generator for workload ``config_index`` (seed 20250515 + k, optional salt)."""
    return np.random.default_rng(BASE_SEED + config_index + 1000003 * salt)


@dataclass
class Scene:
    """Gaussian parameters in SoA layout, float32, C-contiguous.

    mean[3][N], log_scale[3][N], quat[4][N] (w, x, y, z; not normalised),
    opacity_logit[N], sh[K][3][N] with K = (sh_degree + 1)^2.
    """
    mean: np.ndarray
    log_scale: np.ndarray
    quat: np.ndarray
    opacity_logit: np.ndarray
    sh: np.ndarray
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.mean.shape[1])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(np.ascontiguousarray(self.mean[:, idx]),
                     np.ascontiguousarray(self.log_scale[:, idx]),
                     np.ascontiguousarray(self.quat[:, idx]),
                     np.ascontiguousarray(self.opacity_logit[idx]),
                     np.ascontiguousarray(self.sh[:, :, idx]), self.sh_degree)

    def copy(self) -> "Scene":
        return Scene(self.mean.copy(), self.log_scale.copy(), self.quat.copy(),
                     self.opacity_logit.copy(), self.sh.copy(), self.sh_degree)

    def arrays(self):
        return (self.mean, self.log_scale, self.quat, self.opacity_logit, self.sh)


@dataclass
class Camera:
    """Pinhole camera: world_to_cam is 3x4 row-major [R|t]."""
    world_to_cam: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near_z: float = 0.2

    def center(self) -> np.ndarray:
        R = self.world_to_cam[:, :3].astype(np.float64)
        t = self.world_to_cam[:, 3].astype(np.float64)
        return -R.T @ t


@dataclass
class Fovea:
    """Gaze-centred focus circle: full resolution inside radius, linear band outside."""
    gaze_x: float
    gaze_y: float
    radius_px: float
    band_px: float
    periphery_div: int = 2


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _random_params(rng: np.random.Generator, n: int, sh_degree: int, mean: np.ndarray) -> Scene:
    log_scale = rng.normal(-3.5, 0.5, size=(3, n))
    quat = rng.normal(0.0, 1.0, size=(4, n))
    quat /= np.linalg.norm(quat, axis=0, keepdims=True)
    opacity_logit = rng.normal(0.0, 1.0, size=n)
    k = (sh_degree + 1) ** 2
    sh = np.empty((k, 3, n))
    sh[0] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, size=(3, n))
    if k > 1:
        sh[1:] = rng.normal(0.0, 0.2, size=(k - 1, 3, n))
    return Scene(_f32(mean), _f32(log_scale), _f32(quat), _f32(opacity_logit), _f32(sh), sh_degree)


def tiny_scene(n: int = 10_000, rng: np.random.Generator | None = None) -> Scene:
    """Means uniform in [-1,1]^2 x [2,4]; log-scale N(-3.5, 0.5); SH degree 0."""
    rng = rng_for(0) if rng is None else rng
    mean = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 4, n)])
    return _random_params(rng, n, 0, mean)


def shell_scene(n: int, rng: np.random.Generator, sh_degree: int = 3,
                half_size: float = 3.0, jitter: float = 0.05) -> Scene:
    """Room-shaped shell: uniform by area on the six faces of a cube of side 2*half_size
    centred on the head origin, plus N(0, jitter) noise along each axis."""
    face = rng.integers(0, 6, size=n)
    a = rng.uniform(-half_size, half_size, size=n)
    b = rng.uniform(-half_size, half_size, size=n)
    axis = face // 2
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    mean = np.empty((3, n))
    for ax in range(3):
        o1, o2 = [x for x in range(3) if x != ax]
        sel = axis == ax
        mean[ax, sel] = sign[sel] * half_size
        mean[o1, sel] = a[sel]
        mean[o2, sel] = b[sel]
    mean += rng.normal(0.0, jitter, size=mean.shape)
    return _random_params(rng, n, sh_degree, mean)


def focal_for_hfov(width: int, hfov_deg: float) -> float:
    return (width / 2.0) / math.tan(math.radians(hfov_deg) / 2.0)


def open_room_with_landscape(n_room: int, n_far: int, rng: np.random.Generator, sh_degree: int = 3,
                             half_size: float = 3.0, jitter: float = 0.05, far_range=(150.0, 600.0)) -> Scene:
    """A scene with distant content: the room shell without its ceiling (the y = -half
    face; y points down) and its front wall (z = +half), so that part of the view looks
    out, and a landscape of n_far Gaussians around the head at distances uniform in
    far_range, azimuth uniform, elevation uniform in [-10, 30] degrees above the horizon,
    with log-scales N(log(0.012 d), 0.5) (about the angular size of the room's Gaussians).
    The room's Gaussians come first."""
    face = rng.choice(np.array([0, 1, 3, 4]), size=n_room)
    a = rng.uniform(-half_size, half_size, size=n_room)
    b = rng.uniform(-half_size, half_size, size=n_room)
    axis = face // 2
    sign = np.where(face % 2 == 0, -1.0, 1.0)
    mean = np.empty((3, n_room))
    for ax in range(3):
        o1, o2 = [x for x in range(3) if x != ax]
        sel = axis == ax
        mean[ax, sel] = sign[sel] * half_size
        mean[o1, sel] = a[sel]
        mean[o2, sel] = b[sel]
    mean += rng.normal(0.0, jitter, size=mean.shape)
    room = _random_params(rng, n_room, sh_degree, mean)
    d = rng.uniform(far_range[0], far_range[1], size=n_far)
    az = rng.uniform(-math.pi, math.pi, size=n_far)
    el = np.radians(rng.uniform(-10.0, 30.0, size=n_far))
    fmean = np.stack([d * np.cos(el) * np.sin(az), -d * np.sin(el), d * np.cos(el) * np.cos(az)])
    far = _random_params(rng, n_far, sh_degree, fmean)
    far.log_scale = _f32(np.log(0.012 * d)[None, :] + rng.normal(0.0, 0.5, size=(3, n_far)))
    return Scene(*[np.ascontiguousarray(np.concatenate([x, y], axis=-1)) for x, y in zip(room.arrays(), far.arrays())],
                 sh_degree)


def cyclopean_camera(left: Camera, right: Camera) -> Camera:
    """The camera between two eyes: the left eye's rotation and intrinsics, its centre
    at the midpoint of the eye centres."""
    c = 0.5 * (np.asarray(left.center(), dtype=np.float64) + np.asarray(right.center(), dtype=np.float64))
    R = left.world_to_cam[:, :3].astype(np.float64)
    return camera_from_pose(R.T, c, left.width, left.height, left.fx, left.fy, left.near_z, left.cx, left.cy)


def head_rotation(yaw: float, pitch: float = 0.0) -> np.ndarray:
    """Camera-to-world rotation (columns: right, down, forward) for a yaw about the world
    y axis followed by a pitch about the camera x axis."""
    cy_, sy_ = math.cos(yaw), math.sin(yaw)
    Ry = np.array([[cy_, 0, sy_], [0, 1, 0], [-sy_, 0, cy_]])
    cp, sp = math.cos(pitch), math.sin(pitch)
    Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
    return Ry @ Rx


def camera_from_pose(c2w_rot: np.ndarray, position, width: int, height: int,
                     fx: float, fy: float | None = None, near_z: float = 0.2,
                     cx: float | None = None, cy: float | None = None) -> Camera:
    R = np.asarray(c2w_rot, dtype=np.float64).T
    t = -R @ np.asarray(position, dtype=np.float64)
    w2c = np.concatenate([R, t[:, None]], axis=1)
    return Camera(_f32(w2c), float(fx), float(fx if fy is None else fy),
                  float(width / 2.0 if cx is None else cx), float(height / 2.0 if cy is None else cy),
                  int(width), int(height), float(near_z))


def identity_camera(width: int, height: int, hfov_deg: float) -> Camera:
    f = focal_for_hfov(width, hfov_deg)
    return camera_from_pose(np.eye(3), (0, 0, 0), width, height, f)


def stereo_cameras(head_pos, yaw: float, width: int, height: int, hfov_deg: float,
                   ipd: float = 0.064, pitch: float = 0.0) -> list[Camera]:
    """Left and right eye cameras, eyes at -/+ ipd/2 along the head's x axis."""
    Rc2w = head_rotation(yaw, pitch)
    right = Rc2w[:, 0]
    f = focal_for_hfov(width, hfov_deg)
    hp = np.asarray(head_pos, dtype=np.float64)
    return [camera_from_pose(Rc2w, hp + s * 0.5 * ipd * right, width, height, f) for s in (-1.0, 1.0)]


def gaze_in_disc(rng: np.random.Generator, width: int, height: int, frac: float = 0.2):
    r = frac * width * math.sqrt(rng.uniform())
    th = rng.uniform(0, 2 * math.pi)
    return width / 2.0 + r * math.cos(th), height / 2.0 + r * math.sin(th)


def fovea_for(width: int, gaze, radius_frac: float = 0.15, band_frac: float = 0.1,
              periphery_div: int = 2) -> Fovea:
    r = radius_frac * width
    return Fovea(float(gaze[0]), float(gaze[1]), float(r), float(band_frac * r), periphery_div)


def lens_mask(width: int, height: int, eye: int, half_w: float = 0.535, half_h: float = 0.555,
              nasal: float = 0.03) -> np.ndarray:
    """[height, width] uint8 headset visibility mask standing in for an OpenXR hidden-area
    mesh: 1 inside an ellipse with semi-axes half_w * width and half_h * height, its
    centre moved by nasal * width / 2 towards the nose (eye -1 left: right, +1 right:
    left).  With the defaults about 11% of the 32x32 tiles of a 2064x2208 eye have no
    visible pixel."""
    cx = 0.5 * width * (1.0 - nasal * eye)
    cy = 0.5 * height
    y, x = np.mgrid[0:height, 0:width]
    inside = ((x + 0.5 - cx) / (half_w * width)) ** 2 + ((y + 0.5 - cy) / (half_h * height)) ** 2 <= 1.0
    return inside.astype(np.uint8)


@dataclass
class Frame:
    cameras: list
    foveas: list


@dataclass
class VRWorkload:
    """A stereo head trajectory at 72 Hz pose steps: yaw +-45 deg at 0.25 Hz, translation
    +-0.1 m, gaze drawn per frame within 0.2 W of the image centre."""
    width: int = 2064
    height: int = 2208
    hfov_deg: float = 110.0
    frames: list = field(default_factory=list)


def vr_trajectory(n_frames: int, rng: np.random.Generator, width: int = 2064, height: int = 2208,
                  hfov_deg: float = 110.0, rate_hz: float = 72.0) -> VRWorkload:
    wl = VRWorkload(width, height, hfov_deg)
    for f in range(n_frames):
        t = f / rate_hz
        yaw = math.radians(45.0) * math.sin(2 * math.pi * 0.25 * t)
        pos = (0.1 * math.sin(2 * math.pi * 0.25 * t + 1.0), 0.0, 0.1 * math.sin(2 * math.pi * 0.125 * t))
        cams = stereo_cameras(pos, yaw, width, height, hfov_deg)
        gz = gaze_in_disc(rng, width, height)
        fovs = [fovea_for(width, gz), fovea_for(width, gz)]
        wl.frames.append(Frame(cams, fovs))
    return wl


def batched_poses(n_poses: int, rng: np.random.Generator, width: int = 2064, height: int = 2208,
                  hfov_deg: float = 110.0) -> list[Frame]:
    """Smooth yaw/translation path: yaw_k = 20 deg sin(2 pi k / n + phi), translation
    0.15 m (cos, 0, sin)(2 pi k / n); one gaze point per pose shared by both eyes."""
    phi = rng.uniform(0, 2 * math.pi)
    out = []
    for k in range(n_poses):
        a = 2 * math.pi * k / n_poses
        yaw = math.radians(20.0) * math.sin(a + phi)
        pos = (0.15 * math.cos(a), 0.0, 0.15 * math.sin(a))
        cams = stereo_cameras(pos, yaw, width, height, hfov_deg)
        gz = gaze_in_disc(rng, width, height)
        out.append(Frame(cams, [fovea_for(width, gz), fovea_for(width, gz)]))
    return out


def ring_views(n_views: int, width: int, height: int, hfov_deg: float,
               rng: np.random.Generator | None = None) -> list[Camera]:
    """n_views cameras at the head origin, yaws spread evenly over the full turn, with a
    small seeded pitch, used by the fine-tuning workload."""
    f = focal_for_hfov(width, hfov_deg)
    cams = []
    for k in range(n_views):
        pitch = 0.0 if rng is None else rng.uniform(-0.1, 0.1)
        pos = (0.0, 0.0, 0.0) if rng is None else tuple(rng.normal(0, 0.05, 3))
        cams.append(camera_from_pose(head_rotation(2 * math.pi * k / n_views, pitch), pos,
                                     width, height, f))
    return cams


def perturbed(scene: Scene, rng: np.random.Generator, mean_sigma: float = 0.01,
              log_scale_sigma: float = 0.1) -> Scene:
    s = scene.copy()
    s.mean = _f32(s.mean + rng.normal(0, mean_sigma, s.mean.shape))
    s.log_scale = _f32(s.log_scale + rng.normal(0, log_scale_sigma, s.log_scale.shape))
    return s
