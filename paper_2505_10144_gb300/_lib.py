"""ctypes view of the C ABI in include/vrsplat.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "lib" / "libvrsplat.so"

STATUS = {0: "VRS_OK", 1: "VRS_ERR_INVALID", 2: "VRS_ERR_CAPACITY", 3: "VRS_ERR_CUDA", 4: "VRS_ERR_TIMEOUT",
          5: "VRS_ERR_UNSUPPORTED"}


class Gaussians(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p), ("n", C.c_int64), ("sh_degree", C.c_int)]


class GaussianGrads(C.Structure):
    _fields_ = [("mean", C.c_void_p), ("log_scale", C.c_void_p), ("quat", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class Camera(C.Structure):
    _fields_ = [("world_to_cam", C.c_float * 12), ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                ("cy", C.c_float), ("width", C.c_int), ("height", C.c_int), ("near_z", C.c_float)]


class Fovea(C.Structure):
    _fields_ = [("gaze_x", C.c_float), ("gaze_y", C.c_float), ("radius_px", C.c_float), ("band_px", C.c_float),
                ("mode", C.c_int), ("focus_tile", C.c_int), ("visible", C.c_void_p)]


class RenderOpts(C.Structure):
    _fields_ = [("sort_mode", C.c_int), ("win", C.c_int * 3), ("key_tile", C.c_int), ("bg", C.c_float * 3),
                ("stats", C.c_int)]


class Peaks(C.Structure):
    _fields_ = [("sm_count", C.c_int), ("max_sm_clock_khz", C.c_int), ("l2_bytes", C.c_int64),
                ("fp32_tflops", C.c_double), ("exp2_gops", C.c_double), ("logic_gops", C.c_double),
                ("l2_read_gbs", C.c_double), ("dram_read_gbs", C.c_double)]


# every symbol include/vrsplat.h declares
EXPORTED = ["vrs_create", "vrs_destroy", "vrs_reserve", "vrs_render", "vrs_render_backward", "vrs_check_status",
            "vrs_get_stats", "vrs_copy_instances", "vrs_project", "vrs_sort_pairs", "vrs_loss_l1_ssim",
            "vrs_adam_step", "vrs_profile_begin", "vrs_profile_end", "vrs_sort_pairs_noalloc", "vrs_update_views", "vrs_set_tuning",
            "vrs_net_forward", "vrs_net_backward", "vrs_net_periphery", "vrs_mse", "vrs_render_two_pass",
            "vrs_measure_peaks", "vrs_probe_orders", "vrs_test_bounded_wait", "vrs_render_stereo_reuse",
            "vrs_last_error"]

_lib = None


class VrsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load() -> C.CDLL:
    """Load libvrsplat.so; raises when it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(this package has no CPU or PyTorch fallback)")
    lib = C.CDLL(str(LIB_PATH), mode=os.RTLD_NOW | os.RTLD_LOCAL)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
    P = C.POINTER
    lib.vrs_create.argtypes = [P(vp), C.c_size_t]
    lib.vrs_destroy.argtypes = [vp]
    lib.vrs_reserve.argtypes = [vp, i32, i32, i32, i64, i64]
    lib.vrs_render.argtypes = [vp, P(Gaussians), i32, P(i32), P(Camera), P(Fovea), i32, P(RenderOpts), vp, vp, i32, vp]
    lib.vrs_render_two_pass.argtypes = [vp, P(Gaussians), i32, P(i32), P(Camera), P(Fovea), i32, P(RenderOpts), vp, vp]
    lib.vrs_render_stereo_reuse.argtypes = [vp, P(Gaussians), P(Camera), P(RenderOpts), C.c_float, vp, vp]
    lib.vrs_render_backward.argtypes = [vp, P(Gaussians), i32, P(i32), P(Camera), P(Fovea), i32, P(RenderOpts), vp,
                                        P(GaussianGrads), vp]
    lib.vrs_check_status.argtypes = [vp, vp, P(i64)]
    lib.vrs_get_stats.argtypes = [vp, vp, P(i64)]
    lib.vrs_copy_instances.argtypes = [vp, vp, vp, vp, i64, P(i64), vp]
    lib.vrs_project.argtypes = [vp, P(Gaussians), P(Camera), i32, vp, vp, vp, vp]
    lib.vrs_sort_pairs.argtypes = [vp, vp, vp, vp, vp, i64, i32, vp]
    lib.vrs_loss_l1_ssim.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp]
    lib.vrs_adam_step.argtypes = [vp, vp, vp, vp, i64, C.c_float, C.c_float, C.c_float, C.c_float, i32, vp]
    lib.vrs_sort_pairs_noalloc.argtypes = [vp, vp, vp, vp, i64, i32, vp, vp]
    lib.vrs_update_views.argtypes = [vp, P(Camera), P(Fovea), i32]
    lib.vrs_set_tuning.argtypes = [vp, i32]
    lib.vrs_net_forward.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp]
    lib.vrs_net_backward.argtypes = [vp, vp, vp, vp, vp, i32, i32, i32, vp, vp]
    lib.vrs_net_periphery.argtypes = [vp, vp, vp, vp, vp]
    lib.vrs_mse.argtypes = [vp, vp, vp, i64, vp, vp, vp]
    lib.vrs_profile_begin.argtypes = [vp, i32]
    lib.vrs_profile_end.argtypes = [vp, vp, P(C.c_double), P(i64)]
    lib.vrs_measure_peaks.argtypes = [P(Peaks), vp]
    lib.vrs_probe_orders.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp]
    lib.vrs_test_bounded_wait.argtypes = [vp, i32, vp]
    lib.vrs_last_error.argtypes = [vp]
    lib.vrs_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name != "vrs_last_error":
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib
