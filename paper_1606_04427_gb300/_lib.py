"""ctypes declarations of the C ABI in ``include/splotch.h``.

Argument marshalling only: every step of the render runs in the CUDA library.
Loading fails loudly when the library has not been built; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import build as _build

OK, INVALID_ARG, OOM, CUDA, CAPACITY, TIMEOUT, UNSUPPORTED = range(7)
F32, F16, BF16 = 0, 1, 2
STORAGE = {"f32": F32, "f16": F16, "bf16": BF16}
OUT_ACCUM, SYNC, PLAN_GRAPH, TIMING, OUT_ADD, OUT_MAP, STABLE = 1, 2, 4, 8, 16, 32, 64

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class SceneDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_types", C.c_int32), ("type_begin", C.c_void_p),
                ("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("h", C.c_void_p),
                ("intensity", C.c_void_p), ("on_device", C.c_int32), ("storage", C.c_int32),
                ("cmap_rgb", C.c_void_p), ("cmap_len", C.c_void_p), ("brightness", C.c_void_p),
                ("i_min", C.c_void_p), ("i_max", C.c_void_p), ("i_log", C.c_void_p),
                ("allocator", Allocator), ("stream", C.c_void_p),
                ("col_vector", C.c_void_p), ("rgb", C.c_void_p)]


class CameraC(C.Structure):
    _fields_ = [("eye", C.c_double * 3), ("lookat", C.c_double * 3), ("up", C.c_double * 3),
                ("fov_deg", C.c_double), ("z_near", C.c_double), ("width", C.c_int32),
                ("height", C.c_int32), ("z_far", C.c_double)]


class RenderParamsC(C.Structure):
    _fields_ = [("tile", C.c_int32), ("rfac", C.c_float), ("sigma_over_R", C.c_float),
                ("r_min_px", C.c_float), ("block_particles", C.c_int32), ("flags", C.c_int32)]


class SplotchError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


_lib = None
_lock = threading.Lock()

# every symbol include/splotch.h declares, with its ctypes signature
SIGNATURES = {
    "splotch_default_params": ([], RenderParamsC),
    "splotch_create_scene": ([C.POINTER(SceneDesc), C.POINTER(C.c_void_p)], C.c_int),
    "splotch_destroy": ([C.c_void_p], C.c_int),
    "splotch_scene_info": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_camera_params": ([C.POINTER(CameraC), C.c_void_p, C.c_void_p], C.c_int),
    "splotch_render": ([C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(RenderParamsC), C.c_void_p,
                        C.c_void_p], C.c_int),
    "splotch_debug_raster": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC), C.c_void_p,
                              C.c_void_p], C.c_int),
    "splotch_debug_bins": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC), C.c_void_p,
                            C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_int64), C.c_void_p],
                           C.c_int),
    "splotch_plan_create": ([C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(RenderParamsC), C.c_double,
                             C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "splotch_plan_set_cameras": ([C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p], C.c_int),
    "splotch_plan_launch": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_plan_check": ([C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)], C.c_int),
    "splotch_plan_info": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_plan_destroy": ([C.c_void_p], C.c_int),
    "splotch_workspace_bytes": ([C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_int64], C.c_int64),
    "splotch_selftest_bounded_wait": ([C.c_int64, C.c_void_p], C.c_int),
    "splotch_final_transform": ([C.c_void_p, C.c_int64, C.c_void_p], C.c_int),
    "splotch_compose_maps": ([C.c_void_p, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_last_timing": ([C.c_void_p, C.c_void_p], C.c_int),
    "splotch_render_ordered": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC), C.c_void_p, C.c_void_p,
                                C.c_void_p], C.c_int),
    "splotch_debug_sort": ([C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_int32, C.c_void_p], C.c_int),
    "splotch_plan_set_brightness": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_plan_set_colormaps": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_render_streamed": ([C.POINTER(SceneDesc), C.c_int64, C.POINTER(CameraC), C.POINTER(RenderParamsC),
                                 C.c_void_p, C.c_void_p], C.c_int),
    "splotch_render_noalloc": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC), C.c_void_p,
                                C.c_void_p], C.c_int),
    "splotch_frame_fixed_bytes": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC)], C.c_int64),
    "splotch_frame_prepare": ([C.c_void_p, C.POINTER(CameraC), C.POINTER(RenderParamsC), C.c_void_p,
                               C.POINTER(C.c_void_p), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                               C.POINTER(C.c_int64)], C.c_int),
    "splotch_frame_render": ([C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "splotch_frame_destroy": ([C.c_void_p], C.c_int),
    "splotch_status_string": ([C.c_int], C.c_char_p),
    "splotch_last_error": ([], C.c_char_p),
}


def library_path() -> str:
    return _build.LIB_PATH


def load():
    """The loaded CUDA library; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(
                f"Splotch CUDA library not built ({path} missing): run "
                "paper_1606_04427_gb300.build.build() on a machine with nvcc")
        lib = C.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


def check(status: int, where: str) -> None:
    if status != OK:
        lib = load()
        detail = lib.splotch_last_error().decode(errors="replace")
        raise SplotchError(status, where, detail or lib.splotch_status_string(status).decode())


def camera_c(cam) -> CameraC:
    c = CameraC()
    c.eye[:] = [float(v) for v in cam.eye]
    c.lookat[:] = [float(v) for v in cam.lookat]
    c.up[:] = [float(v) for v in cam.up]
    c.fov_deg = float(cam.fov_deg)
    c.z_near = float(cam.z_near)
    c.z_far = float(getattr(cam, "z_far", 0.0) or 0.0)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c
