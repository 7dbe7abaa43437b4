"""ctypes declarations of the C ABI in include/svoanim.h (marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsvoanim.so")

SVO_OK = 0
STATUS_NAMES = {
    0: "SVO_OK", -1: "SVO_ERR_ARG", -2: "SVO_ERR_OOM", -3: "SVO_ERR_HANDLE", -4: "SVO_ERR_CUDA",
    -5: "SVO_ERR_TIMEOUT", -6: "SVO_ERR_ADMIT", -7: "SVO_ERR_NAN", -8: "SVO_ERR_SINGULAR", -9: "SVO_ERR_LIMIT",
    -10: "SVO_ERR_DEVICE",
}

TRACE_CULL = 1
TRACE_SORT = 2
TRACE_FP64_FIX = 4
TRACE_STATS = 8
TRACE_DEFER_FIX = 16
TRACE_ORDER_DIR = 32
TRACE_ORDER_ORIGIN = 64
TRACE_IMAGE_TILES = 128
TRACE_REUSE = 256
TRACE_GRID = 512
TRACE_WAVEFRONT = 1024
TRACE_DEFAULT = TRACE_CULL | TRACE_SORT | TRACE_FP64_FIX


def trace_image(width: int) -> int:
    """Flag bits saying the rays are a row-major image of ``width`` pixels (warps take 8 x 4 tiles)."""
    if not 0 < int(width) < 65536:
        raise ValueError("image width must be in 1..65535")
    return TRACE_IMAGE_TILES | (int(width) << 16)

RAY_UNCERTAIN = 1
RAY_FIXED = 2
RAY_T_REFINED = 4
TILE_ORDER_ROWS = 0
TILE_ORDER_CENTER = 1


def ray_t_bound_exp(flags):
    """Certified error exponent of unfixed T_REFINED rays (SVO_RAY_T_BOUND_EXP):
    |t - t_exact| <= 2^e max(t_exact, leaf diagonal / |d|); 127 = unbounded."""
    import numpy as np

    return ((np.asarray(flags).astype(np.uint32) >> np.uint32(8)) & np.uint32(0xFF)).astype(np.int32) - 128
RAY_REUSED = 8

MAX_DEPTH = 16
MAX_PARTS = 1024
NOALLOC_MAX_RAYS = 262144
COLOR_INVALID = 0xFFFFFFFF

# every symbol include/svoanim.h declares
EXPORTS = [
    "svo_ctx_create", "svo_ctx_destroy", "svo_last_error", "svo_status_string", "svo_check_device",
    "svo_set_trace_config", "svo_get_trace_config", "svo_set_smem_levels", "svo_get_smem_levels",
    "svo_set_tile_order", "svo_get_tile_order",
    "svo_build_host", "svo_upload", "svo_release", "svo_asset_info", "svo_read_asset",
    "scene_create", "scene_destroy", "scene_set_transforms", "scene_set_transforms_device",
    "scene_set_transforms_trs", "scene_refit", "scene_refit_batch",
    "scene_read_poses", "scene_read_clusters", "trace_rays", "trace_batch", "trace_fix_pending",
    "trace_rays_host", "trace_rays_noalloc", "svo_raygen_pinhole", "trace_hit_colors",
    "trace_shade",
]


class SvoDesc(C.Structure):
    _fields_ = [("depth", C.c_int32), ("n_leaves", C.c_uint64), ("leaf_ids", C.c_void_p), ("leaf_rgb", C.c_void_p)]


class SvoTraceStats(C.Structure):
    _fields_ = [(n, C.c_ulonglong) for n in ("rays", "flagged", "fixed", "parts_tested", "parts_entered",
                                             "nodes_visited", "leaves_tested", "passes", "flag_winner",
                                             "flag_overlap", "flag_width", "reused")]


class SvoCamera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3), ("fov_y_deg", C.c_float),
                ("tmin", C.c_float), ("tmax", C.c_float)]


class SvoBatchItem(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("rays", C.c_void_p), ("n", C.c_uint64), ("hits", C.c_void_p),
                ("ray_flags", C.c_void_p), ("image_width", C.c_uint32)]


class SvoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load the compiled library; raises if it is missing (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"libsvoanim.so not built at {p}; run __graft_entry__.build() (no CPU fallback exists)")
    L = C.CDLL(p)
    vp, i32, u32, u64 = C.c_void_p, C.c_int32, C.c_uint32, C.c_uint64
    pvp = C.POINTER(C.c_void_p)
    sig = {
        "svo_ctx_create": ([i32, pvp], i32),
        "svo_ctx_destroy": ([vp], i32),
        "svo_last_error": ([], C.c_char_p),
        "svo_status_string": ([i32], C.c_char_p),
        "svo_check_device": ([vp], i32),
        "svo_set_trace_config": ([vp, i32, i32], i32),
        "svo_get_trace_config": ([vp, C.POINTER(i32), C.POINTER(i32)], i32),
        "svo_set_smem_levels": ([vp, i32], i32),
        "svo_get_smem_levels": ([vp, C.POINTER(i32)], i32),
        "svo_set_tile_order": ([vp, i32], i32),
        "svo_get_tile_order": ([vp, C.POINTER(i32)], i32),
        "svo_build_host": ([C.POINTER(SvoDesc), C.POINTER(u64), C.POINTER(u64), vp, vp], i32),
        "svo_upload": ([vp, C.POINTER(SvoDesc), C.POINTER(u32)], i32),
        "svo_release": ([vp, u32], i32),
        "svo_asset_info": ([vp, u32, C.POINTER(i32), C.POINTER(u64), C.POINTER(u64)], i32),
        "svo_read_asset": ([vp, u32, vp, vp], i32),
        "scene_create": ([vp, i32, vp, vp, pvp], i32),
        "scene_destroy": ([vp], i32),
        "scene_set_transforms": ([vp, vp, vp], i32),
        "scene_set_transforms_device": ([vp, vp, vp], i32),
        "scene_set_transforms_trs": ([vp, vp, vp], i32),
        "scene_refit": ([vp, vp], i32),
        "scene_refit_batch": ([C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), i32, vp], i32),
        "scene_read_poses": ([vp, vp, vp, vp, vp, vp], i32),
        "scene_read_clusters": ([vp, C.POINTER(i32), vp, vp, vp], i32),
        "trace_rays": ([vp, vp, u64, vp, vp, u32, vp, vp], i32),
        "trace_batch": ([vp, C.POINTER(SvoBatchItem), i32, u32, vp, vp], i32),
        "trace_fix_pending": ([vp, vp], i32),
        "trace_rays_host": ([vp, vp, u64, vp, vp, u32, vp], i32),
        "trace_rays_noalloc": ([vp, vp, u64, vp, vp, u32, vp], i32),
        "svo_raygen_pinhole": ([vp, C.POINTER(SvoCamera), u32, u32, vp, vp], i32),
        "trace_hit_colors": ([vp, vp, u64, u32, vp, vp], i32),
        "trace_shade": ([vp, vp, vp, u64, vp, C.c_float, u32, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def check(status: int) -> None:
    if status != SVO_OK:
        msg = load().svo_last_error()
        raise SvoError(status, msg.decode() if msg else "")
