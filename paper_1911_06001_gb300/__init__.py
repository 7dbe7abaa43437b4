"""GB300 (sm_103a) ray casting against scenes of animated sparse voxel octrees.

Thin Python layer over the C ABI of ``libsvoanim.so`` (include/svoanim.h):
argument marshalling only.  PyTorch provides device memory and streams; every
per-frame and per-ray step runs in the library's CUDA kernels.  Importing the
package does not need a GPU; creating a ``Context`` does, and there is no CPU
fallback: a missing library raises ``ImportError``.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (  # noqa: F401
    COLOR_INVALID,
    MAX_DEPTH,
    MAX_PARTS,
    RAY_FIXED,
    RAY_REUSED,
    RAY_T_REFINED,
    TILE_ORDER_CENTER,
    TILE_ORDER_ROWS,
    RAY_UNCERTAIN,
    TRACE_CULL,
    TRACE_DEFAULT,
    TRACE_DEFER_FIX,
    TRACE_ORDER_DIR,
    TRACE_ORDER_ORIGIN,
    TRACE_FP64_FIX,
    TRACE_GRID,
    TRACE_IMAGE_TILES,
    TRACE_REUSE,
    TRACE_WAVEFRONT,
    TRACE_SORT,
    TRACE_STATS,
    SvoError,
    ray_t_bound_exp,
    trace_image,
)

MISS_PART = 0xFFFFFFFF
MISS_VOXEL = 0xFFFFFFFFFFFFFFFF
HIT_BYTES = 16
RAY_FLOATS = 8


def _stream_ptr(stream) -> C.c_void_p:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(int(stream.cuda_stream))


def _ptr(t) -> C.c_void_p:
    return C.c_void_p(0 if t is None else int(t.data_ptr()))


def build_host(depth: int, leaf_ids, rgb=None):
    """Host-only octree build (no GPU): returns (nodes uint32[n_nodes, 2], leaf rgb uint32[n_leaves])."""
    lib = _lib.load()
    ids = np.ascontiguousarray(leaf_ids, dtype=np.uint64)
    col = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint32)
    d = _lib.SvoDesc(depth, ids.shape[0], ids.ctypes.data, 0 if col is None else col.ctypes.data)
    nn, nl = C.c_uint64(0), C.c_uint64(0)
    _lib.check(lib.svo_build_host(C.byref(d), C.byref(nn), C.byref(nl), None, None))
    nodes = np.zeros((nn.value, 2), dtype=np.uint32)
    out_rgb = np.zeros(nl.value, dtype=np.uint32)
    _lib.check(lib.svo_build_host(C.byref(d), C.byref(nn), C.byref(nl), nodes.ctypes.data if nn.value else None,
                                  out_rgb.ctypes.data if nl.value else None))
    return nodes, out_rgb


class Context:
    """A library context on one CUDA device (owns assets, scenes and scratch)."""

    def __init__(self, device: int = 0):
        self.lib = _lib.load()
        h = C.c_void_p()
        _lib.check(self.lib.svo_ctx_create(int(device), C.byref(h)))
        self.h = h
        self.device = device

    def upload(self, depth: int, leaf_ids, rgb=None) -> int:
        ids = np.ascontiguousarray(leaf_ids, dtype=np.uint64)
        col = None if rgb is None else np.ascontiguousarray(rgb, dtype=np.uint32)
        d = _lib.SvoDesc(depth, ids.shape[0], ids.ctypes.data, 0 if col is None else col.ctypes.data)
        out = C.c_uint32(0)
        _lib.check(self.lib.svo_upload(self.h, C.byref(d), C.byref(out)))
        return out.value

    def release(self, handle: int) -> None:
        _lib.check(self.lib.svo_release(self.h, C.c_uint32(handle)))

    def asset_info(self, handle: int):
        d, nn, nl = C.c_int32(0), C.c_uint64(0), C.c_uint64(0)
        _lib.check(self.lib.svo_asset_info(self.h, C.c_uint32(handle), C.byref(d), C.byref(nn), C.byref(nl)))
        return {"depth": d.value, "n_nodes": nn.value, "n_leaves": nl.value}

    def read_asset(self, handle: int):
        """An asset's device data: (nodes uint32[n_nodes, 2], leaf rgb uint32[n_leaves])."""
        info = self.asset_info(handle)
        nodes = np.zeros((info["n_nodes"], 2), dtype=np.uint32)
        rgb = np.zeros(info["n_leaves"], dtype=np.uint32)
        _lib.check(self.lib.svo_read_asset(self.h, C.c_uint32(handle), nodes.ctypes.data, rgb.ctypes.data))
        return nodes, rgb

    def scene(self, part_assets, parent) -> "Scene":
        return Scene(self, part_assets, parent)

    def set_trace_config(self, block: int = 128, rays_per_lane: int = 1) -> None:
        _lib.check(self.lib.svo_set_trace_config(self.h, int(block), int(rays_per_lane)))

    def trace_config(self) -> tuple:
        b, r = C.c_int32(0), C.c_int32(0)
        _lib.check(self.lib.svo_get_trace_config(self.h, C.byref(b), C.byref(r)))
        return b.value, r.value

    def set_smem_levels(self, levels: int) -> None:
        """Top octree levels (0-4) one-scene traces stage in shared memory (speed only)."""
        _lib.check(self.lib.svo_set_smem_levels(self.h, int(levels)))

    def smem_levels(self) -> int:
        v = C.c_int32(0)
        _lib.check(self.lib.svo_get_smem_levels(self.h, C.byref(v)))
        return v.value

    def set_tile_order(self, order: int) -> None:
        """Claim order of image tiles: TILE_ORDER_ROWS or TILE_ORDER_CENTER (speed only)."""
        _lib.check(self.lib.svo_set_tile_order(self.h, int(order)))

    def tile_order(self) -> int:
        v = C.c_int32(0)
        _lib.check(self.lib.svo_get_tile_order(self.h, C.byref(v)))
        return v.value

    def check_device(self) -> None:
        _lib.check(self.lib.svo_check_device(self.h))

    def trace_batch(self, items, flags: int = TRACE_DEFAULT, stats=None, stream=None) -> None:
        """items: list of (scene, rays, hits, ray_flags-or-None[, image_width]) with device tensors;
        image_width > 0 says the item's rays are a row-major image of that width."""
        arr = (_lib.SvoBatchItem * max(len(items), 1))()
        for i, item in enumerate(items):
            sc, rays, hits, rf = item[:4]
            width = int(item[4]) if len(item) > 4 else 0
            arr[i] = _lib.SvoBatchItem(sc.h.value, rays.data_ptr(), rays.shape[0], hits.data_ptr(),
                                       0 if rf is None else rf.data_ptr(), width)
        _lib.check(self.lib.trace_batch(self.h, arr, len(items), int(flags), _ptr(stats), _stream_ptr(stream)))

    def refit_batch(self, scenes, local_dev=None, stream=None) -> None:
        """scene_refit of several scenes in one launch (a block per scene).
        local_dev: None, or one entry per scene, each None or a CUDA float64
        tensor of that scene's [P, 12] local poses."""
        n = len(scenes)
        if n == 0:
            return
        hs = (C.c_void_p * n)(*[sc.h.value for sc in scenes])
        if local_dev is None:
            ptrs = None
        else:
            if len(local_dev) != n:
                raise ValueError("local_dev needs one entry per scene")
            for sc, t in zip(scenes, local_dev):
                if t is not None and (t.dtype.itemsize != 8 or not t.is_cuda or not t.is_contiguous()
                                      or t.numel() != 12 * sc.n_parts):
                    raise ValueError("local_dev entries: contiguous CUDA float64 tensors of n_parts*12")
            ptrs = (C.c_void_p * n)(*[None if t is None else t.data_ptr() for t in local_dev])
        _lib.check(self.lib.scene_refit_batch(hs, ptrs, n, _stream_ptr(stream)))

    def raygen(self, eye, target, width: int, height: int, fov_y_deg: float = 60.0, up=(0.0, 1.0, 0.0),
               tmin: float = 0.0, tmax: float = float("inf"), rays=None, stream=None):
        """Pinhole primary rays generated on the device: returns a CUDA float32 tensor [W*H, 8]."""
        import torch

        if rays is None:
            rays = torch.empty((width * height, RAY_FLOATS), dtype=torch.float32, device=f"cuda:{self.device}")
        cam = _lib.SvoCamera((C.c_float * 3)(*eye), (C.c_float * 3)(*target), (C.c_float * 3)(*up), fov_y_deg, tmin,
                             tmax)
        _lib.check(self.lib.svo_raygen_pinhole(self.h, C.byref(cam), width, height, _ptr(rays), _stream_ptr(stream)))
        return rays

    def fix_pending(self, stream=None) -> None:
        """Run the FP64 pass deferred by a trace issued with TRACE_DEFER_FIX on ``stream``."""
        _lib.check(self.lib.trace_fix_pending(self.h, _stream_ptr(stream)))

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.svo_ctx_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """Parts instancing uploaded assets in a transform tree (parent[i] < i or -1)."""

    def __init__(self, ctx: Context, part_assets, parent):
        self.ctx = ctx
        self.lib = ctx.lib
        a = np.ascontiguousarray(part_assets, dtype=np.uint32)
        p = np.ascontiguousarray(parent, dtype=np.int32)
        h = C.c_void_p()
        _lib.check(self.lib.scene_create(ctx.h, int(a.shape[0]), a.ctypes.data, p.ctypes.data, C.byref(h)))
        self.h = h
        self.n_parts = int(a.shape[0])

    def set_transforms(self, local, stream=None) -> None:
        m = np.ascontiguousarray(local, dtype=np.float64).reshape(self.n_parts, 12)
        _lib.check(self.lib.scene_set_transforms(self.h, m.ctypes.data, _stream_ptr(stream)))

    def set_transforms_trs(self, rts, stream=None) -> None:
        """Poses as rotation, translation and per-axis octree dimensions
        (Sec. III-B): [P, 15] FP64 rows ``R (9, row-major) | t (3) | s (3)``."""
        m = np.ascontiguousarray(rts, dtype=np.float64).reshape(self.n_parts, 15)
        _lib.check(self.lib.scene_set_transforms_trs(self.h, m.ctypes.data, _stream_ptr(stream)))

    def set_transforms_device(self, local_dev, stream=None) -> None:
        _lib.check(self.lib.scene_set_transforms_device(self.h, _ptr(local_dev), _stream_ptr(stream)))

    def refit(self, stream=None) -> None:
        _lib.check(self.lib.scene_refit(self.h, _stream_ptr(stream)))

    def read_poses(self, stream=None) -> dict:
        P = self.n_parts
        w = np.zeros((P, 12))
        iv = np.zeros((P, 12))
        f = np.zeros((P, 12), dtype=np.float32)
        s = np.zeros((P, 4), dtype=np.float32)
        _lib.check(self.lib.scene_read_poses(self.h, w.ctypes.data, iv.ctypes.data, f.ctypes.data, s.ctypes.data,
                                             _stream_ptr(stream)))
        return {"world": w, "inv": iv, "inv_f32": f, "sphere": s}

    def read_clusters(self, stream=None) -> dict:
        n = C.c_int32(0)
        _lib.check(self.lib.scene_read_clusters(self.h, C.byref(n), None, None, _stream_ptr(stream)))
        s = np.zeros((n.value, 4), dtype=np.float32)
        o = np.zeros(self.n_parts, dtype=np.int32)
        _lib.check(self.lib.scene_read_clusters(self.h, C.byref(n), s.ctypes.data, o.ctypes.data,
                                                _stream_ptr(stream)))
        return {"sphere": s, "order": o}

    def trace(self, rays, hits=None, flags: int = TRACE_DEFAULT, ray_flags=None, stats=None, stream=None):
        """rays: CUDA float32 tensor [n, 8]; returns hits (CUDA int64 tensor [n, 2])."""
        import torch

        if rays.dtype != torch.float32 or rays.dim() != 2 or rays.shape[1] != RAY_FLOATS or not rays.is_cuda:
            raise ValueError("rays must be a CUDA float32 tensor [n, 8]")
        rays = rays.contiguous()
        n = rays.shape[0]
        if hits is None:
            hits = torch.empty((n, 2), dtype=torch.int64, device=rays.device)
        _lib.check(self.lib.trace_rays(self.h, _ptr(rays), n, _ptr(hits), _ptr(ray_flags), int(flags), _ptr(stats),
                                       _stream_ptr(stream)))
        return hits

    def hit_colors(self, hits, background: int = 0, out=None, stream=None):
        """Leaf colours (0x00RRGGBB as int32) of hits from ``trace``; ``background`` for misses."""
        import torch

        if hits.dtype != torch.int64 or hits.dim() != 2 or hits.shape[1] != 2 or not hits.is_cuda:
            raise ValueError("hits must be a CUDA int64 tensor [n, 2]")
        n = hits.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=hits.device)
        _lib.check(self.lib.trace_hit_colors(self.h, _ptr(hits), n, int(background), _ptr(out), _stream_ptr(stream)))
        return out

    def shade(self, rays, hits, light, ambient: float = 0.2, background: int = 0, out=None, stream=None):
        """Lambert-shaded 0x00RRGGBB image (int32) of ``hits`` traced from ``rays`` (CUDA tensors)."""
        import torch

        if hits.dtype != torch.int64 or hits.dim() != 2 or hits.shape[1] != 2 or not hits.is_cuda:
            raise ValueError("hits must be a CUDA int64 tensor [n, 2]")
        if rays.dtype != torch.float32 or rays.shape != (hits.shape[0], RAY_FLOATS) or not rays.is_cuda:
            raise ValueError("rays must be a CUDA float32 tensor [n, 8] matching hits")
        n = hits.shape[0]
        if out is None:
            out = torch.empty(n, dtype=torch.int32, device=hits.device)
        lv = (C.c_float * 3)(*[float(x) for x in light])
        _lib.check(self.lib.trace_shade(self.h, _ptr(rays), _ptr(hits), n, lv, float(ambient), int(background),
                                        _ptr(out), _stream_ptr(stream)))
        return out

    def trace_host(self, rays_host, hits_host, flags: int = TRACE_DEFAULT, ray_flags_host=None, stream=None):
        """Trace rays held in host memory (CPU tensors, ideally pinned) into host hits (async on ``stream``)."""
        n = rays_host.shape[0]
        _lib.check(self.lib.trace_rays_host(self.h, _ptr(rays_host), n, _ptr(hits_host), _ptr(ray_flags_host),
                                            int(flags), _stream_ptr(stream)))
        return hits_host

    def close(self) -> None:
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.scene_destroy(self.h)
            self.h = C.c_void_p()


def decode_hits(hits) -> dict:
    """Split packed 16-byte hits (tensor or ndarray) into t / part / voxel numpy arrays."""
    a = hits.detach().cpu().numpy() if hasattr(hits, "detach") else np.asarray(hits)
    a = np.ascontiguousarray(a).view(np.uint32).reshape(-1, 4)
    t = a[:, 0].copy().view(np.float32)
    part = a[:, 1].copy()
    voxel = a[:, 2].astype(np.uint64) | (a[:, 3].astype(np.uint64) << np.uint64(32))
    return {"t": t, "part": part, "voxel": voxel}


def new_stats(device="cuda"):
    import torch

    return torch.zeros(12, dtype=torch.int64, device=device)


def read_stats(stats) -> dict:
    names = ("rays", "flagged", "fixed", "parts_tested", "parts_entered", "nodes_visited", "leaves_tested", "passes",
             "flag_winner", "flag_overlap", "flag_width", "reused")
    v = stats.detach().cpu().numpy().astype(np.uint64)
    return {n: int(x) for n, x in zip(names, v)}
