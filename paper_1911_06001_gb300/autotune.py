"""Autotuner for the trace launch.

Knobs that change only speed, never results: the trace kernel's block size
(64 / 128 / 256 threads), the rays each lane takes per warp tile (1 / 2 / 4 /
8), the number of top octree levels each block stages in shared memory (0-4,
for traces of one scene), the claim order of image tiles (row by row or
centre-out), the ray order (as given, grouped by direction, grouped by origin cell
then direction, or -- for rays that are the pixels of an image -- warp tiles
of 8 x 4 pixels) and the culling structure: the cluster level in one launch,
the cluster level as a culling launch plus a descent launch over the rays it
queued (SVO_TRACE_WAVEFRONT), or -- for scenes of 64 parts or more -- the
scene grid.  ``tune`` times every combination on the caller's rays with
CUDA events (L2 flushed between repetitions), keeps the fastest, and can
remember it in a JSON cache under a caller-chosen key (for example the scene
and ray-batch shape).  ``tune_batch`` does the same for a batch of uneven
scenes traced in one persistent launch (``Context.trace_batch``), keyed by the
batch's shape (``batch_key``).
"""

from __future__ import annotations

import itertools
import json
import os

import numpy as np

from . import (TRACE_CULL, TRACE_DEFAULT, TRACE_GRID, TRACE_IMAGE_TILES, TRACE_ORDER_DIR, TRACE_ORDER_ORIGIN,
               TRACE_REUSE, TRACE_SORT, TRACE_WAVEFRONT, Context, trace_image)

BLOCKS = (64, 128, 256)
RAYS_PER_LANE = (1, 2, 4, 8)
ORDERS = {"none": 0, "dir": TRACE_ORDER_DIR, "origin": TRACE_ORDER_ORIGIN, "image": TRACE_IMAGE_TILES}
_ORDER_BITS = TRACE_ORDER_DIR | TRACE_ORDER_ORIGIN | TRACE_IMAGE_TILES | 0xFFFF0000
CULLS = {"clusters": 0, "grid": TRACE_GRID, "wavefront": TRACE_WAVEFRONT}
_CULL_BITS = TRACE_GRID | TRACE_WAVEFRONT
GRID_MIN_PARTS = 64  # scenes from this size on carry a grid


def _time(ctx: Context, scene, rays, hits, flags: int, reps: int, flush) -> float:
    import torch

    evs = []
    for i in range(reps + 1):
        flush.fill_(i & 0xFF)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record()
        scene.trace(rays, hits, flags=flags)
        e[1].record()
        evs.append(e)
    torch.cuda.synchronize()
    return float(np.median([a.elapsed_time(b) for a, b in evs[1:]]))


def tune(ctx: Context, scene, rays, flags: int = TRACE_DEFAULT, reps: int = 5, blocks=BLOCKS,
         rays_per_lane=RAYS_PER_LANE, orders=None, cache_path: str | None = None,
         key: str | None = None, image_width: int = 0, culls=None, levels=(0,), tile_orders=(1,)) -> dict:
    """Time every (block, rays_per_lane, smem levels, order, cull) on ``rays``
    (CUDA [n, 8]) traced against ``scene``; apply and return the fastest.  The
    "image" order is tried only when ``image_width`` (row-major pixels) is
    given, the "grid" culling only for scenes of GRID_MIN_PARTS parts or more
    traced with CULL | SORT and without REUSE."""
    import torch

    if cache_path and key:
        cached = load(cache_path).get(key)
        if cached:
            apply(ctx, cached)
            return cached
    if orders is None:
        orders = tuple(o for o in ORDERS if o != "image" or image_width > 0)
    if culls is None:
        cs = TRACE_CULL | TRACE_SORT
        two = (flags & cs) == cs and not (flags & TRACE_REUSE)
        grid_ok = two and getattr(scene, "n_parts", 0) >= GRID_MIN_PARTS
        culls = ("clusters", "wavefront") + (("grid",) if grid_ok else ()) if two else ("clusters",)
    hits = torch.empty((rays.shape[0], 2), dtype=torch.int64, device=rays.device)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=rays.device)
    old = ctx.trace_config()
    old_levels = ctx.smem_levels()
    old_tiles = ctx.tile_order()
    table = []
    for b, r, lv, o, c, to in itertools.product(blocks, rays_per_lane, levels, orders, culls, tile_orders):
        if o != "image" and to != tile_orders[0]:
            continue  # the tile order only matters for image tiles
        ctx.set_trace_config(b, r)
        ctx.set_smem_levels(lv)
        ctx.set_tile_order(to)
        f = (flags & ~(_ORDER_BITS | _CULL_BITS)) | _flag(o, image_width) | CULLS[c]
        table.append({"block": b, "rays_per_lane": r, "smem_levels": lv, "order": o, "cull": c, "tile_order": to,
                      "ms": _time(ctx, scene, rays, hits, f, reps, flush)})
    ctx.set_trace_config(*old)
    ctx.set_smem_levels(old_levels)
    ctx.set_tile_order(old_tiles)
    best = min(table, key=lambda x: x["ms"])
    default = next((x for x in table if x["block"] == 128 and x["rays_per_lane"] == 1 and x["order"] == "none"
                    and x["cull"] == "clusters" and x["smem_levels"] == 0 and x["tile_order"] == tile_orders[0]),
                   None)
    result = dict(best)
    result["default_ms"] = default["ms"] if default else None
    result["n_rays"] = int(rays.shape[0])
    result["image_width"] = int(image_width)
    result["table"] = table
    apply(ctx, result)
    if cache_path and key:
        data = load(cache_path)
        data[key] = result
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1)
        os.replace(tmp, cache_path)
    return result


def _flag(order: str, image_width: int) -> int:
    return trace_image(image_width) if order == "image" else ORDERS[order]


def apply(ctx: Context, cfg: dict) -> int:
    """Set the tuned launch shape on ``ctx``; returns the flags (order, culling) to OR into trace flags."""
    ctx.set_trace_config(int(cfg["block"]), int(cfg["rays_per_lane"]))
    ctx.set_smem_levels(int(cfg.get("smem_levels", 0)))
    ctx.set_tile_order(int(cfg.get("tile_order", 1)))
    return order_flag(cfg)


def order_flag(cfg: dict) -> int:
    """The tuned ray-order and culling flags (configurations cached before the
    culling knob existed read as the cluster level)."""
    return _flag(cfg["order"], int(cfg.get("image_width", 0))) | CULLS[cfg.get("cull", "clusters")]


def load(cache_path: str) -> dict:
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            return json.load(f)
    return {}


def batch_key(items) -> str:
    """Cache key of a batch's shape: item count, ray count and part count of
    every item (the workload the tuned launch applies to)."""
    shape = ",".join(f"{int(it[1].shape[0])}x{int(it[0].n_parts)}" for it in items)
    import hashlib

    return f"batch:{len(items)}:{hashlib.sha256(shape.encode()).hexdigest()[:16]}"


def tune_batch(ctx: Context, items, flags: int = TRACE_DEFAULT, reps: int = 3, blocks=BLOCKS,
               rays_per_lane=RAYS_PER_LANE, orders=("none", "dir", "origin"), culls=None,
               cache_path: str | None = None, key: str | None = None, stream=None) -> dict:
    """Time every (block, rays_per_lane, order, cull) on a whole batch traced by
    one ``trace_batch`` launch (``items`` as for ``Context.trace_batch``);
    apply and return the fastest.  The grid is tried when some scene of the
    batch has GRID_MIN_PARTS parts or more.  ``key`` defaults to
    ``batch_key(items)``."""
    import torch

    key = key or batch_key(items)
    if cache_path:
        cached = load(cache_path).get(key)
        if cached:
            apply(ctx, cached)
            return cached
    if culls is None:
        cs = TRACE_CULL | TRACE_SORT
        big = any(getattr(it[0], "n_parts", 0) >= GRID_MIN_PARTS for it in items)
        two = (flags & cs) == cs and not (flags & TRACE_REUSE)
        culls = ("clusters", "wavefront") + (("grid",) if big else ()) if two else ("clusters",)
    dev = items[0][1].device
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    old = ctx.trace_config()
    table = []
    for b, r, o, c in itertools.product(blocks, rays_per_lane, orders, culls):
        ctx.set_trace_config(b, r)
        f = (flags & ~(_ORDER_BITS | _CULL_BITS)) | ORDERS[o] | CULLS[c]
        evs = []
        with torch.cuda.stream(st):
            for i in range(reps + 1):
                flush.fill_(i & 0xFF)
                e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
                e[0].record(st)
                ctx.trace_batch(items, flags=f, stream=st)
                e[1].record(st)
                evs.append(e)
        torch.cuda.synchronize()
        table.append({"block": b, "rays_per_lane": r, "smem_levels": 0, "order": o, "cull": c,
                      "ms": float(np.median([a.elapsed_time(z) for a, z in evs[1:]]))})
    ctx.set_trace_config(*old)
    best = min(table, key=lambda x: x["ms"])
    default = next((x for x in table if x["block"] == 128 and x["rays_per_lane"] == 1 and x["order"] == "none"
                    and x["cull"] == "clusters"), None)
    result = dict(best)
    result["default_ms"] = default["ms"] if default else None
    result["n_rays"] = int(sum(int(it[1].shape[0]) for it in items))
    result["image_width"] = 0
    result["key"] = key
    result["table"] = table
    apply(ctx, result)
    if cache_path:
        data = load(cache_path)
        data[key] = result
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1)
        os.replace(tmp, cache_path)
    return result
