"""FP64 CPU oracle for ray casting against animated sparse voxel octrees.

TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  The CUDA library never calls it and
shares no code with it (see svo_oracle.c for the definition it computes).

Python side: argument marshalling with ctypes plus a convenience wrapper that
runs the per-frame pose pipeline (compose, invert) and the tracer for a scene
built by ``synthetic``.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        up32 = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
        up64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
        L.oracle_compose.argtypes = [C.c_int, ip, dp, dp]
        L.oracle_compose.restype = C.c_int
        L.oracle_invert.argtypes = [C.c_int, dp, dp]
        L.oracle_invert.restype = C.c_int
        L.oracle_part_sphere.argtypes = [C.c_int, dp, C.c_void_p, dp]
        L.oracle_part_sphere.restype = None
        L.oracle_ray_sphere.argtypes = [dp, dp, dp, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.oracle_ray_sphere.restype = C.c_int
        L.oracle_slab.argtypes = [dp, dp, dp, dp, C.c_double, C.c_double, dp]
        L.oracle_slab.restype = C.c_int
        L.oracle_asset_new.argtypes = [C.c_int, C.c_int64, up64]
        L.oracle_asset_new.restype = C.c_void_p
        L.oracle_asset_free.argtypes = [C.c_void_p]
        L.oracle_asset_free.restype = None
        L.oracle_asset_leaves.argtypes = [C.c_void_p]
        L.oracle_asset_leaves.restype = C.c_int64
        L.oracle_trace.argtypes = [C.c_int, C.POINTER(C.c_void_p), dp, C.c_int64, dp, dp, up32, up64, dp, C.c_int,
                                   C.c_int]
        L.oracle_trace.restype = C.c_int
        L.oracle_ray_valid.argtypes = [dp]
        L.oracle_ray_valid.restype = C.c_int
        _lib = L
    return _lib


MISS_PART = 0xFFFFFFFF
MISS_VOXEL = 0xFFFFFFFFFFFFFFFF


def compose(parent, local) -> np.ndarray:
    parent = np.ascontiguousarray(parent, dtype=np.int32)
    local = np.ascontiguousarray(local, dtype=np.float64).reshape(-1, 12)
    world = np.zeros_like(local)
    if lib().oracle_compose(len(parent), parent, local, world) != 0:
        raise ValueError("parent[i] must be < i")
    return world


def invert(world) -> np.ndarray:
    world = np.ascontiguousarray(world, dtype=np.float64).reshape(-1, 12)
    inv = np.zeros_like(world)
    if lib().oracle_invert(world.shape[0], world, inv) != 0:
        raise ValueError("singular pose")
    return inv


def part_spheres(world, boxes=None) -> np.ndarray:
    """Bounding sphere per part (Sec. IV-A) of the local box ``boxes[p] = (lo3,
    hi3)`` of its content, or of the unit cube when ``boxes`` is None."""
    world = np.ascontiguousarray(world, dtype=np.float64).reshape(-1, 12)
    out = np.zeros((world.shape[0], 4))
    bx = None
    if boxes is not None:
        bx = np.ascontiguousarray(boxes, dtype=np.float64).reshape(world.shape[0], 6)
    lib().oracle_part_sphere(world.shape[0], world, None if bx is None else bx.ctypes.data, out)
    return out


def occupied_box(depth: int, leaf_ids) -> np.ndarray:
    """Local box (lo3, hi3) of the occupied leaves of an asset: the cells'
    min and max+1 corners over 2^depth; the unit cube for an empty asset."""
    ids = np.asarray(leaf_ids, dtype=np.uint64)
    if ids.size == 0:
        return np.array([0.0, 0.0, 0.0, 1.0, 1.0, 1.0])
    m = np.uint64((1 << depth) - 1)
    d = np.uint64(depth)
    xyz = np.stack([ids & m, (ids >> d) & m, (ids >> (d + d)) & m], 1).astype(np.float64)
    return np.concatenate([xyz.min(0), xyz.max(0) + 1.0]) / float(1 << depth)


def ray_sphere(o, d, sphere4):
    """Eq. 4 (general direction length).  Returns (hit, t_in, t_out)."""
    ti, to = C.c_double(0), C.c_double(0)
    h = lib().oracle_ray_sphere(np.ascontiguousarray(o, np.float64), np.ascontiguousarray(d, np.float64),
                                np.ascontiguousarray(sphere4, np.float64), C.byref(ti), C.byref(to))
    return bool(h), ti.value, to.value


def slab(o, d, lo, hi, t_lo=0.0, t_hi=float("inf")):
    """Closed-box slab test.  Returns (hit, t0, t1)."""
    out = np.zeros(2)
    h = lib().oracle_slab(*(np.ascontiguousarray(v, np.float64) for v in (o, d, lo, hi)), float(t_lo), float(t_hi),
                          out)
    return bool(h), float(out[0]), float(out[1])


class OracleAsset:
    """The oracle's own octree of one asset (sorted Morton codes of its leaves)."""

    def __init__(self, depth: int, leaf_ids):
        ids = np.ascontiguousarray(leaf_ids, dtype=np.uint64)
        self.depth = depth
        self.handle = lib().oracle_asset_new(depth, ids.shape[0], ids)
        if not self.handle:
            raise ValueError("bad asset")

    @property
    def n_leaves(self) -> int:
        return int(lib().oracle_asset_leaves(self.handle))

    def __del__(self):
        h, self.handle = getattr(self, "handle", None), None
        if h and _lib is not None:
            _lib.oracle_asset_free(h)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def trace(part_assets, inv, rays, mode: int = 1, threads: int | None = None) -> dict:
    """Closest hit of every ray.  ``part_assets``: one OracleAsset per part;
    ``inv``: [P,12] FP64 world->local poses; ``rays``: [n,8] (any float dtype,
    converted exactly to FP64)."""
    rays = np.ascontiguousarray(np.asarray(rays).astype(np.float64)).reshape(-1, 8)
    inv = np.ascontiguousarray(inv, dtype=np.float64).reshape(-1, 12)
    n = rays.shape[0]
    P = len(part_assets)
    handles = (C.c_void_p * max(P, 1))(*[a.handle for a in part_assets])
    out_t = np.zeros(n)
    out_s = np.zeros(n)
    out_p = np.zeros(n, dtype=np.uint32)
    out_v = np.zeros(n, dtype=np.uint64)
    rc = lib().oracle_trace(P, handles, inv, n, rays, out_t, out_p, out_v, out_s, int(mode),
                            int(threads or default_threads()))
    if rc != 0:
        raise ValueError("oracle_trace failed")
    return {"t": out_t, "part": out_p, "voxel": out_v, "second": out_s}


def ray_valid(rays) -> np.ndarray:
    """Per ray, whether it is a ray the method traces (the oracle's rule:
    finite origin and direction, no NaN bound, largest direction component
    magnitude in [2^-60, 2^60]); anything else is reported as a miss."""
    rays = np.ascontiguousarray(np.asarray(rays).astype(np.float64)).reshape(-1, 8)
    return np.array([bool(lib().oracle_ray_valid(np.ascontiguousarray(r))) for r in rays], dtype=bool)


def trs_to_local(rts) -> np.ndarray:
    """Sec. III-B poses (rotation R, translation t, octree dimensions s; rows
    ``R (9, row-major) | t | s``) as local 3x4 affines: x_parent = R (s * x) + t."""
    rts = np.asarray(rts, dtype=np.float64).reshape(-1, 15)
    out = np.zeros((rts.shape[0], 12))
    for p, row in enumerate(rts):
        R, t, s = row[:9].reshape(3, 3), row[9:12], row[12:15]
        out[p] = np.hstack([R @ np.diag(s), t[:, None]]).ravel()
    return out


def trace_octree_dims(part_leaf_ids, part_depth, rts, rays) -> dict:
    """Brute-force closest hit with the pose split as Sec. III-B describes,
    for scenes whose parts are all roots: the ray goes to each part's frame by
    the rigid inverse only (Eq. 2-3: R^T (o - t), R^T d), and the octree keeps
    its dimensions s, so the leaf at cell v of a depth-D asset is the box
    [v s / 2^D, (v + 1) s / 2^D] per axis.  Every leaf of every part is
    slab-tested (closed box, t in [tmin, tmax]); the smallest (t, part,
    voxel) wins.  Small inputs only."""
    rays = np.asarray(rays, dtype=np.float64).reshape(-1, 8)
    rts = np.asarray(rts, dtype=np.float64).reshape(-1, 15)
    n = rays.shape[0]
    best_t = np.full(n, np.inf)
    best_p = np.full(n, MISS_PART, dtype=np.uint32)
    best_v = np.full(n, MISS_VOXEL, dtype=np.uint64)
    valid = ray_valid(rays)
    for p, row in enumerate(rts):
        R, tv, dims = row[:9].reshape(3, 3), row[9:12], row[12:15]
        ids = np.asarray(part_leaf_ids[p], dtype=np.uint64)
        if ids.size == 0:
            continue
        D = int(part_depth[p])
        m = np.uint64((1 << D) - 1)
        cell = np.stack([(ids >> np.uint64(k * D)) & m for k in range(3)], axis=1).astype(np.float64)
        lo = cell * dims / 2.0 ** D
        hi = (cell + 1.0) * dims / 2.0 ** D
        for r in range(n):
            if not valid[r]:
                continue
            o = R.T @ (rays[r, 0:3] - tv)
            d = R.T @ rays[r, 4:7]
            a = np.full(ids.size, rays[r, 3])
            b = np.full(ids.size, rays[r, 7])
            ok = np.ones(ids.size, dtype=bool)
            for k in range(3):
                if d[k] == 0.0:
                    ok &= (lo[:, k] <= o[k]) & (o[k] <= hi[:, k])
                    continue
                ta = (lo[:, k] - o[k]) / d[k]
                tb = (hi[:, k] - o[k]) / d[k]
                a = np.maximum(a, np.minimum(ta, tb))
                b = np.minimum(b, np.maximum(ta, tb))
            ok &= a <= b
            if not ok.any():
                continue
            cand = np.nonzero(ok)[0]
            # lexicographic (t, voxel) within the part; parts are visited in increasing order
            order = np.lexsort((ids[cand], a[cand]))
            j = cand[order[0]]
            if a[j] < best_t[r]:
                best_t[r], best_p[r], best_v[r] = a[j], p, ids[j]
    return {"t": best_t, "part": best_p, "voxel": best_v}


COLOR_INVALID = 0xFFFFFFFF


def hit_colors(leaf_lists, part_asset, part, voxel, background: int = 0) -> np.ndarray:
    """Colour of each hit, as the hit buffer carries it for shading (Sec. IV-C):
    the colour given with the hit voxel's id in the part's asset leaf list (the
    first occurrence when an id is listed twice), ``background`` for a miss,
    COLOR_INVALID when the part or voxel names no leaf.

    ``leaf_lists``: per asset a pair (leaf_ids, rgb or None); ``part_asset``:
    asset index of each part; ``part``/``voxel``: the hits."""
    part = np.asarray(part, dtype=np.uint32)
    voxel = np.asarray(voxel, dtype=np.uint64)
    out = np.full(part.shape, background, dtype=np.uint32)
    hit = part != MISS_PART
    out[hit] = COLOR_INVALID
    for p in np.unique(part[hit]):
        sel = np.nonzero(part == p)[0]
        if int(p) >= len(part_asset):
            continue
        ids, rgb = leaf_lists[int(part_asset[int(p)])]
        ids = np.asarray(ids, dtype=np.uint64)
        if rgb is None:
            rgb = np.zeros(ids.shape, dtype=np.uint32)
        # a stable sort keeps equal ids in list order, so the left end of each
        # run of equal ids is the first occurrence
        order = np.argsort(ids, kind="stable")
        sids = ids[order]
        pos = np.searchsorted(sids, voxel[sel], side="left")
        found = pos < sids.shape[0]
        found[found] = sids[pos[found]] == voxel[sel][found]
        out[sel[found]] = np.asarray(rgb, dtype=np.uint32)[order[pos[found]]]
    return out


def shade(colors, part, voxel, depths, inv, rays, light, ambient: float, background: int = 0):
    """Headless shading of hits (the hit buffer's colour and normal, Sec. IV-C),
    in FP64.  Per hit: the entry face of the hit leaf's closed box (the axis
    whose near-plane t is largest; the lower axis index on a tie) gives the
    local normal -sign(d'_k) e_k, mapped to world space by the inverse
    transpose (row k of A^-1) and normalised; a ray that starts inside the box
    (entry before tmin) takes -d/|d|.  Lambert: s = ambient + (1 - ambient)
    max(0, n . l) with l the unit light direction, and every 8-bit channel c
    becomes min(255, floor(c s + 1/2)).  Misses keep ``background``, invalid
    colours stay invalid.

    ``colors``: hit_colors of the hits; ``depths``: asset depth per part;
    ``inv``: [P,12] world->local poses.  Returns (rgb uint32, ambiguous bool):
    a pixel is ambiguous when its face choice, its inside test or a channel's
    rounding lies within 1e-9 (relative) of a decision boundary, where two
    correct FP64 evaluations may round differently."""
    colors = np.asarray(colors, dtype=np.uint32)
    part = np.asarray(part, dtype=np.uint32)
    voxel = np.asarray(voxel, dtype=np.uint64)
    rays = np.asarray(rays, dtype=np.float64).reshape(-1, 8)
    inv = np.asarray(inv, dtype=np.float64).reshape(-1, 12)
    out = colors.copy()
    amb = np.zeros(part.shape, dtype=bool)
    hit = (part != MISS_PART) & (colors != COLOR_INVALID)
    out[part == MISS_PART] = background
    idx = np.nonzero(hit)[0]
    if idx.size == 0:
        return out, amb
    L = np.asarray(light, dtype=np.float64)
    L = L / np.linalg.norm(L)
    p = part[idx].astype(np.int64)
    D = np.asarray(depths, dtype=np.int64)[p]
    m = (np.uint64(1) << D.astype(np.uint64)) - np.uint64(1)
    v = voxel[idx]
    cell = np.stack([v & m, (v >> D.astype(np.uint64)) & m, (v >> (2 * D).astype(np.uint64)) & m], 1).astype(np.float64)
    size = np.ldexp(1.0, -D)[:, None]
    lo = cell * size
    hi = lo + size
    M = inv[p].reshape(-1, 3, 4)
    o = rays[idx, 0:3]
    d = rays[idx, 4:7]
    tmin = rays[idx, 3]
    ol = np.einsum("nij,nj->ni", M[:, :, :3], o) + M[:, :, 3]
    dl = np.einsum("nij,nj->ni", M[:, :, :3], d)
    near = np.where(dl > 0, lo, hi)
    with np.errstate(divide="ignore", invalid="ignore"):
        tk = np.where(dl != 0, (near - ol) / dl, -np.inf)
    te = tk.max(1)
    k = tk.argmax(1)  # first index of the maximum: the lower axis on a tie
    scale = np.maximum(1.0, np.abs(te))
    second = np.sort(tk, 1)[:, -2]
    amb_face = te - second <= 1e-9 * scale
    inside = te < tmin
    amb_inside = np.abs(te - tmin) <= 1e-9 * np.maximum(1.0, np.abs(tmin))
    sign = np.sign(dl[np.arange(idx.size), k])
    n = -sign[:, None] * M[np.arange(idx.size), k, :3]
    n = np.where(inside[:, None], -d, n)
    n = n / np.linalg.norm(n, axis=1)[:, None]
    s = ambient + (1.0 - ambient) * np.maximum(0.0, n @ L)
    c = colors[idx]
    chans = np.stack([(c >> 16) & 255, (c >> 8) & 255, c & 255], 1).astype(np.float64)
    x = chans * s[:, None] + 0.5
    q = np.minimum(255.0, np.floor(x))
    frac = x - np.floor(x)
    amb_round = (np.minimum(frac, 1.0 - frac) <= 1e-9 * np.maximum(1.0, x)).any(1)
    qi = q.astype(np.uint32)
    out[idx] = (qi[:, 0] << 16) | (qi[:, 1] << 8) | qi[:, 2]
    amb[idx] = amb_face | amb_inside | amb_round
    return out, amb


class SceneOracle:
    """Oracle view of a ``synthetic.Scene``: assets built once, poses per frame."""

    def __init__(self, scene):
        self.scene = scene
        self.assets = [OracleAsset(a.depth, a.leaf_ids) for a in scene.assets]

    def boxes(self) -> np.ndarray:
        """Occupied box of every part's asset, [P, 6]."""
        b = [occupied_box(a.depth, a.leaf_ids) for a in self.scene.assets]
        return np.array([b[int(i)] for i in self.scene.part_asset])

    def poses(self, local=None):
        local = self.scene.local if local is None else local
        world = compose(self.scene.parent, local)
        return world, invert(world)

    def hit_colors(self, hits: dict, background: int = 0) -> np.ndarray:
        leaf_lists = [(a.leaf_ids, a.rgb) for a in self.scene.assets]
        return hit_colors(leaf_lists, self.scene.part_asset, hits["part"], hits["voxel"], background)

    def shade(self, hits: dict, rays, light, ambient: float, background: int = 0, local=None):
        colors = self.hit_colors(hits, background)
        _, inv = self.poses(local)
        depths = [self.scene.assets[int(a)].depth for a in self.scene.part_asset]
        return shade(colors, hits["part"], hits["voxel"], depths, inv, rays, light, ambient, background)

    def trace(self, rays, local=None, mode: int = 1, threads: int | None = None) -> dict:
        world, inv = self.poses(local)
        parts = [self.assets[int(a)] for a in self.scene.part_asset]
        return trace(parts, inv, rays, mode=mode, threads=threads)
