"""Seeded scene, pose and ray generators (inputs only; see the package docstring).

Conventions shared by every consumer of these arrays:

* An asset (one static sparse voxel octree) of depth ``D`` is given by its set of
  occupied leaf cells at the finest level.  A cell ``(x, y, z)`` with integer
  coordinates in ``[0, 2**D)`` is packed as the voxel id
  ``x | y << D | z << 2D`` (uint64).  Leaf lists are sorted and unique.
* Leaf colours are 8-bit RGB packed as ``0x00RRGGBB`` (uint32), one per leaf,
  in the order of the leaf list.
* A part's pose is the affine map from its local frame to its parent's frame,
  stored row-major as 3x4 ``[A | b]`` (12 float64).  ``parent[i] < i`` or ``-1``.
  The asset's local frame is the unit cube ``[0, 1]^3`` with the octree origin at
  a corner (the paper's Fig. 2 and the text around Eq. 3).
* A ray is 8 float32: ``ox, oy, oz, tmin, dx, dy, dz, tmax`` (Eq. 1,
  ``R(t) = r_o + t r_d`` restricted to ``tmin <= t <= tmax``).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1911_06001


def config_seed(config_idx: int, k: int = 0) -> int:
    """Seed for the k-th random stream of a workload (PR1=0, ART=1, BAT=2, PREC=3, SRV=4)."""
    return SEED_BASE + config_idx * 1000 + k


# --------------------------------------------------------------------------- ids

def pack_ids(x, y, z, depth: int) -> np.ndarray:
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    d = np.uint64(depth)
    return x | (y << d) | (z << (d + d))


def unpack_ids(ids, depth: int):
    ids = np.asarray(ids, dtype=np.uint64)
    m = np.uint64((1 << depth) - 1)
    d = np.uint64(depth)
    return (ids & m).astype(np.int64), ((ids >> d) & m).astype(np.int64), ((ids >> (d + d)) & m).astype(np.int64)


def rgb_hash(x, y, z) -> np.ndarray:
    """Deterministic 24-bit colour per cell (a spatial hash; any fixed function would do)."""
    x = np.asarray(x, dtype=np.uint64)
    y = np.asarray(y, dtype=np.uint64)
    z = np.asarray(z, dtype=np.uint64)
    h = (x * np.uint64(73856093)) ^ (y * np.uint64(19349663)) ^ (z * np.uint64(83492791))
    h ^= h >> np.uint64(13)
    return (h & np.uint64(0xFFFFFF)).astype(np.uint32)


# ---------------------------------------------------------------- voxelisation

def _column_shell(n: int, zlo_o, zhi_o, zlo_i, zhi_i, xs, ys):
    """Cells of the outer z-interval minus the inner z-interval, per (x, y) column.

    All bounds are inclusive integer arrays over the columns ``(xs, ys)``; an
    interval with ``lo > hi`` is empty.  Returns (x, y, z) int64 arrays.
    """
    zlo_o = np.maximum(zlo_o, 0)
    zhi_o = np.minimum(zhi_o, n - 1)
    inner_empty = zlo_i > zhi_i
    # first run: [zlo_o, min(zhi_o, zlo_i - 1)]  (whole outer when inner is empty)
    a_lo = zlo_o
    a_hi = np.where(inner_empty, zhi_o, np.minimum(zhi_o, zlo_i - 1))
    # second run: [max(zlo_o, zhi_i + 1), zhi_o]  (none when inner is empty)
    b_lo = np.maximum(zlo_o, zhi_i + 1)
    b_hi = np.where(inner_empty, zlo_o - 1, zhi_o)
    out = []
    for lo, hi in ((a_lo, a_hi), (b_lo, b_hi)):
        cnt = np.maximum(hi - lo + 1, 0)
        tot = int(cnt.sum())
        if tot == 0:
            continue
        rx = np.repeat(xs, cnt)
        ry = np.repeat(ys, cnt)
        start = np.repeat(lo, cnt)
        offs = np.arange(tot, dtype=np.int64) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        out.append((rx, ry, start + offs))
    if not out:
        e = np.zeros(0, dtype=np.int64)
        return e, e, e
    return tuple(np.concatenate([o[k] for o in out]) for k in range(3))


def _zrange(cz, h):
    """Integer cells z with |z + 0.5 - cz| <= h (h may be NaN for empty)."""
    lo = np.ceil(cz - h - 0.5)
    hi = np.floor(cz + h - 0.5)
    bad = ~np.isfinite(h)
    lo = np.where(bad, 1, lo).astype(np.int64)
    hi = np.where(bad, 0, hi).astype(np.int64)
    return lo, hi


def ellipsoid_shell(depth: int, center, axes, thickness: float):
    """Cells whose centre p satisfies  f_out(p) <= 1  and  f_in(p) > 1.

    ``f(p) = sum_k ((p_k - c_k) / a_k)^2`` with outer semi-axes ``axes`` and inner
    semi-axes ``axes - thickness`` (all in cell units).  A sphere shell of radius
    ``r`` and thickness 2 is therefore ``r - 2 < |p - c| <= r``.
    """
    n = 1 << depth
    cx, cy, cz = (float(v) for v in center)
    a, b, c = (float(v) for v in axes)
    ai, bi, ci = a - thickness, b - thickness, c - thickness
    g = np.arange(n, dtype=np.float64) + 0.5
    x0 = max(int(math.floor(cx - a - 1)), 0)
    x1 = min(int(math.ceil(cx + a + 1)), n - 1)
    y0 = max(int(math.floor(cy - b - 1)), 0)
    y1 = min(int(math.ceil(cy + b + 1)), n - 1)
    xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1), indexing="ij")
    xs = xs.ravel().astype(np.int64)
    ys = ys.ravel().astype(np.int64)
    px, py = g[xs], g[ys]
    qo = 1.0 - ((px - cx) / a) ** 2 - ((py - cy) / b) ** 2
    with np.errstate(invalid="ignore"):
        ho = np.where(qo >= 0, c * np.sqrt(np.maximum(qo, 0)), np.nan)
        if ai > 0 and bi > 0 and ci > 0:
            qi = 1.0 - ((px - cx) / ai) ** 2 - ((py - cy) / bi) ** 2
            hi = np.where(qi >= 0, ci * np.sqrt(np.maximum(qi, 0)), np.nan)
        else:
            hi = np.full_like(ho, np.nan)
    zlo_o, zhi_o = _zrange(cz, ho)
    zlo_i, zhi_i = _zrange(cz, hi)
    # the inner test is strict (f_in > 1 keeps the cell): a cell exactly on the
    # inner surface has |z+0.5-cz| == h_in and is removed by the inclusive range.
    return _column_shell(n, zlo_o, zhi_o, zlo_i, zhi_i, xs, ys)


def capsule_shell(depth: int, center, radius: float, half_len: float, thickness: float):
    """Cells within ``radius`` of the z-aligned segment ``center +- half_len e_z`` but
    not within ``radius - thickness`` of it (cell units)."""
    n = 1 << depth
    cx, cy, cz = (float(v) for v in center)
    r_o, r_i = float(radius), float(radius) - thickness
    g = np.arange(n, dtype=np.float64) + 0.5
    x0 = max(int(math.floor(cx - r_o - 1)), 0)
    x1 = min(int(math.ceil(cx + r_o + 1)), n - 1)
    y0 = max(int(math.floor(cy - r_o - 1)), 0)
    y1 = min(int(math.ceil(cy + r_o + 1)), n - 1)
    xs, ys = np.meshgrid(np.arange(x0, x1 + 1), np.arange(y0, y1 + 1), indexing="ij")
    xs = xs.ravel().astype(np.int64)
    ys = ys.ravel().astype(np.int64)
    rho2 = (g[xs] - cx) ** 2 + (g[ys] - cy) ** 2
    with np.errstate(invalid="ignore"):
        ho = np.where(rho2 <= r_o * r_o, half_len + np.sqrt(np.maximum(r_o * r_o - rho2, 0)), np.nan)
        if r_i > 0:
            hi = np.where(rho2 <= r_i * r_i, half_len + np.sqrt(np.maximum(r_i * r_i - rho2, 0)), np.nan)
        else:
            hi = np.full_like(ho, np.nan)
    zlo_o, zhi_o = _zrange(cz, ho)
    zlo_i, zhi_i = _zrange(cz, hi)
    return _column_shell(n, zlo_o, zhi_o, zlo_i, zhi_i, xs, ys)


def noise_voxels(depth: int, p: float, rng: np.random.Generator):
    """Each cell independently occupied with probability p (dense draw; small depths only)."""
    n = 1 << depth
    occ = rng.random(n * n * n) < p
    idx = np.nonzero(occ)[0].astype(np.int64)
    # dense index order is x-fastest: i = x + n*y + n*n*z
    return idx % n, (idx // n) % n, idx // (n * n)


@dataclass
class Asset:
    """One static sparse voxel octree given by its occupied finest-level cells."""

    depth: int
    leaf_ids: np.ndarray  # uint64, sorted, unique
    rgb: np.ndarray  # uint32, per leaf

    @property
    def n_leaves(self) -> int:
        return int(self.leaf_ids.shape[0])


def make_asset(depth: int, *cell_sets) -> Asset:
    xs = np.concatenate([c[0] for c in cell_sets]) if cell_sets else np.zeros(0, np.int64)
    ys = np.concatenate([c[1] for c in cell_sets]) if cell_sets else np.zeros(0, np.int64)
    zs = np.concatenate([c[2] for c in cell_sets]) if cell_sets else np.zeros(0, np.int64)
    ids = np.unique(pack_ids(xs, ys, zs, depth))
    x, y, z = unpack_ids(ids, depth)
    return Asset(depth=depth, leaf_ids=ids, rgb=rgb_hash(x, y, z))


# ------------------------------------------------------------------- poses

def euler_xyz(ax: float, ay: float, az: float) -> np.ndarray:
    """Rotation R = Rz(az) @ Ry(ay) @ Rx(ax) (x applied first)."""
    cx, sx = math.cos(ax), math.sin(ax)
    cy, sy = math.cos(ay), math.sin(ay)
    cz, sz = math.cos(az), math.sin(az)
    rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]], dtype=np.float64)
    ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]], dtype=np.float64)
    rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]], dtype=np.float64)
    return rz @ ry @ rx


def axis_angle(axis, angle: float) -> np.ndarray:
    """Rodrigues rotation about a unit axis."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    kx = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]], dtype=np.float64)
    return np.eye(3) + math.sin(angle) * kx + (1.0 - math.cos(angle)) * (kx @ kx)


def affine12(a3x3, b3) -> np.ndarray:
    """Pack [A | b] row-major into 12 float64."""
    m = np.zeros((3, 4), dtype=np.float64)
    m[:, :3] = a3x3
    m[:, 3] = b3
    return m.reshape(12)


def _h4(m12) -> np.ndarray:
    """3x4 -> 4x4 homogeneous, used only to build poses from named joint pieces."""
    m = np.eye(4)
    m[:3, :] = np.asarray(m12, dtype=np.float64).reshape(3, 4)
    return m


@dataclass
class Scene:
    """A set of parts, each an instance of an asset with a pose relative to its parent."""

    name: str
    assets: list
    part_asset: np.ndarray  # int32[P]
    parent: np.ndarray  # int32[P]
    local: np.ndarray  # float64[P, 12]
    meta: dict = field(default_factory=dict)

    @property
    def n_parts(self) -> int:
        return int(self.part_asset.shape[0])


# -------------------------------------------------------------------- rays

def pinhole_rays(eye, target, width: int, height: int, fov_deg: float = 60.0, up=(0.0, 1.0, 0.0),
                 tmin: float = 0.0, tmax: float = float("inf")) -> np.ndarray:
    """Primary rays of a pinhole camera, row-major pixel order (index = j*W + i).

    ``fov_deg`` is the vertical field of view.  Directions are unit length and
    the result is rounded to float32 (both sides trace these exact float32 rays).
    """
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    upv = np.asarray(up, dtype=np.float64)
    if abs(float(np.dot(upv / np.linalg.norm(upv), f))) > 0.999:
        upv = np.array([1.0, 0.0, 0.0]) if abs(f[0]) < 0.9 else np.array([0.0, 0.0, 1.0])
    r = np.cross(f, upv)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = math.tan(math.radians(fov_deg) * 0.5)
    aspect = width / height
    i = np.arange(width, dtype=np.float64)
    j = np.arange(height, dtype=np.float64)
    sx = (2.0 * (i + 0.5) / width - 1.0) * th * aspect
    sy = (1.0 - 2.0 * (j + 0.5) / height) * th
    d = f[None, None, :] + sx[None, :, None] * r[None, None, :] + sy[:, None, None] * u[None, None, :]
    d /= np.linalg.norm(d, axis=2, keepdims=True)
    n = width * height
    out = np.empty((n, 8), dtype=np.float32)
    out[:, 0:3] = eye[None, :]
    out[:, 3] = tmin
    out[:, 4:7] = d.reshape(n, 3)
    out[:, 7] = tmax
    return out


def random_rays(n: int, rng: np.random.Generator, box_lo, box_hi, tmin: float = 0.0,
                tmax: float = float("inf")) -> np.ndarray:
    """Incoherent rays: origins uniform in a box, directions uniform on the sphere."""
    lo = np.asarray(box_lo, dtype=np.float64)
    hi = np.asarray(box_hi, dtype=np.float64)
    o = lo + (hi - lo) * rng.random((n, 3))
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = np.empty((n, 8), dtype=np.float32)
    out[:, 0:3] = o
    out[:, 3] = tmin
    out[:, 4:7] = d
    out[:, 7] = tmax
    return out


# -------------------------------------------------------------------- PR1

def pr1_scene(seed: int | None = None, depth: int = 6, noise_p: float = 0.05) -> Scene:
    """4 rigid parts in a 2-level hierarchy, each a seeded sphere shell + 5 % noise.

    Root R centred on the world origin; children C1..C3 are placed 1.2 part widths
    from the root centre along the root's +x, -x and +y axes.  Every part gets a
    rotation with Euler angles uniform in [-pi/4, pi/4].
    """
    rng = np.random.default_rng(config_seed(0) if seed is None else seed)
    n = 1 << depth
    half = n / 2.0
    assets = []
    for _ in range(4):
        c = np.array([half, half, half]) + rng.uniform(-2.0, 2.0, 3) * (n / 64.0)
        r = rng.uniform(20.0, 26.0) * (n / 64.0)
        shell = ellipsoid_shell(depth, c, (r, r, r), 2.0)
        noise = noise_voxels(depth, noise_p, rng) if noise_p > 0 else None
        assets.append(make_asset(depth, shell, *( [noise] if noise is not None else [])))
    local = np.zeros((4, 12))
    centre = np.array([0.5, 0.5, 0.5])
    for i in range(4):
        R = euler_xyz(*rng.uniform(-math.pi / 4, math.pi / 4, 3))
        if i == 0:
            t = -R @ centre
        else:
            offs = [np.array([1.2, 0, 0]), np.array([-1.2, 0, 0]), np.array([0, 1.2, 0])][i - 1]
            t = (centre + offs) - R @ centre
        local[i] = affine12(R, t)
    view = rng.standard_normal(3)
    view /= np.linalg.norm(view)
    scene_radius = 1.2 + math.sqrt(3.0) / 2.0
    return Scene(
        name="PR1",
        assets=assets,
        part_asset=np.arange(4, dtype=np.int32),
        parent=np.array([-1, 0, 0, 0], dtype=np.int32),
        local=local,
        meta={"eye": view * 3.0 * scene_radius, "target": np.zeros(3), "scene_radius": scene_radius},
    )


def pr1_rays(scene: Scene, width: int = 128, height: int = 128) -> np.ndarray:
    return pinhole_rays(scene.meta["eye"], scene.meta["target"], width, height, 60.0)


# ------------------------------------------------------- articulated figure

@dataclass
class ArticulatedFigure:
    """16 parts in a 4-level tree animated by seeded sinusoidal joint angles.

    Topology: torso (0) -> 4 limbs (1..4) -> 2 segments each (5..12) -> 3 end
    parts (13..15) on segments 5, 7 and 9.  A part's pose relative to its parent
    is  T(attach) * R_rest * R(axis, theta(t)) * T(-joint)  where ``joint`` is the
    part's own -z end, ``attach`` a point on the parent and
    ``theta(t) = 0.5 sin(2 pi f t + phi)``.
    """

    scene: Scene
    attach: np.ndarray  # [P, 3] parent-local attachment points
    joint: np.ndarray  # [P, 3] own-local joint points
    rest: np.ndarray  # [P, 3, 3]
    axis: np.ndarray  # [P, 3]
    freq: np.ndarray  # [P]
    phase: np.ndarray  # [P]
    amplitude: float = 0.5
    fps: float = 30.0

    def pose(self, frame: int) -> np.ndarray:
        t = frame / self.fps
        P = self.scene.n_parts
        local = np.zeros((P, 12))
        for i in range(P):
            th = self.amplitude * math.sin(2 * math.pi * self.freq[i] * t + self.phase[i]) if i > 0 else 0.0
            Rj = axis_angle(self.axis[i], th)
            A = self.rest[i] @ Rj
            b = self.attach[i] - A @ self.joint[i]
            local[i] = affine12(A, b)
        return local

    def rays(self, width: int = 1920, height: int = 1080) -> np.ndarray:
        m = self.scene.meta
        return pinhole_rays(m["eye"], m["target"], width, height, 60.0)


def _sorted_unique(ids: np.ndarray) -> np.ndarray:
    s = np.sort(ids)
    if s.size == 0:
        return s
    keep = np.empty(s.shape, dtype=bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def static_union(scene: Scene, world, depth: int = 12, origin: float = -4.0, extent: float = 8.0):
    """The posed scene resampled into one static SVO in world space (the
    paper's "static model" comparison scene): every leaf of every part is
    sampled at 4 inset points (alternate corners of its 2x2x2 subcells), each mapped by
    its part's world pose into a 2^depth grid over the cube [origin,
    origin + extent]^3; occupied grid cells become the leaves (colour: the
    spatial hash of the grid cell).  Returns (Asset, world pose of the grid's
    unit cube as 12 float64)."""
    world = np.asarray(world, dtype=np.float64).reshape(-1, 12)
    n = 1 << depth
    cell = extent / n
    # four inset points of a leaf (alternate corners of its 2x2x2 subcells)
    offs = np.array([[0.25, 0.25, 0.25], [0.75, 0.75, 0.25], [0.75, 0.25, 0.75], [0.25, 0.75, 0.75]])
    per_part = []
    for p in range(scene.n_parts):
        a = scene.assets[int(scene.part_asset[p])]
        if a.n_leaves == 0:
            continue
        x, y, z = unpack_ids(a.leaf_ids, a.depth)
        base = np.stack([x, y, z], 1).astype(np.float64)
        W = world[p].reshape(3, 4)
        got = []
        for o in offs:
            loc = (base + o) / float(1 << a.depth)
            g = np.floor((loc @ W[:, :3].T + W[:, 3] - origin) / cell).astype(np.int64)
            ok = np.all((g >= 0) & (g < n), axis=1)
            got.append(pack_ids(g[ok, 0], g[ok, 1], g[ok, 2], depth))
        per_part.append(_sorted_unique(np.concatenate(got)))
    ids = _sorted_unique(np.concatenate(per_part)) if per_part else np.zeros(0, np.uint64)
    pose = affine12(np.eye(3) * extent, np.full(3, origin))
    return Asset(depth=depth, leaf_ids=ids, rgb=rgb_hash(*unpack_ids(ids, depth))), pose


def _rot_z_to(v) -> np.ndarray:
    """A rotation taking +z to the unit vector v."""
    v = np.asarray(v, dtype=np.float64)
    v = v / np.linalg.norm(v)
    z = np.array([0.0, 0.0, 1.0])
    c = float(np.dot(z, v))
    if c > 1 - 1e-12:
        return np.eye(3)
    if c < -1 + 1e-12:
        return axis_angle((1.0, 0.0, 0.0), math.pi)
    return axis_angle(np.cross(z, v), math.acos(c))


def articulated_figure(seed: int | None = None, depth: int = 9) -> ArticulatedFigure:
    rng = np.random.default_rng(config_seed(1) if seed is None else seed)
    n = 1 << depth
    P = 16
    parent = np.array([-1, 0, 0, 0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 5, 7, 9], dtype=np.int32)
    centre_cells = np.array([n / 2.0] * 3)
    assets = []
    semi = np.zeros((P, 3))
    for i in range(P):
        ax = rng.uniform(0.15, 0.45, 3) * n
        kind = "ellipsoid" if (i == 0 or rng.random() < 0.5) else "capsule"
        if kind == "ellipsoid":
            cells = ellipsoid_shell(depth, centre_cells, ax, 2.0)
            semi[i] = ax / n
        else:
            rad = min(ax[0], ax[1])
            hl = max(ax[2] - rad, 0.0)
            cells = capsule_shell(depth, centre_cells, rad, hl, 2.0)
            semi[i] = np.array([rad, rad, hl + rad]) / n
        assets.append(make_asset(depth, cells))
    c = np.array([0.5, 0.5, 0.5])
    attach = np.zeros((P, 3))
    joint = np.zeros((P, 3))
    rest = np.zeros((P, 3, 3))
    axis = np.zeros((P, 3))
    limb_dirs = [np.array([1.0, 0, 0]), np.array([-1.0, 0, 0]), np.array([0, 1.0, 0]), np.array([0, -1.0, 0])]
    for i in range(P):
        joint[i] = c - np.array([0, 0, semi[i][2]])
        a = rng.standard_normal(3)
        axis[i] = a / np.linalg.norm(a)
        if i == 0:
            attach[i] = np.zeros(3)
            rest[i] = np.eye(3)
            joint[i] = c
        elif 1 <= i <= 4:
            dvec = limb_dirs[i - 1]
            attach[i] = c + dvec * semi[0]
            rest[i] = _rot_z_to(dvec)
        else:
            p = parent[i]
            attach[i] = c + np.array([0, 0, semi[p][2]])
            rest[i] = np.eye(3)
    freq = rng.uniform(0.2, 2.0, P)
    phase = rng.uniform(0.0, 2 * math.pi, P)
    view = np.array([0.35, 0.45, 1.0]) + 0.1 * rng.standard_normal(3)
    view /= np.linalg.norm(view)
    # camera framing chosen for this topology: the figure spans about 6 x 4.5
    # cube widths around (0.25, 0.28, -0.1); 5.2 widths away it fills the frame
    target = np.array([0.25, 0.28, -0.1])
    scene = Scene(
        name="ART",
        assets=assets,
        part_asset=np.arange(P, dtype=np.int32),
        parent=parent,
        local=np.zeros((P, 12)),
        meta={"eye": target + view * 5.2, "target": target, "frames": 60},
    )
    fig = ArticulatedFigure(scene=scene, attach=attach, joint=joint, rest=rest, axis=axis, freq=freq, phase=phase)
    scene.local = fig.pose(0)
    return fig


# ------------------------------------------------------ asset pool, BAT, SRV

@dataclass
class PoolAsset:
    asset: Asset
    semi: np.ndarray  # semi-axes in unit-cube units (x, y, z)


def asset_pool(depths, per_depth: int = 4, seed: int = 0, thin_from: int = 11) -> list:
    """Seeded ellipsoid / capsule shells, ``per_depth`` per depth.  Shells are
    two cells thick, one cell from depth ``thin_from`` on (to bound memory)."""
    rng = np.random.default_rng(seed)
    pool = []
    for depth in depths:
        n = 1 << depth
        for _ in range(per_depth):
            ax = rng.uniform(0.15, 0.45, 3) * n
            thick = 1.0 if depth >= thin_from else 2.0
            c = np.array([n / 2.0] * 3)
            if rng.random() < 0.5:
                cells = ellipsoid_shell(depth, c, ax, thick)
                semi = ax / n
            else:
                rad = min(ax[0], ax[1])
                hl = max(ax[2] - rad, 0.0)
                cells = capsule_shell(depth, c, rad, hl, thick)
                semi = np.array([rad, rad, hl + rad]) / n
            pool.append(PoolAsset(make_asset(depth, cells), semi))
    return pool


def _random_rotation(rng) -> np.ndarray:
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


@dataclass
class BatchedScenes:
    """Scenes of uneven size over a shared asset pool, each with its own rays."""

    pool: list
    scenes: list  # Scene (assets = the pool's Asset list; part_asset indexes it)
    rays: list    # float32 [n_s, 8] per scene


def batched_scenes(seed: int | None = None, n_scenes: int = 64, parts=(4, 256), depths=range(6, 12),
                   side=(64, 1024), per_depth: int = 4, thin_from: int = 11, pool=None) -> BatchedScenes:
    """Uneven scenes: P log-uniform in ``parts``; per part a random pool asset
    of a random depth; pose = rotation (uniform) x scale U(0.5, 2) per axis x
    shear U(-0.1, 0.1) on three off-diagonals, translation in a box of side
    4 P^(1/3) part widths.  Rays: side log-uniform in ``side`` (side^2 rays),
    origins uniform in the box, directions uniform on the sphere."""
    rng = np.random.default_rng(config_seed(2) if seed is None else seed)
    depths = list(depths)
    pool_seed = int(rng.integers(1 << 31))
    if pool is None:
        pool = asset_pool(depths, per_depth, seed=pool_seed, thin_from=thin_from)
    assets = [p.asset for p in pool]
    scenes, rays = [], []
    for _ in range(n_scenes):
        P = int(round(math.exp(rng.uniform(math.log(parts[0]), math.log(parts[1])))))
        box = 4.0 * P ** (1.0 / 3.0)
        local = np.zeros((P, 12))
        part_asset = np.zeros(P, dtype=np.int32)
        for i in range(P):
            d = int(rng.integers(len(depths)))
            part_asset[i] = d * per_depth + int(rng.integers(per_depth))
            S = np.diag(rng.uniform(0.5, 2.0, 3))
            H = np.eye(3)
            H[0, 1], H[0, 2], H[1, 2] = rng.uniform(-0.1, 0.1, 3)
            A = _random_rotation(rng) @ S @ H
            t = rng.uniform(-box / 2, box / 2, 3) - A @ np.full(3, 0.5)
            local[i] = affine12(A, t)
        scenes.append(Scene("BAT", assets, part_asset, np.full(P, -1, np.int32), local, {"box": box}))
        s = int(round(math.exp(rng.uniform(math.log(side[0]), math.log(side[1])))))
        rays.append(random_rays(s * s, rng, (-box / 2,) * 3, (box / 2,) * 3))
    return BatchedScenes(pool, scenes, rays)


@dataclass
class ServedScene:
    """One resident scene of the serving workload: a tree of pool assets with
    joints animated like the articulated figure."""

    scene: Scene
    attach: np.ndarray
    joint: np.ndarray
    rest: np.ndarray
    axis: np.ndarray
    radius: float  # rough extent of the figure (camera framing)

    def pose(self, rng: np.random.Generator) -> np.ndarray:
        """A fresh seeded pose: every joint angle uniform in [-0.5, 0.5] rad."""
        P = self.scene.n_parts
        local = np.zeros((P, 12))
        for i in range(P):
            th = rng.uniform(-0.5, 0.5) if i > 0 else 0.0
            A = self.rest[i] @ axis_angle(self.axis[i], th)
            local[i] = affine12(A, self.attach[i] - A @ self.joint[i])
        return local


@dataclass
class RenderRequest:
    scene: int
    local: np.ndarray
    eye: np.ndarray
    target: np.ndarray
    width: int
    height: int
    arrival: float  # seconds from the start of the stream


@dataclass
class ServingWorld:
    pool: list
    scenes: list  # ServedScene

    def requests(self, n: int, rate: float, seed: int, resolutions=((256, 256), (512, 512), (1280, 720),
                                                                     (1920, 1080))) -> list:
        """Poisson arrivals (exponential gaps of mean 1/rate), a uniformly chosen
        scene, resolution and camera direction, and a fresh pose per request."""
        rng = np.random.default_rng(seed)
        t = 0.0
        out = []
        for _ in range(n):
            t += rng.exponential(1.0 / rate)
            s = int(rng.integers(len(self.scenes)))
            sc = self.scenes[s]
            w, h = resolutions[int(rng.integers(len(resolutions)))]
            view = rng.standard_normal(3)
            view /= np.linalg.norm(view)
            eye = view * sc.radius * 2.2
            out.append(RenderRequest(s, sc.pose(rng), eye, np.zeros(3), w, h, t))
        return out


def serving_world(seed: int | None = None, n_scenes: int = 32, parts=(16, 128), depths=range(8, 12),
                  per_depth: int = 4, thin_from: int = 11, pool=None, pool_indices=None) -> ServingWorld:
    """Resident scenes for the serving workload: P uniform in ``parts``, parts
    drawn from a pool of depths ``depths``; each part hangs from a random
    earlier part at a point on its surface and swings about a seeded axis."""
    rng = np.random.default_rng(config_seed(4) if seed is None else seed)
    depths = list(depths)
    pool_seed = int(rng.integers(1 << 31))
    if pool is None:
        pool = asset_pool(depths, per_depth, seed=pool_seed, thin_from=thin_from)
    # the pool entries a part may draw (all of them unless a shared pool is restricted)
    choices = np.arange(len(pool)) if pool_indices is None else np.asarray(pool_indices)
    assets = [p.asset for p in pool]
    scenes = []
    c = np.array([0.5, 0.5, 0.5])
    for _ in range(n_scenes):
        P = int(rng.integers(parts[0], parts[1] + 1))
        part_asset = np.array([int(choices[rng.integers(len(choices))]) for _ in range(P)], dtype=np.int32)
        parent = np.array([-1] + [int(rng.integers(max(0, i - 6), i)) for i in range(1, P)], dtype=np.int32)
        attach = np.zeros((P, 3))
        joint = np.zeros((P, 3))
        rest = np.zeros((P, 3, 3))
        axis = np.zeros((P, 3))
        level = np.zeros(P, dtype=np.int64)
        for i in range(P):
            semi = pool[part_asset[i]].semi
            a = rng.standard_normal(3)
            axis[i] = a / np.linalg.norm(a)
            if i == 0:
                attach[i] = -c
                joint[i] = np.zeros(3)
                rest[i] = np.eye(3)
                continue
            p = parent[i]
            level[i] = level[p] + 1
            u = rng.standard_normal(3)
            u /= np.linalg.norm(u)
            attach[i] = c + u * pool[part_asset[p]].semi
            joint[i] = c - np.array([0.0, 0.0, semi[2]])
            rest[i] = _rot_z_to(u)
        radius = 1.0 + 0.9 * float(level.max() + 1)
        local0 = np.zeros((P, 12))
        sc = Scene("SRV", assets, part_asset, parent, local0)
        served = ServedScene(sc, attach, joint, rest, axis, radius)
        sc.local = served.pose(np.random.default_rng(0))
        scenes.append(served)
    return ServingWorld(pool, scenes)


# ------------------------------------------------------------------ PREC

@dataclass
class PrecisionScene:
    """Precision stress: visible parts at the ends of long rigid chains."""

    scene: Scene
    visible: np.ndarray  # indices of the parts that carry geometry
    eye: np.ndarray
    target: np.ndarray


def precision_scene(seed: int | None = None, n_visible: int = 8, chain: int = 5, depth: int = 13,
                    radius=(150.0, 400.0), max_shift_leaves: float = 1e4) -> PrecisionScene:
    """``n_visible`` parts, each the last link of a ``chain``-level chain of
    rigid transforms whose other links are empty parts; two depth-``depth``
    one-cell sphere shells (radius uniform in ``radius`` cells) shared by the
    visible parts; every link translates by up to ``max_shift_leaves`` leaf
    sizes and rotates by a uniform random rotation."""
    rng = np.random.default_rng(config_seed(3) if seed is None else seed)
    n = 1 << depth
    shells = []
    for _ in range(2):
        r = rng.uniform(*radius)
        c = np.array([n / 2.0] * 3) + rng.uniform(-20, 20, 3)
        shells.append(make_asset(depth, ellipsoid_shell(depth, c, (r, r, r), 1.0)))
    empty = Asset(depth, np.zeros(0, np.uint64), np.zeros(0, np.uint32))
    assets = shells + [empty]
    P = n_visible * chain
    parent = np.zeros(P, dtype=np.int32)
    part_asset = np.zeros(P, dtype=np.int32)
    local = np.zeros((P, 12))
    visible = []
    leaf = 1.0 / n
    for v in range(n_visible):
        for k in range(chain):
            i = v * chain + k
            parent[i] = -1 if k == 0 else i - 1
            R = _random_rotation(rng)
            shift = rng.uniform(-max_shift_leaves, max_shift_leaves, 3) * leaf
            if k == 0:
                shift = shift + rng.uniform(-3.0, 3.0, 3)
            local[i] = affine12(R, shift)
            part_asset[i] = 2 if k < chain - 1 else v % 2
        visible.append(v * chain + chain - 1)
    scene = Scene("PREC", assets, part_asset, parent, local)
    view = rng.standard_normal(3)
    view /= np.linalg.norm(view)
    return PrecisionScene(scene, np.array(visible), view * 14.0, np.zeros(3))


def grazing_rays(world12, depth: int, leaf_ids, n: int, rng: np.random.Generator, max_angle: float = 1e-3,
                 back_off_leaves: float = 100.0) -> np.ndarray:
    """Rays that graze a face of a leaf: pick a leaf and one of its faces, a
    direction inside the face plane tilted by at most ``max_angle`` rad towards
    the face normal, and an origin ``back_off_leaves`` leaf sizes behind a point
    of the face.  Built in the part's local frame and mapped to world space by
    the part's pose ``world12`` (the forward map, given by the caller)."""
    M = np.asarray(world12, dtype=np.float64).reshape(3, 4)
    ids = np.asarray(leaf_ids, dtype=np.uint64)
    pick = ids[rng.integers(0, ids.shape[0], n)]
    x, y, z = unpack_ids(pick, depth)
    s = 1.0 / (1 << depth)
    cell = np.stack([x, y, z], axis=1).astype(np.float64) * s
    axis = rng.integers(0, 3, n)
    side = rng.integers(0, 2, n).astype(np.float64)
    out = np.empty((n, 8), dtype=np.float32)
    for k in range(n):
        a = int(axis[k])
        others = [i for i in range(3) if i != a]
        p = cell[k] + s * 0.5
        p[a] = cell[k][a] + side[k] * s
        p[others[0]] = cell[k][others[0]] + rng.uniform(0.1, 0.9) * s
        p[others[1]] = cell[k][others[1]] + rng.uniform(0.1, 0.9) * s
        phi = rng.uniform(0, 2 * math.pi)
        tilt = rng.uniform(0, max_angle) * (1 if rng.random() < 0.5 else -1)
        d = np.zeros(3)
        d[others[0]] = math.cos(phi)
        d[others[1]] = math.sin(phi)
        d[a] = math.tan(tilt)
        d /= np.linalg.norm(d)
        o = p - d * back_off_leaves * s
        wo = M[:, :3] @ o + M[:, 3]
        wd = M[:, :3] @ d
        wd /= np.linalg.norm(wd)
        out[k, 0:3] = wo
        out[k, 3] = 0.0
        out[k, 4:7] = wd
        out[k, 7] = np.inf
    return out


def precision_rays(prec: PrecisionScene, world, n_total: int = 1 << 20, graze_frac: float = 0.3,
                   seed: int = 13) -> tuple:
    """The precision-stress ray set: ``n_total`` rays of which ``graze_frac``
    graze leaf faces (``grazing_rays``, dealt over the visible parts) and the
    rest are pinhole rays, one square camera per visible part framing its
    shell from three shell radii away.  ``world``: the parts' world poses
    ([P, 12], as the caller composes them), used only to aim the rays.
    Returns (rays [n, 8] float32, number of pinhole rays first)."""
    rng = np.random.default_rng(seed)
    scene = prec.scene
    n_graze = int(graze_frac * n_total)
    per_cam = (n_total - n_graze) // len(prec.visible)
    side = int(np.sqrt(per_cam))
    prim = []
    for v in prec.visible:
        a = scene.assets[int(scene.part_asset[v])]
        x, y, z = unpack_ids(a.leaf_ids, a.depth)
        cells = (np.stack([x, y, z], 1) + 0.5) / (1 << a.depth)
        mid = cells.mean(0)
        r_l = float(np.linalg.norm(cells - mid, axis=1).max())
        W = np.asarray(world[v]).reshape(3, 4)
        c = W[:, :3] @ mid + W[:, 3]  # rigid chain: the shell keeps its size
        view = rng.standard_normal(3)
        view /= np.linalg.norm(view)
        prim.append(pinhole_rays(c + 3.0 * r_l * view, c, side, side, 44.0))
    prim = np.concatenate(prim)
    graze = []
    for k in range(n_graze // 4096 + 1):
        v = int(prec.visible[k % len(prec.visible)])
        a = scene.assets[int(scene.part_asset[v])]
        graze.append(grazing_rays(world[v], a.depth, a.leaf_ids, 4096, rng))
    graze = np.concatenate(graze)[:n_graze]
    return np.ascontiguousarray(np.concatenate([prim, graze]), dtype=np.float32), prim.shape[0]
