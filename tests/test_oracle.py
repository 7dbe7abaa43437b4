"""Pins of the FP64 oracle against facts fixed by the paper and by geometry.

Nothing here compares the oracle with itself: every expected value comes from
a hand derivation (tests/golden), a closed form, an independent algorithm (a
voxel-walking DDA, exact rational arithmetic, brute-force sampling) or an exact
invariant of the method (Eq. 3 moves the ray instead of the model, so moving
model and ray together, or re-expressing one model as aligned pieces, must not
change the hit).
"""

from __future__ import annotations

import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthetic
from golden_cases import case_scene, load_hand_cases


def _random_rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


def _random_affine(rng, shear=0.1, scale=(0.5, 2.0)):
    R = _random_rotation(rng)
    S = np.diag(rng.uniform(*scale, 3))
    H = np.eye(3)
    H[0, 1], H[0, 2], H[1, 2] = rng.uniform(-shear, shear, 3)
    return R @ S @ H


def _random_asset(rng, depth, p):
    n = 1 << depth
    occ = rng.random(n ** 3) < p
    idx = np.nonzero(occ)[0]
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    return synthetic.make_asset(depth, (x, y, z))


def _tiny_scene(rng, n_parts, depth, p=0.15, rigid=False):
    assets = [_random_asset(rng, depth, p) for _ in range(n_parts)]
    parent = np.array([-1] + [int(rng.integers(-1, i)) for i in range(1, n_parts)], dtype=np.int32)
    local = np.zeros((n_parts, 12))
    for i in range(n_parts):
        A = _random_rotation(rng) if rigid else _random_affine(rng)
        local[i] = synthetic.affine12(A, rng.uniform(-1.0, 1.0, 3))
    return synthetic.Scene("tiny", assets, np.arange(n_parts, dtype=np.int32), parent, local)


def _scene_rays(rng, n, half=2.5):
    """Half incoherent rays from the box, half aimed from outside at its centre region."""
    rays = synthetic.random_rays(n, rng, (-half,) * 3, (half,) * 3).astype(np.float64)
    m = n // 2
    org = rng.standard_normal((m, 3))
    org *= (2.0 * half / np.linalg.norm(org, axis=1))[:, None]
    tgt = rng.uniform(-0.6 * half, 0.6 * half, (m, 3))
    rays[:m, 0:3] = org
    rays[:m, 4:7] = tgt - org
    return rays


# ----------------------------------------------------------------- golden

@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("mode", [0, 1])
def test_hand_cases(case, mode):
    scene, rays = case_scene(case)
    res = oracle.SceneOracle(scene).trace(rays, mode=mode, threads=1)
    for i, exp in enumerate(case["hits"]):
        if exp is None:
            assert math.isinf(res["t"][i]) and res["part"][i] == oracle.MISS_PART
            assert res["voxel"][i] == oracle.MISS_VOXEL
        else:
            assert res["t"][i] == exp[0]
            assert int(res["part"][i]) == exp[1]
            assert int(res["voxel"][i]) == exp[2]


# ------------------------------------------------------ descent vs brute force

@pytest.mark.parametrize("seed", range(6))
def test_descent_equals_bruteforce(seed):
    rng = np.random.default_rng(1000 + seed)
    depth = 2 + seed % 4
    scene = _tiny_scene(rng, n_parts=1 + seed % 4, depth=depth, p=0.08 + 0.05 * (seed % 3))
    rays = _scene_rays(rng, 4096)
    o = oracle.SceneOracle(scene)
    a = o.trace(rays, mode=0)
    b = o.trace(rays, mode=1)
    for k in ("t", "part", "voxel", "second"):
        assert np.array_equal(a[k], b[k]), k
    assert (a["part"] != oracle.MISS_PART).sum() >= 30


# --------------------------------------------------------- independent DDA

def _dda_first_hit(grid, o, d):
    """Amanatides-Woo voxel walk over a dense grid in the unit cube.

    Independent of the oracle's hierarchy: it steps cell to cell along the ray
    and stops at the first occupied cell; t is where the ray entered that cell.
    """
    n = grid.shape[0]
    t_enter, t_exit = 0.0, math.inf
    for i in range(3):
        if d[i] == 0.0:
            if not (0.0 <= o[i] <= 1.0):
                return None
            continue
        a, b = (0.0 - o[i]) / d[i], (1.0 - o[i]) / d[i]
        t_enter, t_exit = max(t_enter, min(a, b)), min(t_exit, max(a, b))
    if t_enter > t_exit:
        return None
    p = [o[i] + t_enter * d[i] for i in range(3)]
    cell = [min(max(int(math.floor(p[i] * n)), 0), n - 1) for i in range(3)]
    step, t_max, t_delta = [0] * 3, [math.inf] * 3, [math.inf] * 3
    for i in range(3):
        if d[i] > 0:
            step[i] = 1
            t_max[i] = ((cell[i] + 1) / n - o[i]) / d[i]
            t_delta[i] = 1.0 / (n * d[i])
        elif d[i] < 0:
            step[i] = -1
            t_max[i] = (cell[i] / n - o[i]) / d[i]
            t_delta[i] = -1.0 / (n * d[i])
    t = t_enter
    while True:
        if grid[cell[0], cell[1], cell[2]]:
            return t, cell
        k = int(np.argmin(t_max))
        t = t_max[k]
        if t > t_exit:
            return None
        cell[k] += step[k]
        if not (0 <= cell[k] < n):
            return None
        t_max[k] += t_delta[k]


@pytest.mark.parametrize("depth", [3, 5])
def test_identity_pose_matches_dda(depth):
    rng = np.random.default_rng(77 + depth)
    asset = _random_asset(rng, depth, 0.04)
    n = 1 << depth
    grid = np.zeros((n, n, n), dtype=bool)
    x, y, z = synthetic.unpack_ids(asset.leaf_ids, depth)
    grid[x, y, z] = True
    scene = synthetic.Scene("one", [asset], np.zeros(1, np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None, :])
    # origins outside the cube aimed at random interior points
    m = 1500
    tgt = rng.random((m, 3))
    org = 0.5 + rng.standard_normal((m, 3)) * 2.0
    d = tgt - org
    rays = np.zeros((m, 8))
    rays[:, 0:3] = org
    rays[:, 4:7] = d
    rays[:, 7] = math.inf
    res = oracle.SceneOracle(scene).trace(rays, mode=1, threads=2)
    checked = 0
    for i in range(m):
        ref = _dda_first_hit(grid, org[i], d[i])
        tie = math.isfinite(res["t"][i]) and res["second"][i] - res["t"][i] <= 1e-9 * max(1.0, res["t"][i])
        if ref is None:
            assert res["part"][i] == oracle.MISS_PART or tie
            continue
        t_ref, cell = ref
        assert abs(res["t"][i] - t_ref) <= 1e-12 * max(1.0, t_ref)
        if not tie:
            assert int(res["voxel"][i]) == cell[0] | (cell[1] << depth) | (cell[2] << 2 * depth)
            checked += 1
    assert checked > 200


def test_full_cube_entry_is_analytic():
    """A fully occupied asset returns the cube's entry point, found here by
    intersecting the six face planes and keeping the first point on a face."""
    depth = 3
    n = 1 << depth
    g = np.arange(n)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    asset = synthetic.make_asset(depth, (x.ravel(), y.ravel(), z.ravel()))
    scene = synthetic.Scene("full", [asset], np.zeros(1, np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None, :])
    rng = np.random.default_rng(5)
    m = 800
    org = 0.5 + rng.standard_normal((m, 3)) * 3.0
    tgt = rng.random((m, 3))
    rays = np.zeros((m, 8))
    rays[:, 0:3] = org
    rays[:, 4:7] = tgt - org
    rays[:, 7] = math.inf
    res = oracle.SceneOracle(scene).trace(rays, mode=1, threads=2)
    for i in range(m):
        o, d = org[i], tgt[i] - org[i]
        if np.all((o >= 0) & (o <= 1)):
            exp = 0.0
        else:
            best = math.inf
            for ax in range(3):
                for face in (0.0, 1.0):
                    if d[ax] == 0:
                        continue
                    t = (face - o[ax]) / d[ax]
                    p = o + t * d
                    others = [k for k in range(3) if k != ax]
                    if t >= 0 and all(-1e-12 <= p[k] <= 1 + 1e-12 for k in others):
                        best = min(best, t)
            exp = best
        assert abs(res["t"][i] - exp) <= 1e-12 * max(1.0, exp)


def test_axis_aligned_rays_through_centres():
    """Rays along +x through cell centres hit the first occupied cell of their row at x/2^D - o_x."""
    depth = 4
    n = 1 << depth
    rng = np.random.default_rng(9)
    asset = _random_asset(rng, depth, 0.1)
    x, y, z = synthetic.unpack_ids(asset.leaf_ids, depth)
    scene = synthetic.Scene("one", [asset], np.zeros(1, np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None, :])
    ys, zs = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    rays = np.zeros((n * n, 8))
    rays[:, 0] = -0.5
    rays[:, 1] = (ys.ravel() + 0.5) / n
    rays[:, 2] = (zs.ravel() + 0.5) / n
    rays[:, 4] = 1.0
    rays[:, 7] = math.inf
    res = oracle.SceneOracle(scene).trace(rays, mode=1, threads=1)
    for r in range(n * n):
        yy, zz = int(ys.ravel()[r]), int(zs.ravel()[r])
        row = np.sort(x[(y == yy) & (z == zz)])
        if row.size == 0:
            assert res["part"][r] == oracle.MISS_PART
        else:
            assert res["t"][r] == row[0] / n + 0.5
            assert int(res["voxel"][r]) == int(row[0]) | (yy << depth) | (zz << 2 * depth)


# ------------------------------------------------------------------- poses

def test_invert_roundtrip_and_rigid_closed_form():
    rng = np.random.default_rng(3)
    P = 32
    world = np.array([synthetic.affine12(_random_affine(rng, shear=0.3), rng.uniform(-1e3, 1e3, 3))
                      for _ in range(P)])
    inv = oracle.invert(world)
    for p in range(P):
        W = np.eye(4)
        W[:3] = world[p].reshape(3, 4)
        V = np.eye(4)
        V[:3] = inv[p].reshape(3, 4)
        assert np.max(np.abs(W @ V - np.eye(4))) <= 1e-12 * max(1.0, np.abs(world[p]).max())
    # rigid: inverse = [R^T | -R^T t] (transpose the rotation, negate the translation; Sec. III-A)
    rig = np.array([synthetic.affine12(_random_rotation(rng), rng.uniform(-5, 5, 3)) for _ in range(P)])
    inv = oracle.invert(rig)
    for p in range(P):
        R = rig[p].reshape(3, 4)[:, :3]
        t = rig[p].reshape(3, 4)[:, 3]
        exp = synthetic.affine12(R.T, -R.T @ t)
        assert np.max(np.abs(inv[p] - exp)) <= 1e-14


def test_compose_five_level_chain_exact():
    """Small-integer poses compose exactly; compare with rational arithmetic."""
    rng = np.random.default_rng(11)
    P = 6
    parent = np.array([-1, 0, 1, 2, 3, 4], dtype=np.int32)
    local = rng.integers(-3, 4, (P, 12)).astype(np.float64)
    world = oracle.compose(parent, local)

    def mat(v):
        m = [[Fraction(0)] * 4 for _ in range(4)]
        for i in range(3):
            for j in range(4):
                m[i][j] = Fraction(int(v[i * 4 + j]))
        m[3][3] = Fraction(1)
        return m

    def mul(a, b):
        return [[sum(a[i][k] * b[k][j] for k in range(4)) for j in range(4)] for i in range(4)]

    acc = None
    for i in range(P):
        acc = mat(local[i]) if acc is None else mul(acc, mat(local[i]))
        exp = np.array([[float(acc[r][c]) for c in range(4)] for r in range(3)]).reshape(12)
        assert np.array_equal(world[i], exp)
    with pytest.raises(ValueError):
        oracle.compose(np.array([-1, 1], np.int32), np.zeros((2, 12)))


def test_part_sphere_encloses_and_is_tight():
    rng = np.random.default_rng(4)
    P = 20
    world = np.array([synthetic.affine12(_random_affine(rng), rng.uniform(-3, 3, 3)) for _ in range(P)])
    sph = oracle.part_spheres(world)
    for p in range(P):
        M = world[p].reshape(3, 4)
        c_exp = M[:, :3] @ np.full(3, 0.5) + M[:, 3]
        assert np.allclose(sph[p, :3], c_exp, rtol=0, atol=1e-12)
        corners = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)], dtype=np.float64)
        dist = np.linalg.norm(corners @ M[:, :3].T + M[:, 3] - c_exp, axis=1)
        assert abs(sph[p, 3] - dist.max()) <= 1e-12
    # rigid part of unit size: radius = half the cube diagonal
    rig = synthetic.affine12(_random_rotation(rng), np.zeros(3))
    assert abs(oracle.part_spheres(rig[None])[0, 3] - math.sqrt(3) / 2) <= 1e-15


def test_part_sphere_of_occupied_box():
    """The sphere of a part's occupied box: closed forms for identity and rigid
    poses; under any affine pose it holds every occupied leaf cell and one box
    corner lies on it; the unit-cube box gives the plain part sphere."""
    rng = np.random.default_rng(6)
    # occupied box of a hand-made asset, depth 3: cells (1,2,5) and (6,3,2)
    ids = synthetic.pack_ids(np.array([1, 6]), np.array([2, 3]), np.array([5, 2]), 3)
    box = oracle.occupied_box(3, ids)
    assert box.tolist() == [1 / 8, 2 / 8, 2 / 8, 7 / 8, 4 / 8, 6 / 8]
    assert oracle.occupied_box(3, np.zeros(0, np.uint64)).tolist() == [0, 0, 0, 1, 1, 1]
    lo, hi = box[:3], box[3:]
    s = oracle.part_spheres(synthetic.affine12(np.eye(3), np.zeros(3))[None], box[None])[0]
    assert np.allclose(s[:3], (lo + hi) / 2, rtol=0, atol=1e-15)
    assert abs(s[3] - np.linalg.norm(hi - lo) / 2) <= 1e-15
    R = _random_rotation(rng)
    s = oracle.part_spheres(synthetic.affine12(R, np.array([3.0, -1.0, 2.0]))[None], box[None])[0]
    assert abs(s[3] - np.linalg.norm(hi - lo) / 2) <= 1e-14
    assert np.allclose(s[:3], R @ ((lo + hi) / 2) + np.array([3.0, -1.0, 2.0]), rtol=0, atol=1e-14)
    a = synthetic.make_asset(5, synthetic.noise_voxels(5, 0.01, rng))
    abox = oracle.occupied_box(5, a.leaf_ids)
    for _ in range(10):
        W = synthetic.affine12(_random_affine(rng), rng.uniform(-3, 3, 3))
        s = oracle.part_spheres(W[None], abox[None])[0]
        M = W.reshape(3, 4)
        x, y, z = synthetic.unpack_ids(a.leaf_ids, 5)
        cells = np.stack([x, y, z], 1).astype(np.float64)
        for k in range(8):
            corner = (cells + np.array([k & 1, (k >> 1) & 1, (k >> 2) & 1])) / 32.0
            assert np.all(np.linalg.norm(corner @ M[:, :3].T + M[:, 3] - s[:3], axis=1) <= s[3] * (1 + 1e-12))
        bc = np.array([[abox[3 * (k & 1)], abox[1 + 3 * ((k >> 1) & 1)], abox[2 + 3 * ((k >> 2) & 1)]]
                       for k in range(8)])
        assert abs(np.linalg.norm(bc @ M[:, :3].T + M[:, 3] - s[:3], axis=1).max() - s[3]) <= 1e-12
        assert np.array_equal(oracle.part_spheres(W[None], np.array([[0, 0, 0, 1, 1, 1.0]]))[0],
                              oracle.part_spheres(W[None])[0])


# ------------------------------------------------------------------ Eq. 4

def test_ray_sphere_eq4_against_sampled_distance():
    rng = np.random.default_rng(8)
    for _ in range(400):
        c = rng.uniform(-2, 2, 3)
        r = rng.uniform(0.1, 1.5)
        o = rng.uniform(-4, 4, 3)
        d = rng.standard_normal(3) * rng.uniform(0.2, 3.0)
        ts = np.linspace(0.0, 40.0 / np.linalg.norm(d), 400001)
        pts = o[None, :] + ts[:, None] * d[None, :]
        dist = np.linalg.norm(pts - c[None, :], axis=1)
        k = int(np.argmin(dist))
        hit, t_in, t_out = oracle.ray_sphere(o, d, np.r_[c, r])
        if dist[k] < r * (1 - 1e-3):
            assert hit
            inside = ts[dist <= r]
            step = ts[1] - ts[0]
            assert abs(t_in - inside.min()) <= 2 * step and abs(t_out - inside.max()) <= 2 * step
        elif dist[k] > r * (1 + 1e-3):
            assert not hit


def test_ray_sphere_tangent_and_behind():
    c = np.array([0.0, 0.0, 0.0, 1.0])
    # tangent: the line passes at distance exactly r (dyadic numbers, exact arithmetic)
    hit, t_in, t_out = oracle.ray_sphere([-4.0, 1.0, 0.0], [2.0, 0.0, 0.0], c)
    assert hit and t_in == t_out == 2.0
    # sphere behind the origin: the line meets it but the ray (t >= 0) does not
    hit, _, _ = oracle.ray_sphere([4.0, 0.0, 0.0], [1.0, 0.0, 0.0], c)
    assert not hit
    # origin inside: entry clamps to 0
    hit, t_in, t_out = oracle.ray_sphere([0.5, 0.0, 0.0], [1.0, 0.0, 0.0], c)
    assert hit and t_in == 0.0 and t_out == 0.5


# -------------------------------------------------------------- invariants

def test_aligned_union_invariant():
    """Parts of scale 2^-k on the level-k grid reproduce one static SVO of depth D+k.

    In FP64 every quantity of the two traces is the same rounded value (powers
    of two commute with rounding), so t agrees bit for bit; ids agree up to the
    relabelling part = level-k node, voxel = low D bits per axis.
    """
    rng = np.random.default_rng(21)
    D, k = 3, 1
    big = _random_asset(rng, D + k, 0.05)
    X, Y, Z = synthetic.unpack_ids(big.leaf_ids, D + k)
    union = synthetic.Scene("union", [big], np.zeros(1, np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None, :])
    g = 1 << k
    assets, local = [], []
    for p in range(g ** 3):
        a, b, c = p % g, (p // g) % g, p // (g * g)
        sel = ((X >> D) == a) & ((Y >> D) == b) & ((Z >> D) == c)
        m = (1 << D) - 1
        assets.append(synthetic.make_asset(D, (X[sel] & m, Y[sel] & m, Z[sel] & m)))
        local.append(synthetic.affine12(np.eye(3) / g, np.array([a, b, c], dtype=np.float64) / g))
    parts = synthetic.Scene("parts", assets, np.arange(g ** 3, dtype=np.int32), np.full(g ** 3, -1, np.int32),
                            np.array(local))
    rays = _scene_rays(rng, 3000, half=1.5)
    ru = oracle.SceneOracle(union).trace(rays)
    rp = oracle.SceneOracle(parts).trace(rays)
    assert np.array_equal(ru["t"], rp["t"])
    hit = ru["part"] != oracle.MISS_PART
    assert np.array_equal(hit, rp["part"] != oracle.MISS_PART)
    no_tie = hit & (ru["second"] > ru["t"])
    Xh, Yh, Zh = synthetic.unpack_ids(ru["voxel"][no_tie], D + k)
    m = (1 << D) - 1
    assert np.array_equal(rp["part"][no_tie], (Xh >> D) + g * (Yh >> D) + g * g * (Zh >> D))
    assert np.array_equal(rp["voxel"][no_tie], synthetic.pack_ids(Xh & m, Yh & m, Zh & m, D))
    assert no_tie.sum() > 300


def test_rigid_scene_and_camera_invariant():
    """Moving every root pose and every ray by one rigid map leaves hits unchanged."""
    rng = np.random.default_rng(31)
    scene = _tiny_scene(rng, n_parts=4, depth=4, p=0.1, rigid=False)
    rays = _scene_rays(rng, 4000)
    base = oracle.SceneOracle(scene).trace(rays)
    G = _random_rotation(rng)
    g = rng.uniform(-50, 50, 3)
    moved = scene.local.copy()
    for i in range(scene.n_parts):
        if scene.parent[i] < 0:
            M = scene.local[i].reshape(3, 4)
            moved[i] = synthetic.affine12(G @ M[:, :3], G @ M[:, 3] + g)
    r2 = rays.copy()
    r2[:, 0:3] = rays[:, 0:3] @ G.T + g
    r2[:, 4:7] = rays[:, 4:7] @ G.T
    res = oracle.SceneOracle(scene).trace(r2, local=moved)
    hit = base["part"] != oracle.MISS_PART
    with np.errstate(invalid="ignore"):
        near = np.isfinite(base["t"]) & (base["second"] - base["t"] <= 1e-9 * np.maximum(base["t"], 1.0))
    assert np.array_equal(hit | near, (res["part"] != oracle.MISS_PART) | near)
    ok = hit & ~near
    assert np.all(np.abs(res["t"][ok] - base["t"][ok]) <= 1e-11 * np.maximum(base["t"][ok], 1.0))
    assert np.array_equal(res["part"][ok], base["part"][ok])
    assert np.array_equal(res["voxel"][ok], base["voxel"][ok])
    assert ok.sum() > 300


def test_hit_colors_closed_form_and_first_occurrence():
    """Hit colours (Sec. IV-C): on a hash-coloured scene the colour of every hit
    is the hash of the hit voxel's own coordinates; a duplicated id takes the
    colour listed first; misses take the background; ids that are not leaves
    are invalid."""
    scene = synthetic.pr1_scene(depth=4)
    so = oracle.SceneOracle(scene)
    rays = synthetic.pr1_rays(scene, 48, 48)
    ora = so.trace(rays)
    col = so.hit_colors(ora, background=0x123456)
    hit = ora["part"] != oracle.MISS_PART
    assert hit.sum() > 100 and (~hit).sum() > 100
    assert np.all(col[~hit] == 0x123456)
    for i in np.nonzero(hit)[0]:
        d = scene.assets[int(scene.part_asset[int(ora["part"][i])])].depth
        x, y, z = synthetic.unpack_ids(np.array([ora["voxel"][i]]), d)
        assert col[i] == synthetic.rgb_hash(x, y, z)[0]
    # duplicates: the first listed colour wins; a non-leaf id and an unknown part are invalid
    ids = synthetic.pack_ids(np.array([3, 1, 3, 2]), np.array([0, 0, 0, 5]), np.array([1, 1, 1, 7]), 3)
    rgb = np.array([0xAA0000, 0x00BB00, 0x0000CC, 0x010203], dtype=np.uint32)
    part = np.array([0, 0, 0, 0, 1, oracle.MISS_PART], dtype=np.uint32)
    vox = np.array([ids[0], ids[1], ids[3], synthetic.pack_ids(4, 4, 4, 3), ids[0], 0], dtype=np.uint64)
    got = oracle.hit_colors([(ids, rgb)], [0], part, vox, background=7)
    assert got.tolist() == [0xAA0000, 0x00BB00, 0x010203, oracle.COLOR_INVALID, oracle.COLOR_INVALID, 7]
    # an asset without colours gives 0 for its leaves
    assert oracle.hit_colors([(ids, None)], [0], part[:1], vox[:1]).tolist() == [0]


def _shade_one(depth, cells, rgb, world12, rays, light, ambient, background=0):
    ids = synthetic.pack_ids(*[np.array([c[i] for c in cells]) for i in range(3)], depth)
    inv = oracle.invert(np.asarray(world12, np.float64)[None])
    a = oracle.OracleAsset(depth, ids)
    hits = oracle.trace([a], inv, rays)
    colors = oracle.hit_colors([(ids, np.asarray(rgb, np.uint32))], [0], hits["part"], hits["voxel"], background)
    return oracle.shade(colors, hits["part"], hits["voxel"], [depth], inv, rays, light, ambient, background), hits


def test_shade_closed_forms():
    """Shading of hits (Sec. IV-C hit buffer: colour + normal): an axis-aligned
    ray entering through the -x face is lit fully by a light along -x and only
    by the ambient term from +x; a ray starting inside its voxel faces the
    viewer; a diagonal ray entering through an edge takes the lower axis."""
    ident = synthetic.affine12(np.eye(3), np.zeros(3))
    rgb = [0xC86432]  # (200, 100, 50)
    ray = np.array([[-1.0, 0.3, 0.3, 0.0, 1.0, 0.0, 0.0, np.inf]])  # enters cell (0,0,0) of depth 1 through x = 0
    (full, amb), hits = _shade_one(1, [(0, 0, 0)], rgb, ident, ray, [-1.0, 0.0, 0.0], 0.25)
    assert hits["part"][0] == 0 and full[0] == 0xC86432 and not amb[0]
    (dark, _), _ = _shade_one(1, [(0, 0, 0)], rgb, ident, ray, [1.0, 0.0, 0.0], 0.25)
    assert dark[0] == (50 << 16) | (25 << 8) | 13  # floor(c/4 + 1/2): 50, 25, 12.5 -> 13
    (side, _), _ = _shade_one(1, [(0, 0, 0)], rgb, ident, ray, [-1.0, 1.0, 0.0], 0.0)
    cos45 = 1.0 / math.sqrt(2.0)
    assert side[0] == (int(200 * cos45 + 0.5) << 16) | (int(100 * cos45 + 0.5) << 8) | int(50 * cos45 + 0.5)
    # origin inside the voxel: the normal is -d, fully lit by a light along -d
    inside = np.array([[0.2, 0.2, 0.2, 0.0, 0.0, 0.0, 2.0, np.inf]])
    (ins, _), _ = _shade_one(1, [(0, 0, 0)], rgb, ident, inside, [0.0, 0.0, -1.0], 0.0)
    assert ins[0] == 0xC86432
    # entry through the edge x = y = 0 (equal near-plane t): ambiguous, and the x face is taken
    diag = np.array([[-0.5, -0.5, 0.25, 0.0, 1.0, 1.0, 0.0, np.inf]])
    (dg, amb), _ = _shade_one(1, [(0, 0, 0)], rgb, ident, diag, [-1.0, 0.0, 0.0], 0.0)
    assert amb[0] and dg[0] == 0xC86432
    # a miss keeps the background
    miss = np.array([[-1.0, 5.0, 5.0, 0.0, 1.0, 0.0, 0.0, np.inf]])
    (ms, _), _ = _shade_one(1, [(0, 0, 0)], rgb, ident, miss, [-1.0, 0.0, 0.0], 0.3, background=0x010203)
    assert ms[0] == 0x010203


def test_shade_rigid_invariance_and_scaled_normals():
    """One rigid motion applied to the part, the rays and the light leaves the
    shaded image unchanged; an anisotropic scale keeps face normals on the
    axes (the inverse transpose, not the forward matrix, maps normals)."""
    rng = np.random.default_rng(21)
    scene = synthetic.pr1_scene(depth=4)
    so = oracle.SceneOracle(scene)
    rays = synthetic.pr1_rays(scene, 40, 40).astype(np.float64)
    light = np.array([0.3, -0.8, 0.5])
    hits = so.trace(rays)
    base, amb0 = so.shade(hits, rays, light, 0.2)
    R = _random_rotation(rng)
    t = rng.uniform(-2, 2, 3)
    G = np.eye(4)
    G[:3, :3] = R
    G[:3, 3] = t
    local = scene.local.copy()
    for i in np.nonzero(scene.parent < 0)[0]:
        M = np.eye(4)
        M[:3, :] = local[i].reshape(3, 4)
        local[i] = (G @ M)[:3, :].reshape(12)
    moved = rays.copy()
    moved[:, 0:3] = rays[:, 0:3] @ R.T + t
    moved[:, 4:7] = rays[:, 4:7] @ R.T
    hits2 = so.trace(moved, local=local)
    got, amb1 = so.shade(hits2, moved, R @ light, 0.2, local=local)
    ok = ~(amb0 | amb1) & (hits["part"] == hits2["part"]) & (hits["voxel"] == hits2["voxel"])
    assert ok.sum() > 300 and np.array_equal(got[ok], base[ok])
    # anisotropic scale: a ray along +y into a cell of a part scaled (4, 1, 1) enters through -y
    W = synthetic.affine12(np.diag([4.0, 1.0, 1.0]), np.zeros(3))
    ray = np.array([[0.5, -1.0, 0.25, 0.0, 0.0, 1.0, 0.0, np.inf]])
    (sh, amb), hits = _shade_one(1, [(0, 0, 0)], [0xFFFFFF], W, ray, [0.0, -1.0, 0.0], 0.0)
    assert hits["part"][0] == 0 and sh[0] == 0xFFFFFF and not amb[0]


def test_static_union_closed_forms():
    """The static comparison scene (a posed scene resampled into one world
    grid): a grid-aligned identity part reproduces its own leaves, and a
    whole-cell translation shifts them."""
    a = synthetic.make_asset(4, synthetic.noise_voxels(4, 0.05, np.random.default_rng(3)))
    scene = synthetic.Scene("one", [a], np.array([0], np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None])
    u, pose = synthetic.static_union(scene, scene.local, depth=4, origin=0.0, extent=1.0)
    assert np.array_equal(u.leaf_ids, np.sort(a.leaf_ids))
    assert np.allclose(pose, synthetic.affine12(np.eye(3), np.zeros(3)))
    # translate by (2, 1, 0) cells of 1/16 inside a grid of twice the extent (cells of 1/8 at depth 4)
    shifted = synthetic.affine12(np.eye(3), np.array([2, 1, 0]) / 16.0)[None]
    u2, _ = synthetic.static_union(scene, shifted, depth=5, origin=0.0, extent=2.0)
    x, y, z = synthetic.unpack_ids(a.leaf_ids, 4)
    want = np.unique(synthetic.pack_ids(x + 2, y + 1, z, 5))
    assert np.array_equal(u2.leaf_ids, want)


def _rot(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def test_trs_to_local_closed_forms():
    """Sec. III-B poses: x_parent = R (s * x) + t, so column j of the linear
    part is s_j times column j of R."""
    rz = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    row = np.concatenate([rz.ravel(), [1.0, 2.0, 3.0], [2.0, 3.0, 5.0]])
    m = oracle.trs_to_local(row).reshape(3, 4)
    assert np.array_equal(m[:, :3], np.array([[0.0, -3.0, 0.0], [2.0, 0.0, 0.0], [0.0, 0.0, 5.0]]))
    assert np.array_equal(m[:, 3], [1.0, 2.0, 3.0])
    # the unit cube's far corner lands at R s + t
    assert np.allclose(m[:, :3] @ np.ones(3) + m[:, 3], rz @ np.array([2.0, 3.0, 5.0]) + [1.0, 2.0, 3.0])


def test_octree_dims_closed_form():
    """One leaf, cell (1, 0, 0) of a depth-1 asset, dimensions (2, 4, 8) at
    t = (1, 2, 3): the world box is [2, 3] x [2, 4] x [3, 7]."""
    ids = synthetic.pack_ids(np.array([1]), np.array([0]), np.array([0]), 1)
    row = np.concatenate([np.eye(3).ravel(), [1.0, 2.0, 3.0], [2.0, 4.0, 8.0]])
    rays = np.array([[0.0, 3.0, 5.0, 0.0, 1.0, 0.0, 0.0, np.inf],
                     [0.0, 3.0, 5.0, 0.0, 2.0, 0.0, 0.0, np.inf],
                     [0.0, 4.5, 5.0, 0.0, 1.0, 0.0, 0.0, np.inf],    # above the box: miss
                     [2.5, 3.0, 0.0, 0.0, 0.0, 0.0, 1.0, np.inf],    # along z from below: enters at z = 3
                     [0.0, 3.0, 5.0, 0.0, 1.0, 0.0, 0.0, 1.5]])      # tmax before the box
    out = oracle.trace_octree_dims([ids], [1], row, rays)
    assert list(out["t"][:2]) == [2.0, 1.0]
    assert out["part"][2] == oracle.MISS_PART and out["part"][4] == oracle.MISS_PART
    assert out["t"][3] == 3.0 and out["voxel"][3] == ids[0]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_octree_dims_equal_the_affine_pose(seed):
    """The Sec. III-B form (rigid inverse, octree of dimensions s) and the
    general affine [R diag(s) | t] give the same closest hits: brute force
    over every leaf against the oracle's descent."""
    rng = np.random.default_rng(900 + seed)
    assets, leaf_ids = [], []
    for depth in (2, 3, 4):
        n = 1 << depth
        occ = np.nonzero(rng.random(n ** 3) < 0.15)[0]
        a = synthetic.make_asset(depth, (occ % n, (occ // n) % n, occ // (n * n)))
        assets.append(a)
    P = 5
    part_asset = rng.integers(0, 3, P).astype(np.int32)
    rts = np.zeros((P, 15))
    for p in range(P):
        rts[p, :9] = _rot(rng).ravel()
        rts[p, 9:12] = rng.uniform(-2, 2, 3)
        rts[p, 12:15] = rng.uniform(0.3, 3.0, 3)
    scene = synthetic.Scene("trs", assets, part_asset, np.full(P, -1, np.int32), oracle.trs_to_local(rts))
    rays = synthetic.random_rays(300, rng, (-3,) * 3, (3,) * 3)
    ref = oracle.SceneOracle(scene).trace(rays)
    got = oracle.trace_octree_dims([assets[a].leaf_ids for a in part_asset], [assets[a].depth for a in part_asset],
                                   rts, rays)
    hit = ref["part"] != oracle.MISS_PART
    assert hit.sum() > 30
    assert np.array_equal(got["part"] != oracle.MISS_PART, hit)
    assert np.allclose(got["t"][hit], ref["t"][hit], rtol=1e-12, atol=1e-12)
    with np.errstate(invalid="ignore"):  # inf - inf where a ray meets one leaf
        clear = hit & (ref["second"] - ref["t"] > 1e-9 * np.maximum(np.abs(ref["t"]), 1.0))
    assert np.array_equal(got["part"][clear], ref["part"][clear])
    assert np.array_equal(got["voxel"][clear], ref["voxel"][clear])


def test_ray_validity_rule():
    """Eq. 1 rays have a direction.  The oracle's reading makes that a rule
    with exact bounds: the largest direction component magnitude lies in
    [2^-60, 2^60], origin and direction are finite and neither bound is NaN.
    Anything else is a miss -- even a zero direction whose origin lies inside
    an occupied leaf, which the slab rule alone would report at tmin.  A valid
    tiny or huge direction is traced: t scales as 1 / |d| exactly (the
    entry plane x = 0 is 1 unit away from the origin)."""
    depth = 2
    n = 1 << depth
    g = np.arange(n)
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    asset = synthetic.make_asset(depth, (x.ravel(), y.ravel(), z.ravel()))
    scene = synthetic.Scene("full", [asset], np.zeros(1, np.int32), np.array([-1], np.int32),
                            synthetic.affine12(np.eye(3), np.zeros(3))[None, :])
    inside = [0.3, 0.4, 0.6]
    outside = [-1.0, 0.4, 0.6]
    rows = [
        (inside, [0.0, 0.0, 0.0], 0.0, math.inf, None),                   # zero direction, origin in a leaf
        (outside, [2.0 ** -61, 0.0, 0.0], 0.0, math.inf, None),           # below the range
        (outside, [2.0 ** 61, 0.0, 0.0], 0.0, math.inf, None),            # above the range
        (outside, [math.nan, 1.0, 0.0], 0.0, math.inf, None),             # NaN component
        ([math.inf, 0.4, 0.6], [1.0, 0.0, 0.0], 0.0, math.inf, None),     # infinite origin
        (outside, [1.0, 0.0, 0.0], math.nan, math.inf, None),             # NaN tmin
        (outside, [1.0, 0.0, 0.0], 0.0, math.nan, None),                  # NaN tmax
        (outside, [2.0 ** -60, 0.0, 0.0], 0.0, math.inf, 2.0 ** 60),      # smallest valid |d|
        (outside, [2.0 ** 60, 0.0, 0.0], 0.0, math.inf, 2.0 ** -60),      # largest valid |d|
        (outside, [-(2.0 ** -60), 2.0 ** -70, 0.0], 0.0, math.inf, "miss"),  # valid, pointing away
        (inside, [0.0, 0.0, 2.0 ** -60], 0.25, math.inf, 0.25),           # valid, starts inside: tmin
    ]
    rays = np.zeros((len(rows), 8))
    for i, (o, d, t0, t1, _) in enumerate(rows):
        rays[i, 0:3], rays[i, 3], rays[i, 4:7], rays[i, 7] = o, t0, d, t1
    valid = oracle.ray_valid(rays)
    assert valid.tolist() == [r[4] is not None for r in rows]
    for mode in (0, 1):
        res = oracle.SceneOracle(scene).trace(rays, mode=mode, threads=1)
        for i, (*_, exp) in enumerate(rows):
            if exp is None or exp == "miss":
                assert res["part"][i] == oracle.MISS_PART and math.isinf(res["t"][i]), (mode, i)
            else:
                assert res["part"][i] == 0 and res["t"][i] == exp, (mode, i, res["t"][i])
