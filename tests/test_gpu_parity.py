"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Bar: part and voxel ids bit-exact on every ray the FP32 path does not flag;
hit t within 1e-5 * max(|t|, leaf diagonal); flagged rays re-intersected in
FP64 and compared the same way (mismatches counted, expected zero).
"""

from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
import synthetic
from golden_cases import case_scene, load_hand_cases
from gpu_helpers import GpuScene, compare

pytestmark = pytest.mark.gpu

FLAG_SETS = {
    "plain": 0,
    "cull": 1,
    "cull_sort": 3,
    "fix": 4,
    "cull_fix": 5,
    "default": 7,
}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1911_06001_gb300 as g

    c = g.Context(0)
    yield c
    c.check_device()
    c.close()


@pytest.fixture(scope="module")
def pr1(ctx):
    s = synthetic.pr1_scene()
    return s, GpuScene(ctx, s), oracle.SceneOracle(s)


def test_refit_matches_oracle(ctx, pr1):
    scene, gs, so = pr1
    got = gs.sc.read_poses()
    world, inv = so.poses(gs.local)
    assert np.allclose(got["world"], world, rtol=0, atol=1e-13 * np.abs(world).max())
    assert np.allclose(got["inv"], inv, rtol=0, atol=1e-12 * max(1.0, np.abs(inv).max()))
    A32 = got["inv_f32"].reshape(-1, 3, 4)
    assert np.array_equal(A32[:, :, :3], got["inv"].reshape(-1, 3, 4)[:, :, :3].astype(np.float32))
    # column 3: local coordinates of the FP32 sphere centre (close to the cube centre)
    c32 = got["sphere"][:, :3].astype(np.float64)
    lc = np.einsum("pij,pj->pi", inv.reshape(-1, 3, 4)[:, :, :3], c32) + inv.reshape(-1, 3, 4)[:, :, 3]
    assert np.allclose(A32[:, :, 3], lc, rtol=0, atol=1e-6)
    boxes = so.boxes()
    assert np.allclose(lc, 0.5 * (boxes[:, :3] + boxes[:, 3:]), atol=1e-5)  # the occupied box's centre
    sph = oracle.part_spheres(world, boxes)
    dc = np.linalg.norm(got["sphere"][:, :3].astype(np.float64) - sph[:, :3], axis=1)
    r = got["sphere"][:, 3].astype(np.float64)
    assert np.all(dc + sph[:, 3] <= r)  # the FP32 sphere encloses the exact one
    # the radius is an FP32 upper bound with 2^-20 slack on the corner norms and their rounding scale
    assert np.all(r <= sph[:, 3] * (1 + 4e-6) + 2 * dc + 1e-30)
    cl = gs.sc.read_clusters()
    assert sorted(cl["order"].tolist()) == list(range(scene.n_parts))
    for c in range(cl["sphere"].shape[0]):
        C = cl["sphere"][c].astype(np.float64)
        for p in cl["order"][8 * c: 8 * c + 8]:
            s = got["sphere"][p].astype(np.float64)
            assert np.linalg.norm(s[:3] - C[:3]) + s[3] <= C[3] * (1 + 1e-12)


def test_five_level_chain_compose(ctx):
    """Long transform chains composed in FP64 on the device match the oracle."""
    rng = np.random.default_rng(5)
    asset = synthetic.make_asset(4, (np.array([1, 2]), np.array([3, 3]), np.array([0, 15])))
    P = 6
    parent = np.array([-1, 0, 1, 2, 3, 4], np.int32)
    local = np.array([synthetic.affine12(synthetic.euler_xyz(*rng.uniform(-3, 3, 3)), rng.uniform(-1e4, 1e4, 3) / 8192)
                      for _ in range(P)])
    scene = synthetic.Scene("chain", [asset], np.zeros(P, np.int32), parent, local)
    gs = GpuScene(ctx, scene)
    got = gs.sc.read_poses()
    world = oracle.compose(parent, local)
    inv = oracle.invert(world)
    assert np.allclose(got["world"], world, rtol=0, atol=1e-12)
    assert np.allclose(got["inv"], inv, rtol=0, atol=1e-11)


@pytest.mark.parametrize("case", load_hand_cases(), ids=lambda c: c["name"])
def test_hand_cases_gpu(ctx, case):
    scene, rays = case_scene(case)
    gs = GpuScene(ctx, scene)
    for flags in (0, 4, 7):
        res = gs.trace(rays.astype(np.float32), flags)
        for i, exp in enumerate(case["hits"]):
            uncertain = (res["flags"][i] & 1) != 0
            if exp is None:
                if not uncertain or flags & 4:
                    assert math.isinf(res["t"][i]) and res["part"][i] == oracle.MISS_PART, (flags, res)
            else:
                if not uncertain or flags & 4:
                    assert abs(res["t"][i] - exp[0]) <= 1e-6 * max(1.0, exp[0]), (flags, res)
                    assert int(res["part"][i]) == exp[1] and int(res["voxel"][i]) == exp[2], (flags, res)


@pytest.mark.parametrize("flags", list(FLAG_SETS.values()), ids=list(FLAG_SETS.keys()))
def test_pr1_parity(ctx, pr1, flags):
    scene, gs, so = pr1
    rays = synthetic.pr1_rays(scene)[: 16384 - 77]  # ragged tail
    ora = so.trace(rays)
    res = gs.trace(rays, flags)
    rep = compare(scene, gs.local, rays, res, ora)
    assert rep["hits"] >= 1241  # the oracle hits 1379 of these rays; the floor is 90% of that
    assert rep["flagged"] <= 0.05 * rep["rays"], rep
    print("PR1", flags, rep)


def test_flags_do_not_change_results(ctx, pr1):
    """Culling and depth sorting only save work (Sec. IV; the optimised and
    unoptimised animations are identical): with FP64 re-intersection the hits
    are bit-identical under every flag combination."""
    scene, gs, so = pr1
    rays = synthetic.pr1_rays(scene)
    ref = gs.trace(rays, 4)
    for f in (5, 6, 7):
        res = gs.trace(rays, f)
        for k in ("t", "part", "voxel", "flags"):
            assert np.array_equal(res[k], ref[k]), (f, k)


def test_articulated_reduced_parity(ctx):
    fig = synthetic.articulated_figure(depth=7)
    gs = GpuScene(ctx, fig.scene)
    so = oracle.SceneOracle(fig.scene)
    rays = fig.rays(320, 180)
    for frame in (0, 17, 45):
        local = fig.pose(frame)
        gs.set_pose(local)
        ora = so.trace(rays, local=local)
        res = gs.trace(rays, 7)
        rep = compare(fig.scene, local, rays, res, ora)
        # the oracle hits 3374 / 3668 / 3834 of these seeded rays at frames 0 / 17 / 45;
        # the floor (90% of the smallest) keeps a changed workload from thinning the comparison
        assert rep["hits"] >= 3030
        print("ART-reduced frame", frame, rep)


def test_incoherent_affine_many_parts(ctx):
    """Random affine poses (scale 0.5-2, shear <= 0.1), directions uniform on
    the sphere, 300 parts (beyond the shared-memory part table), mixed depths."""
    rng = np.random.default_rng(2024)
    assets = []
    for depth in (3, 4, 5, 6):
        n = 1 << depth
        occ = rng.random(n ** 3) < 0.04
        idx = np.nonzero(occ)[0]
        assets.append(synthetic.make_asset(depth, (idx % n, (idx // n) % n, idx // (n * n))))
    P = 300
    local = []
    for _ in range(P):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        S = np.diag(rng.uniform(0.5, 2.0, 3))
        H = np.eye(3)
        H[0, 1], H[0, 2], H[1, 2] = rng.uniform(-0.1, 0.1, 3)
        local.append(synthetic.affine12(R @ S @ H, rng.uniform(-8, 8, 3)))
    scene = synthetic.Scene("bat-like", assets, rng.integers(0, 4, P).astype(np.int32),
                            np.full(P, -1, np.int32), np.array(local))
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    rays = synthetic.random_rays(20000 - 3, rng, (-9,) * 3, (9,) * 3)
    ora = so.trace(rays)
    for flags in (7, 4):
        res = gs.trace(rays, flags)
        rep = compare(scene, scene.local, rays, res, ora)
        assert rep["hits"] > 2000
        print("incoherent", flags, rep)


def test_edge_rays(ctx, pr1):
    """Degenerate and extreme rays, every one compared with the oracle.  Both
    sides apply the same rule to inputs that are not rays (Eq. 1 needs a
    direction: its largest component magnitude in [2^-60, 2^60], finite origin
    and direction, no NaN bound): they are misses, even a zero direction whose
    origin lies inside an occupied leaf."""
    scene, gs, so = pr1
    base = synthetic.pr1_rays(scene)[8000:8064].copy()
    ora_base = so.trace(base)
    k = int(np.nonzero(ora_base["part"] != oracle.MISS_PART)[0][0])  # a ray that hits
    rays = base.copy()
    rays[0, 3], rays[0, 7] = 5.0, 1.0          # tmin > tmax: empty segment
    rays[1, 4:7] = 0.0                          # zero direction
    rays[2, 0] = np.nan                         # NaN origin
    rays[3, 7] = 0.0                            # tmax = 0 with origin outside everything
    rays[4, 4:7] = [1.0, 0.0, 0.0]              # axis-aligned
    rays[5, 4:7] = [0.0, -1.0, 0.0]
    rays[6, 4:7] *= 1000.0                      # long direction (t scales)
    rays[7, 4:7] *= 1e-3                        # short direction
    # zero direction from the centre of the leaf ray k hits
    part, vox = int(ora_base["part"][k]), int(ora_base["voxel"][k])
    D = scene.assets[int(scene.part_asset[part])].depth
    cell = np.array([(vox >> (a * D)) & ((1 << D) - 1) for a in range(3)], dtype=np.float64)
    W = oracle.compose(scene.parent, gs.local)[part].reshape(3, 4)
    inside = W[:, :3] @ ((cell + 0.5) / 2.0 ** D) + W[:, 3]
    rays[8, 0:3], rays[8, 3], rays[8, 4:7], rays[8, 7] = inside, 0.0, 0.0, np.inf
    # ray k with its direction rescaled to the ends of the valid range and just beyond
    m = np.float32(np.abs(base[k, 4:7]).max())
    unit = (base[k, 4:7] / m).astype(np.float32)  # largest component exactly 1
    for row, scale in ((9, 2.0 ** -60), (10, 2.0 ** -61), (11, 2.0 ** 60), (12, 2.0 ** 61)):
        rays[row] = base[k]
        rays[row, 4:7] = unit * np.float32(scale)
    rays[13, 3] = np.nan                        # NaN tmin
    rays[14, 7] = np.nan                        # NaN tmax
    rays[15, 4] = np.inf                        # infinite direction component
    valid = oracle.ray_valid(rays)
    assert not valid[[1, 2, 8, 10, 12, 13, 14, 15]].any() and valid[[0, 3, 9, 11]].all()
    ora = so.trace(rays)
    for flags in (0, 4, 7):
        res = gs.trace(rays, flags)
        for i in (0, 1, 2, 3, 8, 10, 12, 13, 14, 15):
            assert res["part"][i] == oracle.MISS_PART and math.isinf(res["t"][i]), (flags, i)
            assert ora["part"][i] == oracle.MISS_PART, i
        for i in (9, 11):  # valid rescaled rays hit the same leaf; t scales with 1 / |d|
            assert ora["part"][i] == ora_base["part"][k] and ora["voxel"][i] == ora_base["voxel"][k]
        compare(scene, gs.local, rays, res, ora)
    # scaling d by s divides t by s
    r6 = gs.trace(base[6:7], 7)
    assert abs(res["t"][6] * 1000.0 - r6["t"][0]) <= 1e-5 * r6["t"][0] or not np.isfinite(r6["t"][0])


def test_empty_and_degenerate_assets(ctx):
    rng = np.random.default_rng(12)
    empty = synthetic.Asset(5, np.zeros(0, np.uint64), np.zeros(0, np.uint32))
    one = synthetic.make_asset(1, (np.array([1]), np.array([0]), np.array([1])))
    deep = synthetic.make_asset(16, (np.array([1, 40000, 65535]), np.array([2, 30000, 65535]),
                                     np.array([3, 20000, 0])))
    dense_n = 8
    g3 = np.arange(dense_n)
    xx, yy, zz = np.meshgrid(g3, g3, g3, indexing="ij")
    full = synthetic.make_asset(3, (xx.ravel(), yy.ravel(), zz.ravel()))
    assets = [empty, one, deep, full]
    local = np.array([synthetic.affine12(synthetic.euler_xyz(*rng.uniform(-1, 1, 3)), rng.uniform(-2, 2, 3))
                      for _ in range(4)])
    scene = synthetic.Scene("degenerate", assets, np.arange(4, dtype=np.int32), np.array([-1, 0, -1, 2], np.int32),
                            local)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    rays = synthetic.random_rays(8192, rng, (-3,) * 3, (3,) * 3)
    ora = so.trace(rays)
    res = gs.trace(rays, 7)
    rep = compare(scene, local, rays, res, ora)
    # the oracle hits 155 of these 8192 seeded rays (three of the four assets are
    # nearly empty); the floor is 90% of that
    assert rep["hits"] >= 139
    # the deep asset is reachable: rays aimed at its leaf centres hit it
    world = oracle.compose(scene.parent, local)
    W = world[2].reshape(3, 4)
    tgt = np.array([[1.5, 2.5, 3.5], [40000.5, 30000.5, 20000.5], [65535.5, 65535.5, 0.5]]) / 65536.0
    pts = tgt @ W[:, :3].T + W[:, 3]
    org = pts + np.array([5.0, 4.0, 3.0])
    r2 = np.zeros((3, 8), np.float32)
    r2[:, 0:3] = org
    r2[:, 4:7] = pts - org
    r2[:, 7] = np.inf
    ora2 = so.trace(r2)
    res2 = gs.trace(r2, 7)
    compare(scene, local, r2, res2, ora2)
    assert (ora2["part"] == 2).sum() >= 2


def test_batch_equals_individual(ctx, pr1):
    import torch

    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    fig = synthetic.articulated_figure(depth=6)
    ga = GpuScene(ctx, fig.scene)
    r1 = synthetic.pr1_rays(scene)
    r2 = fig.rays(200, 120)
    r3 = r1[::7].copy()
    items, outs = [], []
    for sc, r in ((gs, r1), (ga, r2), (gs, r3)):
        rt = torch.from_numpy(np.ascontiguousarray(r)).cuda()
        ht = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
        ft = torch.empty(r.shape[0], dtype=torch.int32, device="cuda")
        items.append((sc.sc, rt, ht, ft))
        outs.append((sc, r, ht, ft))
    ctx.trace_batch(items, flags=7)
    torch.cuda.synchronize()
    for sc, r, ht, ft in outs:
        ref = sc.trace(r, 7)
        got = g.decode_hits(ht)
        for k in ("t", "part", "voxel"):
            assert np.array_equal(got[k], ref[k]), k
        assert np.array_equal(ft.cpu().numpy().astype(np.uint32), ref["flags"])


def test_stats_counters(ctx, pr1):
    import torch

    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    rays = torch.from_numpy(synthetic.pr1_rays(scene)).cuda()
    st = g.new_stats()
    rf = torch.zeros(rays.shape[0], dtype=torch.int32, device="cuda")
    gs.sc.trace(rays, flags=7 | g.TRACE_STATS, ray_flags=rf, stats=st)
    torch.cuda.synchronize()
    s = g.read_stats(st)
    flags = rf.cpu().numpy()
    assert s["rays"] == rays.shape[0]
    assert s["flagged"] == int(((flags & 1) != 0).sum())
    assert s["flag_width"] == int(((flags & 4) != 0).sum())
    assert s["fixed"] == s["flagged"] + s["flag_width"] == int(((flags & 2) != 0).sum())
    assert s["nodes_visited"] > 0 and s["parts_entered"] <= s["parts_tested"]
    assert s["passes"] >= s["rays"]


def test_articulated_full_size_sampled(ctx):
    """The bench workload (1920x1080 rays, depth-9 parts) in the bench's launch
    configuration; the oracle checks a random sample of 20000 rays."""
    fig = synthetic.articulated_figure()
    gs = GpuScene(ctx, fig.scene)
    so = oracle.SceneOracle(fig.scene)
    rays = fig.rays()
    rng = np.random.default_rng(99)
    for frame in (0, 31):
        local = fig.pose(frame)
        gs.set_pose(local)
        res = gs.trace(rays, 7)
        idx = rng.choice(rays.shape[0], 20000, replace=False)
        ora = so.trace(rays[idx], local=local)
        sub = {k: v[idx] for k, v in res.items()}
        rep = compare(fig.scene, local, rays[idx], sub, ora)
        # about 6% of the frame's rays hit: the oracle hits 1184 / 1336 of the
        # sampled rays at frames 0 / 31; the floor is 90% of the smaller
        assert rep["hits"] >= 1065
        print("ART full sampled frame", frame, rep, "flag rate full frame",
              float(((res["flags"] & 1) != 0).mean()))


def test_ray_ordering_does_not_change_results(ctx, pr1):
    """Ray ordering only changes which rays share a warp: hits and flags are
    bit-identical with and without it, for coherent and incoherent rays."""
    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    rng = np.random.default_rng(4)
    cases = [(gs, synthetic.pr1_rays(scene)[:12345]),
             (gs, synthetic.random_rays(9999, rng, (-3,) * 3, (3,) * 3))]
    for sc, rays in cases:
        ref = sc.trace(rays, 7)
        for extra in (g.TRACE_ORDER_DIR, g.TRACE_ORDER_ORIGIN):
            res = sc.trace(rays, 7 | extra)
            for k in ("t", "part", "voxel", "flags"):
                assert np.array_equal(res[k], ref[k]), (extra, k)
    ora = so.trace(cases[1][1])
    compare(scene, gs.local, cases[1][1], gs.trace(cases[1][1], 7 | g.TRACE_ORDER_ORIGIN), ora)


def test_raygen_matches_host_pinhole(ctx):
    import torch

    eye, tgt = (3.0, 2.0, 5.0), (0.2, -0.1, 0.3)
    for w, h in ((128, 128), (333, 77)):
        dev = ctx.raygen(eye, tgt, w, h, 60.0)
        torch.cuda.synchronize()
        got = dev.cpu().numpy()
        ref = synthetic.pinhole_rays(eye, tgt, w, h, 60.0)
        assert got.shape == ref.shape
        assert np.array_equal(got[:, 0:4], ref[:, 0:4])
        assert np.max(np.abs(got[:, 4:7] - ref[:, 4:7])) <= 2e-6
        assert np.all(np.isinf(got[:, 7]))


def _pack_hits(t, part, voxel):
    p = np.zeros((len(t), 4), np.uint32)
    p[:, 0] = np.asarray(t, np.float32).view(np.uint32)
    p[:, 1] = part
    p[:, 2] = (np.asarray(voxel, np.uint64) & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    p[:, 3] = (np.asarray(voxel, np.uint64) >> np.uint64(32)).astype(np.uint32)
    return p.view(np.int64).reshape(-1, 2)


def test_hit_colors_match_oracle(ctx, pr1):
    """Leaf colours of hits (Sec. IV-C hit buffer): the oracle's hits coloured
    on the GPU equal the oracle's colours everywhere; the GPU's own trace gives
    the oracle's colours on every ray whose ids are certified; hits that name
    no leaf come back invalid."""
    import torch

    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    rays = synthetic.pr1_rays(scene)
    ora = so.trace(rays)
    bg = 0x102030
    want = so.hit_colors(ora, background=bg)
    hits = torch.from_numpy(_pack_hits(ora["t"], ora["part"], ora["voxel"])).cuda()
    got = gs.sc.hit_colors(hits, background=bg).cpu().numpy().view(np.uint32)
    assert np.array_equal(got, want)
    assert (ora["part"] != oracle.MISS_PART).sum() > 1000
    r = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32)).cuda()
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    h2 = gs.sc.trace(r, flags=g.TRACE_DEFAULT, ray_flags=rf)
    c2 = gs.sc.hit_colors(h2, background=bg).cpu().numpy().view(np.uint32)
    certified = (rf.cpu().numpy() & g.RAY_UNCERTAIN) == 0
    assert np.array_equal(c2[certified], want[certified])
    # invalid: part out of range, voxel outside the grid, voxel that is not a leaf
    a = scene.assets[int(scene.part_asset[0])]
    occupied = set(a.leaf_ids.tolist())
    free = next(v for v in range(1 << (3 * a.depth)) if v not in occupied)
    bad = _pack_hits([1.0, 1.0, 1.0, np.inf], [scene.n_parts, 0, 0, oracle.MISS_PART],
                     [0, 1 << (3 * a.depth), free, oracle.MISS_VOXEL])
    cb = gs.sc.hit_colors(torch.from_numpy(bad).cuda(), background=bg).cpu().numpy().view(np.uint32)
    assert cb.tolist() == [g.COLOR_INVALID] * 3 + [bg]
    with pytest.raises(g.SvoError):
        gs.sc.hit_colors(hits, background=0x1000000)
    torch.cuda.synchronize()


def _shade_case(ctx, gs, so, rays, light, ambient, bg):
    import torch

    import paper_1911_06001_gb300 as g

    rays = np.ascontiguousarray(rays, dtype=np.float32)
    light32 = np.asarray(light, dtype=np.float32).astype(np.float64)  # what the library receives
    ora = so.trace(rays)
    want, amb = so.shade(ora, rays, light32, float(np.float32(ambient)), bg)
    r = torch.from_numpy(rays).cuda()
    # the oracle's own hits, shaded on the GPU
    oh = torch.from_numpy(_pack_hits(ora["t"], ora["part"], ora["voxel"])).cuda()
    got = gs.sc.shade(r, oh, light, ambient, bg).cpu().numpy().view(np.uint32)
    bad = np.nonzero((got != want) & ~amb)[0]
    assert bad.size == 0, (bad[:5], got[bad[:5]], want[bad[:5]])
    # the GPU's own trace: equal wherever the ids are certified
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    h2 = gs.sc.trace(r, flags=g.TRACE_DEFAULT, ray_flags=rf)
    got2 = gs.sc.shade(r, h2, light, ambient, bg).cpu().numpy().view(np.uint32)
    certified = ((rf.cpu().numpy() & g.RAY_UNCERTAIN) == 0) & ~amb
    assert np.array_equal(got2[certified], want[certified])
    hit = ora["part"] != oracle.MISS_PART
    return int(hit.sum()), int((amb & hit).sum())


def test_shade_matches_oracle(ctx, pr1):
    """Lambert shading from the hit leaf's colour and entry-face normal
    (Sec. IV-C hit buffer): equal to the FP64 oracle on every pixel whose face
    choice and channel rounding are not within rounding distance of a tie;
    also on a sheared, anisotropically scaled scene."""
    import torch

    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    hits, amb = _shade_case(ctx, gs, so, synthetic.pr1_rays(scene), (0.5, -0.75, 0.25), 0.15, 0x203040)
    assert hits > 1000 and amb < 0.01 * hits
    bat = synthetic.batched_scenes(seed=8, n_scenes=1, parts=(8, 12), depths=range(5, 7), side=(96, 96), per_depth=2)
    sc = bat.scenes[0]  # its assets are the pool's
    gs2 = GpuScene(ctx, sc)
    hits2, amb2 = _shade_case(ctx, gs2, oracle.SceneOracle(sc), bat.rays[0], (-0.25, 0.5, 1.0), 0.0, 0)
    assert hits2 > 100 and amb2 < 0.05 * hits2
    # argument checks
    r = torch.zeros((4, 8), dtype=torch.float32, device="cuda")
    h = torch.zeros((4, 2), dtype=torch.int64, device="cuda")
    for light, ambient, bg in (((0, 0, 0), 0.1, 0), ((1, 0, 0), 1.5, 0), ((1, 0, 0), 0.1, 1 << 24)):
        with pytest.raises(g.SvoError):
            gs.sc.shade(r, h, light, ambient, bg)
    torch.cuda.synchronize()


def test_octree_dimension_poses(ctx):
    """Sec. III-B poses (rotation, translation, per-axis octree dimensions)
    through scene_set_transforms_trs: equal to the oracle, and bit-identical
    to the same poses given as [R diag(s) | t] affines; a transform tree of
    such poses composes like any affine one."""
    import paper_1911_06001_gb300 as g

    rng = np.random.default_rng(4040)
    assets = []
    for depth in (4, 5, 6):
        n = 1 << depth
        occ = np.nonzero(rng.random(n ** 3) < 0.05)[0]
        assets.append(synthetic.make_asset(depth, (occ % n, (occ // n) % n, occ // (n * n))))
    P = 24
    parent = np.array([-1 if i < 8 else int(rng.integers(0, i)) for i in range(P)], np.int32)
    rts = np.zeros((P, 15))
    for p in range(P):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        rts[p, :9] = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                               [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                               [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]]).ravel()
        rts[p, 9:12] = rng.uniform(-3, 3, 3) if parent[p] < 0 else rng.uniform(-1, 1, 3)
        rts[p, 12:15] = rng.uniform(0.4, 2.5, 3)
    local = oracle.trs_to_local(rts)
    scene = synthetic.Scene("trs", assets, rng.integers(0, 3, P).astype(np.int32), parent, local)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    rays = synthetic.random_rays(30000, rng, (-5,) * 3, (5,) * 3)
    ref = gs.trace(rays, 7)  # poses set as affines by GpuScene
    gs.sc.set_transforms_trs(rts)
    gs.sc.refit()
    got = gs.trace(rays, 7)
    rep = compare(scene, local, rays, got, so.trace(rays, local=local))
    assert rep["hits"] > 1000
    for k in ("t", "part", "voxel", "flags"):
        assert np.array_equal(got[k], ref[k]), k
    # rejected poses change nothing
    bad = rts.copy()
    bad[3, 0] += 1e-6  # R no longer orthonormal
    with pytest.raises(g.SvoError):
        gs.sc.set_transforms_trs(bad)
    bad = rts.copy()
    bad[5, 13] = 0.0  # a zero dimension
    with pytest.raises(g.SvoError):
        gs.sc.set_transforms_trs(bad)
    bad = rts.copy()
    bad[1, 10] = np.nan
    with pytest.raises(g.SvoError):
        gs.sc.set_transforms_trs(bad)
    gs.sc.refit()
    again = gs.trace(rays, 7)
    assert np.array_equal(again["part"], got["part"]) and np.array_equal(again["t"], got["t"])


def test_animation_never_writes_the_svos(ctx):
    """Animation moves only poses (Sec. III): after 60 frames of poses, refits
    and traces with every trace option, each asset's device data is byte for
    byte what the host build produced."""
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=7)
    gs = GpuScene(ctx, fig.scene)
    before = [ctx.read_asset(h) for h in gs.handles]
    for a, (nodes, rgb) in zip(fig.scene.assets, before):
        hn, hrgb = g.build_host(a.depth, a.leaf_ids, a.rgb)
        assert np.array_equal(nodes, hn) and np.array_equal(rgb, hrgb)
    rays = torch.from_numpy(fig.rays(320, 180)).cuda()
    hits = torch.empty((rays.shape[0], 2), dtype=torch.int64, device="cuda")
    opts = [g.TRACE_DEFAULT, g.TRACE_DEFAULT | g.TRACE_REUSE, g.TRACE_FP64_FIX, g.TRACE_DEFAULT | g.trace_image(320),
            g.TRACE_DEFAULT | g.TRACE_ORDER_ORIGIN]
    for f in range(60):
        gs.sc.set_transforms(fig.pose(f))
        gs.sc.refit()
        gs.sc.trace(rays, hits, flags=opts[f % len(opts)])
    gs.sc.hit_colors(hits)
    torch.cuda.synchronize()
    after = [ctx.read_asset(h) for h in gs.handles]
    for (n0, c0), (n1, c1) in zip(before, after):
        assert n0.tobytes() == n1.tobytes() and c0.tobytes() == c1.tobytes()


def test_batched_ray_ordering_does_not_change_results(ctx, pr1):
    """Ray ordering across a batch (all items sorted by the same launches)
    leaves every item's hits and flags at its rays' own indices, equal to the
    unordered batch."""
    import torch

    import paper_1911_06001_gb300 as g

    scene, gs, so = pr1
    fig = synthetic.articulated_figure(depth=6)
    ga = GpuScene(ctx, fig.scene)
    rng = np.random.default_rng(31)
    sets = [(gs, synthetic.pr1_rays(scene)), (ga, fig.rays(200, 120)), (gs, synthetic.random_rays(5000, rng, (-3,) * 3,
                                                                                                   (3,) * 3)),
            (ga, np.zeros((0, 8), np.float32)), (ga, synthetic.random_rays(777, rng, (-2,) * 3, (2,) * 3))]
    outs = {}
    for order in (0, g.TRACE_ORDER_DIR, g.TRACE_ORDER_ORIGIN):
        items, res = [], []
        for sc, r in sets:
            rt = torch.from_numpy(np.ascontiguousarray(r, dtype=np.float32)).cuda()
            ht = torch.zeros((r.shape[0], 2), dtype=torch.int64, device="cuda")
            ft = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
            items.append((sc.sc, rt, ht, ft))
            res.append((ht, ft))
        ctx.trace_batch(items, flags=7 | order)
        torch.cuda.synchronize()
        outs[order] = [(h.cpu().numpy(), f.cpu().numpy()) for h, f in res]
    for order in (g.TRACE_ORDER_DIR, g.TRACE_ORDER_ORIGIN):
        for (h0, f0), (h1, f1) in zip(outs[0], outs[order]):
            assert np.array_equal(h0, h1) and np.array_equal(f0, f1)
