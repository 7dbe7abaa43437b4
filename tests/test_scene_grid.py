"""Scene-level grid culling (Sec. V-E, the larger structure over many parts) on
the GPU: traces with SVO_TRACE_GRID must equal the FP64 oracle element by
element, like every other trace, on scenes large enough to get a grid and on
the cases where the walk falls back to the cluster level."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import synthetic
from gpu_helpers import GpuScene, compare

pytestmark = pytest.mark.gpu

DEFAULT = 7  # CULL | SORT | FP64_FIX
GRID = 512


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1911_06001_gb300 as g

    assert g.TRACE_GRID == GRID
    c = g.Context(0)
    yield c
    c.check_device()
    c.close()


def _assets(rng, depths=(3, 4, 5, 6), p=0.04):
    out = []
    for depth in depths:
        n = 1 << depth
        occ = rng.random(n ** 3) < p
        idx = np.nonzero(occ)[0]
        if idx.size == 0:
            idx = np.array([0])
        out.append(synthetic.make_asset(depth, (idx % n, (idx // n) % n, idx // (n * n))))
    return out


def _affine_scene(rng, P, box, scale=(0.5, 2.0), offset=0.0, assets=None):
    """P parts of random rotation x scale x shear, placed uniformly in a cube of side ``box``."""
    assets = assets if assets is not None else _assets(rng)
    local = []
    for _ in range(P):
        q = rng.standard_normal(4)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        S = np.diag(rng.uniform(*scale, 3))
        H = np.eye(3)
        H[0, 1], H[0, 2], H[1, 2] = rng.uniform(-0.1, 0.1, 3)
        A = R @ S @ H
        local.append(synthetic.affine12(A, rng.uniform(-box / 2, box / 2, 3) - A @ np.full(3, 0.5) + offset))
    return synthetic.Scene("grid", assets, rng.integers(0, len(assets), P).astype(np.int32),
                           np.full(P, -1, np.int32), np.array(local))


def _outside_camera_rays(box, w, h, offset=0.0):
    eye = np.array([0.9, 0.6, 1.4]) * box + offset
    return synthetic.pinhole_rays(eye, np.full(3, offset), w, h, fov_deg=50.0)


def _stats(gs, rays, flags):
    import torch

    import paper_1911_06001_gb300 as g

    r = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32)).cuda()
    st = g.new_stats()
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    gs.sc.trace(r, flags=flags | g.TRACE_STATS, ray_flags=rf, stats=st)
    torch.cuda.synchronize()
    return g.read_stats(st)


@pytest.mark.parametrize("P", [64, 250, 700, 1024])
def test_grid_matches_oracle(ctx, P):
    rng = np.random.default_rng(7000 + P)
    box = 4.0 * P ** (1.0 / 3.0)
    scene = _affine_scene(rng, P, box)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    inner = synthetic.random_rays(12000 - 5, rng, (-box / 2,) * 3, (box / 2,) * 3)
    cam = _outside_camera_rays(box, 96, 64)
    for rays in (inner, cam):
        ora = so.trace(rays)
        res = gs.trace(rays, DEFAULT | GRID)
        rep = compare(scene, scene.local, rays, res, ora)
        assert rep["hits"] > 0.03 * len(rays)
        # the certified ids of the grid walk are the cluster level's
        ref = gs.trace(rays, DEFAULT)
        both = ((res["flags"] | ref["flags"]) & 1) == 0
        assert np.array_equal(res["part"][both], ref["part"][both])
        assert np.array_equal(res["voxel"][both], ref["voxel"][both])
        print("grid", P, rep)
    s_grid, s_cl = _stats(gs, inner, DEFAULT | GRID), _stats(gs, inner, DEFAULT)
    assert s_grid["rays"] == s_cl["rays"] == len(inner)
    print("parts tested per ray: grid", s_grid["parts_tested"] / len(inner), "clusters",
          s_cl["parts_tested"] / len(inner))


def test_grid_after_pose_changes(ctx):
    """The grid is rebuilt by every refit: new poses move parts between cells."""
    rng = np.random.default_rng(71)
    P = 180
    box = 4.0 * P ** (1.0 / 3.0)
    scene = _affine_scene(rng, P, box)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    rays = _outside_camera_rays(box, 80, 60)
    for k in range(3):
        local = scene.local.copy()
        local[:, [3, 7, 11]] += rng.uniform(-box / 4, box / 4, (P, 3))
        gs.set_pose(local)
        res = gs.trace(rays, DEFAULT | GRID)
        compare(scene, local, rays, res, so.trace(rays, local=local))


def test_grid_edge_rays(ctx):
    rng = np.random.default_rng(72)
    P = 120
    box = 4.0 * P ** (1.0 / 3.0)
    scene = _affine_scene(rng, P, box)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    base = synthetic.random_rays(512, rng, (-box / 2,) * 3, (box / 2,) * 3)
    rays = base.copy()
    n = 64
    # axis-aligned directions (zero components), each sign
    for i in range(6):
        rays[i * n:(i + 1) * n, 4:7] = 0.0
        rays[i * n:(i + 1) * n, 4 + i // 2] = 1.0 if i % 2 == 0 else -1.0
    # origins on lattice planes of the scene's coordinates, diagonal directions (cell-corner ties)
    sl = slice(6 * n, 7 * n)
    rays[sl, 0:3] = np.round(rays[sl, 0:3])
    rays[sl, 4:7] = np.sign(rng.standard_normal((n, 3)))
    # tiny direction components (the walk hands these to the cluster level) and short segments
    sl = slice(7 * n, 8 * n)
    rays[sl, 4] = 1e-30
    rays[sl, 7] = rng.uniform(0.0, box / 2, n)
    rays[::5, 3] = -box  # segments starting behind the origin
    ora = so.trace(rays)
    res = gs.trace(rays, DEFAULT | GRID)
    compare(scene, scene.local, rays, res, ora)


def test_grid_fallbacks(ctx):
    """Cases the grid declines (lists overflowing, a scene far from the origin
    relative to its cells, fewer than 64 parts) still trace exactly."""
    rng = np.random.default_rng(73)
    cases = [
        ("overlapping", _affine_scene(rng, 96, 2.0, scale=(6.0, 9.0))),   # every part meets every cell
        ("far", _affine_scene(rng, 96, 16.0, offset=3.0e4)),            # rounding too coarse for the walk
        ("small", _affine_scene(rng, 40, 10.0)),                         # no grid below 64 parts
    ]
    for name, scene in cases:
        gs = GpuScene(ctx, scene)
        so = oracle.SceneOracle(scene)
        off = 3.0e4 if name == "far" else 0.0
        box = 16.0 if name != "small" else 10.0
        rays = _outside_camera_rays(box, 64, 48, offset=off)
        ora = so.trace(rays)
        res = gs.trace(rays, DEFAULT | GRID)
        rep = compare(scene, scene.local, rays, res, ora)
        ref = gs.trace(rays, DEFAULT)
        for k in ("part", "voxel"):
            assert np.array_equal(res[k], ref[k]), (name, k)
        print(name, rep)


def test_grid_flag_rules(ctx):
    import paper_1911_06001_gb300 as g

    rng = np.random.default_rng(74)
    scene = _affine_scene(rng, 64, 12.0)
    gs = GpuScene(ctx, scene)
    rays = synthetic.random_rays(256, rng, (-6,) * 3, (6,) * 3)
    with pytest.raises(g.SvoError):
        gs.trace(rays, DEFAULT | GRID | g.TRACE_REUSE)
    with pytest.raises(g.SvoError):
        gs.trace(rays, g.TRACE_CULL | g.TRACE_FP64_FIX | GRID)


def test_new_scene_traces_identity_poses(ctx):
    """A new scene holds identity poses (every part in the unit cube, one grid
    cell list per part): its first trace, before any pose is set, is the
    oracle's trace of those poses for the plain trace, the cluster level and
    the grid walk alike."""
    rng = np.random.default_rng(75)
    scene = _affine_scene(rng, 80, 12.0)
    handles = [ctx.upload(a.depth, a.leaf_ids, a.rgb) for a in scene.assets]
    sc = ctx.scene([handles[int(i)] for i in scene.part_asset], scene.parent)
    ident = np.tile(synthetic.affine12(np.eye(3), np.zeros(3)), (scene.n_parts, 1))
    rays = synthetic.random_rays(2048, rng, (-1,) * 3, (2,) * 3)
    ora = oracle.SceneOracle(scene).trace(rays, local=ident)
    import torch

    import paper_1911_06001_gb300 as g

    r = torch.from_numpy(rays).cuda()
    for flags in (0, DEFAULT, DEFAULT | GRID):
        rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
        hits = sc.trace(r, flags=flags, ray_flags=rf)
        torch.cuda.synchronize()
        d = g.decode_hits(hits)
        d["flags"] = rf.cpu().numpy().astype(np.uint32)
        if flags & 4:
            rep = compare(scene, ident, rays, d, ora)
            assert rep["hits"] > 100
        else:  # no FP64 pass: compare where the FP32 trace is certain
            ok = (d["flags"] & 1) == 0
            assert np.array_equal(d["part"][ok], ora["part"][ok])
    sc.close()
    for h in handles:
        ctx.release(h)


def test_autotune_tries_the_grid(ctx):
    import torch

    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300 import autotune

    rng = np.random.default_rng(76)
    P = 100
    box = 4.0 * P ** (1.0 / 3.0)
    scene = _affine_scene(rng, P, box)
    gs = GpuScene(ctx, scene)
    rays_np = _outside_camera_rays(box, 128, 96)
    rays = torch.from_numpy(rays_np).cuda()
    old = ctx.trace_config()
    cfg = autotune.tune(ctx, gs.sc, rays, reps=2, blocks=(128,), rays_per_lane=(1,), orders=("none",))
    assert sorted(x["cull"] for x in cfg["table"]) == ["clusters", "grid", "wavefront"]
    extra = autotune.order_flag(cfg)
    assert bool(extra & g.TRACE_GRID) == (cfg["cull"] == "grid")
    assert bool(extra & g.TRACE_WAVEFRONT) == (cfg["cull"] == "wavefront")
    res = gs.trace(rays_np, DEFAULT | extra)
    compare(scene, scene.local, rays_np, res, oracle.SceneOracle(scene).trace(rays_np))
    # no grid knob for small scenes; neither grid nor wavefront with hit buffer reuse
    small = GpuScene(ctx, _affine_scene(rng, 20, 8.0))
    c2 = autotune.tune(ctx, small.sc, rays, reps=1, blocks=(128,), rays_per_lane=(1,), orders=("none",))
    assert [x["cull"] for x in c2["table"]] == ["clusters", "wavefront"]
    c3 = autotune.tune(ctx, gs.sc, rays, flags=DEFAULT | g.TRACE_REUSE, reps=1, blocks=(128,), rays_per_lane=(1,),
                       orders=("none",))
    assert [x["cull"] for x in c3["table"]] == ["clusters"]
    ctx.set_trace_config(*old)


def test_grid_rebuilt_in_graph_replays(ctx):
    """The grid is rebuilt after every refit whether the refit and the trace
    run eagerly or as CUDA-graph replays: a captured frame, and an eager grid
    trace after a graph that only refits, both see the new poses."""
    import torch

    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300.graphs import FrameGraph

    rng = np.random.default_rng(77)
    P = 150
    box = 4.0 * P ** (1.0 / 3.0)
    scene = _affine_scene(rng, P, box)
    gs = GpuScene(ctx, scene)
    so = oracle.SceneOracle(scene)
    rays_np = _outside_camera_rays(box, 96, 72)
    rays = torch.from_numpy(rays_np).cuda()
    hits = torch.empty((rays.shape[0], 2), dtype=torch.int64, device="cuda")
    rf = torch.zeros(rays.shape[0], dtype=torch.int32, device="cuda")
    fg = FrameGraph(ctx, gs.sc, rays, hits, flags=DEFAULT | GRID, ray_flags=rf)
    poses = []
    for k in range(3):
        local = scene.local.copy()
        local[:, [3, 7, 11]] += rng.uniform(-box / 4, box / 4, (P, 3))
        poses.append(local)
        fg.replay(local)
        torch.cuda.synchronize()
        d = g.decode_hits(hits)
        d["flags"] = rf.cpu().numpy().astype(np.uint32)
        compare(scene, local, rays_np, d, so.trace(rays_np, local=local))
    # a graph holding only the pose upload and the refit, then an eager grid trace
    dev_poses = torch.from_numpy(scene.local.copy()).cuda()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        gs.sc.set_transforms_device(dev_poses)
        gs.sc.refit()
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        gs.sc.set_transforms_device(dev_poses)
        gs.sc.refit()
    for local in (poses[0], poses[1]):
        res = gs.trace(rays_np, DEFAULT | GRID)  # builds the grid for the current poses
        dev_poses.copy_(torch.from_numpy(local))
        graph.replay()
        torch.cuda.synchronize()
        res = gs.trace(rays_np, DEFAULT | GRID)
        compare(scene, local, rays_np, res, so.trace(rays_np, local=local))


def test_grid_in_batches_and_without_allocation(ctx):
    """The grid flag in one persistent launch over scenes with and without a
    grid (and one scene twice: its grid is built once), and through
    trace_rays_noalloc: every result equals the same scene traced alone."""
    import ctypes as C

    import torch

    import paper_1911_06001_gb300 as g

    rng = np.random.default_rng(78)
    specs = [(40, 10.0), (100, 4.0 * 100 ** (1 / 3)), (300, 4.0 * 300 ** (1 / 3))]
    scenes, items, outs = [], [], []
    for P, box in specs:
        sc = _affine_scene(rng, P, box)
        gs = GpuScene(ctx, sc)
        scenes.append((sc, gs, box))
    for k in (0, 1, 2, 1):
        sc, gs, box = scenes[k]
        rays_np = _outside_camera_rays(box, 64 + 16 * k, 48)
        rt = torch.from_numpy(rays_np).cuda()
        ht = torch.empty((rt.shape[0], 2), dtype=torch.int64, device="cuda")
        ft = torch.zeros(rt.shape[0], dtype=torch.int32, device="cuda")
        items.append((gs.sc, rt, ht, ft))
        outs.append((gs, rays_np, ht, ft))
    # new poses after the last trace: the batch must rebuild the grids first
    for sc, gs, box in scenes:
        local = sc.local.copy()
        local[:, [3, 7, 11]] += rng.uniform(-box / 8, box / 8, (sc.n_parts, 3))
        gs.set_pose(local)
    ctx.trace_batch(items, flags=DEFAULT | GRID)
    torch.cuda.synchronize()
    for gs, rays_np, ht, ft in outs:
        got = g.decode_hits(ht)
        got["flags"] = ft.cpu().numpy().astype(np.uint32)
        ref = gs.trace(rays_np, DEFAULT)
        compare(gs.scene, gs.local, rays_np, got, oracle.SceneOracle(gs.scene).trace(rays_np, local=gs.local))
        both = ((got["flags"] | ref["flags"]) & 1) == 0
        assert np.array_equal(got["part"][both], ref["part"][both])
    # the no-allocation entry point with the grid
    lib = g._lib.load()
    sc, gs, box = scenes[2]
    rays_np = _outside_camera_rays(box, 96, 64)
    r = torch.from_numpy(rays_np).cuda()
    hits = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    local = sc.local.copy()
    local[:, [3, 7, 11]] += 0.5
    gs.set_pose(local)
    rc = lib.trace_rays_noalloc(gs.sc.h, C.c_void_p(r.data_ptr()), r.shape[0], C.c_void_p(hits.data_ptr()),
                                C.c_void_p(rf.data_ptr()), DEFAULT | GRID, stream)
    assert rc == 0, lib.svo_last_error()
    torch.cuda.synchronize()
    got = g.decode_hits(hits)
    got["flags"] = rf.cpu().numpy().astype(np.uint32)
    compare(sc, local, rays_np, got, oracle.SceneOracle(sc).trace(rays_np, local=local))
