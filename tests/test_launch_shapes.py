"""Launch-shape knobs (block size, rays per lane, ray order), the autotuner and
the CUDA-graph frame: none of them may change a result."""

from __future__ import annotations

import numpy as np
import pytest

import synthetic
from gpu_helpers import GpuScene

pytestmark = pytest.mark.gpu


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


def _same(a, b):
    for k in ("t", "part", "voxel", "flags"):
        assert np.array_equal(a[k], b[k]), k


def test_every_launch_shape_gives_identical_hits(ctx):
    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    rng = np.random.default_rng(3)
    rays = np.concatenate([synthetic.pr1_rays(s)[:9000], synthetic.random_rays(3001, rng, (-3,) * 3, (3,) * 3)])
    ctx.set_trace_config(128, 4)
    ref = gs.trace(rays, g.TRACE_DEFAULT)
    for block in (64, 128, 256):
        for rpl in (1, 2, 4, 8):
            ctx.set_trace_config(block, rpl)
            _same(gs.trace(rays, g.TRACE_DEFAULT | g.TRACE_ORDER_ORIGIN), ref)
    ctx.set_trace_config(128, 4)
    with pytest.raises(g.SvoError):
        ctx.set_trace_config(96, 4)
    with pytest.raises(g.SvoError):
        ctx.set_trace_config(128, 3)


def test_tile_claim_order_gives_identical_hits(ctx):
    """Image tiles claimed row by row or centre-out (per image shape, ragged
    widths, 1-4 rays per lane, alone and as batch items of two shapes):
    every ray is traced exactly once with the same result."""
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=7)
    gs = GpuScene(ctx, fig.scene)
    gs.set_pose(fig.pose(9))
    assert ctx.tile_order() == g.TILE_ORDER_CENTER
    for w, h in ((333, 201), (640, 360), (7, 50)):
        rays = fig.rays(w, h)
        ctx.set_tile_order(g.TILE_ORDER_ROWS)
        ref = gs.trace(rays, g.TRACE_DEFAULT)
        for rpl in (1, 2, 4):
            ctx.set_trace_config(128, rpl)
            for order in (g.TILE_ORDER_ROWS, g.TILE_ORDER_CENTER):
                ctx.set_tile_order(order)
                _same(gs.trace(rays, g.TRACE_DEFAULT | g.trace_image(w)), ref)
    # batch items of two image shapes, each with its own table
    r1, r2 = fig.rays(320, 180), fig.rays(200, 150)
    ctx.set_tile_order(g.TILE_ORDER_ROWS)
    ctx.set_trace_config(128, 1)
    refs = [gs.trace(r, g.TRACE_DEFAULT) for r in (r1, r2)]
    ctx.set_tile_order(g.TILE_ORDER_CENTER)
    items = []
    for r, w in ((r1, 320), (r2, 200)):
        rt = torch.from_numpy(np.ascontiguousarray(r)).cuda()
        items.append((gs.sc, rt, torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda"),
                      torch.zeros(r.shape[0], dtype=torch.int32, device="cuda"), w))
    ctx.trace_batch(items, flags=g.TRACE_DEFAULT)
    torch.cuda.synchronize()
    for (_, _, h, f, _), ref in zip(items, refs):
        got = g.decode_hits(h)
        got["flags"] = f.cpu().numpy().astype(np.uint32)
        _same(got, ref)
    with pytest.raises(g.SvoError):
        ctx.set_tile_order(2)
    ctx.set_trace_config(128, 4)


def test_shared_memory_top_levels_give_identical_hits(ctx):
    """Staging the top octree levels of every part in shared memory (0-4
    levels; a depth-9 scene of 16 parts and PR1's four depth-6 parts; a batch
    of one scene too) changes only where node descriptors are read from."""
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=9)
    art = GpuScene(ctx, fig.scene)
    art.set_pose(fig.pose(12))
    pr1 = GpuScene(ctx, synthetic.pr1_scene())
    cases = [(art, fig.rays(400, 225), g.trace_image(400)), (pr1, synthetic.pr1_rays(pr1.scene), 0)]
    ctx.set_trace_config(128, 1)
    assert ctx.smem_levels() == 0
    for gs, rays, img in cases:
        ref = gs.trace(rays, g.TRACE_DEFAULT | img)
        assert (ref["part"] != 0xFFFFFFFF).sum() > 1000
        for levels in (1, 2, 3, 4):
            ctx.set_smem_levels(levels)
            _same(gs.trace(rays, g.TRACE_DEFAULT | img), ref)
            # a batch whose items all trace this scene stages the same levels
            r = torch.from_numpy(np.ascontiguousarray(rays)).cuda()
            h = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
            f = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
            ctx.trace_batch([(gs.sc, r[:5000], h[:5000], f[:5000]), (gs.sc, r[5000:], h[5000:], f[5000:])],
                            flags=g.TRACE_DEFAULT)
            torch.cuda.synchronize()
            got = g.decode_hits(h)
            got["flags"] = f.cpu().numpy().astype(np.uint32)
            _same(got, ref)
        ctx.set_smem_levels(0)
    with pytest.raises(g.SvoError):
        ctx.set_smem_levels(5)
    ctx.set_trace_config(128, 4)


def test_image_tiles_give_identical_hits(ctx):
    """Warp tiles of 8 x 4*rays_per_lane pixels (rays given as a row-major
    image) on ragged widths and a ragged last row, alone and per batch item:
    every ray is traced exactly once with the same result."""
    import torch

    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    rng = np.random.default_rng(9)
    rays = np.concatenate([synthetic.pr1_rays(s)[:11000], synthetic.random_rays(2117, rng, (-3,) * 3, (3,) * 3)])
    ctx.set_trace_config(128, 4)
    ref = gs.trace(rays, g.TRACE_DEFAULT)
    for width in (1, 7, 8, 13, 128, 333, 4096, 65535):
        for rpl in (1, 2, 8):
            ctx.set_trace_config(64, rpl)
            _same(gs.trace(rays, g.TRACE_DEFAULT | g.trace_image(width)), ref)
    # the ordering flags take precedence over the image layout
    _same(gs.trace(rays, g.TRACE_DEFAULT | g.TRACE_ORDER_DIR | g.trace_image(128)), ref)
    ctx.set_trace_config(128, 1)
    rt = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32)).cuda()
    items, outs = [], []
    for lo, hi, w in ((0, 5000, 100), (5000, 5001, 8), (5001, rays.shape[0], 0)):
        h = torch.empty((hi - lo, 2), dtype=torch.int64, device="cuda")
        f = torch.zeros(hi - lo, dtype=torch.int32, device="cuda")
        items.append((gs.sc, rt[lo:hi], h, f, w))
    ctx.trace_batch(items)
    torch.cuda.synchronize()
    got = {k: np.concatenate([g.decode_hits(it[2])[k] for it in items]) for k in ("t", "part", "voxel")}
    got["flags"] = np.concatenate([it[3].cpu().numpy().astype(np.uint32) for it in items])
    _same(got, ref)
    ctx.set_trace_config(128, 4)
    with pytest.raises(ValueError):
        g.trace_image(0)


def test_autotune_picks_a_valid_shape_and_caches_it(ctx, tmp_path):
    import torch

    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300 import autotune

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    rays = torch.from_numpy(synthetic.pr1_rays(s, 256, 256)).cuda()
    cache = str(tmp_path / "tune.json")
    cfg = autotune.tune(ctx, gs.sc, rays, reps=2, blocks=(64, 128), rays_per_lane=(2, 4), cache_path=cache,
                        key="pr1-256")
    assert cfg["block"] in (64, 128) and cfg["rays_per_lane"] in (2, 4) and cfg["order"] in autotune.ORDERS
    assert ctx.trace_config() == (cfg["block"], cfg["rays_per_lane"])
    assert len(cfg["table"]) == 2 * 2 * 3 * 2  # 3 orders, the cluster level in one launch or two
    assert autotune.load(cache)["pr1-256"]["block"] == cfg["block"]
    again = autotune.tune(ctx, gs.sc, rays, cache_path=cache, key="pr1-256")  # from the cache
    assert again["ms"] == cfg["ms"]
    ctx.set_trace_config(128, 4)
    assert g.TRACE_ORDER_DIR == autotune.ORDERS["dir"]


def test_frame_graph_replays_match_eager_frames(ctx):
    import torch

    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300.graphs import FrameGraph

    fig = synthetic.articulated_figure(depth=6)
    gs = GpuScene(ctx, fig.scene)
    rays_np = fig.rays(240, 135)
    rays = torch.from_numpy(rays_np).cuda()
    hits = torch.empty((rays.shape[0], 2), dtype=torch.int64, device="cuda")
    fg = FrameGraph(ctx, gs.sc, rays, hits, flags=g.TRACE_DEFAULT)
    for frame in (3, 19, 44):
        local = fig.pose(frame)
        fg.replay(local)
        torch.cuda.synchronize()
        got = g.decode_hits(hits)
        gs.set_pose(local)
        ref = gs.trace(rays_np, g.TRACE_DEFAULT)
        for k in ("t", "part", "voxel"):
            assert np.array_equal(got[k], ref[k]), (frame, k)
        assert (ref["part"] != 0xFFFFFFFF).sum() > 200


def test_host_buffers_equal_device_trace(ctx):
    """trace_rays_host pipelines chunks of rays through copy-in, trace and
    copy-out streams: hits and flags equal the device trace, with and without
    the image layout, pinned or pageable."""
    import torch

    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    rng = np.random.default_rng(12)
    n = 1_300_001  # three chunks and a ragged end
    rays = synthetic.random_rays(n, rng, (-3,) * 3, (3,) * 3)
    rays[: n // 2] = np.resize(synthetic.pr1_rays(s), (n // 2, 8))
    ctx.set_trace_config(128, 1)
    for flags in (g.TRACE_DEFAULT, g.TRACE_DEFAULT | g.trace_image(1000)):
        ref = gs.trace(rays, flags)
        for pinned in (True, False):  # mapped: kernels read/write host memory; pageable: staged chunks
            rh = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32))
            hh = torch.empty((n, 2), dtype=torch.int64)
            fh = torch.zeros(n, dtype=torch.int32)
            if pinned:
                rh, hh, fh = rh.pin_memory(), hh.pin_memory(), fh.pin_memory()
            gs.sc.trace_host(rh, hh, flags=flags, ray_flags_host=fh)
            torch.cuda.synchronize()
            got = g.decode_hits(hh)
            got["flags"] = fh.numpy().astype(np.uint32)
            _same(got, ref)
    # a small pinned batch is traced in place (zero copy)
    m = 100_003
    rh = torch.from_numpy(np.ascontiguousarray(rays[:m], dtype=np.float32)).pin_memory()
    hh = torch.empty((m, 2), dtype=torch.int64).pin_memory()
    gs.sc.trace_host(rh, hh, flags=g.TRACE_DEFAULT)
    torch.cuda.synchronize()
    got, ref = g.decode_hits(hh), gs.trace(rays[:m], g.TRACE_DEFAULT)
    assert np.array_equal(got["part"], ref["part"]) and np.array_equal(got["voxel"], ref["voxel"])
    hp = torch.empty((1000, 2), dtype=torch.int64)  # pageable
    gs.sc.trace_host(torch.from_numpy(np.ascontiguousarray(rays[:1000], dtype=np.float32)), hp)
    torch.cuda.synchronize()
    ref = gs.trace(rays[:1000], g.TRACE_DEFAULT)
    got = g.decode_hits(hp)
    assert np.array_equal(got["part"], ref["part"]) and np.array_equal(got["voxel"], ref["voxel"])
    with pytest.raises(g.SvoError):
        gs.sc.trace_host(torch.zeros((8, 8)), torch.zeros((8, 2), dtype=torch.int64), flags=g.TRACE_DEFAULT | g.TRACE_REUSE)
    ctx.set_trace_config(128, 4)


def test_host_frame_loop_overlaps_calls(ctx):
    """trace_rays_host in a frame loop with no synchronisation between frames:
    each call's copy-in may run while the previous frame is still traced
    (two staging halves).  Every frame, with its own poses, rays and hits,
    must equal the device trace of that frame."""
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=7)
    gs = GpuScene(ctx, fig.scene)
    w, h = 640, 480  # 307,200 rays: above the zero-copy limit, one chunk
    rng = np.random.default_rng(13)
    ray_sets = [fig.rays(w, h), synthetic.random_rays(w * h, rng, (-2,) * 3, (2,) * 3)]
    host_rays = [torch.from_numpy(np.ascontiguousarray(r)).pin_memory() for r in ray_sets]
    frames = [(f, f % 2) for f in range(0, 50, 7)]
    hits = [torch.empty((w * h, 2), dtype=torch.int64).pin_memory() for _ in frames]
    flags = g.TRACE_DEFAULT
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()
    for (f, k), hh in zip(frames, hits):
        gs.sc.set_transforms(fig.pose(f), stream=stream)
        gs.sc.refit(stream=stream)
        gs.sc.trace_host(host_rays[k], hh, flags=flags, stream=stream)
    stream.synchronize()
    for (f, k), hh in zip(frames, hits):
        gs.set_pose(fig.pose(f))
        ref = gs.trace(ray_sets[k], flags)
        got = g.decode_hits(hh)
        for key in ("t", "part", "voxel"):
            assert np.array_equal(got[key], ref[key]), (f, key)


def _small_batch(ctx):
    import torch

    bat = synthetic.batched_scenes(seed=5, n_scenes=6, parts=(4, 80), depths=range(6, 9), side=(48, 128),
                                   per_depth=2)
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in bat.pool]
    items = []
    for s, r in zip(bat.scenes, bat.rays):
        sc = ctx.scene([handles[int(a)] for a in s.part_asset], s.parent)
        sc.set_transforms(s.local)
        sc.refit()
        items.append((sc, torch.from_numpy(r).cuda(), torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda"),
                      torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")))
    return bat, items


@pytest.mark.parametrize("wavefront", [False, True])
def test_batch_graph_replays_match_eager_batches(ctx, wavefront):
    """A batched frame (one pose copy, every scene refitted by one batched
    launch, ordering, the persistent trace and the FP64 pass) replayed from
    one CUDA graph gives bit-identical hits and flags to the eager
    trace_batch of the same poses, over several pose sets."""
    import torch

    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300.graphs import BatchGraph

    bat, items = _small_batch(ctx)
    rng = np.random.default_rng(3)
    flags = g.TRACE_DEFAULT | (g.TRACE_WAVEFRONT if wavefront else g.TRACE_ORDER_ORIGIN)
    graph_items = [(sc, r, torch.empty_like(h), torch.zeros_like(f)) for sc, r, h, f in items]
    bg = BatchGraph(ctx, graph_items, [s.local for s in bat.scenes], flags=flags)
    for rep in range(3):
        local = []
        for s in bat.scenes:  # every root re-posed: a small rigid motion of each scene
            L = s.local.copy()
            for i in np.nonzero(s.parent < 0)[0]:
                A = synthetic.euler_xyz(*rng.uniform(-0.2, 0.2, 3))
                M = L[i].reshape(3, 4)
                L[i] = np.hstack([A @ M[:, :3], (A @ M[:, 3] + rng.uniform(-0.3, 0.3, 3))[:, None]]).ravel()
            local.append(L)
        bg.replay(local)
        torch.cuda.current_stream().wait_stream(bg.stream)  # the eager frame below re-poses the same scenes
        for (sc, _, _, _), L in zip(items, local):
            sc.set_transforms(L)
            sc.refit()
        ctx.trace_batch(items, flags=flags)
        torch.cuda.synchronize()
        hits = 0
        for (_, _, h_ref, f_ref), (_, _, h_g, f_g) in zip(items, graph_items):
            assert torch.equal(h_ref, h_g) and torch.equal(f_ref, f_g), rep
            hits += int((g.decode_hits(h_ref)["part"] != 0xFFFFFFFF).sum())
        # the oracle hits 1660 / 1612 / 1569 of these 33838 seeded rays over the
        # three pose sets; the floor is 90% of the smallest
        assert hits >= 1412


def test_tune_batch_picks_and_caches(ctx, tmp_path):
    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300 import autotune

    _, items = _small_batch(ctx)
    cache = str(tmp_path / "tune.json")
    cfg = autotune.tune_batch(ctx, items, reps=1, blocks=(128,), rays_per_lane=(1, 2), orders=("none", "origin"),
                              cache_path=cache)
    # one launch or two (wavefront), and the grid when some scene is large enough for one
    culls = 3 if any(it[0].n_parts >= autotune.GRID_MIN_PARTS for it in items) else 2
    assert cfg["key"] == autotune.batch_key(items) and len(cfg["table"]) == 2 * 2 * culls
    assert ctx.trace_config() == (cfg["block"], cfg["rays_per_lane"])
    assert autotune.tune_batch(ctx, items, cache_path=cache)["ms"] == cfg["ms"]
    ctx.set_trace_config(128, 4)
    assert g.TRACE_GRID == autotune.CULLS["grid"]
