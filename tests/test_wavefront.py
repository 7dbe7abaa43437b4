"""SVO_TRACE_WAVEFRONT: the trace as a culling launch (every ray's first
culling pass; misses written, the others queued with their candidate parts)
plus a descent launch over the queued rays.  A launch shape only: hits, ray
flags and counters must be bit-identical to the single fused launch, and the
hits must match the FP64 oracle element by element."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import synthetic
from gpu_helpers import GpuScene, compare

pytestmark = pytest.mark.gpu

COUNTERS = ("rays", "flagged", "parts_tested", "parts_entered", "nodes_visited", "leaves_tested", "passes",
            "flag_winner", "flag_overlap", "flag_width", "fixed")


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


def _counted(gs, rays, flags):
    import torch

    import paper_1911_06001_gb300 as g

    r = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32)).cuda()
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    st = g.new_stats("cuda")
    hits = gs.sc.trace(r, flags=flags | g.TRACE_STATS, ray_flags=rf, stats=st)
    torch.cuda.synchronize()
    out = g.decode_hits(hits)
    out["flags"] = rf.cpu().numpy().astype(np.uint32)
    return out, g.read_stats(st)


def test_wavefront_matches_fused_and_oracle_on_one_scene(ctx):
    """PR1 scene: pinhole rays, incoherent rays and edge rays (empty segment,
    NaN, zero direction) in one call of 2^14 + 1013 rays (a ragged last warp),
    at every block size and 1-4 rays per lane; the counters of the two launch
    shapes agree too."""
    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    rng = np.random.default_rng(11)
    rays = np.concatenate([synthetic.pr1_rays(s)[:12000],
                           synthetic.random_rays(4000 + 1013 - 16, rng, (-3,) * 3, (3,) * 3)]).astype(np.float32)
    rays[100, 3], rays[100, 7] = 5.0, 1.0        # tmin > tmax: not a ray
    rays[101, :] = np.nan                         # not a ray
    rays[102, 4:7] = 0.0                          # no direction: not a ray
    rays[103, 4:7] = (0.0, 0.0, 1.0)              # axis-parallel
    fused, c1 = _counted(gs, rays, g.TRACE_DEFAULT)
    wave, c2 = _counted(gs, rays, g.TRACE_DEFAULT | g.TRACE_WAVEFRONT)
    _same(wave, fused)
    for k in COUNTERS:
        assert c1[k] == c2[k], k
    ora = oracle.SceneOracle(s).trace(rays)
    rep = compare(s, s.local, rays, wave, ora)  # every ray, element by element
    assert rep["hits"] > 1000  # the comparison is not vacuous
    for block in (64, 128, 256):
        for rpl in (1, 2, 4):
            ctx.set_trace_config(block, rpl)
            _same(gs.trace(rays, g.TRACE_DEFAULT | g.TRACE_WAVEFRONT | g.TRACE_ORDER_ORIGIN), fused)
    ctx.set_trace_config(128, 1)


def test_wavefront_on_image_tiles_of_the_articulated_figure(ctx):
    """A 640x360 frame of the articulated figure (depth 7 parts), rays as
    image tiles: identical to the fused launch, every ray against the oracle."""
    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=7)
    gs = GpuScene(ctx, fig.scene)
    local = fig.pose(29)
    gs.set_pose(local)
    rays = fig.rays(640, 360)
    flags = g.TRACE_DEFAULT | g.trace_image(640)
    fused, c1 = _counted(gs, rays, flags)
    wave, c2 = _counted(gs, rays, flags | g.TRACE_WAVEFRONT)
    _same(wave, fused)
    for k in COUNTERS:
        assert c1[k] == c2[k], k
    ora = oracle.SceneOracle(fig.scene).trace(rays, local)
    rep = compare(fig.scene, local, rays, wave, ora)
    assert rep["hits"] > 2000


def test_wavefront_batch_matches_fused_and_oracle(ctx):
    """Uneven scenes in one batch (each item has its own queue region): hits
    and flags identical to the fused batch, each item against the oracle; and
    the same again in a second call whose queue still holds the first's."""
    import torch

    import paper_1911_06001_gb300 as g

    bat = synthetic.batched_scenes(seed=5, n_scenes=8, parts=(4, 48), depths=range(6, 9), side=(48, 128),
                                   per_depth=2)
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in bat.pool]
    oassets = [oracle.OracleAsset(p.asset.depth, p.asset.leaf_ids) for p in bat.pool]
    scenes = []
    for s in bat.scenes:
        sc = ctx.scene([handles[int(a)] for a in s.part_asset], s.parent)
        sc.set_transforms(s.local)
        sc.refit()
        scenes.append(sc)
    rays = [torch.from_numpy(r).cuda() for r in bat.rays]

    def run(flags):
        hits = [torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda") for r in rays]
        rfs = [torch.zeros(r.shape[0], dtype=torch.int32, device="cuda") for r in rays]
        ctx.trace_batch([(sc, r, h, f) for sc, r, h, f in zip(scenes, rays, hits, rfs)], flags=flags)
        torch.cuda.synchronize()
        outs = []
        for h, f in zip(hits, rfs):
            d = g.decode_hits(h)
            d["flags"] = f.cpu().numpy().astype(np.uint32)
            outs.append(d)
        return outs

    fused = run(g.TRACE_DEFAULT)
    for flags in (g.TRACE_DEFAULT | g.TRACE_WAVEFRONT, g.TRACE_DEFAULT | g.TRACE_WAVEFRONT | g.TRACE_ORDER_ORIGIN):
        wave = run(flags)
        for a, b in zip(wave, fused):
            _same(a, b)
    hits = 0
    for s, r, res in zip(bat.scenes, bat.rays, wave):
        inv = oracle.invert(oracle.compose(s.parent, s.local))
        ora = oracle.trace([oassets[int(a)] for a in s.part_asset], inv, r)
        rep = compare(s, s.local, r, res, ora)
        hits += rep["hits"]
    assert hits > 2000
    for sc in scenes:
        sc.close()


def test_wavefront_flag_combinations(ctx):
    """WAVEFRONT needs CULL | SORT and excludes REUSE and GRID; the call that
    asks otherwise fails with SVO_ERR_ARG before any device work."""
    import torch

    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    gs = GpuScene(ctx, s)
    r = torch.from_numpy(synthetic.pr1_rays(s, 32, 32)).cuda()
    for bad in (g.TRACE_WAVEFRONT, g.TRACE_CULL | g.TRACE_WAVEFRONT, g.TRACE_DEFAULT | g.TRACE_WAVEFRONT | g.TRACE_REUSE,
                g.TRACE_DEFAULT | g.TRACE_WAVEFRONT | g.TRACE_GRID):
        with pytest.raises(g.SvoError):
            gs.sc.trace(r, flags=bad)
    gs.sc.trace(r, flags=g.TRACE_DEFAULT | g.TRACE_WAVEFRONT)
    torch.cuda.synchronize()
    # the entry point that allocates nothing has no queue: it refuses the shape
    import ctypes as C

    import paper_1911_06001_gb300._lib as L

    lib = L.load()
    h = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
    rc = lib.trace_rays_noalloc(gs.sc.h, C.c_void_p(r.data_ptr()), r.shape[0], C.c_void_p(h.data_ptr()), None,
                                g.TRACE_DEFAULT | g.TRACE_WAVEFRONT, None)
    assert rc == -1 and b"WAVEFRONT" in lib.svo_last_error()
    ctx.check_device()
