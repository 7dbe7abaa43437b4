"""Hit buffer reuse (Sec. IV-C, Fig. 5) on the GPU: with a static camera, a
ray whose only intersected part sphere belongs to the part it hit in the
previous frame, and whose part has not moved since, keeps its previous hit.
The reused frames must still equal the FP64 oracle of the new poses."""

from __future__ import annotations

import numpy as np
import pytest

import oracle
import synthetic
from gpu_helpers import compare

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


def _decode(g, hits, rf):
    d = g.decode_hits(hits)
    d["flags"] = rf.cpu().numpy().astype(np.uint32)
    return d


def test_reuse_keeps_unmoved_hits_and_matches_oracle(ctx):
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=7)
    scene = fig.scene
    so = oracle.SceneOracle(scene)
    handles = [ctx.upload(a.depth, a.leaf_ids, a.rgb) for a in scene.assets]
    sc = ctx.scene(handles, scene.parent)
    rays_np = fig.rays(480, 270)
    rays = torch.from_numpy(rays_np).cuda()
    n = rays.shape[0]
    hits = torch.empty((n, 2), dtype=torch.int64, device="cuda")
    rf = torch.zeros(n, dtype=torch.int32, device="cuda")
    flags = g.TRACE_DEFAULT | g.TRACE_REUSE

    pose0 = fig.pose(0)
    sc.set_transforms(pose0)
    sc.refit()
    sc.trace(rays, hits, flags=g.TRACE_DEFAULT, ray_flags=rf)
    # frame 1: only the end parts 13 and 15 move (leaves of the transform tree)
    pose1 = pose0.copy()
    later = fig.pose(20)
    for p in (13, 15):
        pose1[p] = later[p]
    sc.set_transforms(pose1)
    sc.refit()
    st = g.new_stats()
    sc.trace(rays, hits, flags=flags | g.TRACE_STATS, ray_flags=rf, stats=st)
    torch.cuda.synchronize()
    s = g.read_stats(st)
    got = _decode(g, hits, rf)
    rep = compare(scene, pose1, rays_np, got, so.trace(rays_np, local=pose1))
    reused = (got["flags"] & g.RAY_REUSED) != 0
    assert s["reused"] == int(reused.sum())
    assert 0.02 * rep["hits"] < s["reused"] < n
    # reused rays carry exactly the hit a fresh trace of the same frame finds
    fresh = torch.empty_like(hits)
    rf2 = torch.zeros_like(rf)
    sc.trace(rays, fresh, flags=g.TRACE_DEFAULT, ray_flags=rf2)
    f2 = _decode(g, fresh, rf2)
    same = reused & ((f2["flags"] & g.RAY_UNCERTAIN) == 0)
    assert np.array_equal(got["part"][same], f2["part"][same])
    assert np.array_equal(got["voxel"][same], f2["voxel"][same])

    # frame 2: a root translation moves every part -> nothing is reused
    pose2 = fig.pose(40)
    pose2[0] = pose2[0].copy()
    pose2[0][[3, 7, 11]] += (0.01, -0.02, 0.015)
    sc.set_transforms(pose2)
    sc.refit()
    st = g.new_stats()
    sc.trace(rays, hits, flags=flags | g.TRACE_STATS, ray_flags=rf, stats=st)
    torch.cuda.synchronize()
    assert g.read_stats(st)["reused"] == 0
    compare(scene, pose2, rays_np, _decode(g, hits, rf), so.trace(rays_np, local=pose2))

    # frame 3: two refits before the trace; the first one's change must not be forgotten
    pose3a = pose2.copy()
    pose3a[13] = fig.pose(50)[13]
    sc.set_transforms(pose3a)
    sc.refit()
    pose3b = pose3a.copy()
    pose3b[15] = fig.pose(50)[15]
    sc.set_transforms(pose3b)
    sc.refit()
    sc.trace(rays, hits, flags=flags, ray_flags=rf)
    torch.cuda.synchronize()
    got3 = _decode(g, hits, rf)
    compare(scene, pose3b, rays_np, got3, so.trace(rays_np, local=pose3b))
    assert ((got3["flags"] & g.RAY_REUSED) != 0).sum() > 0

    # reuse composes with the ray order and the image layout (hits stay at each ray's own index)
    for extra in (g.TRACE_ORDER_ORIGIN, g.trace_image(480)):
        pose4 = pose3b.copy()
        pose4[14] = fig.pose(60)[14]
        sc.set_transforms(pose3b)
        sc.refit()
        sc.trace(rays, hits, flags=g.TRACE_DEFAULT | extra, ray_flags=rf)
        sc.set_transforms(pose4)
        sc.refit()
        sc.trace(rays, hits, flags=flags | extra, ray_flags=rf)
        torch.cuda.synchronize()
        got4 = _decode(g, hits, rf)
        compare(scene, pose4, rays_np, got4, so.trace(rays_np, local=pose4))
        assert ((got4["flags"] & g.RAY_REUSED) != 0).sum() > 0

    with pytest.raises(g.SvoError):
        sc.trace(rays, hits, flags=g.TRACE_CULL | g.TRACE_FP64_FIX | g.TRACE_REUSE)
    sc.close()
    for h in handles:
        ctx.release(h)
