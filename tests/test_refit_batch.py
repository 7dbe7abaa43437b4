"""scene_refit_batch: many scenes composed, inverted and refitted in one
launch (a thread block per scene).  Every scene's result -- world and
inverse poses, FP32 rows, spheres, clusters, part order, change flags as
seen by hit buffer reuse -- must be bit-identical to scene_refit of the same
poses, whichever way the poses arrive (host poses of small scenes, device
poses, staged poses of a scene above 256 parts)."""

from __future__ import annotations

import numpy as np
import pytest

import synthetic

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


def _scenes(ctx, rng):
    """(scene spec, [handle pairs]) of 12 uneven scenes: trees and flat sets of
    4-300 parts (one above the 256-part inline-pose limit)."""
    pool = synthetic.asset_pool(range(4, 7), 2, seed=5)
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in pool]
    specs = []
    for P in (4, 7, 16, 33, 64, 5, 128, 300, 9, 21, 50, 2):
        parent = np.array([-1] + [int(rng.integers(0, i)) if rng.random() < 0.7 else -1 for i in range(1, P)],
                          dtype=np.int32)
        assets = rng.integers(0, len(pool), P)
        specs.append((parent, assets))
    return handles, specs


def _poses(rng, parent):
    local = []
    for _ in range(len(parent)):
        A = synthetic.euler_xyz(*rng.uniform(-np.pi, np.pi, 3)) @ np.diag(rng.uniform(0.5, 2.0, 3))
        local.append(synthetic.affine12(A, rng.uniform(-3.0, 3.0, 3)))
    return np.array(local)


def _state(sc):
    p = sc.read_poses()
    c = sc.read_clusters()
    return {**p, **{"cl_" + k: v for k, v in c.items()}}


def _equal(a, b):
    for k in a:
        assert np.array_equal(a[k].view(np.uint8), b[k].view(np.uint8)), k


def test_refit_batch_equals_single_refits(ctx):
    import torch

    rng = np.random.default_rng(41)
    handles, specs = _scenes(ctx, rng)
    single = [ctx.scene([handles[int(a)] for a in assets], parent) for parent, assets in specs]
    batched = [ctx.scene([handles[int(a)] for a in assets], parent) for parent, assets in specs]
    for rnd in range(3):  # repeated rounds reuse the staging buffers and the change flags
        poses = [_poses(rng, parent) for parent, _ in specs]
        for sc, L in zip(single, poses):
            sc.set_transforms(L)
            sc.refit()
        # half the scenes get host poses, half device poses
        dev = []
        for k, (sc, L) in enumerate(zip(batched, poses)):
            if (k + rnd) % 2 == 0:  # every scene takes both paths over the rounds
                sc.set_transforms(L)
                dev.append(None)
            else:
                dev.append(torch.from_numpy(np.ascontiguousarray(L)).cuda())
        ctx.refit_batch(batched, dev)
        torch.cuda.synchronize()
        for a, b in zip(single, batched):
            _equal(_state(a), _state(b))
        ctx.check_device()
    # scenes whose poses did not change keep them (no new poses given)
    ctx.refit_batch(batched)
    torch.cuda.synchronize()
    for a, b in zip(single, batched):
        _equal(_state(a), _state(b))
    for sc in single + batched:
        sc.close()


def test_refit_batch_then_trace_equals_single(ctx):
    """Traces after a batched refit equal those after single refits, and hit
    buffer reuse sees the same changed parts."""
    import torch

    import paper_1911_06001_gb300 as g

    fig = synthetic.articulated_figure(depth=6)
    hs = [ctx.upload(a.depth, a.leaf_ids, a.rgb) for a in fig.scene.assets]
    a = ctx.scene([hs[int(i)] for i in fig.scene.part_asset], fig.scene.parent)
    b = ctx.scene([hs[int(i)] for i in fig.scene.part_asset], fig.scene.parent)
    rays = torch.from_numpy(fig.rays(320, 240)).cuda()
    flags = g.TRACE_DEFAULT | g.TRACE_REUSE
    ha = torch.empty((rays.shape[0], 2), dtype=torch.int64, device="cuda")
    hb = torch.empty_like(ha)
    fa = torch.zeros(rays.shape[0], dtype=torch.int32, device="cuda")
    fb = torch.zeros_like(fa)
    base = fig.pose(0)
    for f in range(4):
        L = base.copy()
        if f > 0:  # parts 13-15 move, the rest keep their poses
            L[13:] = fig.pose(5 * f)[13:]
        a.set_transforms(L)
        a.refit()
        b.set_transforms(L)
        ctx.refit_batch([b])
        a.trace(rays, ha, flags=flags if f > 0 else g.TRACE_DEFAULT, ray_flags=fa)
        b.trace(rays, hb, flags=flags if f > 0 else g.TRACE_DEFAULT, ray_flags=fb)
        torch.cuda.synchronize()
        assert torch.equal(ha, hb) and torch.equal(fa, fb), f
        if f > 0:
            assert int(((fb.cpu().numpy() & g.RAY_REUSED) != 0).sum()) > 0
    a.close()
    b.close()


def test_refit_batch_rejects_bad_lists(ctx):
    import paper_1911_06001_gb300 as g

    s = synthetic.pr1_scene()
    hs = [ctx.upload(a.depth, a.leaf_ids, a.rgb) for a in s.assets]
    sc = ctx.scene([hs[int(i)] for i in s.part_asset], s.parent)
    sc.set_transforms(s.local)
    with pytest.raises(g.SvoError):
        ctx.refit_batch([sc, sc])  # the same scene twice
    ctx.refit_batch([])  # nothing to do
    ctx.refit_batch([sc])
    ctx.check_device()
    sc.close()


def test_refit_batch_more_scenes_than_one_launch_takes(ctx):
    """70 scenes: two launches (64 + 6), each scene as scene_refit leaves it."""
    import torch

    rng = np.random.default_rng(7)
    pool = synthetic.asset_pool(range(4, 6), 2, seed=9)
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in pool]
    single, batched = [], []
    for k in range(70):
        P = int(rng.integers(1, 12))
        parent = np.array([-1] + [int(rng.integers(0, i)) for i in range(1, P)], dtype=np.int32)
        assets = [handles[int(a)] for a in rng.integers(0, len(handles), P)]
        L = _poses(rng, parent)
        a = ctx.scene(assets, parent)
        b = ctx.scene(assets, parent)
        a.set_transforms(L)
        a.refit()
        b.set_transforms(L)
        single.append(a)
        batched.append(b)
    ctx.refit_batch(batched)
    torch.cuda.synchronize()
    for a, b in zip(single, batched):
        _equal(_state(a), _state(b))
    for sc in single + batched:
        sc.close()
