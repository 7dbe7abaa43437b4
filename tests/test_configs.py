"""Parity on the batched and precision-stress workloads.

Batched: many uneven scenes over a shared asset pool, affine poses with shear,
incoherent rays, all traced in one persistent launch.  Precision stress:
depth-13 assets at the ends of five-level rigid chains with translations of
up to 10^4 leaf sizes, with rays that graze leaf faces at < 1e-3 rad.
"""

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


def _batched_trace(ctx, bat, handles, flags):
    import torch

    import paper_1911_06001_gb300 as g

    scenes, items, outs = [], [], []
    for s, r in zip(bat.scenes, bat.rays):
        sc = ctx.scene([handles[int(a)] for a in s.part_asset], s.parent)
        sc.set_transforms(s.local)
        sc.refit()
        rt = torch.from_numpy(r).cuda()
        ht = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
        ft = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
        scenes.append(sc)
        items.append((sc, rt, ht, ft))
    ctx.trace_batch(items, flags=flags)
    torch.cuda.synchronize()
    for sc, rt, ht, ft in items:
        d = g.decode_hits(ht)
        d["flags"] = ft.cpu().numpy().astype(np.uint32)
        outs.append(d)
    return scenes, outs


def test_batched_reduced_parity(ctx):
    import paper_1911_06001_gb300 as g

    bat = synthetic.batched_scenes(seed=5, n_scenes=8, parts=(4, 48), depths=range(6, 9), side=(48, 128),
                                   per_depth=2)
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in bat.pool]
    oassets = [oracle.OracleAsset(p.asset.depth, p.asset.leaf_ids) for p in bat.pool]
    _, outs = _batched_trace(ctx, bat, handles, g.TRACE_DEFAULT | g.TRACE_ORDER_ORIGIN)
    hits = 0
    for s, r, res in zip(bat.scenes, bat.rays, outs):
        inv = oracle.invert(oracle.compose(s.parent, s.local))
        ora = oracle.trace([oassets[int(a)] for a in s.part_asset], inv, r)
        rep = compare(s, s.local, r, res, ora)
        hits += rep["hits"]
    assert hits > 2000


def test_batched_full_size_sampled(ctx):
    """The batched workload at full size (64 scenes, ~10^7 rays, depths 6-11) in
    one persistent launch; the oracle checks 400 random rays of every scene."""
    import paper_1911_06001_gb300 as g

    bat = synthetic.batched_scenes()
    handles = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in bat.pool]
    oassets = [oracle.OracleAsset(p.asset.depth, p.asset.leaf_ids) for p in bat.pool]
    _, outs = _batched_trace(ctx, bat, handles, g.TRACE_DEFAULT | g.TRACE_ORDER_ORIGIN)
    rng = np.random.default_rng(17)
    hits = flagged = total = 0
    for s, r, res in zip(bat.scenes, bat.rays, outs):
        idx = rng.choice(r.shape[0], min(400, r.shape[0]), replace=False)
        inv = oracle.invert(oracle.compose(s.parent, s.local))
        ora = oracle.trace([oassets[int(a)] for a in s.part_asset], inv, r[idx])
        rep = compare(s, s.local, r[idx], {k: v[idx] for k, v in res.items()}, ora)
        hits += rep["hits"]
        flagged += rep["flagged"]
        total += rep["rays"]
    print("BAT full sampled: rays", total, "hits", hits, "flagged", flagged)
    assert total == 64 * 400 and hits > 1000


def test_precision_stress(ctx):
    """Depth-13 parts behind five-level chains, 2^20 rays of which 30% graze
    leaf faces.  Unflagged rays must match the oracle exactly; flagged ones
    are re-intersected in FP64 and must match too."""
    import torch

    import paper_1911_06001_gb300 as g
    from gpu_helpers import GpuScene

    prec = synthetic.precision_scene()
    scene = prec.scene
    gs = GpuScene(ctx, scene)
    world = oracle.compose(scene.parent, scene.local)
    got = gs.sc.read_poses()
    assert np.allclose(got["world"], world, rtol=0, atol=1e-12 * max(1.0, np.abs(world).max()))
    n_total = 1 << 20
    rays, n_prim = synthetic.precision_rays(prec, world, n_total)
    prim = rays[:n_prim]
    ora = oracle.SceneOracle(scene).trace(rays)
    res = gs.trace(rays, g.TRACE_DEFAULT)
    rep = compare(scene, scene.local, rays, res, ora)
    g_flag = ((res["flags"][len(prim):] & 1) != 0).mean()
    print("PREC", rep, "grazing flagged fraction", float(g_flag))
    assert rep["hits"] > 0.5 * n_total
    assert rep["flagged_id_mismatch"] == 0
