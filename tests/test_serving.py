"""Continuous-batching server: results equal the same request rendered alone;
admission by memory; queued requests complete once memory frees up."""

from __future__ import annotations

import numpy as np
import pytest

import synthetic
from gpu_helpers import TOL_T

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def world_ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1911_06001_gb300 as g

    ctx = g.Context(0)
    world = synthetic.serving_world(seed=77, n_scenes=4, parts=(12, 40), depths=range(6, 9), per_depth=2)
    pool_h = [ctx.upload(p.asset.depth, p.asset.leaf_ids, p.asset.rgb) for p in world.pool]
    scenes = [([pool_h[int(a)] for a in s.scene.part_asset], s.scene.parent) for s in world.scenes]
    yield ctx, world, scenes
    ctx.check_device()
    ctx.close()


def _decode(h):
    import paper_1911_06001_gb300 as g

    return g.decode_hits(h)


def test_served_results_equal_rendered_alone(world_ctx):
    import torch

    from paper_1911_06001_gb300.serving import Server, render_alone

    ctx, world, scenes = world_ctx
    server = Server(ctx, scenes, n_slots=3, max_batch_rays=1 << 19, instances_per_scene=2)
    reqs = world.requests(48, rate=4000.0, seed=5, resolutions=((64, 64), (128, 96), (200, 150)))
    got = {}

    def keep(t):
        got[id(t.request)] = t.hits.cpu().numpy().copy()

    tickets = server.run(reqs, on_done=keep)
    assert len(tickets) == len(reqs) and all(t.done >= t.arrival for t in tickets)
    # several requests must have shared a batch or overlapped in time (not a queue of singles)
    assert max(len([u for u in tickets if u.submitted == t.submitted]) for t in tickets) > 1 or \
        any(a.submitted < b.done and b.submitted < a.done and a.slot != b.slot for a in tickets for b in tickets)
    alone = [ctx.scene(h, p) for h, p in scenes]
    hits_total = 0
    for r in reqs:
        _, h = render_alone(ctx, alone[r.scene], r)
        torch.cuda.synchronize()
        ref = _decode(h)
        res = _decode(got[id(r)])
        assert np.array_equal(res["part"], ref["part"])
        assert np.array_equal(res["voxel"], ref["voxel"])
        hit = ref["part"] != 0xFFFFFFFF
        hits_total += int(hit.sum())
        ta, tb = res["t"].astype(np.float64), ref["t"].astype(np.float64)
        assert np.all(np.abs(ta[hit] - tb[hit]) <= TOL_T * np.abs(tb[hit]))
    assert hits_total > 1000


def test_admission_by_memory(world_ctx):
    from paper_1911_06001_gb300.serving import HIT_BYTES, RAY_BYTES, SCRATCH_BYTES_PER_RAY, AdmissionError, Server

    ctx, world, scenes = world_ctx
    per_ray = RAY_BYTES + HIT_BYTES + SCRATCH_BYTES_PER_RAY
    # a budget of 32768 rays: one 160x160 request (25600 rays) at a time
    small = Server(ctx, scenes, n_slots=2, max_batch_rays=1 << 16, memory_budget=(1 << 15) * per_ray,
                   instances_per_scene=1)
    big = world.requests(1, 100.0, seed=9, resolutions=((512, 512),))[0]
    with pytest.raises(AdmissionError):
        small.submit(big)
    # requests that fit only one at a time still all complete (they queue for memory)
    reqs = world.requests(10, rate=1e6, seed=10, resolutions=((160, 160),))
    tickets = small.run(reqs)
    assert len(tickets) == 10 and all(t.done > 0 for t in tickets)
    starts = sorted(t.submitted for t in tickets)
    dones = sorted(t.done for t in tickets)
    # never two in flight at once: each launch happens after the previous completion
    assert all(starts[i + 1] >= dones[i] - 1e-9 for i in range(len(starts) - 1))


def test_requests_time_out_in_the_queue(world_ctx):
    """With a maximum queue wait, requests that cannot start in time end with
    status "timeout" and never reach the GPU; the others complete normally."""
    from paper_1911_06001_gb300.serving import HIT_BYTES, RAY_BYTES, SCRATCH_BYTES_PER_RAY, Server

    ctx, world, scenes = world_ctx
    per_ray = RAY_BYTES + HIT_BYTES + SCRATCH_BYTES_PER_RAY
    srv = Server(ctx, scenes, n_slots=1, max_batch_rays=1 << 16, memory_budget=(1 << 16) * per_ray,
                 instances_per_scene=1, max_wait=0.0)
    reqs = world.requests(40, rate=1e7, seed=11, resolutions=((200, 200),))
    tickets = srv.run(reqs)
    status = [t.status for t in tickets]
    assert set(status) <= {"done", "timeout"}
    assert "done" in status and "timeout" in status
    assert all(t.hits is None and t.slot == -1 for t in tickets if t.status == "timeout")
    assert all(t.done >= t.arrival for t in tickets)
