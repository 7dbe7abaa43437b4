"""trace_rays_noalloc: the trace for callers that cannot allocate device memory.

Some callers must not trigger cudaMalloc: a frame loop with a hard deadline
(an allocation may synchronise the whole device) or an application whose own
allocator owns all device memory.  trace_rays_noalloc gives them the same
trace with its scratch in a fixed static device array.  Here it is called
through the C ABI twice in a row -- the second call reuses the scratch the
first one left behind -- and each result must equal trace_rays' on the same
inputs within the parity tolerance the other GPU tests use.
"""

from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import synthetic
from gpu_helpers import TOL_T, GpuScene

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


def _noalloc(lib, scene, rays_np, flags):
    import torch

    import paper_1911_06001_gb300 as g

    r = torch.from_numpy(np.ascontiguousarray(rays_np, dtype=np.float32)).cuda()
    hits = torch.empty((r.shape[0], 2), dtype=torch.int64, device="cuda")
    rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
    stream = C.c_void_p(int(torch.cuda.current_stream().cuda_stream))
    rc = lib.trace_rays_noalloc(scene.sc.h, C.c_void_p(r.data_ptr()), r.shape[0], C.c_void_p(hits.data_ptr()),
                                C.c_void_p(rf.data_ptr()), flags, stream)
    assert rc == 0, lib.svo_last_error()
    torch.cuda.synchronize()
    out = g.decode_hits(hits)
    out["flags"] = rf.cpu().numpy().astype(np.uint32)
    return out


def _same(a, b):
    assert np.array_equal(a["part"], b["part"])
    assert np.array_equal(a["voxel"], b["voxel"])
    assert np.array_equal(a["flags"], b["flags"])
    hit = b["part"] != 0xFFFFFFFF
    ta, tb = a["t"].astype(np.float64), b["t"].astype(np.float64)
    assert np.all(np.abs(ta[hit] - tb[hit]) <= TOL_T * np.abs(tb[hit]))
    assert np.all(np.isinf(ta[~hit]))


def test_noalloc_matches_trace_rays_on_two_calls(ctx):
    import paper_1911_06001_gb300._lib as L

    lib = L.load()
    pr1 = synthetic.pr1_scene()
    fig = synthetic.articulated_figure(depth=7)
    s1 = GpuScene(ctx, pr1)
    s2 = GpuScene(ctx, fig.scene)
    s2.set_pose(fig.pose(23))
    r1 = synthetic.pr1_rays(pr1)[: 16384 - 77]
    r2 = fig.rays(320, 180)
    flags = L.TRACE_DEFAULT
    first = _noalloc(lib, s1, r1, flags)
    second = _noalloc(lib, s2, r2, flags)
    _same(first, s1.trace(r1, flags))
    _same(second, s2.trace(r2, flags))
    assert (first["part"] != 0xFFFFFFFF).sum() > 1000
    assert (second["part"] != 0xFFFFFFFF).sum() > 2000


def test_noalloc_rejects_oversized_batches(ctx):
    import torch

    import paper_1911_06001_gb300._lib as L

    lib = L.load()
    pr1 = synthetic.pr1_scene()
    s1 = GpuScene(ctx, pr1)
    r = torch.zeros((16, 8), dtype=torch.float32, device="cuda")
    h = torch.zeros((16, 2), dtype=torch.int64, device="cuda")
    # the size check comes before any device work, so the small buffers are never read
    rc = lib.trace_rays_noalloc(s1.sc.h, C.c_void_p(r.data_ptr()), L.NOALLOC_MAX_RAYS + 1, C.c_void_p(h.data_ptr()),
                                None, L.TRACE_DEFAULT, None)
    assert rc == -9
    assert b"limit" in lib.svo_last_error()
