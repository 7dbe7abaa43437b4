"""Host-side error handling of the C ABI: every failure is a status code and a
message, never an abort, and the context stays usable afterwards."""

from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()
    import paper_1911_06001_gb300 as g

    c = g.Context(0)
    a = synthetic.make_asset(3, (np.array([1, 2]), np.array([1, 2]), np.array([1, 5])))
    h = c.upload(a.depth, a.leaf_ids, a.rgb)
    yield g, c, h
    c.close()


def test_bad_arguments_are_status_codes(env):
    g, ctx, h = env
    with pytest.raises(g.SvoError) as e:
        ctx.scene([h, h], [-1, 1])  # parent not before child
    assert e.value.status == -1
    with pytest.raises(g.SvoError) as e:
        ctx.scene([h, 12345], [-1, 0])  # unknown asset
    assert e.value.status == -3
    with pytest.raises(g.SvoError) as e:
        ctx.upload(0, np.zeros(1, np.uint64))
    assert e.value.status == -1
    with pytest.raises(g.SvoError) as e:
        ctx.scene([h] * (g.MAX_PARTS + 1), [-1] * (g.MAX_PARTS + 1))
    assert e.value.status == -9


def test_nan_pose_is_rejected_before_any_device_work(env):
    g, ctx, h = env
    sc = ctx.scene([h], [-1])
    bad = synthetic.affine12(np.eye(3), np.zeros(3))
    bad[5] = np.nan
    with pytest.raises(g.SvoError) as e:
        sc.set_transforms(bad[None])
    assert e.value.status == -7
    sc.close()


def test_asset_in_use_cannot_be_released(env):
    g, ctx, h = env
    sc = ctx.scene([h], [-1])
    with pytest.raises(g.SvoError) as e:
        ctx.release(h)
    assert e.value.status == -1 and "used" in str(e.value)
    sc.close()
    a = synthetic.make_asset(2, (np.array([0]), np.array([0]), np.array([0])))
    h2 = ctx.upload(a.depth, a.leaf_ids)
    ctx.release(h2)
    with pytest.raises(g.SvoError) as e:
        ctx.release(h2)
    assert e.value.status == -3


def test_singular_pose_reports_a_device_error_and_context_survives(env):
    import torch

    g, ctx, h = env
    sc = ctx.scene([h], [-1])
    sc.set_transforms(np.zeros((1, 12)))  # A = 0: not invertible
    sc.refit()
    with pytest.raises(g.SvoError) as e:
        ctx.check_device()
    assert e.value.status == -10 and "singular" in str(e.value)
    ctx.check_device()  # cleared
    # the part is skipped (its sphere is disabled); tracing still works
    rays = torch.from_numpy(synthetic.random_rays(256, np.random.default_rng(1), (-2,) * 3, (2,) * 3)).cuda()
    hits = g.decode_hits(sc.trace(rays))
    assert np.all(hits["part"] == 0xFFFFFFFF)
    sc.set_transforms(synthetic.affine12(np.eye(3), np.zeros(3))[None])
    sc.refit()
    ctx.check_device()
    sc.close()


def test_misaligned_and_null_buffers(env):
    import torch

    g, ctx, h = env
    sc = ctx.scene([h], [-1])
    lib = g._lib.load()
    buf = torch.zeros(1024, dtype=torch.float32, device="cuda")
    hits = torch.zeros(256, dtype=torch.int64, device="cuda")
    rc = lib.trace_rays(sc.h, C.c_void_p(buf.data_ptr() + 4), 8, C.c_void_p(hits.data_ptr()), None, 0, None, None)
    assert rc == -1 and b"aligned" in lib.svo_last_error()
    rc = lib.trace_rays(sc.h, None, 8, C.c_void_p(hits.data_ptr()), None, 0, None, None)
    assert rc == -1
    rc = lib.trace_rays(sc.h, C.c_void_p(buf.data_ptr()), 8, C.c_void_p(hits.data_ptr()), None, g.TRACE_STATS, None,
                        None)
    assert rc == -1 and b"stats" in lib.svo_last_error()
    sc.close()
