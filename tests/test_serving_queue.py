"""The render server's admission and batching policy, on the host (no GPU):
refusal of requests that can never run, batches bounded by the slot and the
memory budget, order kept for requests whose scene is busy, expiry after a
maximum wait and cancellation (both end the request with a status and never
reach the GPU)."""

from __future__ import annotations

import gc
from dataclasses import dataclass

import pytest

from paper_1911_06001_gb300.serving import AdmissionError, RequestQueue, Ticket, gc_paused


@dataclass
class Req:
    scene: int


def _t(n, scene=0, arrival=0.0):
    return Ticket(Req(scene), n, arrival)


def test_refuses_requests_that_can_never_run():
    q = RequestQueue(slot_rays=1000, budget_bytes=800 * 10, bytes_per_ray=10)
    with pytest.raises(AdmissionError):
        q.submit(_t(1001))  # larger than a slot
    with pytest.raises(AdmissionError):
        q.submit(_t(900))  # larger than the whole budget
    q.submit(_t(800))
    assert len(q) == 1


def test_batches_fill_slots_in_order_and_respect_memory():
    q = RequestQueue(slot_rays=1000, budget_bytes=1500 * 10, bytes_per_ray=10)
    ts = [q.submit(_t(n)) for n in (400, 400, 400, 700, 100)]
    b1, n1 = q.take_batch(1000, lambda t: object())
    assert b1 == ts[:2] and n1 == 800 and [t.offset for t in b1] == [0, 400]
    assert all(t.status == "running" for t in b1)
    # 800 rays in flight: 700 more would pass the budget of 1500, so the next
    # batch stops before the 700-ray request (it does not jump the queue)
    b2, n2 = q.take_batch(1000, lambda t: object())
    assert b2 == [ts[2]] and n2 == 400
    b3, _ = q.take_batch(1000, lambda t: object())
    assert b3 == []
    q.release(b1)
    b4, n4 = q.take_batch(1000, lambda t: object())
    assert b4 == [ts[3], ts[4]] and n4 == 800
    q.release(b2)
    q.release(b4)
    assert q.in_flight_bytes == 0 and len(q) == 0


def test_busy_scene_keeps_its_place():
    q = RequestQueue(slot_rays=1000, budget_bytes=10 ** 9, bytes_per_ray=1)
    a, b, c = q.submit(_t(100, scene=0)), q.submit(_t(100, scene=1)), q.submit(_t(100, scene=0))
    free = {0: 1, 1: 1}  # one instance of each scene

    def lease(t):
        if free[t.request.scene] == 0:
            return None
        free[t.request.scene] -= 1
        return "inst"

    batch, _ = q.take_batch(1000, lease)
    assert batch == [a, b]  # c's scene is taken by a: c waits, first in line
    assert list(q.waiting) == [c]


def test_expiry_and_cancellation():
    q = RequestQueue(slot_rays=1000, budget_bytes=10 ** 9, bytes_per_ray=1, max_wait=0.5)
    old, new, gone = q.submit(_t(10, arrival=0.0)), q.submit(_t(10, arrival=0.8)), q.submit(_t(10, arrival=0.9))
    assert q.cancel(gone, now=1.0) and gone.status == "cancelled" and gone.done == 1.0
    assert not q.cancel(gone, now=1.1)
    expired = q.expire(now=1.0)
    assert expired == [old] and old.status == "timeout" and old.done == 1.0
    batch, _ = q.take_batch(1000, lambda t: object())
    assert batch == [new]
    # no maximum wait: nothing expires
    q2 = RequestQueue(slot_rays=10, budget_bytes=100, bytes_per_ray=1)
    q2.submit(_t(5, arrival=-1e9))
    assert q2.expire(now=0.0) == [] and len(q2) == 1



def test_gc_paused_restores_the_collector_state():
    was = gc.isenabled()
    try:
        gc.enable()
        with gc_paused():
            assert not gc.isenabled()
        assert gc.isenabled()
        with pytest.raises(RuntimeError):
            with gc_paused():
                raise RuntimeError("a failing serving loop")
        assert gc.isenabled()
        with gc_paused(False):
            assert gc.isenabled()
        gc.disable()
        with gc_paused():
            assert not gc.isenabled()
        assert not gc.isenabled()  # a collector that was off stays off
    finally:
        (gc.enable if was else gc.disable)()
