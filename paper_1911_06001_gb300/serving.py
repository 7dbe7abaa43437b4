"""Continuous-batching render server over resident animated scenes.

Requests (scene, pose, camera, resolution) arrive over time.  The server keeps
every scene's SVO assets resident on the device, admits requests by memory
(the ray and hit bytes of everything in flight must fit a budget), and packs
the admitted requests that are waiting into one persistent trace launch
(``trace_batch``) per free *slot*.  Slots are CUDA streams with preallocated
ray / hit buffers, so a batch formed from requests that arrived while earlier
batches were still on the GPU runs concurrently with them.

Per request, on its slot's stream: the request's pose goes to a leased
*instance* of its scene (a scene object sharing the assets but owning its own
pose tables, so concurrent requests of one scene can carry different poses),
the instance is refitted, and the camera's primary rays are generated on the
device.  Latency is measured from the request's arrival to the host observing
its batch's completion event.  The serving loops run with Python's cyclic
garbage collector paused (reference counting still frees what they drop): a
full collection in a process holding many objects stops the host for tens to
hundreds of milliseconds, and every request in flight would wait it out.

Host-side scheduling only; every per-ray and per-frame step runs in the
library's kernels.
"""

from __future__ import annotations

import collections
import contextlib
import gc
import time
from dataclasses import dataclass, field

import numpy as np

from . import TRACE_DEFAULT, TRACE_STATS, Context, trace_image

RAY_BYTES = 32
HIT_BYTES = 16
# per-ray scratch the library keeps per stream (FP64 list and pool offsets, the FP64 pass's
# leaf pool of 3 entries of 16 B per ray, ray ordering)
SCRATCH_BYTES_PER_RAY = 8 + 4 + 48 + 10


class AdmissionError(RuntimeError):
    """A request can never be admitted (larger than a slot or than the memory budget)."""


@dataclass
class Ticket:
    request: object
    n_rays: int
    arrival: float          # host clock (perf_counter) of arrival
    submitted: float = 0.0  # host clock when its batch was launched
    done: float = 0.0       # host clock when its completion (or expiry, or cancellation) was observed
    slot: int = -1
    offset: int = 0         # first ray of the request in its slot's buffers
    instance: object = None
    hits: object = None     # CUDA int64 view [n, 2] into the slot's hit buffer (valid until the slot is reused)
    status: str = "queued"  # queued -> running -> done, or queued -> timeout / cancelled
    device_ms: float = 0.0  # device time of its batch (first kernel of the batch to completion)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


class RequestQueue:
    """The server's admission and batching policy (host only, no GPU).

    * A request is refused at submission if it could never run: more rays
      than a slot holds, or more bytes than the whole memory budget.
    * Requests wait in arrival order.  A batch takes requests from the front
      while they fit the slot and the bytes still free in the budget; a
      request whose scene has no free instance keeps its place and the ones
      behind it may go first.
    * A request that has waited longer than ``max_wait`` seconds leaves the
      queue with status "timeout"; ``cancel`` removes one with status
      "cancelled".  Neither ever reaches the GPU.
    """

    def __init__(self, slot_rays: int, budget_bytes: int, bytes_per_ray: int, max_wait: float | None = None):
        self.slot_rays = int(slot_rays)
        self.budget = int(budget_bytes)
        self.per_ray = int(bytes_per_ray)
        self.max_wait = max_wait
        self.waiting = collections.deque()
        self.in_flight_bytes = 0

    def __len__(self) -> int:
        return len(self.waiting)

    def submit(self, ticket: Ticket) -> Ticket:
        if ticket.n_rays > self.slot_rays or ticket.n_rays * self.per_ray > self.budget:
            raise AdmissionError(f"request of {ticket.n_rays} rays exceeds the slot capacity or the memory budget")
        self.waiting.append(ticket)
        return ticket

    def cancel(self, ticket: Ticket, now: float) -> bool:
        """Remove a waiting request; False if it is no longer waiting."""
        try:
            self.waiting.remove(ticket)
        except ValueError:
            return False
        ticket.status, ticket.done = "cancelled", now
        return True

    def expire(self, now: float) -> list:
        """Remove and return the requests that waited longer than max_wait."""
        if self.max_wait is None:
            return []
        out = [t for t in self.waiting if now - t.arrival > self.max_wait]
        for t in out:
            self.waiting.remove(t)
            t.status, t.done = "timeout", now
        return out

    def take_batch(self, capacity: int, lease) -> tuple:
        """Requests for one slot of ``capacity`` rays: (tickets, total rays).
        ``lease(ticket)`` returns an instance of the ticket's scene, or None
        if all are busy; the taken tickets' bytes count as in flight."""
        batch, total, skipped = [], 0, []
        while self.waiting:
            t = self.waiting[0]
            if total + t.n_rays > capacity or self.in_flight_bytes + (total + t.n_rays) * self.per_ray > self.budget:
                break
            self.waiting.popleft()
            inst = lease(t)
            if inst is None:
                skipped.append(t)  # keeps its place
                continue
            t.instance, t.offset, t.status = inst, total, "running"
            total += t.n_rays
            batch.append(t)
        for t in reversed(skipped):
            self.waiting.appendleft(t)
        self.in_flight_bytes += total * self.per_ray
        return batch, total

    def release(self, tickets) -> None:
        """The tickets' batch has finished: their bytes are free again."""
        for t in tickets:
            self.in_flight_bytes -= t.n_rays * self.per_ray


@dataclass
class _Slot:
    stream: object
    rays: object
    hits: object
    capacity: int
    event: object = None
    start: object = None    # timing event recorded before the batch's first kernel
    tickets: list = field(default_factory=list)
    busy: bool = False


class Server:
    """Render server over scenes given as (part asset handles, parent) pairs."""

    def __init__(self, ctx: Context, scenes, n_slots: int = 3, max_batch_rays: int = 8 << 20,
                 memory_budget: int | None = None, instances_per_scene: int = 3, flags: int = TRACE_DEFAULT,
                 max_wait: float | None = None, pause_gc: bool = True):
        import torch

        self.ctx = ctx
        self.pause_gc = bool(pause_gc)
        self.flags = int(flags)
        self.dev = torch.device("cuda", ctx.device)
        self.instances = []
        for handles, parent in scenes:
            self.instances.append(collections.deque(ctx.scene(handles, parent) for _ in range(instances_per_scene)))
        self.slots = []
        for _ in range(n_slots):
            st = torch.cuda.Stream(device=self.dev)
            rays = torch.empty((max_batch_rays, 8), dtype=torch.float32, device=self.dev)
            hits = torch.empty((max_batch_rays, 2), dtype=torch.int64, device=self.dev)
            self.slots.append(_Slot(st, rays, hits, max_batch_rays))
        per_ray = RAY_BYTES + HIT_BYTES + SCRATCH_BYTES_PER_RAY
        self.budget = memory_budget if memory_budget is not None else n_slots * max_batch_rays * per_ray
        self.per_ray = per_ray
        self.queue = RequestQueue(max_batch_rays, self.budget, per_ray, max_wait)
        self.completed = []
        self.max_batch_rays = max_batch_rays
        self.on_done = None  # called for every completed ticket before its slot is reused
        self.stats = None    # a stats tensor (new_stats): every batch accumulates its counters into it
        self._warm()

    def _warm(self) -> None:
        """Grow every slot stream's library scratch to full size before serving."""
        import torch

        for s in self.slots:
            inst = self.instances[0][0]
            with torch.cuda.stream(s.stream):
                s.rays.zero_()
                s.rays[:, 7] = -1.0  # empty segments: tmax < tmin
            self.ctx.trace_batch([(inst, s.rays, s.hits, None)], flags=self.flags, stream=s.stream)
            s.stream.synchronize()

    # ------------------------------------------------------------- requests
    def submit(self, request, arrival: float | None = None) -> Ticket:
        n = int(request.width) * int(request.height)
        return self.queue.submit(Ticket(request, n, time.perf_counter() if arrival is None else arrival))

    def cancel(self, ticket: Ticket) -> bool:
        """Withdraw a request that is still waiting (status "cancelled")."""
        ok = self.queue.cancel(ticket, time.perf_counter())
        if ok:
            self.completed.append(ticket)
        return ok

    def poll(self) -> list:
        """Retire finished batches; returns the tickets completed by this call."""
        out = []
        now = time.perf_counter()
        for s in self.slots:
            if s.busy and s.event.query():
                dev_ms = s.start.elapsed_time(s.event)
                for t in s.tickets:
                    t.done = now
                    t.status = "done"
                    t.device_ms = dev_ms
                    self.instances[t.request.scene].append(t.instance)
                    out.append(t)
                self.queue.release(s.tickets)
                s.busy = False
                s.tickets = []
        self.completed.extend(out)
        if self.on_done is not None:
            for t in out:
                self.on_done(t)
        return out

    def step(self) -> int:
        """Poll, launch batches on free slots, then expire the requests still
        waiting past the maximum wait; returns the number of batches launched."""
        self.poll()
        launched = 0

        def lease(t):
            free = self.instances[t.request.scene]
            return free.popleft() if free else None

        for si, s in enumerate(self.slots):
            if s.busy or not len(self.queue):
                continue
            batch, total = self.queue.take_batch(s.capacity, lease)
            if batch:
                self._launch(si, s, batch, total)
                launched += 1
        expired = self.queue.expire(time.perf_counter())
        self.completed.extend(expired)
        if self.on_done is not None:
            for t in expired:
                self.on_done(t)
        return launched

    def _launch(self, si: int, s: _Slot, batch: list, total: int) -> None:
        import torch

        items = []
        now = time.perf_counter()
        s.start = torch.cuda.Event(enable_timing=True)
        s.start.record(s.stream)
        # every request's scene instance is posed, then all are refitted by one
        # launch (a block per instance; a batch leases distinct instances)
        for t in batch:
            t.instance.set_transforms(t.request.local, stream=s.stream)
        self.ctx.refit_batch([t.instance for t in batch], stream=s.stream)
        for t in batch:
            r = t.request
            inst = t.instance
            rays = s.rays[t.offset:t.offset + t.n_rays]
            hits = s.hits[t.offset:t.offset + t.n_rays]
            self.ctx.raygen(tuple(float(v) for v in r.eye), tuple(float(v) for v in r.target), int(r.width),
                            int(r.height), 60.0, rays=rays, stream=s.stream)
            items.append((inst, rays, hits, None, int(r.width)))
            t.hits = hits
            t.slot = si
            t.submitted = now
        if self.stats is not None:
            self.ctx.trace_batch(items, flags=self.flags | TRACE_STATS, stats=self.stats, stream=s.stream)
        else:
            self.ctx.trace_batch(items, flags=self.flags, stream=s.stream)
        s.event = torch.cuda.Event(enable_timing=True)
        s.event.record(s.stream)
        s.tickets = batch
        s.busy = True

    def idle(self) -> bool:
        return not len(self.queue) and not any(s.busy for s in self.slots)

    # --------------------------------------------------------------- drivers
    def run(self, requests, on_done=None) -> list:
        """Replay requests at their arrival times (seconds from now); returns
        the tickets in completion order.  ``on_done(ticket)`` runs for every
        completed ticket while its hits are still valid."""
        self.on_done = on_done
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        tickets = []
        with gc_paused(self.pause_gc):
            t0 = time.perf_counter()
            while pending or not self.idle():
                now = time.perf_counter()
                while pending and t0 + pending[0].arrival <= now:
                    r = pending.popleft()
                    tickets.append(self.submit(r, arrival=t0 + r.arrival))
                before = len(self.completed)
                launched = self.step()
                if not launched and len(self.completed) == before:
                    time.sleep(20e-6)
        self.on_done = None
        return tickets


def render_alone(ctx: Context, scene_handle, request, flags: int = TRACE_DEFAULT, stream=None):
    """One request by itself (no batching) on the current or given stream: pose,
    refit, device raygen and a single-scene trace.  Returns (rays, hits)."""
    scene_handle.set_transforms(request.local, stream=stream)
    scene_handle.refit(stream=stream)
    rays = ctx.raygen(tuple(float(v) for v in request.eye), tuple(float(v) for v in request.target),
                      int(request.width), int(request.height), 60.0, stream=stream)
    hits = scene_handle.trace(rays, flags=flags | trace_image(int(request.width)), stream=stream)
    return rays, hits


def run_unbatched(ctx: Context, scene_handles, requests, flags: int = TRACE_DEFAULT, pause_gc: bool = True) -> list:
    """The baseline: the same request stream served one request at a time, each
    traced alone as soon as it has arrived and the previous one has finished.
    Returns (arrival, done, n_rays, device ms) per request."""
    import torch

    out = []
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    order = sorted(requests, key=lambda q: q.arrival)
    with gc_paused(pause_gc):
        t0 = time.perf_counter()
        for r in order:
            while time.perf_counter() < t0 + r.arrival:
                pass
            ev[0].record(stream)
            render_alone(ctx, scene_handles[r.scene], r, flags=flags, stream=stream)
            ev[1].record(stream)
            stream.synchronize()
            out.append((t0 + r.arrival, time.perf_counter(), int(r.width) * int(r.height),
                        ev[0].elapsed_time(ev[1])))
    return out


@contextlib.contextmanager
def gc_paused(pause: bool = True):
    """Pause Python's cyclic garbage collector for the duration (when it is on
    and ``pause`` is set), and put it back as it was afterwards, also on an
    exception."""
    was = gc.isenabled()
    if pause and was:
        gc.disable()
    try:
        yield
    finally:
        if pause and was:
            gc.enable()


def latency_stats(pairs) -> dict:
    """pairs: iterable of (arrival, done, n_rays[, device_ms]).  p50/p99 latency
    in ms and Mrays/s over the window; with device times also their p50/p99
    and those of the rest of the latency (waiting, host work, polling)."""
    a = np.array(list(pairs), dtype=np.float64)
    if a.size == 0:
        return {"requests": 0}
    lat = (a[:, 1] - a[:, 0]) * 1e3
    span = a[:, 1].max() - a[:, 0].min()
    out = {"requests": int(a.shape[0]), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
           "mrays_per_s": float(a[:, 2].sum() / span / 1e6)}
    if a.shape[1] > 3:
        dev = a[:, 3]
        out.update({"device_p50_ms": float(np.percentile(dev, 50)), "device_p99_ms": float(np.percentile(dev, 99)),
                    "host_and_wait_p50_ms": float(np.percentile(lat - dev, 50)),
                    "host_and_wait_p99_ms": float(np.percentile(lat - dev, 99))})
    return out
