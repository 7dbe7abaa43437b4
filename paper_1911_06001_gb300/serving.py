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
its batch's completion event.

Host-side scheduling only; every per-ray and per-frame step runs in the
library's kernels.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import TRACE_DEFAULT, Context, trace_image

RAY_BYTES = 32
HIT_BYTES = 16
# per-ray scratch the library keeps per stream (FP64 list + contenders / 8 + ordering)
SCRATCH_BYTES_PER_RAY = 8 + 16 + 10


class AdmissionError(RuntimeError):
    """A request can never be admitted (larger than a slot or than the memory budget)."""


@dataclass
class Ticket:
    request: object
    n_rays: int
    arrival: float          # host clock (perf_counter) of arrival
    submitted: float = 0.0  # host clock when its batch was launched
    done: float = 0.0       # host clock when its completion was observed
    slot: int = -1
    offset: int = 0         # first ray of the request in its slot's buffers
    instance: object = None
    hits: object = None     # CUDA int64 view [n, 2] into the slot's hit buffer (valid until the slot is reused)

    @property
    def latency(self) -> float:
        return self.done - self.arrival


@dataclass
class _Slot:
    stream: object
    rays: object
    hits: object
    capacity: int
    event: object = None
    tickets: list = field(default_factory=list)
    busy: bool = False


class Server:
    """Render server over scenes given as (part asset handles, parent) pairs."""

    def __init__(self, ctx: Context, scenes, n_slots: int = 3, max_batch_rays: int = 8 << 20,
                 memory_budget: int | None = None, instances_per_scene: int = 3, flags: int = TRACE_DEFAULT):
        import torch

        self.ctx = ctx
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
        self.in_flight_bytes = 0
        self.queue = collections.deque()
        self.completed = []
        self.max_batch_rays = max_batch_rays
        self.on_done = None  # called for every completed ticket before its slot is reused
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
        if n > self.max_batch_rays or n * self.per_ray > self.budget:
            raise AdmissionError(f"request of {n} rays exceeds the slot capacity or the memory budget")
        t = Ticket(request, n, time.perf_counter() if arrival is None else arrival)
        self.queue.append(t)
        return t

    def poll(self) -> list:
        """Retire finished batches; returns the tickets completed by this call."""
        out = []
        now = time.perf_counter()
        for s in self.slots:
            if s.busy and s.event.query():
                for t in s.tickets:
                    t.done = now
                    self.instances[t.request.scene].append(t.instance)
                    self.in_flight_bytes -= t.n_rays * self.per_ray
                    out.append(t)
                s.busy = False
                s.tickets = []
        self.completed.extend(out)
        if self.on_done is not None:
            for t in out:
                self.on_done(t)
        return out

    def step(self) -> int:
        """Poll, then launch batches on free slots; returns the number of batches launched."""
        self.poll()
        launched = 0
        for si, s in enumerate(self.slots):
            if s.busy or not self.queue:
                continue
            batch, total, skipped = [], 0, collections.deque()
            while self.queue:
                t = self.queue[0]
                fits = total + t.n_rays <= s.capacity and \
                    self.in_flight_bytes + (total + t.n_rays) * self.per_ray <= self.budget
                if not fits:
                    break
                self.queue.popleft()
                if not self.instances[t.request.scene]:
                    skipped.append(t)  # every instance of its scene is busy: keep its place
                    continue
                t.instance = self.instances[t.request.scene].popleft()
                t.offset = total
                total += t.n_rays
                batch.append(t)
            while skipped:
                self.queue.appendleft(skipped.pop())
            if batch:
                self._launch(si, s, batch, total)
                launched += 1
        return launched

    def _launch(self, si: int, s: _Slot, batch: list, total: int) -> None:
        import torch

        items = []
        now = time.perf_counter()
        for t in batch:
            r = t.request
            inst = t.instance
            inst.set_transforms(r.local, stream=s.stream)
            inst.refit(stream=s.stream)
            rays = s.rays[t.offset:t.offset + t.n_rays]
            hits = s.hits[t.offset:t.offset + t.n_rays]
            self.ctx.raygen(tuple(float(v) for v in r.eye), tuple(float(v) for v in r.target), int(r.width),
                            int(r.height), 60.0, rays=rays, stream=s.stream)
            items.append((inst, rays, hits, None, int(r.width)))
            t.hits = hits
            t.slot = si
            t.submitted = now
        self.ctx.trace_batch(items, flags=self.flags, stream=s.stream)
        s.event = torch.cuda.Event()
        s.event.record(s.stream)
        s.tickets = batch
        s.busy = True
        self.in_flight_bytes += total * self.per_ray

    def idle(self) -> bool:
        return not self.queue and not any(s.busy for s in self.slots)

    # --------------------------------------------------------------- drivers
    def run(self, requests, on_done=None) -> list:
        """Replay requests at their arrival times (seconds from now); returns
        the tickets in completion order.  ``on_done(ticket)`` runs for every
        completed ticket while its hits are still valid."""
        self.on_done = on_done
        t0 = time.perf_counter()
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        tickets = []
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


def run_unbatched(ctx: Context, scene_handles, requests, flags: int = TRACE_DEFAULT) -> list:
    """The baseline: the same request stream served one request at a time, each
    traced alone as soon as it has arrived and the previous one has finished.
    Returns (arrival, done, n_rays) per request."""
    import torch

    t0 = time.perf_counter()
    out = []
    stream = torch.cuda.current_stream()
    for r in sorted(requests, key=lambda q: q.arrival):
        while time.perf_counter() < t0 + r.arrival:
            pass
        render_alone(ctx, scene_handles[r.scene], r, flags=flags, stream=stream)
        stream.synchronize()
        out.append((t0 + r.arrival, time.perf_counter(), int(r.width) * int(r.height)))
    return out


def latency_stats(pairs) -> dict:
    """pairs: iterable of (arrival, done, n_rays).  p50/p99 latency in ms and Mrays/s over the window."""
    a = np.array(list(pairs), dtype=np.float64)
    if a.size == 0:
        return {"requests": 0}
    lat = (a[:, 1] - a[:, 0]) * 1e3
    span = a[:, 1].max() - a[:, 0].min()
    return {"requests": int(a.shape[0]), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "mrays_per_s": float(a[:, 2].sum() / span / 1e6)}
