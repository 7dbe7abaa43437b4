"""One animation frame captured as a CUDA graph.

A frame of the path -- copy the frame's local poses from a device buffer into
the scene, compose / invert / refit, trace the rays, re-intersect the flagged
rays in FP64 -- is launched as one graph, removing the per-kernel launch cost
from the frame loop.  The graph reads the poses from ``self.poses`` (a device
tensor), so a new frame only needs the poses copied there before ``replay``.
Capture happens once, after an eager warm-up frame has grown the library's
per-stream scratch (no allocation may happen while capturing).
"""

from __future__ import annotations

import numpy as np

from . import TRACE_DEFAULT, Context


class FrameGraph:
    def __init__(self, ctx: Context, scene, rays, hits, flags: int = TRACE_DEFAULT, ray_flags=None):
        import torch

        self.ctx = ctx
        self.scene = scene
        self.rays = rays
        self.hits = hits
        self.flags = int(flags)
        self.ray_flags = ray_flags
        dev = rays.device
        self.stream = torch.cuda.Stream(device=dev)
        self.poses = torch.zeros((scene.n_parts, 12), dtype=torch.float64, device=dev)
        self.poses[:, 0] = 1.0
        self.poses[:, 5] = 1.0
        self.poses[:, 10] = 1.0
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self._frame()  # eager warm-up on the capture stream: grows its scratch
        self.stream.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._frame()

    def _frame(self) -> None:
        self.scene.set_transforms_device(self.poses)
        self.scene.refit()
        self.scene.trace(self.rays, self.hits, flags=self.flags, ray_flags=self.ray_flags)

    def replay(self, local=None) -> None:
        """Run one frame; ``local`` ([P, 12] FP64 host poses) replaces the poses first."""
        import torch

        if local is not None:
            host = torch.from_numpy(np.ascontiguousarray(local, dtype=np.float64).reshape(-1, 12))
            self.poses.copy_(host, non_blocking=False)
        self.graph.replay()


class BatchGraph:
    """A batched frame of many scenes captured as one CUDA graph.

    One replay copies every scene's local poses from a pinned host buffer to
    the device, composes / inverts / refits every scene, and runs
    ``trace_batch`` over all items (its ray-ordering launches, the persistent
    trace kernel and the FP64 pass included).  The refits are one launch
    (``Context.refit_batch``: a thread block per scene, each reading its
    poses straight from the copied buffer), so they run side by side on the
    device instead of one after another.

    ``items``: (scene, rays, hits, ray_flags-or-None[, image_width]) as for
    ``Context.trace_batch``; ``local``: one [P, 12] FP64 pose array per
    distinct scene, in order of first appearance in ``items``.  Capture
    happens once, after an eager warm-up on the same streams has grown the
    library's per-stream scratch."""

    def __init__(self, ctx: Context, items, local, flags: int = TRACE_DEFAULT):
        import torch

        self.ctx = ctx
        self.items = list(items)
        self.flags = int(flags)
        dev = self.items[0][1].device
        self.scenes = []
        for it in self.items:
            if all(it[0] is not s for s in self.scenes):
                self.scenes.append(it[0])
        sizes = [12 * s.n_parts for s in self.scenes]
        self.offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        n = int(self.offsets[-1])
        self.host = torch.empty(n, dtype=torch.float64).pin_memory()
        self.dev = torch.empty(n, dtype=torch.float64, device=dev)
        self.stream = torch.cuda.Stream(device=dev)
        self.pose_views = [self.dev[int(self.offsets[k]):int(self.offsets[k + 1])] for k in range(len(self.scenes))]
        self.done = torch.cuda.Event()
        self.set_poses(local)
        torch.cuda.synchronize()
        with torch.cuda.stream(self.stream):
            self._frame()  # eager warm-up on the capture streams: grows their scratch
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=self.stream):
            self._frame()

    def set_poses(self, local) -> None:
        """Write the next replay's poses (waits until the previous replay has read them)."""
        self.done.synchronize()
        h = self.host.numpy()
        for k, sc in enumerate(self.scenes):
            h[self.offsets[k]:self.offsets[k + 1]] = np.ascontiguousarray(local[k], dtype=np.float64).ravel()

    def _frame(self) -> None:
        s = self.stream
        self.dev.copy_(self.host, non_blocking=True)
        self.ctx.refit_batch(self.scenes, self.pose_views, stream=s)
        self.ctx.trace_batch(self.items, flags=self.flags, stream=s)

    def replay(self, local=None) -> None:
        """Run one batched frame on ``self.stream`` (asynchronously: the caller
        orders its own stream after it, e.g. ``wait_stream``); ``local`` (per
        scene [P, 12] poses) replaces the poses first."""
        import torch

        if local is not None:
            self.set_poses(local)
        with torch.cuda.stream(self.stream):  # a graph launches on the current stream
            self.graph.replay()
        self.done.record(self.stream)
