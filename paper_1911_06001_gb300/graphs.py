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
