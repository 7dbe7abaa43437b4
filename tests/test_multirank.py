"""Multi-rank host logic of the benchmark, on CPU with the gloo backend.

Rays are independent and the assets read-only, so N GPUs render disjoint
frames with no collective on the data path; the only cross-rank step is the
max of the per-rank times.  Two gloo ranks check the frame sharding and the
reduction.
"""

from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    frames = [bench.frame_of(s, world, rank) for s in range(30)]
    local_ms = 10.0 + 5.0 * rank
    slowest = bench.max_over_ranks(local_ms)
    dist.barrier()
    q.put((rank, frames, slowest))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_frames_are_sharded_and_times_max_reduced(world):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    # every rank sees the slowest rank's time
    assert all(abs(o[2] - (10.0 + 5.0 * (world - 1))) < 1e-12 for o in out)
    # at each step the ranks render distinct frames, and consecutive steps advance by world
    for s in range(30):
        fs = [o[1][s] for o in out]
        assert len(set(fs)) == world
        assert fs == [(s * world + r) % 60 for r in range(world)]


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5) == 3.5
    assert [bench.frame_of(s, 1, 0) for s in range(3)] == [0, 1, 2]
