"""Host-side logic (no GPU): the autotuner's mapping from a tuned
configuration to trace flags, and the bench's lookup of measured DRAM
traffic."""

from __future__ import annotations


def test_autotune_flag_mapping():
    """The autotuner's tuned configuration maps to trace flags on the host:
    ray order and culling structure; configurations cached before the culling
    knob existed read as the cluster level."""
    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300 import autotune

    assert autotune.order_flag({"order": "none", "cull": "clusters"}) == 0
    assert autotune.order_flag({"order": "origin", "cull": "grid"}) == g.TRACE_ORDER_ORIGIN | g.TRACE_GRID
    assert autotune.order_flag({"order": "image", "image_width": 640}) == g.trace_image(640)
    assert autotune.order_flag({"order": "dir"}) == g.TRACE_ORDER_DIR


def test_bench_reports_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    """bench.py takes the trace kernel's DRAM traffic from the committed ncu
    summary only while that summary's recorded source hash matches the
    kernel source; otherwise it reports none, with the reason."""
    import hashlib

    import bench

    src = tmp_path / "k_trace.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    sha = hashlib.sha256(src.read_bytes()).hexdigest()
    prof = tmp_path / "profile.md"
    prof.write_text(f"# x\n\n`k_trace_source_sha256: {sha}`\n\n`traffic_bytes_per_launch: 82762496`\n")
    monkeypatch.setattr(bench, "TRACE_SOURCE", str(src))
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    value, why = bench.measured_traffic()
    assert value == 82762496.0 and sha[:12] in why
    src.write_bytes(b"__global__ void k() { }\n")  # the kernel changed since the capture
    assert bench.measured_traffic() == (None, "kernel changed since the ncu capture")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(tmp_path / "missing.md"))
    assert bench.measured_traffic() == (None, "no ncu summary")
