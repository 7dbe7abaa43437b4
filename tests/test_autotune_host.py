"""The autotuner's host-side mapping from a tuned configuration to trace
flags (no GPU)."""

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
