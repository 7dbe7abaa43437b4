"""C ABI checks that need no GPU: exported symbols, host octree layout, host-side argument checks."""

from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np
import pytest

import synthetic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1911_06001_gb300 import build as b

    b.build()
    import paper_1911_06001_gb300._lib as L

    return L.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "svoanim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", src,
                                 flags=re.M)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 18
    import paper_1911_06001_gb300._lib as L

    assert sorted(L.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    lib.svo_status_string.restype = C.c_char_p
    assert lib.svo_status_string(0) == b"SVO_OK"
    assert lib.svo_status_string(-7) == b"SVO_ERR_NAN"


def _decode(nodes, depth):
    """Walk the breadth-first node array and return the sorted leaf ids it encodes."""
    out = []
    stack = [(0, 0, 0, 0, 0)]  # node index, level, x, y, z
    while stack:
        idx, lvl, x, y, z = stack.pop()
        first, masks = int(nodes[idx, 0]), int(nodes[idx, 1])
        cm, lm = masks & 0xFF, (masks >> 8) & 0xFF
        assert (masks >> 16) == 0
        assert lm == (cm if lvl == depth - 1 else 0)
        assert cm != 0
        for k in range(8):
            if not (cm >> k) & 1:
                continue
            rank = bin(cm & ((1 << k) - 1)).count("1")
            cx, cy, cz = 2 * x + (k & 1), 2 * y + ((k >> 1) & 1), 2 * z + ((k >> 2) & 1)
            if lvl == depth - 1:
                out.append((first + rank, cx | (cy << depth) | (cz << 2 * depth)))
            else:
                stack.append((first + rank, lvl + 1, cx, cy, cz))
    return out


@pytest.mark.parametrize("depth,p", [(1, 0.5), (3, 0.2), (5, 0.03), (7, 0.001)])
def test_host_build_layout_roundtrip(lib, depth, p):
    import paper_1911_06001_gb300 as g

    rng = np.random.default_rng(depth)
    n = 1 << depth
    occ = rng.random(n ** 3) < p
    idx = np.nonzero(occ)[0]
    x, y, z = idx % n, (idx // n) % n, idx // (n * n)
    ids = synthetic.pack_ids(x, y, z, depth)
    dup = np.concatenate([ids, ids[: len(ids) // 3]])  # duplicates are allowed
    rng.shuffle(dup)
    rgb = synthetic.rgb_hash(*synthetic.unpack_ids(dup, depth))
    nodes, leaf_rgb = g.build_host(depth, dup, rgb)
    leaves = _decode(nodes, depth)
    slots = sorted(s for s, _ in leaves)
    assert slots == list(range(len(np.unique(ids))))  # leaf payload indices are a permutation
    got = np.array(sorted(v for _, v in leaves), dtype=np.uint64)
    assert np.array_equal(got, np.unique(ids))
    # payload follows the leaves
    for s, v in leaves:
        assert leaf_rgb[s] == synthetic.rgb_hash(*synthetic.unpack_ids(np.array([v], np.uint64), depth))[0]
    # breadth first: every child index is larger than its parent's
    for i in range(nodes.shape[0]):
        lvl_leaf = (nodes[i, 1] >> 8) & 0xFF
        if not lvl_leaf:
            assert nodes[i, 0] > i


def test_host_build_rejects_bad_input(lib):
    import paper_1911_06001_gb300 as g
    from paper_1911_06001_gb300._lib import SvoError

    with pytest.raises(SvoError):
        g.build_host(0, np.zeros(1, np.uint64))
    with pytest.raises(SvoError):
        g.build_host(17, np.zeros(1, np.uint64))
    with pytest.raises(SvoError):
        g.build_host(2, np.array([1 << 6], np.uint64))  # z = 4 >= 2^2
    nodes, rgb = g.build_host(3, np.zeros(0, np.uint64))
    assert nodes.shape[0] == 0 and rgb.shape[0] == 0


def test_null_arguments_return_errors(lib):
    import paper_1911_06001_gb300._lib as L

    lib = L.load()
    assert lib.svo_ctx_create(0, None) == -1
    assert lib.svo_upload(None, None, None) == -1
    assert lib.scene_create(None, 1, None, None, None) == -1
    assert lib.trace_rays(None, None, 0, None, None, 0, None, None) == -1
    assert lib.scene_destroy(None) == 0
    assert lib.svo_ctx_destroy(None) == 0
    assert b"NULL" in lib.svo_last_error()
