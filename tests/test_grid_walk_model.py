"""The scene grid's coverage argument (Sec. V-E structure), checked on the
host: a float32 model of the grid build (sphere boxes widened by 2^-10 cells,
directed rounding of the box) and of the walk (crossings recomputed from each
cell plane as (plane - o) * (1/d), rays refused when their rounding allowance
exceeds half the widening) must visit, for every ray it accepts, a cell that
lists each part whose sphere box the exact (float64) segment meets.  This is
the property the GPU walk relies on to lose no hit; the GPU tests compare its
results with the oracle.  No GPU.

What this can and cannot show: a wrong far plane for negative directions, a
wrong stepping axis, an early stop or a clip that ignores tmin each fail
every case below.  The 2^-10-cell widening matters only for rays within
rounding distance of a cell edge, which random inputs do not reach (these
cases pass without it, because the directed rounding of the sphere boxes
already lists a box that touches a plane on both sides).  Its margin rests
on the error bound stated with the walk."""

from __future__ import annotations

import math

import numpy as np
import pytest

F = np.float32
U = 2.0 ** -24


def _rd(x: float) -> np.float32:
    f = F(x)
    return np.nextafter(f, F(-np.inf)) if float(f) > x else f


def _ru(x: float) -> np.float32:
    f = F(x)
    return np.nextafter(f, F(np.inf)) if float(f) < x else f


def _fma(a, b, c) -> np.float32:
    return F(float(a) * float(b) + float(c))


def build(spheres, G):
    """Grid corner, cell size, 1/cell size and the cell lists (dict cell -> parts), or None if refused."""
    box = grid_box(spheres, G)
    return None if box is None else (*box, cell_lists(spheres, *box, G))


def grid_box(spheres, G):
    lo = np.zeros(3, F)
    cs = np.zeros(3, F)
    inv = np.zeros(3, F)
    for k in range(3):
        l0 = min(_rd(float(c[k]) - float(c[3])) for c in spheres)
        h0 = max(_ru(float(c[k]) + float(c[3])) for c in spheres)
        m = max(_ru(float(_ru((float(h0) - float(l0)) / G)) * 2.0 ** -10), F(1e-30))
        lo[k] = _rd(float(l0) - float(m))
        cs[k] = max(_ru(float(_ru(float(h0) + float(m)) - float(lo[k])) / G), F(1e-30))
        inv[k] = F(1.0) / cs[k]
        if not 16 * U * (abs(float(lo[k])) + G * float(cs[k])) <= float(cs[k]) * 2.0 ** -12:
            return None
    return lo, cs, inv


def cell_lists(spheres, lo, cs, inv, G):
    pad = F(2.0 ** -10 + 2.0 ** -12)
    lists = {}
    for p, c in enumerate(spheres):
        rng = []
        for k in range(3):
            f0 = F(F(_rd(float(c[k]) - float(c[3])) - lo[k]) * inv[k]) - pad
            f1 = F(F(_ru(float(c[k]) + float(c[3])) - lo[k]) * inv[k]) + pad
            i0 = int(math.floor(max(float(f0), 0.0)))
            i1 = int(math.floor(min(float(f1), G - 0.5)))
            i0 = min(max(i0, 0), G - 1)
            i1 = min(max(i1, i0), G - 1)
            rng.append(range(i0, i1 + 1))
        for x in rng[0]:
            for y in rng[1]:
                for z in rng[2]:
                    lists.setdefault((x, y, z), set()).add(p)
    return lists


def walk(ray, lo, cs, inv, G):
    """Cells the float32 walk visits (in order), or None if it refuses the ray."""
    o = ray[0:3].astype(F)
    d = ray[4:7].astype(F)
    t0, t1 = F(ray[3]), F(ray[7])
    ok = True
    for a in range(3):
        blo, bhi = lo[a], _fma(F(G), cs[a], lo[a])
        if d[a] == 0:
            if o[a] < blo or o[a] > bhi:
                t1 = F(-np.inf)
            continue
        ta, tb = F(F(blo - o[a]) / d[a]), F(F(bhi - o[a]) / d[a])
        ok = ok and abs(float(ta)) < 1e38 and abs(float(tb)) < 1e38
        ta, tb = min(ta, tb), max(ta, tb)
        t0, t1 = max(t0, ta), min(t1, tb)
    if not ok:
        return None
    cur, step, rd, tn = [0] * 3, [0] * 3, [F(0)] * 3, [F(np.inf)] * 3
    for a in range(3):
        mag = abs(float(o[a])) + abs(float(lo[a])) + G * float(cs[a]) + abs(float(t0) * float(d[a]))
        if not 8 * U * mag <= float(cs[a]) * 2.0 ** -11:
            return None
        f = F(F(_fma(t0, d[a], o[a]) - lo[a]) * inv[a])
        i = int(math.floor(min(max(float(f), 0.0), float(G))))
        cur[a] = min(i, G - 1)
        step[a] = 1 if d[a] > 0 else (-1 if d[a] < 0 else 0)
        if d[a] != 0:
            rd[a] = F(F(1.0) / d[a])
            tn[a] = F(F(_fma(F(cur[a] + (1 if step[a] > 0 else 0)), cs[a], lo[a]) - o[a]) * rd[a])
    if not t0 <= t1:
        return []
    cells = []
    for _ in range(3 * G + 1):
        cells.append(tuple(cur))
        ax = (0 if tn[0] <= tn[2] else 2) if tn[0] <= tn[1] else (1 if tn[1] <= tn[2] else 2)
        if not tn[ax] < t1:
            break
        cur[ax] += step[ax]
        if cur[ax] < 0 or cur[ax] > G - 1:
            break
        tn[ax] = F(F(_fma(F(cur[ax] + (1 if step[ax] > 0 else 0)), cs[ax], lo[ax]) - o[ax]) * rd[ax])
    else:
        raise AssertionError("walk did not end")
    return cells


def meets_box(ray, c):
    """The exact (float64) segment meets the sphere's box [c - r, c + r]."""
    o, d = ray[0:3].astype(np.float64), ray[4:7].astype(np.float64)
    a, b = float(ray[3]), float(ray[7])
    for k in range(3):
        lo, hi = float(c[k]) - float(c[3]), float(c[k]) + float(c[3])
        if d[k] == 0.0:
            if o[k] < lo or o[k] > hi:
                return False
            continue
        ta, tb = (lo - o[k]) / d[k], (hi - o[k]) / d[k]
        a, b = max(a, min(ta, tb)), min(b, max(ta, tb))
    return a <= b


def _rays(rng, n, box, offset):
    o = rng.uniform(-box, box, (n, 3)) + offset
    d = rng.standard_normal((n, 3))
    # grazing and axis-aligned directions
    d[: n // 8, rng.integers(0, 3)] = 0.0
    d[n // 8: n // 4] *= np.array([1.0, 1e-4, 1e-4])
    d[n // 4: n // 3, 1] = 0.0
    d[n // 4: n // 3, 2] = 0.0
    r = np.zeros((n, 8), np.float32)
    r[:, 0:3] = o
    r[:, 4:7] = d
    r[:, 3] = rng.choice([0.0, -box, 0.5], n)
    r[:, 7] = rng.choice([np.inf, box, 3 * box], n)
    # origins exactly on lattice values of the scene coordinates
    r[n // 3: n // 2, 0:3] = np.round(r[n // 3: n // 2, 0:3])
    return r


@pytest.mark.parametrize("seed,P,offset", [(0, 64, 0.0), (1, 200, 0.0), (2, 120, 37.0), (3, 80, -500.0),
                                           (4, 80, -5000.0)])
def test_walk_visits_every_part_the_segment_meets(seed, P, offset):
    rng = np.random.default_rng(5100 + seed)
    box = 4.0 * P ** (1.0 / 3.0)
    G = 2
    while G < 16 and G ** 3 < 8 * P:
        G += 1
    centres = rng.uniform(-box / 2, box / 2, (P, 3)) + offset
    radii = rng.uniform(0.3, 2.0, P)
    spheres = np.concatenate([centres, radii[:, None]], 1).astype(np.float32)
    grid = build(spheres, G)
    if offset == -5000.0:
        # far from the origin relative to its cells: the grid is refused
        assert grid is None
        return
    assert grid is not None
    lo, cs, inv, lists = grid
    rays = _rays(rng, 1500, box, offset)
    walked = 0
    for ray in rays:
        cells = walk(ray, lo, cs, inv, G)
        if cells is None:
            continue  # refused: the cluster level takes the ray
        walked += 1
        found = set()
        for c in cells:
            found |= lists.get(c, set())
        for p, s in enumerate(spheres):
            if meets_box(ray, s):
                assert p in found, (p, ray, cells)
    assert walked > 0.9 * len(rays)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_walk_covers_boxes_touching_cell_planes(seed):
    """Sphere boxes that end exactly on a cell plane, and rays lying in that
    plane: where the cell index of a point on the plane rounds either way,
    the widened lists must still name the part in the cell the walk visits."""
    rng = np.random.default_rng(5200 + seed)
    P, G = 120, 10
    box = 4.0 * P ** (1.0 / 3.0)
    centres = rng.uniform(-box / 2, box / 2, (P, 3))
    radii = rng.uniform(0.3, 2.0, P)
    spheres = np.concatenate([centres, radii[:, None]], 1).astype(np.float32)
    lo, cs, inv = grid_box(spheres, G)
    # parts 8.. (well inside the box) moved to touch a plane from below or above
    touch = []
    for p in range(8, P):
        k = int(rng.integers(0, 3))
        i = int(rng.integers(2, G - 2))
        plane = _fma(F(i), cs[k], lo[k])
        r = spheres[p, 3]
        spheres[p, k] = F(float(plane) - float(r)) if p % 2 else F(float(plane) + float(r))
        touch.append((p, k, plane))
    assert grid_box(spheres, G) is not None
    lists = cell_lists(spheres, lo, cs, inv, G)
    checked = 0
    for p, k, plane in touch:
        # rays in the plane x_k = plane through the part's centre, random in-plane direction
        for _ in range(4):
            ray = np.zeros(8, np.float32)
            ray[0:3] = spheres[p, 0:3]
            ray[k] = plane
            d = rng.standard_normal(3)
            d[k] = 0.0
            ray[4:7] = d
            ray[3], ray[7] = -3 * box, 3 * box
            if not meets_box(ray, spheres[p]):
                continue
            cells = walk(ray, lo, cs, inv, G)
            assert cells is not None
            found = set()
            for c in cells:
                found |= lists.get(c, set())
            assert p in found, (p, k, ray)
            checked += 1
    assert checked > 100
