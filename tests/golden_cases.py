"""Parser for tests/golden/hand_cases.txt (hand-derived closest hits)."""

from __future__ import annotations

import os

import numpy as np

from synthetic import Asset, Scene, pack_ids, rgb_hash

HERE = os.path.dirname(os.path.abspath(__file__))


def load_hand_cases(path: str | None = None):
    path = path or os.path.join(HERE, "golden", "hand_cases.txt")
    cases = []
    cur = None
    with open(path) as f:
        for raw in f:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "case":
                cur = {"name": tok[1], "parts": [], "rays": [], "hits": []}
            elif tok[0] == "part":
                parent, depth = int(tok[1]), int(tok[2])
                pose = np.array([float(v) for v in tok[3:15]])
                leaves = [tuple(int(c) for c in s.split(",")) for s in tok[15].split(";")]
                cur["parts"].append((parent, depth, pose, leaves))
            elif tok[0] == "ray":
                cur["rays"].append([float(v) for v in tok[1:9]])
            elif tok[0] == "hit":
                if tok[1] == "miss":
                    cur["hits"].append(None)
                else:
                    cur["hits"].append((float(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "end":
                cases.append(cur)
                cur = None
    return cases


def case_scene(case) -> tuple[Scene, np.ndarray]:
    assets, parent, local = [], [], []
    for p, depth, pose, leaves in case["parts"]:
        xs, ys, zs = (np.array([l[k] for l in leaves]) for k in range(3))
        ids = np.unique(pack_ids(xs, ys, zs, depth))
        assets.append(Asset(depth=depth, leaf_ids=ids, rgb=rgb_hash(xs, ys, zs)))
        parent.append(p)
        local.append(pose)
    P = len(assets)
    scene = Scene(name=case["name"], assets=assets, part_asset=np.arange(P, dtype=np.int32),
                  parent=np.array(parent, dtype=np.int32), local=np.array(local))
    rays = np.array(case["rays"], dtype=np.float64)
    return scene, rays
