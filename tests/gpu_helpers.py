"""Shared helpers for the GPU parity tests: upload synthetic scenes through the
C ABI, trace, and compare with the FP64 oracle element by element."""

from __future__ import annotations

import numpy as np

import oracle

# the hit-t tolerance the method is held to: |t_gpu - t_oracle| <= TOL_T * max(|t_oracle|, h)
# with h the world length of the hit part's leaf diagonal in units of t
TOL_T = 1e-5


class GpuScene:
    def __init__(self, ctx, scene):
        self.scene = scene
        self.handles = [ctx.upload(a.depth, a.leaf_ids, a.rgb) for a in scene.assets]
        self.sc = ctx.scene([self.handles[int(i)] for i in scene.part_asset], scene.parent)
        self.set_pose(scene.local)

    def set_pose(self, local):
        self.local = np.asarray(local, dtype=np.float64)
        self.sc.set_transforms(self.local)
        self.sc.refit()

    def trace(self, rays, flags):
        import torch

        import paper_1911_06001_gb300 as g

        r = torch.from_numpy(np.ascontiguousarray(rays, dtype=np.float32)).cuda()
        rf = torch.zeros(r.shape[0], dtype=torch.int32, device="cuda")
        hits = self.sc.trace(r, flags=flags, ray_flags=rf)
        torch.cuda.synchronize()
        out = g.decode_hits(hits)
        out["flags"] = rf.cpu().numpy().astype(np.uint32)
        return out


def leaf_h(scene, local, part, rays):
    """Leaf diagonal length of the hit part, in units of t (1 for misses)."""
    world = oracle.compose(scene.parent, local)
    depth = np.array([scene.assets[int(a)].depth for a in scene.part_asset])
    diag = np.array([np.linalg.norm(world[p].reshape(3, 4)[:, :3] @ np.ones(3)) * 2.0 ** -depth[p]
                     for p in range(scene.n_parts)])
    dn = np.linalg.norm(np.asarray(rays, dtype=np.float64)[:, 4:7], axis=1)
    h = np.ones(len(part))
    hit = part != oracle.MISS_PART
    h[hit] = diag[part[hit]] / np.maximum(dn[hit], 1e-300)
    return h


def compare(scene, local, rays, gpu, ora, allow_flagged_mismatch=0):
    """Element-wise parity.  Unflagged rays: ids bit-exact, t within TOL_T.
    Flagged rays (re-intersected in FP64): same checks, mismatches counted;
    rays whose oracle top-2 gap is below FP64 resolution are ties with
    several correct answers and only their t is compared."""
    import paper_1911_06001_gb300 as g

    flagged = (gpu["flags"] & g.RAY_UNCERTAIN) != 0
    fixed = (gpu["flags"] & g.RAY_FIXED) != 0
    # ids certified, t left to the FP64 pass: its t is only held to the bound once refined
    t_refined = (gpu["flags"] & g.RAY_T_REFINED) != 0
    t_o = ora["t"]
    hit_o = ora["part"] != oracle.MISS_PART
    with np.errstate(invalid="ignore"):
        fp64_tie = hit_o & (ora["second"] - t_o <= 1e-9 * np.maximum(np.abs(t_o), 1.0))
    id_eq = (gpu["part"] == ora["part"]) & (gpu["voxel"] == ora["voxel"])
    h = leaf_h(scene, local, ora["part"], rays)
    t_g = gpu["t"].astype(np.float64)
    with np.errstate(invalid="ignore"):
        t_eq = np.where(hit_o, np.abs(t_g - t_o) <= TOL_T * np.maximum(np.abs(t_o), h), np.isinf(t_g))
    unf = ~flagged
    bad_unf_id = np.nonzero(unf & ~id_eq)[0]
    bad_unf_t = np.nonzero(unf & ~t_eq & (~t_refined | fixed))[0]
    # t-refined rays the FP64 pass did not fix: held to the certified bound
    # their flag word carries, |t - t_exact| <= 2^e max(t_exact, h) (1 + 2^-18)
    loose = unf & t_refined & ~fixed
    e = g.ray_t_bound_exp(gpu["flags"])
    with np.errstate(invalid="ignore", over="ignore"):
        lim = np.ldexp(1.0, np.minimum(e, 1000)) * np.maximum(np.abs(t_o), h) * (1.0 + 2.0 ** -18)
        loose_err = np.where(loose, np.abs(t_g - t_o), 0.0)
    assert np.all(e[loose] >= -16), "a t-refined ray carries no bound exponent"
    bad_loose = np.nonzero(loose & (e < 127) & ~(loose_err <= lim))[0]
    assert bad_loose.size == 0, f"t-refined rays outside their certified bound at {bad_loose[:10]}: " \
                                f"{t_g[bad_loose[:5]]} vs {t_o[bad_loose[:5]]}, e {e[bad_loose[:5]]}"
    assert bad_unf_id.size == 0, f"unflagged id mismatches at {bad_unf_id[:10]}: gpu part {gpu['part'][bad_unf_id[:5]]} " \
                                 f"vox {gpu['voxel'][bad_unf_id[:5]]} vs ora {ora['part'][bad_unf_id[:5]]} " \
                                 f"{ora['voxel'][bad_unf_id[:5]]}; t {t_g[bad_unf_id[:5]]} vs {t_o[bad_unf_id[:5]]}"
    assert bad_unf_t.size == 0, f"unflagged t mismatches at {bad_unf_t[:10]}: {t_g[bad_unf_t[:5]]} vs {t_o[bad_unf_t[:5]]}"
    flag_id_bad = flagged & ~id_eq & ~fp64_tie
    flag_t_bad = flagged & ~t_eq
    rep = {
        "rays": int(len(t_o)),
        "hits": int(hit_o.sum()),
        "flagged": int(flagged.sum()),
        "t_refined": int(t_refined.sum()),
        "fixed": int(fixed.sum()),
        "flagged_id_mismatch": int(flag_id_bad.sum()),
        "flagged_t_mismatch": int(flag_t_bad.sum()),
        "fp64_ties": int(fp64_tie.sum()),
        "t_refined_unfixed": int(loose.sum()),
        "t_refined_unfixed_max_rel_err": float(np.max(loose_err[loose] / np.maximum(np.abs(t_o[loose]), h[loose])))
        if loose.any() else 0.0,
        "t_refined_unfixed_unbounded": int((loose & (e >= 127)).sum()),
        "max_rel_t_err": float(np.max(np.abs(t_g[hit_o] - t_o[hit_o]) / np.maximum(np.abs(t_o[hit_o]), h[hit_o])))
        if hit_o.any() else 0.0,
    }
    if fixed.any():
        assert rep["flagged_id_mismatch"] <= allow_flagged_mismatch, rep
        assert rep["flagged_t_mismatch"] <= allow_flagged_mismatch, rep
    return rep
