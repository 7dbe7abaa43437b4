"""Seeded synthetic inputs for ray casting against animated sparse voxel octrees.

This package only *constructs inputs*: voxelised shapes (leaf lists), per-part
local poses, transform-tree topology and rays.  It holds none of the method's
arithmetic (no transform composition or inversion, no ray transform, no sphere
or box intersection, no traversal), so that the CUDA library and the CPU
oracle can both consume its arrays without sharing any computation.
"""

from .scenes import (  # noqa: F401
    Asset,
    Scene,
    pack_ids,
    unpack_ids,
    rgb_hash,
    ellipsoid_shell,
    capsule_shell,
    noise_voxels,
    make_asset,
    euler_xyz,
    axis_angle,
    affine12,
    pinhole_rays,
    config_seed,
    pr1_scene,
    pr1_rays,
    ArticulatedFigure,
    articulated_figure,
    static_union,
    random_rays,
    PoolAsset,
    asset_pool,
    BatchedScenes,
    batched_scenes,
    ServedScene,
    RenderRequest,
    ServingWorld,
    serving_world,
    PrecisionScene,
    precision_scene,
    grazing_rays,
    precision_rays,
)
