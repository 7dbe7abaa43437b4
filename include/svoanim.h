/*
 * svoanim.h -- C ABI of the GB300 (sm_103a) library for ray casting against
 * scenes of animated sparse voxel octrees.
 *
 * Method (Espe, Gjermundnes, Hendseth, "Efficient Animation of Sparse Voxel
 * Octrees for Real-Time Ray Tracing"): a scene is a set of static SVOs, each
 * with a pose that changes per frame (Sec. III); instead of moving voxels,
 * every ray is moved into a part's local frame by the inverse pose (Eq. 2-3);
 * parts are culled by bounding spheres (Sec. IV-A, Eq. 4) and traced front to
 * back with an early exit once the closest hit lies before the next part
 * (Sec. IV-B).
 *
 * Conventions used by every call:
 *  - Status: every call returns svo_status (0 = success, < 0 = error) and never
 *    aborts.  svo_last_error() gives a thread-local message for the last error.
 *  - Pointers are host pointers unless the comment says "device".  Host arrays
 *    are copied before the call returns; the caller keeps ownership of every
 *    array it passes.  Device buffers passed in (rays, hits, flags, stats)
 *    belong to the caller and must stay valid until the work on `stream`
 *    completes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls marked "async" only enqueue work on it.
 *  - An asset's local frame is the unit cube [0,1]^3 with the octree origin at
 *    a corner (Fig. 2).  A leaf cell (x,y,z) of a depth-D asset has voxel id
 *    x | y<<D | z<<2D.
 *  - A pose is an affine map stored row-major as 3x4 doubles [A | b]
 *    (y = A x + b).  A part's pose is relative to its parent part;
 *    parent[i] < i, or -1 for a root.  World pose = parent's world pose o local.
 *  - A ray is 8 floats: ox oy oz tmin dx dy dz tmax (Eq. 1; t in
 *    [tmin, tmax]); d need not be unit length and is never renormalised, so
 *    t means the same point in world and local space.
 *  - Device memory: the library allocates device memory for assets, scene
 *    tables and its own scratch (cudaMalloc) in svo_upload, scene_create and,
 *    when a larger ray count than before is traced, in trace_rays /
 *    trace_batch (outside any stream capture; see trace_rays).
 */
#ifndef SVOANIM_H
#define SVOANIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t svo_status;

#define SVO_OK 0
#define SVO_ERR_ARG (-1)      /* bad argument (null pointer, size, depth, parent order) */
#define SVO_ERR_OOM (-2)      /* device or host allocation failed */
#define SVO_ERR_HANDLE (-3)   /* unknown or released asset handle / scene */
#define SVO_ERR_CUDA (-4)     /* a CUDA runtime call failed (message has the CUDA error) */
#define SVO_ERR_TIMEOUT (-5)  /* reserved: a request waited past its limit.  No call of this library
                                 returns it today (no kernel waits on another); request queues built
                                 on the library (the Python server) report timeouts themselves */
#define SVO_ERR_ADMIT (-6)    /* reserved: a request does not fit the memory budget.  No call of this
                                 library returns it today; admission is the server's host policy */
#define SVO_ERR_NAN (-7)      /* NaN or infinity in a pose */
#define SVO_ERR_SINGULAR (-8) /* a composed pose is not invertible */
#define SVO_ERR_LIMIT (-9)    /* a size exceeds a documented library limit */
#define SVO_ERR_DEVICE (-10)  /* a kernel reported an internal check failure */

/* Rays (Eq. 1).  A ray must have a direction: the largest magnitude of its
 * direction's components must lie in [2^-60, 2^60], its origin and direction
 * must be finite and neither tmin nor tmax may be NaN.  Any other input is
 * not a ray and is reported as a miss (not an error). */
#define SVO_RAY_DIR_MIN 0x1p-60
#define SVO_RAY_DIR_MAX 0x1p60

/* Limits. */
#define SVO_MAX_DEPTH 16        /* octree depth of an asset (leaf level) */
#define SVO_MAX_PARTS 1024      /* parts per scene */
#define SVO_NOALLOC_MAX_RAYS 262144 /* rays per trace_rays_noalloc call (size of its fixed scratch) */

/* trace flags (bitmask).  With none set the call is the plain trace: every
 * part in index order, no sphere culling, no cross-part early exit. */
#define SVO_TRACE_CULL 1u     /* bounding-sphere culling of parts (Sec. IV-A, Eq. 4) */
#define SVO_TRACE_SORT 2u     /* visit parts by sphere entry t, stop once the hit is nearer (Sec. IV-B) */
#define SVO_TRACE_FP64_FIX 4u /* re-intersect flagged rays in FP64 and overwrite their hits */
#define SVO_TRACE_STATS 8u    /* accumulate counters into *stats (device) */
#define SVO_TRACE_DEFER_FIX 16u /* with FP64_FIX: collect flagged rays but leave the FP64 pass to
                                   trace_fix_pending (lets a caller time the two passes apart) */
#define SVO_TRACE_ORDER_DIR 32u    /* trace rays in an order grouped by direction (results unchanged) */
#define SVO_TRACE_ORDER_ORIGIN 64u /* ... grouped by origin cell, then direction (results unchanged) */
#define SVO_TRACE_IMAGE_TILES 128u /* rays are the pixels of a row-major image whose width is in bits
                                      16..31 of flags: warps take 8 x 4 pixel tiles instead of 32
                                      consecutive rays (results unchanged; ignored with ORDER_*) */
#define SVO_TRACE_IMAGE(width) (SVO_TRACE_IMAGE_TILES | ((uint32_t)(width) << 16))
#define SVO_TRACE_GRID 512u  /* cull through the scene-level grid (scenes of 64+ parts, built by every
                                refit; Sec. V-E): each ray walks the grid cells it crosses front to back,
                                tests the parts listed there once each, descends them as found and stops
                                once the next cell starts beyond its best hit.  Needs CULL | SORT; not
                                with REUSE.  Falls back to the cluster level for smaller scenes or when
                                the grid's lists overflowed (results are the same either way). */
#define SVO_TRACE_REUSE 256u /* hit buffer reuse (Sec. IV-C, Fig. 5): the hits buffer holds this scene's
                                result for the same rays from the scene's previous trace (a static
                                camera); a ray whose intersected part spheres (at most 4) all belong to
                                parts whose poses have not changed in any refit since that trace, and
                                whose previous hit was a miss or on such a part, keeps its hit without a
                                descent (ray flag SVO_RAY_REUSED).  Needs CULL | SORT | FP64_FIX, as the previous trace
                                must have had; every trace of a scene restarts its change tracking. */
#define SVO_TRACE_WAVEFRONT 1024u /* launch shape (results unchanged): the trace runs as two launches.  The
                                     first runs every ray's first culling pass (Sec. IV-A/B), writes the
                                     miss of each ray whose part spheres are all missed and queues the
                                     others with their candidate parts; the second traces the queued rays
                                     only, 32 to a warp, from those candidates on.  Pays where few rays
                                     meet a part (incoherent rays in sparse scenes), so that a warp of the
                                     fused launch descends with few lanes.  Needs CULL | SORT; not with
                                     REUSE or GRID.  The queue (64 bytes per ray of the largest launch) is
                                     per-stream scratch, grown like the FP64 list. */
#define SVO_TRACE_DEFAULT (SVO_TRACE_CULL | SVO_TRACE_SORT | SVO_TRACE_FP64_FIX)

/* per-ray flags written when ray_flags != NULL */
#define SVO_RAY_UNCERTAIN 1u /* FP32 could not certify which leaf is hit first (near tie / grazing) */
#define SVO_RAY_FIXED 2u     /* the hit was recomputed in FP64 */
#define SVO_RAY_T_REFINED 4u /* the ids were certified but the FP32 t interval was wider than 2^-17 of
                                max(t, leaf diagonal / |d|): t is recomputed in FP64 (FP64_FIX), else
                                bits 8-15 hold a certified error bound (SVO_RAY_T_BOUND_EXP) */
/* For a ray flagged SVO_RAY_T_REFINED and not SVO_RAY_FIXED: with e = SVO_RAY_T_BOUND_EXP(flags),
 * |t - t_exact| <= 2^e * max(t_exact, h / |d|) * (1 + 2^-18), h being the world length of the hit
 * part's leaf diagonal (t_exact: the closed-box entry in exact arithmetic; the bound comes from
 * the FP32 pass's rounding-error analysis; the last factor covers the FP32 evaluation of h / |d|).
 * A biased value of 255 means no finite bound. */
#define SVO_RAY_T_BOUND_EXP(flags) ((int32_t)(((flags) >> 8) & 0xFFu) - 128)
#define SVO_RAY_REUSED 8u    /* SVO_TRACE_REUSE kept the previous hit (no descent) */

typedef struct svo_ctx svo_ctx;
typedef struct svo_scene svo_scene;
typedef uint32_t svo_handle;

/* One static SVO given by its occupied finest-level cells. */
typedef struct {
  int32_t depth;              /* 1..SVO_MAX_DEPTH */
  uint64_t n_leaves;          /* number of entries in leaf_ids (duplicates allowed) */
  const uint64_t *leaf_ids;   /* host; voxel ids x | y<<D | z<<2D */
  const uint32_t *leaf_rgb;   /* host, may be NULL; 0x00RRGGBB per entry of leaf_ids */
} svo_desc;

/* Closest hit of one ray: 16 bytes.  Miss: t = +inf, part = 0xFFFFFFFF,
 * voxel = UINT64_MAX.  Equal t is broken by smaller part, then smaller voxel. */
typedef struct {
  float t;
  uint32_t part;
  uint64_t voxel;
} svo_hit;

/* Counters accumulated (atomically, on the device) when SVO_TRACE_STATS is set. */
typedef struct {
  unsigned long long rays;          /* rays traced */
  unsigned long long flagged;       /* rays flagged SVO_RAY_UNCERTAIN (ids not certified) */
  unsigned long long fixed;         /* rays recomputed in FP64 */
  unsigned long long parts_tested;  /* (ray, part) sphere tests */
  unsigned long long parts_entered; /* (ray, part) traversals started */
  unsigned long long nodes_visited; /* interior node descriptors fetched (8 B each) */
  unsigned long long leaves_tested; /* leaf cells slab-tested */
  unsigned long long passes;        /* candidate-list passes (> rays when lists overflow) */
  unsigned long long flag_winner;   /* flagged because the nearest candidate was not certainly hit */
  unsigned long long flag_overlap;  /* flagged because another candidate's entry bound reached it */
  unsigned long long flag_width;    /* ids certified, but the winner's t interval was too wide (T_REFINED) */
  unsigned long long reused;        /* rays that kept their previous hit (SVO_TRACE_REUSE) */
} svo_trace_stats;

/* A pinhole camera for svo_raygen_pinhole. */
typedef struct {
  float eye[3];     /* centre of projection */
  float target[3];  /* a point on the optical axis */
  float up[3];      /* approximate up direction */
  float fov_y_deg;  /* vertical field of view, degrees, in (0, 180) */
  float tmin, tmax; /* ray segment written into every ray */
} svo_camera;

/* One entry of a batched trace (trace_batch). */
typedef struct {
  svo_scene *scene;
  const float *rays;   /* device, 8 floats per ray */
  uint64_t n;          /* number of rays */
  svo_hit *hits;       /* device, n entries */
  uint32_t *ray_flags; /* device, n entries, or NULL */
  uint32_t image_width; /* rays are a row-major image of this width (0: no image layout); it
                           replaces the width bits of the trace_batch flags for this item */
} svo_batch_item;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` (makes it current for the calling
 * thread).  *out receives the context; destroy it with svo_ctx_destroy. */
svo_status svo_ctx_create(int32_t device, svo_ctx **out);
/* Release every asset, scene and buffer of the context.  NULL is allowed. */
svo_status svo_ctx_destroy(svo_ctx *ctx);
/* Thread-local message of the last failing call of this thread ("" if none).
 * It takes no context: a call can fail before any context exists (a NULL or
 * bad context, svo_ctx_create itself), and one thread's message must not be
 * overwritten by another thread's call on the same context. */
const char *svo_last_error(void);
/* Static name of a status code. */
const char *svo_status_string(svo_status s);
/* Launch shape of the trace kernel for this context's later traces: threads
 * per block (64, 128 or 256) and rays per lane of a warp's tile (1, 2, 4 or 8;
 * a warp takes 32 * rays_per_lane rays at a time from the work counter).
 * Results do not depend on it; the autotuner picks it.  Default 128 / 1. */
svo_status svo_set_trace_config(svo_ctx *ctx, int32_t block, int32_t rays_per_lane);
svo_status svo_get_trace_config(svo_ctx *ctx, int32_t *block, int32_t *rays_per_lane);
/* Top octree levels (0..4) that each thread block of a one-scene trace
 * (trace_rays, or trace_batch whose items all trace one scene of at most
 * 256 parts) copies into shared memory at start, so that the first node
 * fetches of every descent are served on chip (the paper's traversal starts
 * every ray at the root, Sec. IV-B).  Fewer levels are staged when a scene's
 * top nodes would exceed 16 KB.  Results do not depend on it; the autotuner
 * picks it.  Default 0. */
svo_status svo_set_smem_levels(svo_ctx *ctx, int32_t levels);
/* The order in which the persistent trace kernel's warps claim the 8 x 4
 * pixel tiles of image rays (SVO_TRACE_IMAGE, or a batch item's
 * image_width): row by row, or centre-out (tiles sorted by the distance of
 * their centres from the image centre).  A tile's cost is set by its slowest
 * ray, and the kernel ends when its last tile does; claiming the tiles where
 * the scene usually is (a camera aimed at it) first leaves cheap tiles to fill
 * the end of the launch.  Results do not depend on it; the autotuner picks
 * it.  The centre-out table of each image shape is built once per context
 * (cudaMalloc on the first trace of that shape).  Default centre-out. */
#define SVO_TILE_ORDER_ROWS 0
#define SVO_TILE_ORDER_CENTER 1
svo_status svo_set_tile_order(svo_ctx *ctx, int32_t order);
svo_status svo_get_tile_order(svo_ctx *ctx, int32_t *order);
svo_status svo_get_smem_levels(svo_ctx *ctx, int32_t *levels);
/* Read and clear the context's device error word (synchronises the device).
 * Returns SVO_OK, or SVO_ERR_DEVICE with the failing check in the message. */
svo_status svo_check_device(svo_ctx *ctx);

/* ----------------------------------------------------------------- assets */

/* Host-only octree build of the node layout, for inspection (no GPU needed).
 * Node layout (a simplified Laine-Karras child descriptor, Sec. II-B, V):
 * 8 bytes per interior node, nodes in breadth-first order, root first:
 *   uint32 first_child; uint8 child_mask; uint8 leaf_mask; uint16 zero.
 * Bit k of child_mask is octant k (bit0 = +x half, bit1 = +y, bit2 = +z).
 * The children of a node are stored contiguously in ascending octant order;
 * child k is at first_child + popcount(child_mask & ((1<<k)-1)).  At level
 * D-1 the children are leaves: leaf_mask == child_mask and first_child indexes
 * the leaf payload array (one 0x00RRGGBB per leaf, same order).
 * Call with nodes == NULL to get *n_nodes and *n_leaves; then call again with
 * nodes (n_nodes * 8 bytes) and rgb (n_leaves entries, may be NULL). */
svo_status svo_build_host(const svo_desc *desc, uint64_t *n_nodes, uint64_t *n_leaves, void *nodes,
                          uint32_t *rgb);
/* Build an asset from a leaf list and upload it (synchronous).  The library
 * owns the device copy until svo_release.  *out receives the handle. */
svo_status svo_upload(svo_ctx *ctx, const svo_desc *desc, svo_handle *out);
/* Free an asset.  Scenes that still reference it must be destroyed first
 * (SVO_ERR_ARG otherwise). */
svo_status svo_release(svo_ctx *ctx, svo_handle h);
/* Depth, interior node count and leaf count of an asset (any pointer may be NULL). */
svo_status svo_asset_info(svo_ctx *ctx, svo_handle h, int32_t *depth, uint64_t *n_nodes, uint64_t *n_leaves);
/* Copy an asset's device data back to the host (synchronous; the device
 * synchronises with the copy): its n_nodes interior node descriptors (8 bytes
 * each, the svo_build_host layout) into `nodes` and its n_leaves leaf colours
 * into `rgb`.  Either pointer may be NULL to skip it.  Poses, refits and
 * traces never write an asset: the data read back is what svo_upload stored. */
svo_status svo_read_asset(svo_ctx *ctx, svo_handle h, void *nodes, uint32_t *rgb);

/* ----------------------------------------------------------------- scenes */

/* A scene of n_parts parts; part i instances asset[i] and hangs below
 * parent[i] (< i, or -1).  Poses start as identities. */
svo_status scene_create(svo_ctx *ctx, int32_t n_parts, const svo_handle *asset, const int32_t *parent,
                        svo_scene **out);
svo_status scene_destroy(svo_scene *scene);
/* Set every part's local pose (host, n_parts*12 doubles, parent <- part).
 * The array is copied before return.  Scenes of up to 256 parts pass the
 * poses to the device inside the next scene_refit launch (kernel
 * parameters, no separate copy); larger scenes copy them to the device on
 * `stream` through pinned staging.  SVO_ERR_NAN if any entry is NaN/inf. */
svo_status scene_set_transforms(svo_scene *scene, const double *local_3x4, void *stream);
/* Same from a device array (n_parts*12 doubles); no check for NaN. */
svo_status scene_set_transforms_device(svo_scene *scene, const double *local_3x4_dev, void *stream);
/* Poses in the form of Sec. III-B: a rigid motion plus per-axis octree
 * dimensions.  Per part 15 doubles (host, copied before return): R (3x3,
 * row-major, orthonormal: every entry of R R^T - I within 1e-9), t (3),
 * s (3, each > 0): the part's octree spans [0,s_x] x [0,s_y] x [0,s_z] in the
 * frame rotated by R and moved by t, i.e. the local pose is
 * [R diag(s) | t] (x_parent = R (s * x_unit) + t).  The animation transform
 * stays rigid (its inverse is R^T and -R^T t, Sec. III-A); the dimensions
 * are the traversal's octree dimensions, which for the parametric descent
 * equal scaling the rigidly mapped ray by 1/s per axis.  Results equal
 * scene_set_transforms with that local pose.  SVO_ERR_NAN if any entry is
 * not finite, SVO_ERR_ARG if R is not orthonormal or a dimension is not
 * positive; nothing is changed then. */
svo_status scene_set_transforms_trs(svo_scene *scene, const double *rts_15, void *stream);
/* Per-frame pose pipeline (async, one small kernel): compose the transform
 * tree in FP64 (W_i = W_parent o L_i), invert in FP64 (Eq. 3; adjugate /
 * determinant, which reduces to transpose-and-negate for a rigid pose), emit
 * the FP32 world->local rows used by tracing, refit the part bounding spheres
 * (centre = image of the cube centre, radius = farthest image corner,
 * Sec. IV-A) and rebuild the cluster level of the sphere hierarchy.  A
 * singular pose sets the device error word (svo_check_device). */
svo_status scene_refit(svo_scene *scene, void *stream);
/* scene_refit of n scenes of one context in one launch, a thread block per
 * scene (async; Sec. III, Eq. 3, Sec. IV-A as scene_refit).  Each scene's
 * refit is the same as scene_refit's, so the results are identical; the
 * batch runs the scenes side by side on the GPU instead of one launch after
 * another, for a frame that poses many scenes (a server's batch of
 * requests, a batched trace).  scenes: n distinct scene handles.  local_dev:
 * NULL, or n pointers, each NULL or a device array of that scene's
 * n_parts*12 local poses (as scene_set_transforms_device, read by the
 * launch, which also keeps the scene's own copy); a scene without one uses
 * the poses its last scene_set_transforms / _device call set (host poses of
 * a scene of at most 256 parts are read by the launch from the scene's
 * page-locked staging buffer).  Launches of up to 64 scenes each. */
svo_status scene_refit_batch(svo_scene *const *scenes, const double *const *local_dev, int32_t n, void *stream);
/* Copy the last refit's per-part data to host arrays (any may be NULL) and
 * synchronise `stream`: world and inverse poses (n_parts*12 doubles each,
 * [A | b] rows), the FP32 rows used by tracing (n_parts*12 floats: the
 * inverse matrix rounded to FP32 in columns 0-2 and, in column 3, the local
 * coordinates of the FP32 sphere centre), FP32 spheres (n_parts*4 floats:
 * cx cy cz r). */
svo_status scene_read_poses(svo_scene *scene, double *world, double *inv, float *inv_f32, float *sphere,
                            void *stream);
/* Number of clusters of the sphere hierarchy and, if the arrays are not NULL,
 * the cluster spheres (n_clusters*4 floats) and the part order
 * (n_parts ints; cluster c holds order[8c .. 8c+7]).  Synchronises `stream`. */
svo_status scene_read_clusters(svo_scene *scene, int32_t *n_clusters, float *sphere, int32_t *order,
                               void *stream);

/* ------------------------------------------------------------------ trace */

/* Closest hit (t, part, voxel) of n rays (async).  rays: device, 8 floats per
 * ray; hits: device, n svo_hit; ray_flags: device, n uint32 or NULL;
 * stats: device svo_trace_stats or NULL (used with SVO_TRACE_STATS; the caller
 * zeroes it).  Traversal runs in FP32; a ray whose closest hit FP32 cannot
 * certify (the error-bounded intervals of two candidates overlap) is flagged
 * SVO_RAY_UNCERTAIN; a ray whose ids are certified but whose winner's t
 * interval is wider than 2^-17 of max(t, leaf diagonal / |d|) is flagged
 * SVO_RAY_T_REFINED; with SVO_TRACE_FP64_FIX both are re-intersected in FP64.  The scene must have been
 * refitted since its last scene_set_transforms.  If n exceeds the largest n
 * traced so far on this context the call grows the context's scratch with
 * cudaMalloc, so call it once at full size before capturing a CUDA graph. */
svo_status trace_rays(svo_scene *scene, const float *rays, uint64_t n, svo_hit *hits, uint32_t *ray_flags,
                      uint32_t flags, svo_trace_stats *stats, void *stream);
/* (With SVO_TRACE_ORDER_DIR / _ORIGIN the rays are first counting-sorted by a
 * 14-bit direction / origin-cell key into per-stream scratch, grown like the
 * FP64 list; hits still land at each ray's own index.) */
/* Batched trace: every item's rays against its own scene, in one persistent
 * launch whose thread blocks take fixed-size tiles of rays from a device work
 * counter (async), or -- with SVO_TRACE_WAVEFRONT -- in a culling launch and a
 * descent launch over all items' queued rays.  Items may reference different
 * scenes of the context; flags and per-stream scratch are those of
 * trace_rays, sized to the batch's total ray count. */
svo_status trace_batch(svo_ctx *ctx, const svo_batch_item *items, int32_t n_items, uint32_t flags,
                       svo_trace_stats *stats, void *stream);

/* trace_rays for rays and hits in HOST memory (async on `stream`).
 *   * Batches of at most 262144 rays in page-locked buffers mapped into the
 *     device's address space (e.g. cudaHostAlloc'ed; on GB300 reached over
 *     the chip-to-chip link) are read and written by the kernels directly,
 *     with no staging copy: the lowest latency for one call.
 *   * Larger batches are copied in by the copy engines, to one of two
 *     per-stream staging halves that successive calls alternate between.  A
 *     call's copy-in waits only until its half is free (the call two before
 *     has finished with it), not for earlier work on `stream`, so in a frame
 *     loop the next frame's rays stream in while the current frame is
 *     traced.  The trace waits for earlier work on `stream` (poses, refit).
 *     The rays are therefore read at some time between the call and the
 *     completion of its work on `stream`: leave them unchanged until then.
 *     - Mapped page-locked hits (and ray_flags, if not NULL) are written by
 *       the kernels directly, and the rays are traced in one launch.
 *     - Other hits buffers are staged as well: chunks of about 512 K rays
 *       (whole image rows with SVO_TRACE_IMAGE) are copied in, traced and
 *       copied back through three internal streams, so that one chunk's
 *       copies overlap another's trace.  Pageable buffers make the copies
 *       block the host.
 *     `stream` resumes once every hit is back.  The staging grows with
 *     cudaMalloc when n exceeds the largest n staged so far on this stream.
 * The call returns before the work finishes: synchronise `stream` before
 * reading hits.  SVO_TRACE_STATS and SVO_TRACE_REUSE are not supported here
 * (SVO_ERR_ARG); SVO_TRACE_DEFER_FIX is ignored. */
svo_status trace_rays_host(svo_scene *scene, const float *rays_host, uint64_t n, svo_hit *hits_host,
                           uint32_t *ray_flags_host, uint32_t flags, void *stream);

/* trace_rays for callers that cannot allocate device memory -- for example a
 * frame loop with a hard deadline, where cudaMalloc may synchronise the
 * device, or a host application whose own allocator owns all device memory.
 * (The paper has no counterpart; this is a deployment variant.)  Same
 * arguments and results as trace_rays without `stats`; SVO_TRACE_STATS,
 * SVO_TRACE_DEFER_FIX, the ray-order flags SVO_TRACE_ORDER_DIR /
 * SVO_TRACE_ORDER_ORIGIN and SVO_TRACE_WAVEFRONT (which need per-ray scratch)
 * are rejected (SVO_ERR_ARG).  It never calls cudaMalloc
 * or cudaFree: its scratch (about 15.7 MB) is a static device array inside the
 * library that every GPU loading the library holds until the process exits.
 * n above SVO_NOALLOC_MAX_RAYS returns SVO_ERR_LIMIT.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array: the
 * counters are cleared on `stream` at every call, and two calls whose work
 * overlaps on the GPU (other streams or host threads) race -- serialise
 * them.  The looked-up address is kept for the life of the process: do not
 * reset the device (cudaDeviceReset) while the library is loaded. */
svo_status trace_rays_noalloc(svo_scene *scene, const float *rays, uint64_t n, svo_hit *hits,
                              uint32_t *ray_flags, uint32_t flags, void *stream);

/* Primary rays of a pinhole camera, one per pixel (async): pixel (i, j) of a
 * width x height image -> ray j*width + i in `rays` (device, 8 floats per
 * ray, 16-byte aligned) with unit directions through the pixel centres.  This
 * prepares inputs on the device (e.g. for served render requests); it is not
 * part of the paper's method. */
svo_status svo_raygen_pinhole(svo_ctx *ctx, const svo_camera *cam, uint32_t width, uint32_t height, float *rays,
                              void *stream);

/* Colour of hits (async): rgb[i] = the 0x00RRGGBB payload of the leaf that
 * hits[i] names in part hits[i].part of `scene` (the colour the paper's hit
 * buffer carries for shading, Sec. IV-C), or `background` for a miss.  The
 * leaf's colour is the one given for the first occurrence of its id in the
 * svo_desc leaf list (0 if the asset was uploaded without colours).
 *   hits: device, n svo_hit (16-byte aligned), e.g. the output of trace_rays
 *         once its FP64 pass has run (issue both on the same stream);
 *   rgb:  device, n uint32 (4-byte aligned), written by the library.
 * A hit that names no occupied leaf of the scene (part out of range, voxel
 * outside the asset's grid or not a leaf) gets SVO_COLOR_INVALID.
 * SVO_ERR_ARG for NULL or misaligned buffers with n > 0, or a background
 * above 0x00FFFFFF. */
#define SVO_COLOR_INVALID 0xFFFFFFFFu
svo_status trace_hit_colors(svo_scene *scene, const svo_hit *hits, uint64_t n, uint32_t background, uint32_t *rgb,
                            void *stream);

/* Shaded image of hits (async): rgb[i] = the hit leaf's colour lit by a
 * directional light, as 0x00RRGGBB; `background` for a miss; SVO_COLOR_INVALID
 * where trace_hit_colors gives it.  The normal is the face of the leaf's box
 * through which ray i enters (the axis whose near-plane parameter is largest,
 * the lower axis on a tie), mapped to world space by the inverse transpose of
 * the part's pose; a ray that starts inside the leaf takes -d.  Each channel c
 * becomes min(255, floor(c * s + 1/2)) with s = ambient + (1 - ambient) *
 * max(0, n . l), l = light / |light|, evaluated in FP64 (the shading inputs the
 * paper's hit buffer carries, Sec. IV-C).
 *   rays: device, n rays (8 floats, 16-byte aligned), those that were traced;
 *   hits: device, n svo_hit (16-byte aligned), trace_rays' output after its
 *         FP64 pass (issue both on the same stream);
 *   light: host, 3 floats, the direction towards the light (any length > 0);
 *   rgb:  device, n uint32 (4-byte aligned).
 * SVO_ERR_ARG for NULL or misaligned buffers with n > 0, a zero or
 * non-finite light, an ambient outside [0, 1] or a background above
 * 0x00FFFFFF. */
svo_status trace_shade(svo_scene *scene, const float *rays, const svo_hit *hits, uint64_t n, const float *light,
                       float ambient, uint32_t background, uint32_t *rgb, void *stream);

/* Run the FP64 re-intersection pass left pending by the last trace_rays /
 * trace_batch issued on `stream` with SVO_TRACE_FP64_FIX | SVO_TRACE_DEFER_FIX
 * (async).  No-op (SVO_OK) if nothing is pending on that stream. */
svo_status trace_fix_pending(svo_ctx *ctx, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* SVOANIM_H */
