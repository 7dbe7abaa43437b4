// svo_internal.h -- device data layouts shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "svoanim.h"

namespace svo {

constexpr uint32_t kMissPart = 0xFFFFFFFFu;
constexpr unsigned long long kMissVoxel = 0xFFFFFFFFFFFFFFFFull;
constexpr int kMaxDepth = SVO_MAX_DEPTH;
constexpr int kMaxParts = SVO_MAX_PARTS;
constexpr int kClusterSize = 8;                 // parts per sphere-hierarchy cluster
constexpr int kMaxClusters = kMaxParts / kClusterSize;
constexpr int kMaxBatchItems = 128;             // items per trace launch (kernel parameter space)
constexpr int kContenders = 16;                 // contender leaves kept per flagged ray
constexpr unsigned long long kPoolPerRay = 3;   // FP64-pass leaf pool entries per ray of scratch capacity
constexpr int kInlinePoseParts = 256;           // poses up to this many parts go by kernel parameter
constexpr int kMaxSmemLevels = 4;               // top octree levels a trace block may stage in shared memory
constexpr size_t kTopCapBytes = 16384;          // at most this many bytes of staged top-level nodes per block

// Device error word bits (svo_check_device reports them).
constexpr unsigned int kErrNodeIndex = 1u;      // a child index fell outside the node array
constexpr unsigned int kErrFixOverflow = 2u;    // the FP64 re-intersection list overflowed
constexpr unsigned int kErrSingular = 4u;       // a composed pose was not invertible
constexpr unsigned int kErrStack = 8u;          // traversal stack exceeded kMaxDepth

// Static per-part data written at scene_create.
struct PartStatic {
  const uint2 *nodes;   // asset's interior nodes (8 B each, breadth-first)
  uint32_t n_nodes;
  int32_t depth;
  int32_t parent;
  int32_t pad;
  const uint32_t *rgb;  // leaf payload, indexed like the leaf-level children
  unsigned long long n_leaves;
  float box_lo[3];      // local box of the occupied leaves (exact: multiples of 2^-depth);
  float box_hi[3];      // the bounding sphere is fitted to it (empty asset: lo = hi = 0)
};

// Per-frame FP32 data of a part used by the trace kernel (64 B, staged in
// shared memory).  rows .xyz: the FP32 world->local matrix Ainv; rows .w: the
// local coordinates of the FP32 sphere centre (computed in FP64), so that a
// world point q maps to Ainv (q - c) + rows.w with only small numbers
// cancelling; sphere: conservative bounding sphere (c, r) in world space.
struct PartHot {
  float4 r0, r1, r2;
  float4 sphere;
};

// Per-frame scalars of a part (64 B).  In a trace block's shared-memory
// copy, spare0 / spare1 carry (as bits) the first and the count of the part's
// nodes staged in shared memory; in global memory both are 0.
struct PartAux {
  const uint2 *nodes;
  uint32_t n_nodes;
  int32_t depth;
  float n_ainv;      // upper bound of ||Ainv||_inf (max abs row sum of the FP32 rows)
  float hdiag;       // world length of a leaf's diagonal, |A (1,1,1)| 2^-depth
  float spare0, spare1;
  float box_lo[3];   // local box of the occupied leaves (PartStatic), where the descent starts
  float box_hi[3];
  float pad[2];
};
static_assert(sizeof(PartAux) == 64, "PartAux is 64 bytes");

// Cluster of up to kClusterSize parts (consecutive in `order`).
struct Cluster {
  float4 sphere;  // encloses the member spheres
  float4 aux;     // .x max n_ainv of the members, .w bits: first | count << 16
};

// Scene-level grid over the parts (the "larger structure" the paper suggests
// for scenes of many parts, Sec. V-E): a uniform G^3 grid over the part
// spheres, rebuilt on demand after each refit (k_grid.cu).  Cell c lists, in
// increasing part order, the parts whose sphere box comes within 2^-10 cells
// of it: cell_parts[cell_start[c] .. cell_start[c + 1]).
struct SceneGrid {
  float lo[3];      // grid corner
  float cs[3];      // cell size per axis
  float inv_cs[3];  // 1 / cs
  int32_t G;        // cells per axis
  int32_t valid;    // 0: the lists overflowed or the grid is too far from the origin: trace by clusters
  int32_t cap;      // capacity of cell_parts
  int32_t stale;    // 1: a refit changed the spheres since the last build
  int32_t *cell_start;  // G^3 + 1
  int32_t *cell_parts;
};
constexpr int kGridMinParts = 64;  // scenes from this size on get a grid
constexpr int kGridMaxG = 16;

// One item of a trace launch (by value in the kernel parameters).
struct TraceItem {
  const PartHot *hot;
  const PartAux *aux;
  const Cluster *clusters;
  const int32_t *order;
  const double *inv64;  // FP64 world->local rows (12 per part)
  const float4 *rays;   // 2 float4 per ray
  uint4 *hits;          // svo_hit per ray
  uint32_t *ray_flags;  // or nullptr
  const uint32_t *perm; // visiting order of the rays (nullptr = index order)
  const uint8_t *dirty; // per part: pose changed since the scene's previous trace (SVO_TRACE_REUSE)
  const SceneGrid *grid;  // scene-level grid (SVO_TRACE_GRID), or nullptr
  unsigned long long n;
  unsigned long long tile_begin;
  int32_t n_parts;
  int32_t n_clusters;
  int32_t max_depth;  // deepest asset among the scene's parts
  uint32_t width;     // rays are a row-major image of this width (tiles of 8 x 4*rays_per_lane pixels), or 0
  uint32_t tiles_x;   // tiles per image row band (width > 0)
  int32_t pad;
  const uint32_t *tile_order;  // image tiles: claim order, entry tx | ty << 16 (nullptr: row by row)
  unsigned long long qbase;    // SVO_TRACE_WAVEFRONT: the item's first entry in the ray queue
};

// SVO_TRACE_WAVEFRONT: a ray whose first culling pass found candidate parts,
// queued by the culling launch for the descent launch (64 B).
struct QueueEntry {
  uint4 id;   // .x | .y << 32: the ray's index in its item; .z: bits of the smallest sphere entry that
              // did not fit the list (infinity: none); .w: unused
  float4 ct;  // sphere entry t of up to four candidates, increasing (infinity: no candidate)
  float4 ce;  // the reference parameter of each candidate's descent
  int4 cp;    // the candidates' part ids
};
static_assert(sizeof(QueueEntry) == 64, "QueueEntry is 64 bytes");
constexpr int kQueueCountWords = 4;  // per-stream counters before the per-item queue counts (64-bit words)

// Warp tiles of every item, laid out one item after another: sets each
// item's tile_begin (and tiles_x) and returns the total.  A tile is
// 32 * rays_per_lane consecutive rays, or, for an image of width >= 8, a block
// of 8 x 4*rays_per_lane pixels (the last row band and column may be partial).
template <typename Item>
inline unsigned long long layout_tiles(Item *items, int n_items, int rays_per_lane) {
  unsigned long long tiles = 0;
  const unsigned long long tile = 32ull * (unsigned long long)rays_per_lane;
  for (int i = 0; i < n_items; ++i) {
    Item &it = items[i];
    it.tile_begin = tiles;
    it.tiles_x = 0;
    unsigned long long t = (it.n + tile - 1) / tile;
    if (it.width >= 8u && !it.perm) {
      const unsigned long long tx = (it.width + 7ull) / 8ull, rows = (it.n + it.width - 1) / it.width;
      const unsigned long long band = 4ull * (unsigned long long)rays_per_lane;
      const unsigned long long t2 = tx * ((rows + band - 1) / band);
      if (t2 < (1ull << 32)) {
        t = t2;
        it.tiles_x = (uint32_t)tx;
      }
    }
    tiles += t;
  }
  return tiles;
}

struct TraceLaunch {
  TraceItem items[kMaxBatchItems];
  int32_t n_items;
  uint32_t flags;
  unsigned long long n_tiles;
  unsigned long long *tile_counter;   // zeroed before the launch
  unsigned long long *fix_list;       // (count << 48) | (item << 40) | ray, capacity fix_capacity
  unsigned int *fix_count;            // zeroed before the launch
  unsigned long long fix_capacity;
  uint4 *fix_cand;                    // pool of the leaves stored per list slot (fix_off)
  unsigned long long cand_capacity;   // pool entries
  unsigned int *cand_count;           // pool entries taken; zeroed before the launch
  uint32_t *fix_off;                  // per list slot: first pool entry, or 0xFFFFFFFF
  svo_trace_stats *stats;
  unsigned int *err;
  int32_t block;          // trace kernel block size: 64, 128 or 256
  int32_t rays_per_lane;  // warp tile = 32 * rays_per_lane rays
  const int2 *top;        // per part (first, count) of its staged top-level nodes, or nullptr
  int32_t top_nodes;      // nodes staged in shared memory per block (0: none)
  int32_t top_levels;     // the top levels of every part that are staged
  QueueEntry *queue;                  // SVO_TRACE_WAVEFRONT: entries of every item, item i from items[i].qbase
  unsigned int *queue_count;          // SVO_TRACE_WAVEFRONT: per item, entries queued; zeroed before the launch
  unsigned long long *queue_tile;     // SVO_TRACE_WAVEFRONT: tile counter of the descent launch; zeroed
};

// Kernel launchers (k_trace.cu, k_refit.cu).
cudaError_t launch_trace(const TraceLaunch &L, int n_sm, cudaStream_t stream);
cudaError_t launch_fix(const TraceLaunch &L, int n_sm, cudaStream_t stream);

// Leaf colours of n hits (k_color.cu); see trace_hit_colors.
cudaError_t launch_hit_colors(const uint4 *hits, unsigned long long n, const PartStatic *stat, int n_parts,
                              uint32_t background, uint32_t *rgb, int n_sm, cudaStream_t stream);

// Lambert shading of n hits (k_color.cu); see trace_shade.
struct ShadeArgs {
  double light[3];  // unit direction towards the light
  double ambient;   // in [0, 1]
  uint32_t background;
};
cudaError_t launch_shade(const float4 *rays, const uint4 *hits, unsigned long long n, const PartStatic *stat,
                         const double *inv64, int n_parts, const ShadeArgs &sa, uint32_t *rgb, int n_sm,
                         cudaStream_t stream);

struct RaygenArgs {
  float eye[3], f[3], r[3], u[3];  // camera origin and unit forward / right / up
  float tan_x, tan_y, inv_w, inv_h, tmin, tmax;
  uint32_t width, height;
};
cudaError_t launch_raygen(const RaygenArgs &a, float *rays, int n_sm, cudaStream_t stream);
size_t order_scratch_bytes(unsigned long long n);
// mode 1: by direction, 2: by origin cell then direction; *perm_out points into scratch.
cudaError_t launch_order(const float *rays, unsigned long long n, int mode, const float4 *bound, void *scratch,
                         uint32_t **perm_out, int n_sm, cudaStream_t stream);
// One item of a batched ordering: its rays, its scene bound and its part of
// the scratch (order_scratch_bytes(n) bytes, carved by order_item).
struct OrderItem {
  const float4 *rays;
  unsigned long long n;
  const float4 *bound;
  unsigned int *hist;
  uint16_t *keys;
  uint32_t *perm;  // the item's permutation once the launches have run
};
OrderItem order_item(const float *rays, unsigned long long n, const float4 *bound, void *scratch);
// The orderings of up to kMaxBatchItems items in four launches in all.
cudaError_t launch_order_batch(const OrderItem *items, int n_items, int mode, int n_sm, cudaStream_t stream);

struct RefitArgs {
  int32_t n_parts;
  int32_t n_levels;
  const int32_t *level_order;  // parts grouped by tree level
  const int32_t *level_start;  // n_levels + 1
  const PartStatic *stat;
  const double *local;         // parent <- part, 12 per part
  double *world;
  double *inv64;
  PartHot *hot;
  PartAux *aux;
  Cluster *clusters;
  int32_t *order;
  int32_t n_clusters;
  float4 *bound;  // sphere enclosing every part sphere (ray-ordering frame)
  uint8_t *dirty; // set to 1 for every part whose world pose changes (cleared by each trace)
  SceneGrid *grid;        // marked stale by the refit (nullptr: no grid)
  unsigned int *err;
};
// host_local: when not NULL and n_parts <= kInlinePoseParts, the local poses
// travel in the kernel parameters instead of through a device copy.
cudaError_t launch_refit(const RefitArgs &a, const double *host_local, cudaStream_t stream);
// Scenes per launch of scene_refit_batch (kernel parameter space).
constexpr int kRefitBatch = 64;
// n <= kRefitBatch scenes in one launch, one block each; src[i]: where scene
// i's local poses are read from (device or mapped host memory), or nullptr
// for args[i].local.
cudaError_t launch_refit_batch(const RefitArgs *args, const double *const *src, int n, cudaStream_t stream);

// Grid (re)builds before a trace with SVO_TRACE_GRID: one block per distinct
// scene, each a no-op unless the scene's grid is stale.
struct GridJob {
  const PartHot *hot;
  SceneGrid *grid;
  int32_t n_parts;
  int32_t G;
};
struct GridLaunch {
  GridJob jobs[kMaxBatchItems];
  int32_t n_jobs;
};
size_t grid_smem_bytes(int G);
cudaError_t launch_grid(const GridLaunch &L, cudaStream_t stream);

// Cells per axis of a scene's grid: about 2 P^(1/3) (8 cells per part), at
// most kGridMaxG; 0 (no grid) below kGridMinParts parts.
inline int grid_cells_per_axis(int n_parts) {
  if (n_parts < kGridMinParts) return 0;
  int G = 2;
  while (G < kGridMaxG && G * G * G < 8 * n_parts) ++G;
  return G;
}

// The grid jobs of a trace launch's items: one per distinct scene grid.
inline int grid_jobs(const TraceItem *items, int n_items, GridLaunch &g) {
  g.n_jobs = 0;
  for (int i = 0; i < n_items; ++i) {
    if (items[i].grid == nullptr) continue;
    bool seen = false;
    for (int j = 0; j < g.n_jobs; ++j) seen = seen || g.jobs[j].grid == items[i].grid;
    if (seen) continue;
    GridJob &job = g.jobs[g.n_jobs++];
    job.hot = items[i].hot;
    job.grid = const_cast<SceneGrid *>(items[i].grid);
    job.n_parts = items[i].n_parts;
    job.G = grid_cells_per_axis(items[i].n_parts);
  }
  return g.n_jobs;
}

}  // namespace svo
