// svo_api.cu -- C ABI of the library (declared in include/svoanim.h).
//
// Host-side responsibilities: argument checks, asset and scene tables,
// device memory, staging of per-frame poses, and kernel launches.  Every
// per-ray step runs in the kernels of k_trace.cu; the per-frame pose
// pipeline runs in k_refit.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "svo_build.h"
#include "svo_internal.h"

namespace svo {
cudaError_t init_trace_tables(cudaStream_t stream);
}

using namespace svo;

namespace {

thread_local std::string g_last_error;

svo_status fail(svo_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

svo_status ok() { return SVO_OK; }

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(SVO_ERR_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                                       __FILE__, __LINE__);                                        \
  } while (0)

struct AssetRec {
  bool live = false;
  int depth = 0;
  uint64_t n_nodes = 0, n_leaves = 0;
  uint2 *d_nodes = nullptr;
  uint32_t *d_rgb = nullptr;
  float box_lo[3] = {0.f, 0.f, 0.f}, box_hi[3] = {0.f, 0.f, 0.f};  // occupied leaves, local units
  uint32_t top_nodes[kMaxSmemLevels + 1] = {};  // interior nodes in its top 0..kMaxSmemLevels levels
  int refs = 0;
};

// trace_rays_host: batches up to this size in mapped page-locked memory are
// traced in place (zero copy); larger ones go through the staged pipeline
constexpr unsigned long long kZeroCopyMaxRays = 1ull << 18;

// One staging half of trace_rays_host for n rays: rays | hits | flags,
// rounded so that the second half starts 256-byte aligned.
inline size_t stage_half_bytes(unsigned long long n) { return ((size_t)n * (32 + 16 + 4) + 255) & ~(size_t)255; }

constexpr size_t kCounterWords = kQueueCountWords + kMaxBatchItems / 2;

// Scratch of one stream: launch counters and the FP64 re-intersection list.
struct Slot {
  // [0] tile counter, [1] fix count (low 32 bits), [2] pool count, [3] tile counter of the wavefront
  // descent launch, then kMaxBatchItems 32-bit queue counts
  unsigned long long *d_counters = nullptr;
  unsigned long long *d_fix = nullptr;
  unsigned long long cap = 0;
  uint4 *d_cand = nullptr;                   // pool of leaves stored for the FP64 pass
  unsigned long long cand_cap = 0;           // pool entries (kPoolPerRay per ray of capacity)
  uint32_t *d_off = nullptr;                 // per list slot: its first pool entry
  TraceLaunch *pending = nullptr;            // launch whose FP64 pass is deferred
  char *d_stage = nullptr;                   // trace_rays_host: two halves of rays | hits | flags
  cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};  // trace_rays_host: copy in, trace, copy out
  std::vector<cudaEvent_t> pipe_ev;                    // 2 per chunk + 2
  cudaEvent_t stage_free[2] = {nullptr, nullptr};      // a half's last reader (the copy out) is done
  int stage_turn = 0;                                  // the half the next call uses
  unsigned long long stage_rays = 0;                   // capacity of each half
  void *d_order = nullptr;                   // ray-ordering keys, histogram and permutations
  size_t order_cap = 0;
  QueueEntry *d_queue = nullptr;             // SVO_TRACE_WAVEFRONT: the ray queue
  unsigned long long queue_cap = 0;          // entries
};

}  // namespace

struct svo_ctx {
  int device = 0;
  int n_sm = 1;
  int block = 128;         // trace kernel block size
  int rays_per_lane = 1;   // warp tile = 32 * rays_per_lane rays (1: finest load balance)
  int smem_levels = 0;     // top octree levels staged in shared memory by one-scene traces
  int tile_order = SVO_TILE_ORDER_CENTER;  // claim order of image tiles
  std::unordered_map<unsigned long long, uint32_t *> tile_orders;  // (tiles_x, tiles_y) -> device table
  std::mutex mu;
  std::vector<AssetRec> assets;
  std::unordered_set<svo_scene *> scenes;
  std::unordered_map<void *, Slot> slots;
  unsigned int *d_err = nullptr;
};

struct svo_scene {
  svo_ctx *ctx = nullptr;
  int P = 0, L = 0, NC = 0;
  int grid_G = 0, grid_cap = 0;  // scene-level grid (0: none)
  int max_depth = 1;
  std::vector<int32_t> parent;
  std::vector<svo_handle> asset;
  char *d_mem = nullptr;
  double *d_local = nullptr, *d_world = nullptr, *d_inv64 = nullptr;
  PartHot *d_hot = nullptr;
  PartAux *d_aux = nullptr;
  Cluster *d_cl = nullptr;
  int32_t *d_order = nullptr;
  PartStatic *d_stat = nullptr;
  int32_t *d_level_order = nullptr, *d_level_start = nullptr;
  float4 *d_bound = nullptr;
  uint8_t *d_dirty = nullptr;  // per part: world pose changed since the scene's previous trace
  SceneGrid *d_grid = nullptr;  // scene-level grid header, cell starts and part lists
  int32_t *d_cell_start = nullptr, *d_cell_parts = nullptr;
  int2 *d_top = nullptr;  // [kMaxSmemLevels][P] (first, count) of each part's top-level nodes
  size_t top_total[kMaxSmemLevels + 1] = {};  // staged nodes of all parts, per level count
  double *h_stage = nullptr;
  cudaEvent_t ev_stage = nullptr;
  bool stage_pending = false;
  std::vector<double> h_local;  // poses set from the host, not yet composed
  bool host_pending = false;
};

namespace {

AssetRec *find_asset(svo_ctx *ctx, svo_handle h) {
  if (h == 0 || h > ctx->assets.size()) return nullptr;
  AssetRec *a = &ctx->assets[h - 1];
  return a->live ? a : nullptr;
}

svo_status get_slot(svo_ctx *ctx, void *stream, unsigned long long need, Slot **out) {
  std::lock_guard<std::mutex> g(ctx->mu);
  Slot &s = ctx->slots[stream];
  if (!s.d_counters) CK(cudaMalloc(&s.d_counters, kCounterWords * sizeof(unsigned long long)));
  if (need > s.cap) {
    unsigned long long cap = need < 65536 ? 65536 : need;
    unsigned long long *p = nullptr;
    if (s.d_fix) {
      // the old lists may still be read by queued work on this stream
      CK(cudaStreamSynchronize((cudaStream_t)stream));
      CK(cudaFree(s.d_fix));
      CK(cudaFree(s.d_cand));
      CK(cudaFree(s.d_off));
      s.d_fix = nullptr;
      s.d_cand = nullptr;
      s.d_off = nullptr;
      s.cap = 0;
      s.cand_cap = 0;
    }
    // a flagged ray takes 1 pool entry (the winner, or the re-trace bound) or
    // its contenders (at most kContenders); the pool holds kPoolPerRay per ray
    // of capacity, and a ray it cannot hold falls back to a full FP64 re-trace
    const unsigned long long ccap = cap * kPoolPerRay;
    uint4 *c = nullptr;
    uint32_t *o = nullptr;
    cudaError_t e = cudaMalloc(&p, cap * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c, ccap * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&o, cap * sizeof(uint32_t));
    if (e != cudaSuccess) {
      if (p) cudaFree(p);
      if (c) cudaFree(c);
      return fail(SVO_ERR_OOM, "scratch for %llu rays: %s", cap, cudaGetErrorString(e));
    }
    s.d_fix = p;
    s.cap = cap;
    s.d_cand = c;
    s.cand_cap = ccap;
    s.d_off = o;
  }
  *out = &s;
  return SVO_OK;
}

// The launch record of trace_rays / trace_batch (about 16 KB): one per host
// thread, allocated on its first trace, so no call allocates it afresh.
TraceLaunch &launch_record() {
  thread_local std::unique_ptr<TraceLaunch> p;
  if (!p) p.reset(new TraceLaunch());
  return *p;
}

TraceItem make_item(svo_scene *s, const float *rays, uint64_t n, svo_hit *hits, uint32_t *flags) {
  TraceItem it;
  it.hot = s->d_hot;
  it.aux = s->d_aux;
  it.clusters = s->d_cl;
  it.order = s->d_order;
  it.inv64 = s->d_inv64;
  it.rays = reinterpret_cast<const float4 *>(rays);
  it.hits = reinterpret_cast<uint4 *>(hits);
  it.ray_flags = flags;
  it.perm = nullptr;
  it.dirty = s->d_dirty;
  it.grid = s->grid_G > 0 ? s->d_grid : nullptr;
  it.n = n;
  it.tile_begin = 0;
  it.n_parts = s->P;
  it.n_clusters = s->NC;
  it.max_depth = s->max_depth;
  it.width = 0;
  it.tiles_x = 0;
  it.pad = 0;
  it.tile_order = nullptr;
  it.qbase = 0;
  return it;
}

// Top levels of a one-scene launch staged in shared memory: the most levels
// up to the context's setting whose nodes fit kTopCapBytes.
void set_top_levels(svo_ctx *ctx, const svo_scene *only, TraceLaunch &L) {
  L.top = nullptr;
  L.top_nodes = 0;
  L.top_levels = 0;
  if (!only || only->P > 256) return;  // the trace kernel stages part tables up to 256 parts
  for (int l = ctx->smem_levels; l >= 1; --l) {
    if (only->top_total[l] * sizeof(uint2) <= kTopCapBytes && only->top_total[l] > 0) {
      L.top = only->d_top + (size_t)(l - 1) * only->P;
      L.top_nodes = (int32_t)only->top_total[l];
      L.top_levels = l;
      return;
    }
  }
}

// The centre-out claim order of a tiles_x x tiles_y grid of image tiles,
// each tile tw x th pixels: tiles sorted by the distance of their centres from
// the image centre (ties by row-major index), as tx | ty << 16.  Built on the
// host once per shape and kept on the device for the context's life.
svo_status tile_order_table(svo_ctx *ctx, uint32_t tiles_x, uint32_t tiles_y, uint32_t tw, uint32_t th,
                            uint32_t width, uint32_t height, const uint32_t **out) {
  *out = nullptr;
  if (tiles_x == 0 || tiles_y == 0 || tiles_x > 65535u || tiles_y > 65535u) return SVO_OK;  // row by row
  const unsigned long long key = ((unsigned long long)tiles_x << 32) | tiles_y;
  std::lock_guard<std::mutex> g(ctx->mu);
  auto f = ctx->tile_orders.find(key);
  if (f != ctx->tile_orders.end()) {
    *out = f->second;
    return SVO_OK;
  }
  const size_t n = (size_t)tiles_x * tiles_y;
  std::vector<std::pair<double, uint32_t>> d(n);
  const double cx = 0.5 * width, cy = 0.5 * height;
  for (uint32_t ty = 0; ty < tiles_y; ++ty)
    for (uint32_t tx = 0; tx < tiles_x; ++tx) {
      const double x = (tx + 0.5) * tw - cx, y = (ty + 0.5) * th - cy;
      d[(size_t)ty * tiles_x + tx] = {x * x + y * y, tx | (ty << 16)};
    }
  std::stable_sort(d.begin(), d.end(), [](const std::pair<double, uint32_t> &a, const std::pair<double, uint32_t> &b) {
    return a.first < b.first;
  });
  std::vector<uint32_t> h(n);
  for (size_t i = 0; i < n; ++i) h[i] = d[i].second;
  uint32_t *dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, n * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMemcpy(dev, h.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (dev) cudaFree(dev);
    return fail(SVO_ERR_CUDA, "tile order table: %s", cudaGetErrorString(e));
  }
  ctx->tile_orders[key] = dev;
  *out = dev;
  return SVO_OK;
}

// bounds[i]: scene bound of item i (frame of origin-based ray ordering).
// only: the scene every item traces, or nullptr (items of several scenes).
svo_status run_trace(svo_ctx *ctx, TraceLaunch &L, unsigned long long total_rays, const float4 *const *bounds,
                     const svo_scene *only, void *stream) {
  constexpr uint32_t kReuseNeeds = SVO_TRACE_CULL | SVO_TRACE_SORT | SVO_TRACE_FP64_FIX;
  if ((L.flags & SVO_TRACE_REUSE) && (L.flags & kReuseNeeds) != kReuseNeeds)
    return fail(SVO_ERR_ARG, "SVO_TRACE_REUSE needs CULL | SORT | FP64_FIX");
  if ((L.flags & SVO_TRACE_GRID) &&
      ((L.flags & SVO_TRACE_REUSE) || (L.flags & (SVO_TRACE_CULL | SVO_TRACE_SORT)) != (SVO_TRACE_CULL | SVO_TRACE_SORT)))
    return fail(SVO_ERR_ARG, "SVO_TRACE_GRID needs CULL | SORT and excludes REUSE");
  const bool wave = (L.flags & SVO_TRACE_WAVEFRONT) != 0;
  if (wave && ((L.flags & (SVO_TRACE_REUSE | SVO_TRACE_GRID)) ||
               (L.flags & (SVO_TRACE_CULL | SVO_TRACE_SORT)) != (SVO_TRACE_CULL | SVO_TRACE_SORT)))
    return fail(SVO_ERR_ARG, "SVO_TRACE_WAVEFRONT needs CULL | SORT and excludes REUSE and GRID");
  cudaStream_t st = (cudaStream_t)stream;
  Slot *slot = nullptr;
  svo_status rc = get_slot(ctx, stream, total_rays, &slot);
  if (rc != SVO_OK) return rc;
  const int order_mode = (L.flags & SVO_TRACE_ORDER_ORIGIN) ? 2 : ((L.flags & SVO_TRACE_ORDER_DIR) ? 1 : 0);
  if (order_mode) {
    size_t need = 0;
    for (int i = 0; i < L.n_items; ++i) need += (order_scratch_bytes(L.items[i].n) + 255) & ~size_t(255);
    if (need > slot->order_cap) {
      std::lock_guard<std::mutex> g(ctx->mu);
      if (slot->d_order) {
        CK(cudaStreamSynchronize(st));
        CK(cudaFree(slot->d_order));
        slot->d_order = nullptr;
        slot->order_cap = 0;
      }
      cudaError_t e = cudaMalloc(&slot->d_order, need);
      if (e != cudaSuccess) return fail(SVO_ERR_OOM, "ray-order scratch: %s", cudaGetErrorString(e));
      slot->order_cap = need;
    }
    size_t off = 0;
    if (L.n_items == 1) {
      uint32_t *perm = nullptr;
      CK(launch_order(reinterpret_cast<const float *>(L.items[0].rays), L.items[0].n, order_mode, bounds[0],
                      slot->d_order, &perm, ctx->n_sm, st));
      L.items[0].perm = perm;
    } else {
      // every item sorted by the same four launches
      std::vector<OrderItem> oi((size_t)L.n_items);
      for (int i = 0; i < L.n_items; ++i) {
        oi[i] = order_item(reinterpret_cast<const float *>(L.items[i].rays), L.items[i].n, bounds[i],
                           static_cast<char *>(slot->d_order) + off);
        L.items[i].perm = oi[i].perm;
        off += (order_scratch_bytes(L.items[i].n) + 255) & ~size_t(255);
      }
      CK(launch_order_batch(oi.data(), L.n_items, order_mode, ctx->n_sm, st));
    }
  }
  L.n_tiles = layout_tiles(L.items, L.n_items, ctx->rays_per_lane);
  for (int i = 0; i < L.n_items; ++i) {  // image items: the claim order of their tiles
    TraceItem &it = L.items[i];
    it.tile_order = nullptr;
    if (!it.tiles_x || ctx->tile_order != SVO_TILE_ORDER_CENTER) continue;
    const unsigned long long next = i + 1 < L.n_items ? L.items[i + 1].tile_begin : L.n_tiles;
    const unsigned long long band = 4ull * (unsigned long long)ctx->rays_per_lane;
    const uint32_t rows = (uint32_t)((it.n + it.width - 1) / it.width);
    svo_status rc = tile_order_table(ctx, it.tiles_x, (uint32_t)((next - it.tile_begin) / it.tiles_x), 8u,
                                     (uint32_t)band, it.width, rows, &it.tile_order);
    if (rc != SVO_OK) return rc;
  }
  L.queue = nullptr;
  L.queue_count = reinterpret_cast<unsigned int *>(slot->d_counters + kQueueCountWords);
  L.queue_tile = slot->d_counters + 3;
  if (wave) {
    if (total_rays > slot->queue_cap) {
      std::lock_guard<std::mutex> g(ctx->mu);
      if (slot->d_queue) {
        CK(cudaStreamSynchronize(st));  // queued work on this stream may still read the old queue
        CK(cudaFree(slot->d_queue));
        slot->d_queue = nullptr;
        slot->queue_cap = 0;
      }
      cudaError_t e = cudaMalloc(&slot->d_queue, total_rays * sizeof(QueueEntry));
      if (e != cudaSuccess) return fail(SVO_ERR_OOM, "ray queue: %s", cudaGetErrorString(e));
      slot->queue_cap = total_rays;
    }
    L.queue = slot->d_queue;
    unsigned long long q = 0;
    for (int i = 0; i < L.n_items; ++i) {
      L.items[i].qbase = q;
      q += L.items[i].n;
    }
  }
  L.tile_counter = slot->d_counters;
  L.fix_count = reinterpret_cast<unsigned int *>(slot->d_counters + 1);
  L.fix_list = slot->d_fix;
  L.fix_capacity = slot->cap;
  L.fix_cand = slot->d_cand;
  L.cand_capacity = slot->cand_cap;
  L.cand_count = reinterpret_cast<unsigned int *>(slot->d_counters + 2);
  L.fix_off = slot->d_off;
  L.err = ctx->d_err;
  L.block = ctx->block;
  L.rays_per_lane = ctx->rays_per_lane;
  set_top_levels(ctx, only, L);
  CK(cudaMemsetAsync(slot->d_counters, 0,
                     wave ? kQueueCountWords * sizeof(unsigned long long) + (size_t)L.n_items * sizeof(unsigned int)
                          : 3 * sizeof(unsigned long long),
                     st));
  if (L.flags & SVO_TRACE_GRID) {
    GridLaunch gl;
    if (grid_jobs(L.items, L.n_items, gl) > 0) CK(launch_grid(gl, st));
  }
  CK(launch_trace(L, ctx->n_sm, st));
  // pose changes are tracked relative to each scene's latest trace
  for (int i = 0; i < L.n_items; ++i) {
    bool seen = false;
    for (int j = 0; j < i; ++j) seen = seen || L.items[j].dirty == L.items[i].dirty;
    if (!seen) CK(cudaMemsetAsync(const_cast<uint8_t *>(L.items[i].dirty), 0, (size_t)L.items[i].n_parts, st));
  }
  delete slot->pending;
  slot->pending = nullptr;
  if (L.flags & SVO_TRACE_FP64_FIX) {
    if (L.flags & SVO_TRACE_DEFER_FIX)
      slot->pending = new TraceLaunch(L);
    else
      CK(launch_fix(L, ctx->n_sm, st));
  }
  return SVO_OK;
}

}  // namespace

// Accessors for trace_rays_noalloc (svo_noalloc.cu), which keeps its scratch
// in a static device array of its own translation unit.
namespace svo {
int scene_device(const svo_scene *s) { return s->ctx->device; }
TraceItem scene_item(svo_scene *s, const float *rays, uint64_t n, svo_hit *hits, uint32_t *flags) {
  return make_item(s, rays, n, hits, flags);
}
unsigned int *scene_err_word(const svo_scene *s) { return s->ctx->d_err; }
int scene_sm_count(const svo_scene *s) { return s->ctx->n_sm; }
void scene_trace_config(const svo_scene *s, int *block, int *rays_per_lane) {
  *block = s->ctx->block;
  *rays_per_lane = s->ctx->rays_per_lane;
}
svo_status set_last_error(svo_status code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace svo

// Kernel arguments of one scene's refit.
static RefitArgs refit_args(const svo_scene *s) {
  RefitArgs a;
  a.n_parts = s->P;
  a.n_levels = s->L;
  a.level_order = s->d_level_order;
  a.level_start = s->d_level_start;
  a.stat = s->d_stat;
  a.local = s->d_local;
  a.world = s->d_world;
  a.inv64 = s->d_inv64;
  a.hot = s->d_hot;
  a.aux = s->d_aux;
  a.clusters = s->d_cl;
  a.order = s->d_order;
  a.n_clusters = s->NC;
  a.bound = s->d_bound;
  a.dirty = s->d_dirty;
  a.grid = s->grid_G > 0 ? s->d_grid : nullptr;
  a.err = s->ctx->d_err;
  return a;
}

extern "C" {

const char *svo_last_error(void) { return g_last_error.c_str(); }

const char *svo_status_string(svo_status s) {
  switch (s) {
    case SVO_OK: return "SVO_OK";
    case SVO_ERR_ARG: return "SVO_ERR_ARG";
    case SVO_ERR_OOM: return "SVO_ERR_OOM";
    case SVO_ERR_HANDLE: return "SVO_ERR_HANDLE";
    case SVO_ERR_CUDA: return "SVO_ERR_CUDA";
    case SVO_ERR_TIMEOUT: return "SVO_ERR_TIMEOUT";
    case SVO_ERR_ADMIT: return "SVO_ERR_ADMIT";
    case SVO_ERR_NAN: return "SVO_ERR_NAN";
    case SVO_ERR_SINGULAR: return "SVO_ERR_SINGULAR";
    case SVO_ERR_LIMIT: return "SVO_ERR_LIMIT";
    case SVO_ERR_DEVICE: return "SVO_ERR_DEVICE";
    default: return "SVO_ERR_UNKNOWN";
  }
}

svo_status svo_ctx_create(int32_t device, svo_ctx **out) {
  if (!out) return fail(SVO_ERR_ARG, "svo_ctx_create: out is NULL");
  *out = nullptr;
  int n_dev = 0;
  CK(cudaGetDeviceCount(&n_dev));
  if (device < 0 || device >= n_dev) return fail(SVO_ERR_ARG, "svo_ctx_create: device %d of %d", device, n_dev);
  CK(cudaSetDevice(device));
  svo_ctx *c = new svo_ctx();
  c->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(unsigned int));
  if (e == cudaSuccess) e = init_trace_tables(nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    if (c->d_err) cudaFree(c->d_err);
    delete c;
    return fail(SVO_ERR_CUDA, "svo_ctx_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return ok();
}

svo_status scene_destroy(svo_scene *s);

svo_status svo_ctx_destroy(svo_ctx *ctx) {
  if (!ctx) return ok();
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  std::vector<svo_scene *> sc(ctx->scenes.begin(), ctx->scenes.end());
  for (svo_scene *s : sc) scene_destroy(s);
  for (AssetRec &a : ctx->assets) {
    if (a.d_nodes) cudaFree(a.d_nodes);
    if (a.d_rgb) cudaFree(a.d_rgb);
  }
  for (auto &kv : ctx->slots) {
    if (kv.second.d_counters) cudaFree(kv.second.d_counters);
    if (kv.second.d_fix) cudaFree(kv.second.d_fix);
    if (kv.second.d_cand) cudaFree(kv.second.d_cand);
    if (kv.second.d_off) cudaFree(kv.second.d_off);
    if (kv.second.d_stage) cudaFree(kv.second.d_stage);
    if (kv.second.d_order) cudaFree(kv.second.d_order);
    if (kv.second.d_queue) cudaFree(kv.second.d_queue);
    for (cudaStream_t ps : kv.second.pipe)
      if (ps) cudaStreamDestroy(ps);
    for (cudaEvent_t e : kv.second.pipe_ev) cudaEventDestroy(e);
    for (cudaEvent_t e : kv.second.stage_free)
      if (e) cudaEventDestroy(e);
    delete kv.second.pending;
  }
  for (auto &kv : ctx->tile_orders) cudaFree(kv.second);
  if (ctx->d_err) cudaFree(ctx->d_err);
  delete ctx;
  return ok();
}

svo_status svo_set_trace_config(svo_ctx *ctx, int32_t block, int32_t rays_per_lane) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_set_trace_config: ctx is NULL");
  if (block != 64 && block != 128 && block != 256)
    return fail(SVO_ERR_ARG, "svo_set_trace_config: block %d (64, 128 or 256)", block);
  if (rays_per_lane != 1 && rays_per_lane != 2 && rays_per_lane != 4 && rays_per_lane != 8)
    return fail(SVO_ERR_ARG, "svo_set_trace_config: rays_per_lane %d (1, 2, 4 or 8)", rays_per_lane);
  ctx->block = block;
  ctx->rays_per_lane = rays_per_lane;
  return ok();
}

svo_status svo_set_smem_levels(svo_ctx *ctx, int32_t levels) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_set_smem_levels: ctx is NULL");
  if (levels < 0 || levels > kMaxSmemLevels)
    return fail(SVO_ERR_ARG, "svo_set_smem_levels: %d levels (0..%d)", levels, kMaxSmemLevels);
  ctx->smem_levels = levels;
  return ok();
}

svo_status svo_set_tile_order(svo_ctx *ctx, int32_t order) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_set_tile_order: ctx is NULL");
  if (order != SVO_TILE_ORDER_ROWS && order != SVO_TILE_ORDER_CENTER)
    return fail(SVO_ERR_ARG, "svo_set_tile_order: %d (SVO_TILE_ORDER_ROWS or SVO_TILE_ORDER_CENTER)", order);
  ctx->tile_order = order;
  return ok();
}

svo_status svo_get_tile_order(svo_ctx *ctx, int32_t *order) {
  if (!ctx || !order) return fail(SVO_ERR_ARG, "svo_get_tile_order: NULL argument");
  *order = ctx->tile_order;
  return ok();
}

svo_status svo_get_smem_levels(svo_ctx *ctx, int32_t *levels) {
  if (!ctx || !levels) return fail(SVO_ERR_ARG, "svo_get_smem_levels: NULL argument");
  *levels = ctx->smem_levels;
  return ok();
}

svo_status svo_get_trace_config(svo_ctx *ctx, int32_t *block, int32_t *rays_per_lane) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_get_trace_config: ctx is NULL");
  if (block) *block = ctx->block;
  if (rays_per_lane) *rays_per_lane = ctx->rays_per_lane;
  return ok();
}

svo_status svo_check_device(svo_ctx *ctx) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_check_device: ctx is NULL");
  CK(cudaSetDevice(ctx->device));
  CK(cudaDeviceSynchronize());
  unsigned int e = 0;
  CK(cudaMemcpy(&e, ctx->d_err, sizeof(e), cudaMemcpyDeviceToHost));
  CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned int)));
  if (e == 0) return ok();
  return fail(SVO_ERR_DEVICE, "device checks failed: 0x%x%s%s%s%s", e, (e & kErrNodeIndex) ? " node-index" : "",
              (e & kErrFixOverflow) ? " fix-list-overflow" : "", (e & kErrSingular) ? " singular-pose" : "",
              (e & kErrStack) ? " stack" : "");
}

svo_status svo_build_host(const svo_desc *d, uint64_t *n_nodes, uint64_t *n_leaves, void *nodes, uint32_t *rgb) {
  if (!d) return fail(SVO_ERR_ARG, "svo_build_host: desc is NULL");
  BuiltOctree b;
  int rc = build_octree(d->depth, d->n_leaves, d->leaf_ids, d->leaf_rgb, &b);
  if (rc != SVO_OK) return fail(rc, "svo_build_host: bad leaf list (depth %d, %llu leaves)", d->depth,
                                (unsigned long long)d->n_leaves);
  if (n_nodes) *n_nodes = b.n_nodes;
  if (n_leaves) *n_leaves = b.n_leaves;
  if (nodes && b.n_nodes) memcpy(nodes, b.nodes.data(), b.n_nodes * 8);
  if (rgb && b.n_leaves) memcpy(rgb, b.rgb.data(), b.n_leaves * 4);
  return ok();
}

svo_status svo_upload(svo_ctx *ctx, const svo_desc *d, svo_handle *out) {
  if (!ctx || !d || !out) return fail(SVO_ERR_ARG, "svo_upload: NULL argument");
  BuiltOctree b;
  int rc = build_octree(d->depth, d->n_leaves, d->leaf_ids, d->leaf_rgb, &b);
  if (rc != SVO_OK) return fail(rc, "svo_upload: bad leaf list (depth %d)", d->depth);
  CK(cudaSetDevice(ctx->device));
  AssetRec a;
  a.depth = b.depth;
  a.n_nodes = b.n_nodes;
  a.n_leaves = b.n_leaves;
  for (int l = 0; l <= kMaxSmemLevels; ++l)  // breadth first: the top l levels are the first nodes
    a.top_nodes[l] = (uint32_t)(b.n_nodes ? b.level_start[l < b.depth ? l : b.depth] : 0);
  for (int k = 0; k < 3; ++k) {
    a.box_lo[k] = (float)std::ldexp((double)b.box_lo[k], -b.depth);
    a.box_hi[k] = (float)std::ldexp((double)b.box_hi[k], -b.depth);
  }
  if (b.n_nodes) {
    cudaError_t e = cudaMalloc(&a.d_nodes, b.n_nodes * 8);
    if (e != cudaSuccess) return fail(SVO_ERR_OOM, "svo_upload: %llu nodes: %s", (unsigned long long)b.n_nodes,
                                      cudaGetErrorString(e));
    e = cudaMalloc(&a.d_rgb, b.n_leaves * 4);
    if (e != cudaSuccess) {
      cudaFree(a.d_nodes);
      return fail(SVO_ERR_OOM, "svo_upload: leaf payload: %s", cudaGetErrorString(e));
    }
    CK(cudaMemcpy(a.d_nodes, b.nodes.data(), b.n_nodes * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(a.d_rgb, b.rgb.data(), b.n_leaves * 4, cudaMemcpyHostToDevice));
  }
  a.live = true;
  std::lock_guard<std::mutex> g(ctx->mu);
  ctx->assets.push_back(a);
  *out = (svo_handle)ctx->assets.size();
  return ok();
}

svo_status svo_release(svo_ctx *ctx, svo_handle h) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_release: ctx is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  AssetRec *a = find_asset(ctx, h);
  if (!a) return fail(SVO_ERR_HANDLE, "svo_release: unknown handle %u", h);
  if (a->refs > 0) return fail(SVO_ERR_ARG, "svo_release: asset %u is used by %d scene part(s)", h, a->refs);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (a->d_nodes) cudaFree(a->d_nodes);
  if (a->d_rgb) cudaFree(a->d_rgb);
  *a = AssetRec();
  return ok();
}

svo_status svo_asset_info(svo_ctx *ctx, svo_handle h, int32_t *depth, uint64_t *n_nodes, uint64_t *n_leaves) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_asset_info: ctx is NULL");
  std::lock_guard<std::mutex> g(ctx->mu);
  AssetRec *a = find_asset(ctx, h);
  if (!a) return fail(SVO_ERR_HANDLE, "svo_asset_info: unknown handle %u", h);
  if (depth) *depth = a->depth;
  if (n_nodes) *n_nodes = a->n_nodes;
  if (n_leaves) *n_leaves = a->n_leaves;
  return ok();
}

svo_status svo_read_asset(svo_ctx *ctx, svo_handle h, void *nodes, uint32_t *rgb) {
  if (!ctx) return fail(SVO_ERR_ARG, "svo_read_asset: ctx is NULL");
  uint2 *d_nodes = nullptr;
  uint32_t *d_rgb = nullptr;
  uint64_t n_nodes = 0, n_leaves = 0;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    AssetRec *a = find_asset(ctx, h);
    if (!a) return fail(SVO_ERR_HANDLE, "svo_read_asset: unknown handle %u", h);
    d_nodes = a->d_nodes;
    d_rgb = a->d_rgb;
    n_nodes = a->n_nodes;
    n_leaves = a->n_leaves;
  }
  CK(cudaSetDevice(ctx->device));
  if (nodes && n_nodes) CK(cudaMemcpy(nodes, d_nodes, n_nodes * sizeof(uint2), cudaMemcpyDeviceToHost));
  if (rgb && n_leaves) CK(cudaMemcpy(rgb, d_rgb, n_leaves * sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return ok();
}

svo_status scene_create(svo_ctx *ctx, int32_t n_parts, const svo_handle *asset, const int32_t *parent,
                        svo_scene **out) {
  if (!ctx || !asset || !parent || !out) return fail(SVO_ERR_ARG, "scene_create: NULL argument");
  *out = nullptr;
  if (n_parts < 1 || n_parts > kMaxParts)
    return fail(SVO_ERR_LIMIT, "scene_create: %d parts (1..%d)", n_parts, kMaxParts);
  std::vector<int32_t> level(n_parts, 0);
  for (int i = 0; i < n_parts; ++i) {
    if (parent[i] >= i || parent[i] < -1)
      return fail(SVO_ERR_ARG, "scene_create: parent[%d] = %d (must be -1 or < %d)", i, parent[i], i);
    level[i] = parent[i] < 0 ? 0 : level[parent[i]] + 1;
  }
  std::vector<PartStatic> stat(n_parts);
  std::vector<uint32_t> top_cnt((size_t)(kMaxSmemLevels + 1) * n_parts, 0u);
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    for (int i = 0; i < n_parts; ++i) {
      AssetRec *a = find_asset(ctx, asset[i]);
      if (!a) return fail(SVO_ERR_HANDLE, "scene_create: part %d: unknown asset %u", i, asset[i]);
      for (int l = 0; l <= kMaxSmemLevels; ++l) top_cnt[(size_t)l * n_parts + i] = a->top_nodes[l];
      stat[i].nodes = a->d_nodes;
      stat[i].n_nodes = (uint32_t)a->n_nodes;
      stat[i].depth = a->depth;
      stat[i].parent = parent[i];
      stat[i].pad = 0;
      stat[i].rgb = a->d_rgb;
      stat[i].n_leaves = a->n_leaves;
      for (int k = 0; k < 3; ++k) {
        stat[i].box_lo[k] = a->box_lo[k];
        stat[i].box_hi[k] = a->box_hi[k];
      }
    }
  }
  int L = 0;
  for (int i = 0; i < n_parts; ++i) L = level[i] + 1 > L ? level[i] + 1 : L;
  std::vector<int32_t> lorder, lstart(L + 1, 0);
  for (int l = 0; l < L; ++l) {
    lstart[l] = (int32_t)lorder.size();
    for (int i = 0; i < n_parts; ++i)
      if (level[i] == l) lorder.push_back(i);
  }
  lstart[L] = n_parts;
  const int P = n_parts;
  const int NC = (P + kClusterSize - 1) / kClusterSize;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off_local = 0;
  size_t off_world = al(off_local + P * 12 * sizeof(double));
  size_t off_inv = al(off_world + P * 12 * sizeof(double));
  size_t off_hot = al(off_inv + P * 12 * sizeof(double));
  size_t off_aux = al(off_hot + P * sizeof(PartHot));
  size_t off_cl = al(off_aux + P * sizeof(PartAux));
  size_t off_order = al(off_cl + NC * sizeof(Cluster));
  size_t off_stat = al(off_order + P * sizeof(int32_t));
  size_t off_lo = al(off_stat + P * sizeof(PartStatic));
  size_t off_ls = al(off_lo + P * sizeof(int32_t));
  size_t off_bd = al(off_ls + (L + 1) * sizeof(int32_t));
  size_t off_dirty = al(off_bd + sizeof(float4));
  // scene-level grid for scenes of kGridMinParts parts or more; lists sized
  // for about 32 cells per part
  const int grid_G = grid_cells_per_axis(P);
  const int grid_cap = grid_G > 0 ? 32 * P + grid_G * grid_G * grid_G : 0;
  size_t off_top = al(off_dirty + P);
  size_t off_grid = al(off_top + (size_t)kMaxSmemLevels * P * sizeof(int2));
  size_t off_cstart = al(off_grid + sizeof(SceneGrid));
  size_t off_cparts = al(off_cstart + (grid_G > 0 ? (size_t)(grid_G * grid_G * grid_G + 1) * sizeof(int32_t) : 0));
  size_t total = al(off_cparts + (size_t)grid_cap * sizeof(int32_t));
  CK(cudaSetDevice(ctx->device));
  svo_scene *s = new svo_scene();
  s->ctx = ctx;
  s->P = P;
  s->L = L;
  s->NC = NC;
  s->parent.assign(parent, parent + P);
  s->asset.assign(asset, asset + P);
  for (int i = 0; i < P; ++i) s->max_depth = stat[i].depth > s->max_depth ? stat[i].depth : s->max_depth;
  cudaError_t e = cudaMalloc(&s->d_mem, total);
  if (e != cudaSuccess) {
    delete s;
    return fail(SVO_ERR_OOM, "scene_create: %zu bytes: %s", total, cudaGetErrorString(e));
  }
  s->d_local = reinterpret_cast<double *>(s->d_mem + off_local);
  s->d_world = reinterpret_cast<double *>(s->d_mem + off_world);
  s->d_inv64 = reinterpret_cast<double *>(s->d_mem + off_inv);
  s->d_hot = reinterpret_cast<PartHot *>(s->d_mem + off_hot);
  s->d_aux = reinterpret_cast<PartAux *>(s->d_mem + off_aux);
  s->d_cl = reinterpret_cast<Cluster *>(s->d_mem + off_cl);
  s->d_order = reinterpret_cast<int32_t *>(s->d_mem + off_order);
  s->d_stat = reinterpret_cast<PartStatic *>(s->d_mem + off_stat);
  s->d_level_order = reinterpret_cast<int32_t *>(s->d_mem + off_lo);
  s->d_level_start = reinterpret_cast<int32_t *>(s->d_mem + off_ls);
  s->d_bound = reinterpret_cast<float4 *>(s->d_mem + off_bd);
  s->d_dirty = reinterpret_cast<uint8_t *>(s->d_mem + off_dirty);
  s->d_grid = reinterpret_cast<SceneGrid *>(s->d_mem + off_grid);
  s->d_cell_start = reinterpret_cast<int32_t *>(s->d_mem + off_cstart);
  s->d_cell_parts = reinterpret_cast<int32_t *>(s->d_mem + off_cparts);
  s->d_top = reinterpret_cast<int2 *>(s->d_mem + off_top);
  std::vector<int2> top((size_t)kMaxSmemLevels * P);
  for (int l = 1; l <= kMaxSmemLevels; ++l) {
    size_t first = 0;
    for (int i = 0; i < P; ++i) {
      const uint32_t c = top_cnt[(size_t)l * P + i];
      top[(size_t)(l - 1) * P + i] = make_int2((int)first, (int)c);
      first += c;
    }
    s->top_total[l] = first;
  }
  s->grid_G = grid_G;
  s->grid_cap = grid_cap;
  std::vector<double> ident(P * 12, 0.0);
  for (int i = 0; i < P; ++i) ident[12 * i + 0] = ident[12 * i + 5] = ident[12 * i + 10] = 1.0;
  e = cudaMallocHost(&s->h_stage, P * 12 * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_stage, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_local, ident.data(), P * 12 * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && grid_G > 0) {  // built before the first grid trace
    SceneGrid g = {};
    g.G = grid_G;
    g.cap = grid_cap;
    g.stale = 1;
    g.cell_start = s->d_cell_start;
    g.cell_parts = s->d_cell_parts;
    e = cudaMemcpy(s->d_grid, &g, sizeof(g), cudaMemcpyHostToDevice);
  }
  // no pose yet: NaN world poses make the first refit mark every part changed
  if (e == cudaSuccess) e = cudaMemset(s->d_world, 0xFF, P * 12 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemset(s->d_dirty, 1, P);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_stat, stat.data(), P * sizeof(PartStatic), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_top, top.data(), top.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_level_order, lorder.data(), P * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(s->d_level_start, lstart.data(), (L + 1) * sizeof(int32_t), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (s->h_stage) cudaFreeHost(s->h_stage);
    if (s->ev_stage) cudaEventDestroy(s->ev_stage);
    cudaFree(s->d_mem);
    delete s;
    return fail(SVO_ERR_CUDA, "scene_create: %s", cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    for (int i = 0; i < P; ++i) find_asset(ctx, asset[i])->refs++;
    ctx->scenes.insert(s);
  }
  svo_status rc = scene_refit(s, nullptr);
  if (rc == SVO_OK) {
    cudaError_t e2 = cudaStreamSynchronize(nullptr);
    if (e2 != cudaSuccess) rc = fail(SVO_ERR_CUDA, "scene_create: %s", cudaGetErrorString(e2));
  }
  if (rc != SVO_OK) {
    scene_destroy(s);
    return rc;
  }
  *out = s;
  return ok();
}

svo_status scene_destroy(svo_scene *s) {
  if (!s) return ok();
  svo_ctx *ctx = s->ctx;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    if (!ctx->scenes.count(s)) return fail(SVO_ERR_HANDLE, "scene_destroy: unknown scene");
    ctx->scenes.erase(s);
    for (svo_handle h : s->asset) {
      AssetRec *a = find_asset(ctx, h);
      if (a && a->refs > 0) a->refs--;
    }
  }
  if (s->h_stage) cudaFreeHost(s->h_stage);
  if (s->ev_stage) cudaEventDestroy(s->ev_stage);
  if (s->d_mem) cudaFree(s->d_mem);
  delete s;
  return ok();
}

svo_status scene_set_transforms(svo_scene *s, const double *local, void *stream) {
  if (!s || !local) return fail(SVO_ERR_ARG, "scene_set_transforms: NULL argument");
  const int n = s->P * 12;
  for (int i = 0; i < n; ++i)
    if (!std::isfinite(local[i])) return fail(SVO_ERR_NAN, "scene_set_transforms: entry %d is not finite", i);
  if (s->P <= kInlinePoseParts) {
    // small scenes: the poses ride in the next scene_refit's kernel parameters
    s->h_local.assign(local, local + n);
    s->host_pending = true;
    return ok();
  }
  CK(cudaSetDevice(s->ctx->device));
  if (s->stage_pending) CK(cudaEventSynchronize(s->ev_stage));  // previous copy out of the staging buffer
  memcpy(s->h_stage, local, n * sizeof(double));
  CK(cudaMemcpyAsync(s->d_local, s->h_stage, n * sizeof(double), cudaMemcpyHostToDevice, (cudaStream_t)stream));
  CK(cudaEventRecord(s->ev_stage, (cudaStream_t)stream));
  s->stage_pending = true;
  return ok();
}

svo_status scene_set_transforms_trs(svo_scene *s, const double *rts, void *stream) {
  if (!s || !rts) return fail(SVO_ERR_ARG, "scene_set_transforms_trs: NULL argument");
  const int P = s->P;
  for (int i = 0; i < P * 15; ++i)
    if (!std::isfinite(rts[i])) return fail(SVO_ERR_NAN, "scene_set_transforms_trs: entry %d is not finite", i);
  std::vector<double> local((size_t)P * 12);
  for (int p = 0; p < P; ++p) {
    const double *R = rts + 15 * p, *t = R + 9, *d = R + 12;
    for (int i = 0; i < 3; ++i) {
      if (!(d[i] > 0.0)) return fail(SVO_ERR_ARG, "scene_set_transforms_trs: part %d: dimension %d is not positive", p, i);
      for (int j = 0; j < 3; ++j) {
        const double rr = R[3 * i] * R[3 * j] + R[3 * i + 1] * R[3 * j + 1] + R[3 * i + 2] * R[3 * j + 2];
        if (std::fabs(rr - (i == j ? 1.0 : 0.0)) > 1e-9)
          return fail(SVO_ERR_ARG, "scene_set_transforms_trs: part %d: R is not orthonormal", p);
      }
    }
    // x_parent = R (d * x) + t: column j of the linear part is d_j R[:, j]
    double *m = local.data() + 12 * p;
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) m[4 * i + j] = R[3 * i + j] * d[j];
      m[4 * i + 3] = t[i];
    }
  }
  return scene_set_transforms(s, local.data(), stream);
}

svo_status scene_set_transforms_device(svo_scene *s, const double *local_dev, void *stream) {
  if (!s || !local_dev) return fail(SVO_ERR_ARG, "scene_set_transforms_device: NULL argument");
  CK(cudaSetDevice(s->ctx->device));
  s->host_pending = false;
  CK(cudaMemcpyAsync(s->d_local, local_dev, s->P * 12 * sizeof(double), cudaMemcpyDeviceToDevice,
                     (cudaStream_t)stream));
  return ok();
}

svo_status scene_refit_batch(svo_scene *const *scenes, const double *const *local_dev, int32_t n, void *stream) {
  if (n < 0 || (n > 0 && !scenes)) return fail(SVO_ERR_ARG, "scene_refit_batch: bad scene list");
  if (n == 0) return ok();
  for (int i = 0; i < n; ++i) {
    if (!scenes[i]) return fail(SVO_ERR_ARG, "scene_refit_batch: scene %d is NULL", i);
    if (scenes[i]->ctx != scenes[0]->ctx) return fail(SVO_ERR_ARG, "scene_refit_batch: scene %d belongs to another context", i);
    for (int j = 0; j < i; ++j)
      if (scenes[j] == scenes[i]) return fail(SVO_ERR_ARG, "scene_refit_batch: scene %d appears twice", i);
  }
  CK(cudaSetDevice(scenes[0]->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  for (int b = 0; b < n; b += kRefitBatch) {
    const int cnt = (n - b) < kRefitBatch ? (n - b) : kRefitBatch;
    RefitArgs args[kRefitBatch];
    const double *src[kRefitBatch];
    for (int k = 0; k < cnt; ++k) {
      svo_scene *s = scenes[b + k];
      args[k] = refit_args(s);
      src[k] = local_dev ? local_dev[b + k] : nullptr;
      if (src[k]) {
        s->host_pending = false;  // the given device poses replace any set from the host
      } else if (s->host_pending) {
        // poses set from the host (small scenes): the kernel reads them from
        // the scene's page-locked staging buffer through its device mapping
        if (s->stage_pending) CK(cudaEventSynchronize(s->ev_stage));
        memcpy(s->h_stage, s->h_local.data(), s->h_local.size() * sizeof(double));
        void *mapped = nullptr;
        CK(cudaHostGetDevicePointer(&mapped, s->h_stage, 0));
        src[k] = static_cast<const double *>(mapped);
        s->host_pending = false;
      }
    }
    CK(launch_refit_batch(args, src, cnt, st));
    for (int k = 0; k < cnt; ++k) {  // the staging buffers read by this launch stay untouched until it is done
      svo_scene *s = scenes[b + k];
      if (!local_dev || !local_dev[b + k]) {
        CK(cudaEventRecord(s->ev_stage, st));
        s->stage_pending = true;
      }
    }
  }
  return ok();
}

svo_status scene_refit(svo_scene *s, void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "scene_refit: scene is NULL");
  CK(cudaSetDevice(s->ctx->device));
  const RefitArgs a = refit_args(s);
  CK(launch_refit(a, s->host_pending ? s->h_local.data() : nullptr, (cudaStream_t)stream));
  s->host_pending = false;
  return ok();
}

svo_status scene_read_poses(svo_scene *s, double *world, double *inv, float *inv_f32, float *sphere, void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "scene_read_poses: scene is NULL");
  CK(cudaSetDevice(s->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  const int P = s->P;
  if (world) CK(cudaMemcpyAsync(world, s->d_world, P * 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
  if (inv) CK(cudaMemcpyAsync(inv, s->d_inv64, P * 12 * sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<PartHot> hot;
  if (inv_f32 || sphere) {
    hot.resize(P);
    CK(cudaMemcpyAsync(hot.data(), s->d_hot, P * sizeof(PartHot), cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  for (int i = 0; i < P && (inv_f32 || sphere); ++i) {
    if (inv_f32) {
      const float4 r[3] = {hot[i].r0, hot[i].r1, hot[i].r2};
      for (int k = 0; k < 3; ++k) {
        inv_f32[12 * i + 4 * k + 0] = r[k].x;
        inv_f32[12 * i + 4 * k + 1] = r[k].y;
        inv_f32[12 * i + 4 * k + 2] = r[k].z;
        inv_f32[12 * i + 4 * k + 3] = r[k].w;
      }
    }
    if (sphere) {
      sphere[4 * i + 0] = hot[i].sphere.x;
      sphere[4 * i + 1] = hot[i].sphere.y;
      sphere[4 * i + 2] = hot[i].sphere.z;
      sphere[4 * i + 3] = hot[i].sphere.w;
    }
  }
  return ok();
}

svo_status scene_read_clusters(svo_scene *s, int32_t *n_clusters, float *sphere, int32_t *order, void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "scene_read_clusters: scene is NULL");
  CK(cudaSetDevice(s->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  if (n_clusters) *n_clusters = s->NC;
  std::vector<Cluster> cl;
  if (sphere) {
    cl.resize(s->NC);
    CK(cudaMemcpyAsync(cl.data(), s->d_cl, s->NC * sizeof(Cluster), cudaMemcpyDeviceToHost, st));
  }
  if (order) CK(cudaMemcpyAsync(order, s->d_order, s->P * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  for (int c = 0; c < s->NC && sphere; ++c) {
    sphere[4 * c + 0] = cl[c].sphere.x;
    sphere[4 * c + 1] = cl[c].sphere.y;
    sphere[4 * c + 2] = cl[c].sphere.z;
    sphere[4 * c + 3] = cl[c].sphere.w;
  }
  return ok();
}

svo_status trace_rays(svo_scene *s, const float *rays, uint64_t n, svo_hit *hits, uint32_t *ray_flags,
                      uint32_t flags, svo_trace_stats *stats, void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "trace_rays: scene is NULL");
  if (n == 0) return ok();
  if (!rays || !hits) return fail(SVO_ERR_ARG, "trace_rays: rays/hits is NULL");
  if ((reinterpret_cast<uintptr_t>(rays) & 15) || (reinterpret_cast<uintptr_t>(hits) & 15))
    return fail(SVO_ERR_ARG, "trace_rays: rays and hits must be 16-byte aligned");
  if (n >= (1ull << 40)) return fail(SVO_ERR_LIMIT, "trace_rays: %llu rays", (unsigned long long)n);
  if ((flags & SVO_TRACE_STATS) && !stats) return fail(SVO_ERR_ARG, "trace_rays: STATS without stats buffer");
  CK(cudaSetDevice(s->ctx->device));
  TraceLaunch *L = &launch_record();
  L->items[0] = make_item(s, rays, n, hits, ray_flags);
  if (flags & SVO_TRACE_IMAGE_TILES) L->items[0].width = flags >> 16;
  L->n_items = 1;
  L->flags = flags;
  L->stats = (flags & SVO_TRACE_STATS) ? stats : nullptr;
  const float4 *bounds[1] = {s->d_bound};
  return run_trace(s->ctx, *L, n, bounds, s, stream);
}

svo_status trace_batch(svo_ctx *ctx, const svo_batch_item *items, int32_t n_items, uint32_t flags,
                       svo_trace_stats *stats, void *stream) {
  if (!ctx || (n_items > 0 && !items)) return fail(SVO_ERR_ARG, "trace_batch: NULL argument");
  if (n_items < 0) return fail(SVO_ERR_ARG, "trace_batch: n_items < 0");
  if ((flags & SVO_TRACE_STATS) && !stats) return fail(SVO_ERR_ARG, "trace_batch: STATS without stats buffer");
  CK(cudaSetDevice(ctx->device));
  for (int b = 0; b < n_items; b += kMaxBatchItems) {
    const int cnt = (n_items - b) < kMaxBatchItems ? (n_items - b) : kMaxBatchItems;
    TraceLaunch *L = &launch_record();
    L->n_items = 0;
    unsigned long long total = 0;
    const float4 *bounds[kMaxBatchItems];
    svo_scene *only = nullptr;
    bool one = true;
    for (int i = 0; i < cnt; ++i) {
      const svo_batch_item &it = items[b + i];
      if (!it.scene) return fail(SVO_ERR_ARG, "trace_batch: item %d has no scene", b + i);
      if (it.scene->ctx != ctx) return fail(SVO_ERR_ARG, "trace_batch: item %d belongs to another context", b + i);
      if (it.n == 0) continue;
      if (!it.rays || !it.hits || (reinterpret_cast<uintptr_t>(it.rays) & 15) ||
          (reinterpret_cast<uintptr_t>(it.hits) & 15))
        return fail(SVO_ERR_ARG, "trace_batch: item %d rays/hits NULL or not 16-byte aligned", b + i);
      TraceItem ti = make_item(it.scene, it.rays, it.n, it.hits, it.ray_flags);
      ti.width = it.image_width;
      total += it.n;
      bounds[L->n_items] = it.scene->d_bound;
      L->items[L->n_items++] = ti;
      one = one && (only == nullptr || only == it.scene);
      only = it.scene;
    }
    if (L->n_items > 0) {
      L->flags = flags;
      L->stats = (flags & SVO_TRACE_STATS) ? stats : nullptr;
      svo_status rc = run_trace(ctx, *L, total, bounds, one ? only : nullptr, stream);
      if (rc != SVO_OK) return rc;
    }
  }
  return ok();
}

// Device address of page-locked host memory mapped into the device's address
// space, or nullptr (pageable memory, or not mapped).
static void *mapped_device_pointer(const void *host) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, host) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unregistered pointer
    return nullptr;
  }
  if (at.type != cudaMemoryTypeHost || at.devicePointer == nullptr) return nullptr;
  return at.devicePointer;
}

svo_status trace_rays_host(svo_scene *s, const float *rays_host, uint64_t n, svo_hit *hits_host,
                           uint32_t *ray_flags_host, uint32_t flags, void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "trace_rays_host: scene is NULL");
  if (n == 0) return ok();
  if (!rays_host || !hits_host) return fail(SVO_ERR_ARG, "trace_rays_host: rays/hits is NULL");
  if (flags & SVO_TRACE_STATS) return fail(SVO_ERR_ARG, "trace_rays_host: STATS needs a device stats buffer");
  if (flags & SVO_TRACE_REUSE) return fail(SVO_ERR_ARG, "trace_rays_host: REUSE needs the previous hits on the device");
  if (n > 0xFFFFFFFFull) return fail(SVO_ERR_LIMIT, "trace_rays_host: %llu rays", (unsigned long long)n);
  CK(cudaSetDevice(s->ctx->device));
  cudaStream_t st = (cudaStream_t)stream;
  // Small batches in page-locked buffers that the device can address (on
  // GB300 over the chip-to-chip link) are read and written by the kernels
  // directly, with no staging copy: the lowest latency for one call.
  if (n <= kZeroCopyMaxRays) {
    const void *dev_rays = mapped_device_pointer(rays_host);
    void *dev_hits = mapped_device_pointer(hits_host);
    void *dev_flags = ray_flags_host ? mapped_device_pointer(ray_flags_host) : nullptr;
    if (dev_rays && dev_hits && (!ray_flags_host || dev_flags) && !(reinterpret_cast<uintptr_t>(dev_rays) & 15) &&
        !(reinterpret_cast<uintptr_t>(dev_hits) & 15))
      return trace_rays(s, static_cast<const float *>(dev_rays), n, static_cast<svo_hit *>(dev_hits),
                        static_cast<uint32_t *>(dev_flags), flags & ~SVO_TRACE_DEFER_FIX, nullptr, stream);
  }
  // Otherwise the rays are copied in by the copy engines, to one of two
  // staging halves that successive calls alternate between.  A call's
  // copy-in waits only for its half to be free, not for the caller's earlier
  // work, so in a frame loop the next frame's rays stream in while this
  // frame is traced.
  //   * Mapped page-locked hits (and flags) are written by the kernels
  //     directly, and the rays are traced in one launch (split launches would
  //     run their load-imbalance tails one after another).
  //   * Other hits buffers are staged too: chunks of ~512 K rays (whole image
  //     rows with SVO_TRACE_IMAGE) are copied in, traced (with their FP64
  //     pass) and copied out on three streams, so that the copies of one
  //     chunk overlap the trace of another.
  void *dev_hits = mapped_device_pointer(hits_host);
  void *dev_flags = ray_flags_host ? mapped_device_pointer(ray_flags_host) : nullptr;
  const bool out_direct =
      dev_hits && !(reinterpret_cast<uintptr_t>(dev_hits) & 15) && (!ray_flags_host || dev_flags);
  constexpr unsigned long long kChunk = 1ull << 19;
  unsigned long long chunk = out_direct ? n : kChunk;
  if (!out_direct && (flags & SVO_TRACE_IMAGE_TILES)) {
    const unsigned long long w = flags >> 16;
    if (w > 0) chunk = (kChunk / w > 0 ? kChunk / w : 1) * w;
  }
  const unsigned long long n_chunks = (n + chunk - 1) / chunk;
  char *stage = nullptr;
  Slot *slp = nullptr;
  int half = 0;
  {
    std::lock_guard<std::mutex> g(s->ctx->mu);
    Slot &sl = s->ctx->slots[stream];
    if (n > sl.stage_rays) {
      if (sl.d_stage) {
        CK(cudaStreamSynchronize(st));
        for (cudaStream_t ps : sl.pipe)
          if (ps) CK(cudaStreamSynchronize(ps));
        CK(cudaFree(sl.d_stage));
        sl.d_stage = nullptr;
        sl.stage_rays = 0;
      }
      cudaError_t e = cudaMalloc(&sl.d_stage, 2 * stage_half_bytes(n));
      if (e != cudaSuccess) return fail(SVO_ERR_OOM, "trace_rays_host: staging: %s", cudaGetErrorString(e));
      sl.stage_rays = n;
    }
    for (cudaEvent_t &e : sl.stage_free)
      if (!e) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    for (cudaStream_t &ps : sl.pipe)
      if (!ps) CK(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
    while (sl.pipe_ev.size() < 2 * n_chunks + 2) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      sl.pipe_ev.push_back(e);
    }
    stage = sl.d_stage;
    slp = &sl;
    half = sl.stage_turn;
    sl.stage_turn ^= 1;
  }
  const unsigned long long cap = slp->stage_rays;
  stage += (size_t)half * stage_half_bytes(cap);
  float *d_rays = reinterpret_cast<float *>(stage);
  svo_hit *d_hits = reinterpret_cast<svo_hit *>(stage + cap * 32);
  uint32_t *d_flags = ray_flags_host ? reinterpret_cast<uint32_t *>(stage + cap * 48) : nullptr;
  // with direct hit writes there is one trace, run on the caller's stream
  cudaStream_t h2d = slp->pipe[0], comp = out_direct ? st : slp->pipe[1], d2h = slp->pipe[2];
  cudaEvent_t *ev = slp->pipe_ev.data();
  // the copy-in waits for its staging half only; the traces wait for the
  // caller's earlier work (poses, refit) ...
  CK(cudaStreamWaitEvent(h2d, slp->stage_free[half], 0));
  if (!out_direct) {
    CK(cudaEventRecord(ev[0], st));
    CK(cudaStreamWaitEvent(comp, ev[0], 0));
    CK(cudaStreamWaitEvent(d2h, ev[0], 0));
  }
  for (unsigned long long k = 0; k < n_chunks; ++k) {
    const unsigned long long off = k * chunk, m = (n - off) < chunk ? (n - off) : chunk;
    CK(cudaMemcpyAsync(d_rays + off * 8, rays_host + off * 8, m * 32, cudaMemcpyHostToDevice, h2d));
    CK(cudaEventRecord(ev[2 + 2 * k], h2d));
    CK(cudaStreamWaitEvent(comp, ev[2 + 2 * k], 0));
    svo_hit *hits_k = out_direct ? static_cast<svo_hit *>(dev_hits) + off : d_hits + off;
    uint32_t *flags_k = out_direct ? (dev_flags ? static_cast<uint32_t *>(dev_flags) + off : nullptr)
                                   : (d_flags ? d_flags + off : nullptr);
    svo_status rc = trace_rays(s, d_rays + off * 8, m, hits_k, flags_k, flags & ~SVO_TRACE_DEFER_FIX, nullptr, comp);
    if (rc != SVO_OK) return rc;
    if (out_direct) continue;
    CK(cudaEventRecord(ev[3 + 2 * k], comp));
    CK(cudaStreamWaitEvent(d2h, ev[3 + 2 * k], 0));
    CK(cudaMemcpyAsync(hits_host + off, d_hits + off, m * 16, cudaMemcpyDeviceToHost, d2h));
    if (d_flags) CK(cudaMemcpyAsync(ray_flags_host + off, d_flags + off, m * 4, cudaMemcpyDeviceToHost, d2h));
  }
  // ... and the caller's stream continues once every hit is back
  if (out_direct) {
    CK(cudaEventRecord(slp->stage_free[half], st));
    return ok();
  }
  CK(cudaEventRecord(ev[1], d2h));
  CK(cudaEventRecord(slp->stage_free[half], d2h));
  CK(cudaStreamWaitEvent(st, ev[1], 0));
  return ok();
}

svo_status trace_hit_colors(svo_scene *s, const svo_hit *hits, uint64_t n, uint32_t background, uint32_t *rgb,
                            void *stream) {
  if (!s) return fail(SVO_ERR_ARG, "trace_hit_colors: scene is NULL");
  if (background > 0x00FFFFFFu) return fail(SVO_ERR_ARG, "trace_hit_colors: background 0x%x is not 0x00RRGGBB", background);
  if (n == 0) return ok();
  if (!hits || !rgb) return fail(SVO_ERR_ARG, "trace_hit_colors: NULL buffer");
  if (reinterpret_cast<uintptr_t>(hits) & 15) return fail(SVO_ERR_ARG, "trace_hit_colors: hits not 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(rgb) & 3) return fail(SVO_ERR_ARG, "trace_hit_colors: rgb not 4-byte aligned");
  CK(cudaSetDevice(s->ctx->device));
  CK(launch_hit_colors(reinterpret_cast<const uint4 *>(hits), n, s->d_stat, s->P, background, rgb, s->ctx->n_sm,
                       (cudaStream_t)stream));
  return ok();
}

svo_status trace_shade(svo_scene *s, const float *rays, const svo_hit *hits, uint64_t n, const float *light,
                       float ambient, uint32_t background, uint32_t *rgb, void *stream) {
  if (!s || !light) return fail(SVO_ERR_ARG, "trace_shade: NULL argument");
  if (background > 0x00FFFFFFu) return fail(SVO_ERR_ARG, "trace_shade: background 0x%x is not 0x00RRGGBB", background);
  if (!(ambient >= 0.f && ambient <= 1.f)) return fail(SVO_ERR_ARG, "trace_shade: ambient outside [0, 1]");
  ShadeArgs sa;
  const double lx = light[0], ly = light[1], lz = light[2];
  const double ll = std::sqrt(lx * lx + ly * ly + lz * lz);
  if (!(ll > 0.0) || !std::isfinite(ll)) return fail(SVO_ERR_ARG, "trace_shade: light must be finite and non-zero");
  sa.light[0] = lx / ll;
  sa.light[1] = ly / ll;
  sa.light[2] = lz / ll;
  sa.ambient = ambient;
  sa.background = background;
  if (n == 0) return ok();
  if (!rays || !hits || !rgb) return fail(SVO_ERR_ARG, "trace_shade: NULL buffer");
  if ((reinterpret_cast<uintptr_t>(rays) & 15) || (reinterpret_cast<uintptr_t>(hits) & 15))
    return fail(SVO_ERR_ARG, "trace_shade: rays and hits must be 16-byte aligned");
  if (reinterpret_cast<uintptr_t>(rgb) & 3) return fail(SVO_ERR_ARG, "trace_shade: rgb not 4-byte aligned");
  CK(cudaSetDevice(s->ctx->device));
  CK(launch_shade(reinterpret_cast<const float4 *>(rays), reinterpret_cast<const uint4 *>(hits), n, s->d_stat,
                  s->d_inv64, s->P, sa, rgb, s->ctx->n_sm, (cudaStream_t)stream));
  return ok();
}

svo_status svo_raygen_pinhole(svo_ctx *ctx, const svo_camera *cam, uint32_t width, uint32_t height, float *rays,
                              void *stream) {
  if (!ctx || !cam || !rays) return fail(SVO_ERR_ARG, "svo_raygen_pinhole: NULL argument");
  if (width == 0 || height == 0) return ok();
  if (reinterpret_cast<uintptr_t>(rays) & 15) return fail(SVO_ERR_ARG, "svo_raygen_pinhole: rays not 16-byte aligned");
  if (!(cam->fov_y_deg > 0.f && cam->fov_y_deg < 180.f)) return fail(SVO_ERR_ARG, "svo_raygen_pinhole: fov out of (0,180)");
  double f[3] = {(double)cam->target[0] - cam->eye[0], (double)cam->target[1] - cam->eye[1],
                 (double)cam->target[2] - cam->eye[2]};
  double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  if (!(fl > 0.0)) return fail(SVO_ERR_ARG, "svo_raygen_pinhole: eye == target");
  for (double &v : f) v /= fl;
  double up[3] = {cam->up[0], cam->up[1], cam->up[2]};
  double ul = std::sqrt(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
  if (!(ul > 0.0) || std::fabs((up[0] * f[0] + up[1] * f[1] + up[2] * f[2]) / ul) > 0.999) {
    up[0] = std::fabs(f[0]) < 0.9 ? 1.0 : 0.0;
    up[1] = 0.0;
    up[2] = std::fabs(f[0]) < 0.9 ? 0.0 : 1.0;
  }
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (double &v : r) v /= rl;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  RaygenArgs a;
  for (int k = 0; k < 3; ++k) {
    a.eye[k] = cam->eye[k];
    a.f[k] = (float)f[k];
    a.r[k] = (float)r[k];
    a.u[k] = (float)u[k];
  }
  const double th = std::tan(cam->fov_y_deg * 3.14159265358979323846 / 360.0);
  a.tan_y = (float)th;
  a.tan_x = (float)(th * width / height);
  a.inv_w = 1.0f / (float)width;
  a.inv_h = 1.0f / (float)height;
  a.tmin = cam->tmin;
  a.tmax = cam->tmax;
  a.width = width;
  a.height = height;
  CK(cudaSetDevice(ctx->device));
  CK(launch_raygen(a, rays, ctx->n_sm, (cudaStream_t)stream));
  return ok();
}

svo_status trace_fix_pending(svo_ctx *ctx, void *stream) {
  if (!ctx) return fail(SVO_ERR_ARG, "trace_fix_pending: ctx is NULL");
  CK(cudaSetDevice(ctx->device));
  TraceLaunch *L = nullptr;
  {
    std::lock_guard<std::mutex> g(ctx->mu);
    auto it = ctx->slots.find(stream);
    if (it == ctx->slots.end() || !it->second.pending) return ok();
    L = it->second.pending;
    it->second.pending = nullptr;
  }
  cudaError_t e = launch_fix(*L, ctx->n_sm, (cudaStream_t)stream);
  delete L;
  if (e != cudaSuccess) return fail(SVO_ERR_CUDA, "trace_fix_pending: %s", cudaGetErrorString(e));
  return ok();
}

}  // extern "C"
