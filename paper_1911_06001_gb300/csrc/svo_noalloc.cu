// svo_noalloc.cu -- trace_rays for callers that cannot allocate device memory.
//
// trace_rays keeps its scratch (the tile counter, the list of flagged rays and
// their contender leaves) in per-stream buffers that it grows with cudaMalloc
// the first time a larger ray count arrives.  Some callers cannot let that
// happen: a frame loop with a hard deadline, where cudaMalloc may synchronise
// the whole device, or a host application whose own allocator owns all device
// memory and forbids other allocations.  trace_rays_noalloc runs the same
// trace and FP64 kernels on a fixed scratch area that lives in this file as a
// static __device__ array: the library never calls cudaMalloc, cudaFree or an
// allocating library routine on this path.
//
// The array is part of the loaded module, so every GPU that loads the library
// holds it (kNoallocScratchBytes, about 15.7 MB) until the process exits.  All
// calls share it and it keeps the previous call's contents; the counters that
// must start at zero are cleared on `stream` at the start of every call.  Two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) therefore race on the array and must be serialised by the caller.
//
// The array's device address is looked up once per device and kept for the
// life of the process.  A cudaDeviceReset (or anything else that destroys the
// device's primary context) while the library is loaded would leave that
// address stale, so it is not supported.
//
// Ray ordering (SVO_TRACE_ORDER_DIR / _ORIGIN) and the two-launch wavefront
// shape (SVO_TRACE_WAVEFRONT) need per-ray scratch of their own and are
// rejected here, as are STATS and DEFER_FIX.  The launch record
// lives in static storage under a lock of its own, so the call puts nothing
// large on the caller's stack.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>
#include <string>

#include "svo_internal.h"

using namespace svo;

namespace {

constexpr unsigned long long kNoallocMaxRays = SVO_NOALLOC_MAX_RAYS;
constexpr unsigned long long kCounterBytes = 256;
constexpr unsigned long long kFixBytes = kNoallocMaxRays * sizeof(unsigned long long);
constexpr unsigned long long kOffBytes = kNoallocMaxRays * sizeof(uint32_t);
constexpr unsigned long long kCandEntries = kNoallocMaxRays * kPoolPerRay;
constexpr unsigned long long kCandBytes = kCandEntries * sizeof(uint4);
constexpr unsigned long long kNoallocScratchBytes = kCounterBytes + kFixBytes + kOffBytes + kCandBytes;

// The shared scratch: [counters | flagged-ray list | pool offsets | leaf pool].
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
std::mutex g_launch_mu;  // guards the static launch record of trace_rays_noalloc
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device, looked up once
// per device.  In host code the symbol itself is only a host-side stand-in, so
// the kernels must be given this address.
cudaError_t scratch_address(int device, unsigned char **out) {
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_ptr[device]);
  return cudaSuccess;
}

}  // namespace

// The scene's layout is private to svo_api.cu; these accessors live there.
namespace svo {
int scene_device(const svo_scene *s);
TraceItem scene_item(svo_scene *s, const float *rays, uint64_t n, svo_hit *hits, uint32_t *flags);
unsigned int *scene_err_word(const svo_scene *s);
int scene_sm_count(const svo_scene *s);
void scene_trace_config(const svo_scene *s, int *block, int *rays_per_lane);
svo_status set_last_error(svo_status code, const char *msg);
}

extern "C" svo_status trace_rays_noalloc(svo_scene *s, const float *rays, uint64_t n, svo_hit *hits,
                                         uint32_t *ray_flags, uint32_t flags, void *stream) {
  if (!s) return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: scene is NULL");
  if (n == 0) return SVO_OK;
  if (!rays || !hits) return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: rays/hits is NULL");
  if (n > kNoallocMaxRays) {
    char buf[160];
    snprintf(buf, sizeof(buf), "trace_rays_noalloc: %llu rays exceed the fixed scratch limit of %llu rays",
             (unsigned long long)n, kNoallocMaxRays);
    return set_last_error(SVO_ERR_LIMIT, buf);
  }
  if ((reinterpret_cast<uintptr_t>(rays) & 15) || (reinterpret_cast<uintptr_t>(hits) & 15))
    return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: rays and hits must be 16-byte aligned");
  if (flags & (SVO_TRACE_STATS | SVO_TRACE_DEFER_FIX | SVO_TRACE_ORDER_DIR | SVO_TRACE_ORDER_ORIGIN |
               SVO_TRACE_WAVEFRONT))
    return set_last_error(SVO_ERR_ARG,
                          "trace_rays_noalloc: STATS, DEFER_FIX, the ORDER flags and WAVEFRONT are not supported");
  constexpr uint32_t kReuseNeeds = SVO_TRACE_CULL | SVO_TRACE_SORT | SVO_TRACE_FP64_FIX;
  if ((flags & SVO_TRACE_REUSE) && (flags & kReuseNeeds) != kReuseNeeds)
    return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: SVO_TRACE_REUSE needs CULL | SORT | FP64_FIX");
  if ((flags & SVO_TRACE_GRID) &&
      ((flags & SVO_TRACE_REUSE) || (flags & (SVO_TRACE_CULL | SVO_TRACE_SORT)) != (SVO_TRACE_CULL | SVO_TRACE_SORT)))
    return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: SVO_TRACE_GRID needs CULL | SORT and excludes REUSE");
  const int dev = scene_device(s);
  if (dev < 0 || dev >= kMaxDevices) return set_last_error(SVO_ERR_ARG, "trace_rays_noalloc: bad device");
  cudaError_t e = cudaSetDevice(dev);
  unsigned char *base = nullptr;
  if (e == cudaSuccess) e = scratch_address(dev, &base);
  if (e != cudaSuccess) {
    std::string m = std::string("trace_rays_noalloc: ") + cudaGetErrorString(e);
    return set_last_error(SVO_ERR_CUDA, m.c_str());
  }
  cudaStream_t st = (cudaStream_t)stream;
  // static launch record (about 16 KB): neither the host heap nor the caller's stack
  static TraceLaunch launch;
  std::lock_guard<std::mutex> guard(g_launch_mu);
  TraceLaunch *L = &launch;
  L->items[0] = scene_item(s, rays, n, hits, ray_flags);
  if (flags & SVO_TRACE_IMAGE_TILES) L->items[0].width = flags >> 16;
  L->n_items = 1;
  L->flags = flags;
  L->stats = nullptr;
  int block = 128, rpl = 1;
  scene_trace_config(s, &block, &rpl);
  L->block = block;
  L->rays_per_lane = rpl;
  L->n_tiles = layout_tiles(L->items, 1, rpl);
  L->tile_counter = reinterpret_cast<unsigned long long *>(base);
  L->fix_count = reinterpret_cast<unsigned int *>(base + sizeof(unsigned long long));
  L->fix_list = reinterpret_cast<unsigned long long *>(base + kCounterBytes);
  L->fix_capacity = kNoallocMaxRays;
  L->fix_off = reinterpret_cast<uint32_t *>(base + kCounterBytes + kFixBytes);
  L->fix_cand = reinterpret_cast<uint4 *>(base + kCounterBytes + kFixBytes + kOffBytes);
  L->cand_capacity = kCandEntries;
  L->cand_count = reinterpret_cast<unsigned int *>(base + 2 * sizeof(unsigned long long));
  L->err = scene_err_word(s);
  L->top = nullptr;  // no shared-memory top levels on this path
  L->top_nodes = 0;
  L->top_levels = 0;
  L->queue = nullptr;  // no wavefront shape on this path
  L->queue_count = nullptr;
  L->queue_tile = nullptr;
  // clear what the kernels expect at zero: the tile counter, the list count and the pool count
  e = cudaMemsetAsync(base, 0, 3 * sizeof(unsigned long long), st);
  if (e == cudaSuccess && (flags & SVO_TRACE_GRID)) {
    GridLaunch gl;
    if (grid_jobs(L->items, 1, gl) > 0) e = launch_grid(gl, st);
  }
  if (e == cudaSuccess) e = launch_trace(*L, scene_sm_count(s), st);
  if (e == cudaSuccess)  // pose changes are tracked relative to the scene's latest trace
    e = cudaMemsetAsync(const_cast<uint8_t *>(L->items[0].dirty), 0, (size_t)L->items[0].n_parts, st);
  if (e == cudaSuccess && (flags & SVO_TRACE_FP64_FIX)) e = launch_fix(*L, scene_sm_count(s), st);
  if (e != cudaSuccess) {
    std::string m = std::string("trace_rays_noalloc: ") + cudaGetErrorString(e);
    return set_last_error(SVO_ERR_CUDA, m.c_str());
  }
  return SVO_OK;
}
