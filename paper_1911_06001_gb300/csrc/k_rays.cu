// k_rays.cu -- primary-ray generation and ray ordering.
//
// k_raygen: one ray per pixel of a pinhole camera (the paper's renderer casts
// one primary ray per pixel, Sec. V), written as the 8-float ray records the
// trace reads.  Pixel (i, j) -> ray index j*W + i.
//
// Ray ordering: rays are permuted so that a warp traces rays that are close in
// direction (and, optionally, origin) and therefore walk the same spheres and
// octree nodes.  A 14-bit key per ray, a counting sort (histogram, exclusive
// scan, scatter), and the trace kernel reads rays through the permutation and
// writes every hit back at its ray's own index -- results do not change.
#include <cuda_runtime.h>

#include <cstdint>

#include "svo_internal.h"

namespace svo {

namespace {

constexpr int kKeyBits = 14;  // 16384 bins: the histogram (64 KiB) stays in L1 during the scan
constexpr int kBins = 1 << kKeyBits;

__global__ void k_raygen(RaygenArgs a, float4 *__restrict__ rays) {
  const unsigned long long n = (unsigned long long)a.width * a.height;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < n;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    const uint32_t i = (uint32_t)(k % a.width), j = (uint32_t)(k / a.width);
    const float sx = (2.0f * ((float)i + 0.5f) * a.inv_w - 1.0f) * a.tan_x;
    const float sy = (1.0f - 2.0f * ((float)j + 0.5f) * a.inv_h) * a.tan_y;
    float dx = a.f[0] + sx * a.r[0] + sy * a.u[0];
    float dy = a.f[1] + sx * a.r[1] + sy * a.u[1];
    float dz = a.f[2] + sx * a.r[2] + sy * a.u[2];
    const float inv = rsqrtf(dx * dx + dy * dy + dz * dz);
    dx *= inv;
    dy *= inv;
    dz *= inv;
    rays[2 * k] = make_float4(a.eye[0], a.eye[1], a.eye[2], a.tmin);
    rays[2 * k + 1] = make_float4(dx, dy, dz, a.tmax);
  }
}

__device__ __forceinline__ uint32_t spread2(uint32_t v) {  // 8 bits -> even bits of 16
  v &= 0xFFu;
  v = (v | (v << 4)) & 0x0F0Fu;
  v = (v | (v << 2)) & 0x3333u;
  v = (v | (v << 1)) & 0x5555u;
  return v;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 3 bits -> every third bit
  v &= 7u;
  return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}

// Cube-map face of a direction (3 bits) and its face coordinates in [0, 1).
__device__ __forceinline__ uint32_t dir_face(float dx, float dy, float dz, float &u, float &v) {
  const float ax = fabsf(dx), ay = fabsf(dy), az = fabsf(dz);
  uint32_t face;
  float m, a, b;
  if (ax >= ay && ax >= az) {
    face = dx >= 0.f ? 0u : 1u;
    m = ax;
    a = dy;
    b = dz;
  } else if (ay >= az) {
    face = dy >= 0.f ? 2u : 3u;
    m = ay;
    a = dx;
    b = dz;
  } else {
    face = dz >= 0.f ? 4u : 5u;
    m = az;
    a = dx;
    b = dy;
  }
  const float im = m > 0.f ? 1.0f / m : 0.f;
  u = fminf(fmaxf(0.5f * (a * im + 1.0f), 0.f), 0.999999f);
  v = fminf(fmaxf(0.5f * (b * im + 1.0f), 0.f), 0.999999f);
  return face;
}

// mode 1 (direction): face (3 bits) | 2D Morton of (u, v) at 5+5 bits.
// mode 2 (origin): face | Morton of the origin cell in a 4^3 grid over the
// scene's bounding sphere (6 bits) | 2D Morton of (u, v) at 2+2 bits.
__device__ __forceinline__ uint32_t ray_key(float4 o, float4 d, int mode, float4 bound) {
  float u, v;
  const uint32_t face = dir_face(d.x, d.y, d.z, u, v);
  if (mode == 1) {
    const uint32_t qu = (uint32_t)(u * 32.f), qv = (uint32_t)(v * 32.f);
    return (face << 10) | spread2(qu) | (spread2(qv) << 1);
  }
  const float s = bound.w > 0.f ? 2.0f / bound.w : 0.f;  // 4 cells across the diameter
  const int cx = min(max((int)floorf((o.x - bound.x) * s + 2.0f), 0), 3);
  const int cy = min(max((int)floorf((o.y - bound.y) * s + 2.0f), 0), 3);
  const int cz = min(max((int)floorf((o.z - bound.z) * s + 2.0f), 0), 3);
  const uint32_t cell = spread3((uint32_t)cx) | (spread3((uint32_t)cy) << 1) | (spread3((uint32_t)cz) << 2);
  const uint32_t qu = (uint32_t)(u * 4.f), qv = (uint32_t)(v * 4.f);
  return (face << 10) | (cell << 4) | spread2(qu) | (spread2(qv) << 1);
}

// Warp-uniform grid-stride loops (blockDim is a multiple of 32): every lane of a
// warp runs the same iterations, lanes past the end carry an out-of-range key,
// so the warp-wide match below always sees the full warp.
__global__ void k_order_keys(const float4 *__restrict__ rays, unsigned long long n, int mode,
                             const float4 *__restrict__ bound, uint16_t *__restrict__ keys,
                             unsigned int *__restrict__ hist) {
  const float4 b = *bound;
  const int lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w < n; w += stride) {
    const unsigned long long i = w + lane;
    const bool valid = i < n;
    uint32_t k = kBins;  // out of range: never counted
    if (valid) {
      const float4 o = __ldcs(&rays[2 * i]), d = __ldcs(&rays[2 * i + 1]);
      k = ray_key(o, d, mode, b) & (kBins - 1);
      keys[i] = (uint16_t)k;
    }
    // warp-aggregated histogram update: one atomic per distinct key in the warp
    const unsigned int peers = __match_any_sync(0xffffffffu, k);
    if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&hist[k], (unsigned int)__popc(peers));
  }
}

// Exclusive scan of kBins counters by one block of 1024 threads.
__device__ __forceinline__ void scan_bins(unsigned int *__restrict__ hist) {
  constexpr int kPer = kBins / 1024;
  __shared__ unsigned int part[1024];
  unsigned int local[kPer];
  unsigned int sum = 0;
  const int base = threadIdx.x * kPer;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    local[k] = sum;
    sum += hist[base + k];
  }
  part[threadIdx.x] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const unsigned int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  const unsigned int prefix = part[threadIdx.x] - sum;
#pragma unroll
  for (int k = 0; k < kPer; ++k) hist[base + k] = prefix + local[k];
}

__global__ void __launch_bounds__(1024) k_order_scan(unsigned int *__restrict__ hist) { scan_bins(hist); }

// The same counting sort for every item of a batch in one set of launches:
// each item keeps its own histogram, keys and permutation; warps run over the
// concatenation of the items' rays, and the warp-aggregated atomics group
// lanes by (item, key).
struct OrderBatch {
  OrderItem items[kMaxBatchItems];
  unsigned long long begin[kMaxBatchItems + 1];  // first ray of each item in the concatenation
  int n_items;
  int mode;
};

__device__ __forceinline__ int order_item_of(const OrderBatch &B, unsigned long long g) {
  int lo = 0, hi = B.n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.begin[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__global__ void k_order_zero_batch(const __grid_constant__ OrderBatch B) {
  unsigned int *h = B.items[blockIdx.x].hist;
  for (int k = threadIdx.x; k < kBins; k += blockDim.x) h[k] = 0u;
}

__global__ void k_order_keys_batch(const __grid_constant__ OrderBatch B) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = B.begin[B.n_items];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w < total;
       w += stride) {
    const unsigned long long g = w + lane;
    const bool valid = g < total;
    uint32_t tag = 0xFFFFFFFFu, k = 0;  // out of range: never counted
    int it = 0;
    if (valid) {
      it = order_item_of(B, g);
      const OrderItem &I = B.items[it];
      const unsigned long long i = g - B.begin[it];
      const float4 o = __ldcs(&I.rays[2 * i]), d = __ldcs(&I.rays[2 * i + 1]);
      k = ray_key(o, d, B.mode, *I.bound) & (kBins - 1);
      I.keys[i] = (uint16_t)k;
      tag = ((uint32_t)it << 16) | k;
    }
    const unsigned int peers = __match_any_sync(0xffffffffu, tag);
    if (valid && (__ffs(peers) - 1) == lane) atomicAdd(&B.items[it].hist[k], (unsigned int)__popc(peers));
  }
}

__global__ void __launch_bounds__(1024) k_order_scan_batch(const __grid_constant__ OrderBatch B) {
  scan_bins(B.items[blockIdx.x].hist);
}

__global__ void k_order_scatter_batch(const __grid_constant__ OrderBatch B) {
  const int lane = threadIdx.x & 31;
  const unsigned long long total = B.begin[B.n_items];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w < total;
       w += stride) {
    const unsigned long long g = w + lane;
    const bool valid = g < total;
    uint32_t tag = 0xFFFFFFFFu, k = 0;
    int it = 0;
    unsigned long long i = 0;
    if (valid) {
      it = order_item_of(B, g);
      i = g - B.begin[it];
      k = (uint32_t)B.items[it].keys[i];
      tag = ((uint32_t)it << 16) | k;
    }
    const unsigned int peers = __match_any_sync(0xffffffffu, tag);
    const int leader = __ffs(peers) - 1;
    unsigned int base = 0;
    if (valid && lane == leader) base = atomicAdd(&B.items[it].hist[k], (unsigned int)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) B.items[it].perm[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

__global__ void k_order_scatter(const uint16_t *__restrict__ keys, unsigned long long n,
                                unsigned int *__restrict__ offs, uint32_t *__restrict__ perm) {
  const int lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long w = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) - lane; w < n; w += stride) {
    const unsigned long long i = w + lane;
    const bool valid = i < n;
    const uint32_t k = valid ? (uint32_t)keys[i] : (uint32_t)kBins;
    const unsigned int peers = __match_any_sync(0xffffffffu, k);
    const int leader = __ffs(peers) - 1;
    unsigned int base = 0;
    if (valid && lane == leader) base = atomicAdd(&offs[k], (unsigned int)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) perm[base + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)i;
  }
}

}  // namespace

cudaError_t launch_raygen(const RaygenArgs &a, float *rays, int n_sm, cudaStream_t stream) {
  const unsigned long long n = (unsigned long long)a.width * a.height;
  unsigned long long blocks = (n + 255) / 256;
  if (blocks > (unsigned long long)n_sm * 16) blocks = (unsigned long long)n_sm * 16;
  if (blocks == 0) return cudaSuccess;
  k_raygen<<<(unsigned int)blocks, 256, 0, stream>>>(a, reinterpret_cast<float4 *>(rays));
  return cudaGetLastError();
}

size_t order_scratch_bytes(unsigned long long n) {
  return (size_t)kBins * sizeof(unsigned int) + ((n * sizeof(uint16_t) + 255) & ~255ull) + n * sizeof(uint32_t);
}

OrderItem order_item(const float *rays, unsigned long long n, const float4 *bound, void *scratch) {
  unsigned char *p = static_cast<unsigned char *>(scratch);
  OrderItem it;
  it.rays = reinterpret_cast<const float4 *>(rays);
  it.n = n;
  it.bound = bound;
  it.hist = reinterpret_cast<unsigned int *>(p);
  it.keys = reinterpret_cast<uint16_t *>(p + kBins * sizeof(unsigned int));
  it.perm = reinterpret_cast<uint32_t *>(p + kBins * sizeof(unsigned int) + ((n * sizeof(uint16_t) + 255) & ~255ull));
  return it;
}

cudaError_t launch_order_batch(const OrderItem *items, int n_items, int mode, int n_sm, cudaStream_t stream) {
  if (n_items <= 0 || n_items > kMaxBatchItems) return cudaErrorInvalidValue;
  OrderBatch *B = new OrderBatch();  // large: off the host stack
  B->n_items = n_items;
  B->mode = mode;
  B->begin[0] = 0;
  for (int i = 0; i < n_items; ++i) {
    B->items[i] = items[i];
    B->begin[i + 1] = B->begin[i] + items[i].n;
  }
  const unsigned long long total = B->begin[n_items];
  unsigned long long blocks = (total + 255) / 256;
  if (blocks > (unsigned long long)n_sm * 8) blocks = (unsigned long long)n_sm * 8;
  if (blocks == 0) blocks = 1;
  k_order_zero_batch<<<(unsigned int)n_items, 256, 0, stream>>>(*B);
  k_order_keys_batch<<<(unsigned int)blocks, 256, 0, stream>>>(*B);
  k_order_scan_batch<<<(unsigned int)n_items, 1024, 0, stream>>>(*B);
  k_order_scatter_batch<<<(unsigned int)blocks, 256, 0, stream>>>(*B);
  delete B;
  return cudaGetLastError();
}

cudaError_t launch_order(const float *rays, unsigned long long n, int mode, const float4 *bound, void *scratch,
                         uint32_t **perm_out, int n_sm, cudaStream_t stream) {
  unsigned char *p = static_cast<unsigned char *>(scratch);
  unsigned int *hist = reinterpret_cast<unsigned int *>(p);
  uint16_t *keys = reinterpret_cast<uint16_t *>(p + kBins * sizeof(unsigned int));
  uint32_t *perm = reinterpret_cast<uint32_t *>(p + kBins * sizeof(unsigned int) + ((n * sizeof(uint16_t) + 255) & ~255ull));
  cudaError_t e = cudaMemsetAsync(hist, 0, kBins * sizeof(unsigned int), stream);
  if (e != cudaSuccess) return e;
  unsigned long long blocks = (n + 255) / 256;
  if (blocks > (unsigned long long)n_sm * 8) blocks = (unsigned long long)n_sm * 8;
  k_order_keys<<<(unsigned int)blocks, 256, 0, stream>>>(reinterpret_cast<const float4 *>(rays), n, mode, bound, keys,
                                                          hist);
  k_order_scan<<<1, 1024, 0, stream>>>(hist);
  k_order_scatter<<<(unsigned int)blocks, 256, 0, stream>>>(keys, n, hist, perm);
  *perm_out = perm;
  return cudaGetLastError();
}

}  // namespace svo
