// k_color.cu -- colour lookup of closest hits.
//
// The hit buffer of the paper (Sec. IV-C) carries, per pixel, what shading
// needs of the closest hit; for a voxel model that is the hit leaf's colour.
// Here a hit (part, voxel id) is resolved to its leaf by walking the part's
// octree from the root along the voxel's coordinate bits: at level l the
// child octant is bit D-1-l of x, y and z (bit 0 of the octant = +x).  The
// leaf-level node's first_child indexes the leaf payload array directly.
#include <cuda_runtime.h>

#include <cstdint>

#include "svo_internal.h"

namespace svo {

namespace {

__global__ void k_hit_colors(const uint4 *__restrict__ hits, unsigned long long n,
                             const PartStatic *__restrict__ stat, int n_parts, uint32_t background,
                             uint32_t *__restrict__ rgb) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 h = __ldcs(&hits[i]);
    uint32_t out = background;
    if (h.y != kMissPart) {
      out = SVO_COLOR_INVALID;
      if (h.y < (uint32_t)n_parts) {
        const PartStatic ps = stat[h.y];
        const int D = ps.depth;
        const unsigned long long vox = ((unsigned long long)h.w << 32) | h.z;
        const unsigned long long mask = (1ull << D) - 1ull;
        if (ps.n_nodes > 0 && (vox >> (3 * D)) == 0ull) {
          const uint32_t x = (uint32_t)(vox & mask), y = (uint32_t)((vox >> D) & mask),
                         z = (uint32_t)((vox >> (2 * D)) & mask);
          uint32_t node = 0;
          for (int l = 0; l < D; ++l) {
            const int b = D - 1 - l;
            const uint32_t k = ((x >> b) & 1u) | (((y >> b) & 1u) << 1) | (((z >> b) & 1u) << 2);
            const uint2 d = __ldg(&ps.nodes[node]);
            const uint32_t cmask = d.y & 0xFFu;
            if (!((cmask >> k) & 1u)) break;  // not occupied
            const uint32_t idx = d.x + __popc(cmask & ((1u << k) - 1u));
            if (l == D - 1) {
              if (idx < ps.n_leaves) out = __ldg(&ps.rgb[idx]);
            } else {
              if (idx >= ps.n_nodes) break;
              node = idx;
            }
          }
        }
      }
    }
    __stcs(&rgb[i], out);
  }
}

}  // namespace

cudaError_t launch_hit_colors(const uint4 *hits, unsigned long long n, const PartStatic *stat, int n_parts,
                              uint32_t background, uint32_t *rgb, int n_sm, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  constexpr int kThreads = 256;
  const unsigned long long want = (n + kThreads - 1) / kThreads;
  const unsigned long long cap = (unsigned long long)n_sm * 8ull;  // 8 resident blocks per SM
  const unsigned int grid = (unsigned int)(want < cap ? want : cap);
  k_hit_colors<<<grid, kThreads, 0, stream>>>(hits, n, stat, n_parts, background, rgb);
  return cudaGetLastError();
}

}  // namespace svo
