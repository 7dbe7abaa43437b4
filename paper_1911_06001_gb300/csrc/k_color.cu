// k_color.cu -- what shading needs of the closest hits.
//
// The hit buffer of the paper (Sec. IV-C) carries, per pixel, the closest
// hit's colour and normal for shading.  For a voxel model:
//   * colour: the hit leaf's payload.  A hit (part, voxel id) is resolved to
//     its leaf by walking the part's octree from the root along the voxel's
//     coordinate bits: at level l the child octant is bit D-1-l of x, y and z
//     (bit 0 of the octant = +x); the leaf-level node's first_child indexes
//     the leaf payload array directly;
//   * normal: the face of the leaf's box through which the ray enters, mapped
//     to world space by the inverse transpose of the part's pose (so that
//     shear and anisotropic scale keep it perpendicular to the face).
// trace_shade combines both into a Lambert-lit 8-bit image.  Its decisions
// (entry face, rounding of each channel) are taken in FP64, like the FP64
// re-intersection pass, so that they match an FP64 evaluation of the same
// rule except within rounding distance of a tie.
#include <cuda_runtime.h>

#include <cstdint>

#include "svo_internal.h"

namespace svo {

namespace {

// Payload of the leaf (part, vox) names, SVO_COLOR_INVALID if it names none.
__device__ __forceinline__ uint32_t leaf_color(const PartStatic &ps, unsigned long long vox) {
  const int D = ps.depth;
  const unsigned long long mask = (1ull << D) - 1ull;
  if (ps.n_nodes == 0 || (vox >> (3 * D)) != 0ull) return SVO_COLOR_INVALID;
  const uint32_t x = (uint32_t)(vox & mask), y = (uint32_t)((vox >> D) & mask), z = (uint32_t)((vox >> (2 * D)) & mask);
  uint32_t node = 0;
  for (int l = 0; l < D; ++l) {
    const int b = D - 1 - l;
    const uint32_t k = ((x >> b) & 1u) | (((y >> b) & 1u) << 1) | (((z >> b) & 1u) << 2);
    const uint2 d = __ldg(&ps.nodes[node]);
    const uint32_t cmask = d.y & 0xFFu;
    if (!((cmask >> k) & 1u)) return SVO_COLOR_INVALID;  // not occupied
    const uint32_t idx = d.x + __popc(cmask & ((1u << k) - 1u));
    if (l == D - 1) return idx < ps.n_leaves ? __ldg(&ps.rgb[idx]) : SVO_COLOR_INVALID;
    if (idx >= ps.n_nodes) return SVO_COLOR_INVALID;
    node = idx;
  }
  return SVO_COLOR_INVALID;
}

__device__ __forceinline__ uint32_t hit_color(const uint4 h, const PartStatic *__restrict__ stat, int n_parts,
                                              uint32_t background) {
  if (h.y == kMissPart) return background;
  if (h.y >= (uint32_t)n_parts) return SVO_COLOR_INVALID;
  return leaf_color(stat[h.y], ((unsigned long long)h.w << 32) | h.z);
}

__global__ void k_hit_colors(const uint4 *__restrict__ hits, unsigned long long n,
                             const PartStatic *__restrict__ stat, int n_parts, uint32_t background,
                             uint32_t *__restrict__ rgb) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    __stcs(&rgb[i], hit_color(__ldcs(&hits[i]), stat, n_parts, background));
}

// One 8-bit channel scaled by s and rounded half up, at most 255.
__device__ __forceinline__ uint32_t shade_channel(uint32_t c, double s) {
  const double x = floor((double)c * s + 0.5);
  return x >= 255.0 ? 255u : (uint32_t)x;
}

__global__ void k_shade(const float4 *__restrict__ rays, const uint4 *__restrict__ hits, unsigned long long n,
                        const PartStatic *__restrict__ stat, const double *__restrict__ inv64, int n_parts,
                        ShadeArgs sa, uint32_t *__restrict__ rgb) {
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 h = __ldcs(&hits[i]);
    uint32_t out = hit_color(h, stat, n_parts, sa.background);
    if (h.y != kMissPart && out != SVO_COLOR_INVALID) {
      const float4 o = __ldcs(&rays[2 * i]), d = __ldcs(&rays[2 * i + 1]);
      const PartStatic ps = stat[h.y];
      const double *m = inv64 + 12 * (size_t)h.y;
      const unsigned long long vox = ((unsigned long long)h.w << 32) | h.z;
      const int D = ps.depth;
      const unsigned long long mask = (1ull << D) - 1ull;
      const double size = __longlong_as_double((long long)(1023 - D) << 52);  // 2^-D
      const double ro[3] = {o.x, o.y, o.z}, rd[3] = {d.x, d.y, d.z};
      // entry face: the axis whose near-plane t is largest (lower axis on a tie)
      double te = -__longlong_as_double(0x7ff0000000000000ll);
      int kf = 0;
      double sgn = 0.0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double ol = m[4 * k] * ro[0] + m[4 * k + 1] * ro[1] + m[4 * k + 2] * ro[2] + m[4 * k + 3];
        const double dl = m[4 * k] * rd[0] + m[4 * k + 1] * rd[1] + m[4 * k + 2] * rd[2];
        if (dl == 0.0) continue;
        const double lo = (double)((vox >> (k * D)) & mask) * size;
        const double t = ((dl > 0.0 ? lo : lo + size) - ol) / dl;
        if (t > te) {
          te = t;
          kf = k;
          sgn = dl > 0.0 ? 1.0 : -1.0;
        }
      }
      double nx, ny, nz;
      if (te < (double)o.w || sgn == 0.0) {  // the ray starts inside the leaf: face the viewer
        nx = -rd[0];
        ny = -rd[1];
        nz = -rd[2];
      } else {  // outward face normal -sign(d'_k) e_k, through the inverse transpose
        nx = -sgn * m[4 * kf];
        ny = -sgn * m[4 * kf + 1];
        nz = -sgn * m[4 * kf + 2];
      }
      const double len = sqrt(nx * nx + ny * ny + nz * nz);
      const double cosl = (nx * sa.light[0] + ny * sa.light[1] + nz * sa.light[2]) / len;
      const double s = sa.ambient + (1.0 - sa.ambient) * (cosl > 0.0 ? cosl : 0.0);
      out = (shade_channel((out >> 16) & 255u, s) << 16) | (shade_channel((out >> 8) & 255u, s) << 8) |
            shade_channel(out & 255u, s);
    }
    __stcs(&rgb[i], out);
  }
}

unsigned int grid_for(unsigned long long n, int threads, int n_sm) {
  const unsigned long long want = (n + threads - 1) / threads;
  const unsigned long long cap = (unsigned long long)n_sm * 8ull;  // 8 resident blocks per SM
  return (unsigned int)(want < cap ? want : cap);
}

}  // namespace

cudaError_t launch_hit_colors(const uint4 *hits, unsigned long long n, const PartStatic *stat, int n_parts,
                              uint32_t background, uint32_t *rgb, int n_sm, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_hit_colors<<<grid_for(n, 256, n_sm), 256, 0, stream>>>(hits, n, stat, n_parts, background, rgb);
  return cudaGetLastError();
}

cudaError_t launch_shade(const float4 *rays, const uint4 *hits, unsigned long long n, const PartStatic *stat,
                         const double *inv64, int n_parts, const ShadeArgs &sa, uint32_t *rgb, int n_sm,
                         cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  k_shade<<<grid_for(n, 256, n_sm), 256, 0, stream>>>(rays, hits, n, stat, inv64, n_parts, sa, rgb);
  return cudaGetLastError();
}

}  // namespace svo
