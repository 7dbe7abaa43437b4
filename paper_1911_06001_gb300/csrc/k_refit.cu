// k_refit.cu -- per-frame pose pipeline of a scene, one thread block.
//
//  1. compose the transform tree in FP64, parents first: W_i = W_parent(i) o L_i
//     (the paper gives one transform per SVO, Sec. III; the tree is a
//     generalisation in which a root part has W_i = L_i);
//  2. invert each W_i in FP64 (Eq. 3): A^-1 = adj(A)/det(A), b' = -A^-1 b,
//     which for a rigid pose equals the transposed rotation and the negated,
//     rotated translation (Sec. III-A);
//  3. emit the FP32 world->local matrix the trace kernel uses, the local
//     coordinates of the FP32 sphere centre (FP64-accurate), and bounds on
//     norms for the trace kernel's rounding-error bound;
//  4. refit the part bounding spheres (Sec. IV-A: centre and radius follow
//     from the pose).  The sphere bounds the asset's occupied box (the
//     smallest grid-aligned box holding its leaves, found at upload) rather
//     than its whole unit cube: centre = image of the box centre, radius =
//     farthest image of a box corner, rounded outward to FP32.  Any sphere
//     that holds every leaf culls no hit; the tighter one culls more rays;
//  5. rebuild the cluster level of the sphere hierarchy: parts sorted by the
//     Morton code of their sphere centres, runs of 8 enclosed by one sphere
//     (the scene-level structure the paper proposes for many parts, Sec. V-E).
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>

#include "svo_internal.h"

namespace svo {

namespace {

constexpr int kRefitThreads = 256;  // block size for large scenes; one warp for <= 32 parts

// Poses passed by value in the kernel parameters (no host-to-device copy),
// in size classes so that a small scene's launch carries a small parameter
// block (the whole block is fetched before the kernel starts).
template <int CAP>
struct InlinePoses {
  double local[CAP * 12];
};

__device__ __forceinline__ void compose_affine(const double *p, const double *q, double *out) {
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    double r0 = p[i * 4 + 0] * q[0] + p[i * 4 + 1] * q[4] + p[i * 4 + 2] * q[8];
    double r1 = p[i * 4 + 0] * q[1] + p[i * 4 + 1] * q[5] + p[i * 4 + 2] * q[9];
    double r2 = p[i * 4 + 0] * q[2] + p[i * 4 + 1] * q[6] + p[i * 4 + 2] * q[10];
    double r3 = p[i * 4 + 0] * q[3] + p[i * 4 + 1] * q[7] + p[i * 4 + 2] * q[11] + p[i * 4 + 3];
    out[i * 4 + 0] = r0;
    out[i * 4 + 1] = r1;
    out[i * 4 + 2] = r2;
    out[i * 4 + 3] = r3;
  }
}

__device__ __forceinline__ unsigned int spread10(unsigned int v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Shared-memory layout of one refit: every per-part intermediate stays on
// chip, so the phases below chain no global-memory round trips (the block
// is alone on its SM and latency-bound).
struct RefitSmem {
  double *world;             // P x 12
  float4 *sph;               // P
  float4 *cl;                // clusters
  unsigned long long *key;   // P
  float *na;                 // P
  int32_t *ord;              // P
  int32_t *parent;           // P
  int32_t *lorder;           // P
  int32_t *lstart;           // levels + 1
  float *red;                // 6 x threads
};

__host__ __device__ inline size_t refit_smem_bytes(int P, int NC, int L, int nthr) {
  return (size_t)P * (12 * sizeof(double) + sizeof(unsigned long long) + sizeof(float4) + sizeof(float) +
                      3 * sizeof(int32_t)) +
         (size_t)NC * sizeof(float4) + (size_t)(L + 1) * sizeof(int32_t) + 6 * (size_t)nthr * sizeof(float) + 64;
}

__device__ inline RefitSmem carve(unsigned char *base, int P, int NC, int L, int nthr) {
  RefitSmem m;
  // 16-byte items first: every offset stays aligned for any P
  m.world = reinterpret_cast<double *>(base);
  m.sph = reinterpret_cast<float4 *>(m.world + 12 * P);
  m.cl = m.sph + P;
  m.key = reinterpret_cast<unsigned long long *>(m.cl + NC);
  m.na = reinterpret_cast<float *>(m.key + P);
  m.ord = reinterpret_cast<int32_t *>(m.na + P);
  m.parent = m.ord + P;
  m.lorder = m.parent + P;
  m.lstart = m.lorder + P;
  m.red = reinterpret_cast<float *>(m.lstart + L + 1);
  return m;
}

template <bool INLINE, int CAP>
__global__ void __launch_bounds__(kRefitThreads) k_refit(RefitArgs a, const __grid_constant__ InlinePoses<CAP> poses) {
  const int P = a.n_parts;
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  extern __shared__ __align__(16) unsigned char refit_smem[];
  const RefitSmem sm = carve(refit_smem, P, a.n_clusters, a.n_levels, nthr);
  if (INLINE) {
    // keep the device copy of the local poses in step with what is composed
    for (int k = tid; k < P * 12; k += nthr) const_cast<double *>(a.local)[k] = poses.local[k];
  }
  const double *local = INLINE ? poses.local : a.local;
  // tree topology to shared memory (independent loads, one round trip)
  for (int i = tid; i < P; i += nthr) {
    sm.parent[i] = a.stat[i].parent;
    sm.lorder[i] = a.level_order[i];
  }
  for (int i = tid; i <= a.n_levels; i += nthr) sm.lstart[i] = a.level_start[i];
  __syncthreads();

  // 1. compose, level by level (parents are on earlier levels)
  for (int L = 0; L < a.n_levels; ++L) {
    const int b = sm.lstart[L], e = sm.lstart[L + 1];
    for (int j = b + tid; j < e; j += nthr) {
      const int i = sm.lorder[j];
      const int p = sm.parent[i];
      const double *Li = local + 12 * i;
      double *Wi = sm.world + 12 * i;
      double out[12];
      if (p < 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = Li[k];
      } else {
        double Wp[12], L12[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          Wp[k] = sm.world[12 * p + k];
          L12[k] = Li[k];
        }
        compose_affine(Wp, L12, out);
      }
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        Wi[k] = out[k];
        a.world[12 * i + k] = out[k];
      }
    }
    __syncthreads();
  }

  // 2-4. per part: invert, FP32 rows, norms, sphere
  float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int i = tid; i < P; i += nthr) {
    double m[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) m[k] = sm.world[12 * i + k];
    const double A0 = m[0], A1 = m[1], A2 = m[2], A3 = m[4], A4 = m[5], A5 = m[6], A6 = m[8], A7 = m[9],
                 A8 = m[10];
    const double c00 = A4 * A8 - A5 * A7, c01 = A5 * A6 - A3 * A8, c02 = A3 * A7 - A4 * A6;
    const double det = A0 * c00 + A1 * c01 + A2 * c02;
    double inv[12];
    bool ok = isfinite(det) && fabs(det) > 0.0;
    if (ok) {
      const double rd = 1.0 / det;
      inv[0] = c00 * rd;
      inv[1] = (A2 * A7 - A1 * A8) * rd;
      inv[2] = (A1 * A5 - A2 * A4) * rd;
      inv[4] = c01 * rd;
      inv[5] = (A0 * A8 - A2 * A6) * rd;
      inv[6] = (A2 * A3 - A0 * A5) * rd;
      inv[8] = c02 * rd;
      inv[9] = (A1 * A6 - A0 * A7) * rd;
      inv[10] = (A0 * A4 - A1 * A3) * rd;
#pragma unroll
      for (int r = 0; r < 3; ++r)
        inv[r * 4 + 3] = -(inv[r * 4 + 0] * m[3] + inv[r * 4 + 1] * m[7] + inv[r * 4 + 2] * m[11]);
      for (int k = 0; k < 12; ++k) ok = ok && isfinite(inv[k]);
    }
    if (!ok) {
      atomicOr(a.err, kErrSingular);
      for (int k = 0; k < 12; ++k) inv[k] = 0.0;
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) a.inv64[12 * i + k] = inv[k];

    float f[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) f[k] = (float)inv[k];
    double rowsum = 0.0;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      double s = fabs((double)f[r * 4]) + fabs((double)f[r * 4 + 1]) + fabs((double)f[r * 4 + 2]);
      rowsum = fmax(rowsum, s);
    }
    // sphere of the occupied box [lo, hi] (it holds every leaf of the part):
    // centre = W (lo + hi) / 2, radius = farthest image of a box corner
    const PartStatic &ps = a.stat[i];
    double mid[3], ext[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      mid[q] = 0.5 * ((double)ps.box_lo[q] + (double)ps.box_hi[q]);
      ext[q] = 0.5 * ((double)ps.box_hi[q] - (double)ps.box_lo[q]);
    }
    double c[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) c[r] = m[r * 4] * mid[0] + m[r * 4 + 1] * mid[1] + m[r * 4 + 2] * mid[2] + m[r * 4 + 3];
    double r2 = 0.0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double qx = (k & 1) ? ext[0] : -ext[0], qy = (k & 2) ? ext[1] : -ext[1], qz = (k & 4) ? ext[2] : -ext[2];
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double v = m[r * 4] * qx + m[r * 4 + 1] * qy + m[r * 4 + 2] * qz;
        s += v * v;
      }
      r2 = fmax(r2, s);
    }
    const float cfx = (float)c[0], cfy = (float)c[1], cfz = (float)c[2];
    const double dcx = c[0] - cfx, dcy = c[1] - cfy, dcz = c[2] - cfz;
    const double rr = (sqrt(r2) + sqrt(dcx * dcx + dcy * dcy + dcz * dcz)) * (1.0 + 1e-12);
    // local coordinates of the FP32 centre (close to the box centre)
    float lc[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      lc[q] = (float)(inv[q * 4] * (double)cfx + inv[q * 4 + 1] * (double)cfy + inv[q * 4 + 2] * (double)cfz +
                      inv[q * 4 + 3]);
    PartHot h;
    h.r0 = make_float4(f[0], f[1], f[2], lc[0]);
    h.r1 = make_float4(f[4], f[5], f[6], lc[1]);
    h.r2 = make_float4(f[8], f[9], f[10], lc[2]);
    // a singular pose or an empty asset disables the sphere: no ray tests the part
    h.sphere = make_float4(cfx, cfy, cfz, (ok && ps.n_nodes > 0) ? __double2float_ru(rr) : -1.0f);
    a.hot[i] = h;
    sm.sph[i] = h.sphere;
    PartAux x;
    x.nodes = a.stat[i].nodes;
    x.n_nodes = a.stat[i].n_nodes;
    x.depth = a.stat[i].depth;
    x.n_ainv = __double2float_ru(rowsum * (1.0 + 1e-12));
    x.spare0 = 0.f;
    x.spare1 = 0.f;
    {
      double dg = 0.0;
#pragma unroll
      for (int rr2 = 0; rr2 < 3; ++rr2) {
        const double v = m[rr2 * 4] + m[rr2 * 4 + 1] + m[rr2 * 4 + 2];
        dg += v * v;
      }
      x.hdiag = (float)(sqrt(dg) * ldexp(1.0, -a.stat[i].depth));
    }
    a.aux[i] = x;
    sm.na[i] = x.n_ainv;
    mn[0] = fminf(mn[0], cfx);
    mn[1] = fminf(mn[1], cfy);
    mn[2] = fminf(mn[2], cfz);
    mx[0] = fmaxf(mx[0], cfx);
    mx[1] = fmaxf(mx[1], cfy);
    mx[2] = fmaxf(mx[2], cfz);
  }
  // bounding box of the sphere centres (block reduction)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    sm.red[k * nthr + tid] = mn[k];
    sm.red[(3 + k) * nthr + tid] = mx[k];
  }
  __syncthreads();
  for (int w = nthr / 2; w > 0; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        sm.red[k * nthr + tid] = fminf(sm.red[k * nthr + tid], sm.red[k * nthr + tid + w]);
        sm.red[(3 + k) * nthr + tid] = fmaxf(sm.red[(3 + k) * nthr + tid], sm.red[(3 + k) * nthr + tid + w]);
      }
    }
    __syncthreads();
  }
  const float bx0 = sm.red[0], by0 = sm.red[nthr], bz0 = sm.red[2 * nthr];
  const float bx1 = sm.red[3 * nthr], by1 = sm.red[4 * nthr], bz1 = sm.red[5 * nthr];
  const float ex = fmaxf(bx1 - bx0, 1e-30f), ey = fmaxf(by1 - by0, 1e-30f), ez = fmaxf(bz1 - bz0, 1e-30f);
  // 5. Morton keys and a rank sort (P <= kMaxParts)
  for (int i = tid; i < P; i += nthr) {
    const float4 s = sm.sph[i];
    const unsigned int qx = (unsigned int)fminf(fmaxf((s.x - bx0) / ex * 1023.0f, 0.0f), 1023.0f);
    const unsigned int qy = (unsigned int)fminf(fmaxf((s.y - by0) / ey * 1023.0f, 0.0f), 1023.0f);
    const unsigned int qz = (unsigned int)fminf(fmaxf((s.z - bz0) / ez * 1023.0f, 0.0f), 1023.0f);
    const unsigned int mc = spread10(qx) | (spread10(qy) << 1) | (spread10(qz) << 2);
    sm.key[i] = ((unsigned long long)mc << 11) | (unsigned long long)i;
  }
  __syncthreads();
  for (int i = tid; i < P; i += nthr) {
    const unsigned long long k = sm.key[i];
    int rank = 0;
    for (int j = 0; j < P; ++j) rank += (sm.key[j] < k) ? 1 : 0;
    sm.ord[rank] = i;
    a.order[rank] = i;
  }
  __syncthreads();
  for (int cidx = tid; cidx < a.n_clusters; cidx += nthr) {
    const int first = cidx * kClusterSize;
    const int cnt = min(kClusterSize, P - first);
    double lo[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, hi[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    float na = 0.f;
    bool any = false;
    for (int k = 0; k < cnt; ++k) {
      const int p = sm.ord[first + k];
      const float4 s = sm.sph[p];
      if (s.w < 0.f) continue;
      any = true;
      lo[0] = fmin(lo[0], (double)s.x - s.w);
      lo[1] = fmin(lo[1], (double)s.y - s.w);
      lo[2] = fmin(lo[2], (double)s.z - s.w);
      hi[0] = fmax(hi[0], (double)s.x + s.w);
      hi[1] = fmax(hi[1], (double)s.y + s.w);
      hi[2] = fmax(hi[2], (double)s.z + s.w);
      na = fmaxf(na, sm.na[p]);
    }
    Cluster cl;
    if (any) {
      double C[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
      const float Cx = (float)C[0], Cy = (float)C[1], Cz = (float)C[2];
      double R = 0.0;
      for (int k = 0; k < cnt; ++k) {
        const int p = sm.ord[first + k];
        const float4 s = sm.sph[p];
        if (s.w < 0.f) continue;
        const double dx = (double)s.x - Cx, dy = (double)s.y - Cy, dz = (double)s.z - Cz;
        R = fmax(R, sqrt(dx * dx + dy * dy + dz * dz) + (double)s.w);
      }
      cl.sphere = make_float4(Cx, Cy, Cz, __double2float_ru(R * (1.0 + 1e-12)));
    } else {
      cl.sphere = make_float4(0.f, 0.f, 0.f, -1.0f);
    }
    cl.aux = make_float4(na, 0.f, 0.f, __uint_as_float((unsigned int)first | ((unsigned int)cnt << 16)));
    a.clusters[cidx] = cl;
    sm.cl[cidx] = cl.sphere;
  }
  __syncthreads();
  if (tid == 0) {
    // a sphere around all cluster spheres: the frame of origin-based ray ordering
    const float Cx = 0.5f * (bx0 + bx1), Cy = 0.5f * (by0 + by1), Cz = 0.5f * (bz0 + bz1);
    float R = 0.f;
    for (int c = 0; c < a.n_clusters; ++c) {
      const float4 s = sm.cl[c];
      if (s.w < 0.f) continue;
      const float dx = s.x - Cx, dy = s.y - Cy, dz = s.z - Cz;
      R = fmaxf(R, sqrtf(dx * dx + dy * dy + dz * dz) + s.w);
    }
    *a.bound = make_float4(Cx, Cy, Cz, R);
  }
}

}  // namespace

template <bool INLINE, int CAP>
cudaError_t launch_refit_t(const RefitArgs &a, const double *host_local, int threads, size_t smem,
                           cudaStream_t stream) {
  InlinePoses<CAP> p;
  if (INLINE)
    for (int k = 0; k < a.n_parts * 12; ++k) p.local[k] = host_local[k];
  cudaError_t e = cudaFuncSetAttribute(k_refit<INLINE, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_refit<INLINE, CAP><<<1, threads, smem, stream>>>(a, p);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitArgs &a, const double *host_local, cudaStream_t stream) {
  static_assert(kInlinePoseParts == 256, "size classes below");
  const int threads = a.n_parts <= 32 ? 32 : kRefitThreads;
  const size_t smem = refit_smem_bytes(a.n_parts, a.n_clusters, a.n_levels, threads);
  if (host_local && a.n_parts <= 16) return launch_refit_t<true, 16>(a, host_local, threads, smem, stream);
  if (host_local && a.n_parts <= 64) return launch_refit_t<true, 64>(a, host_local, threads, smem, stream);
  if (host_local && a.n_parts <= 256) return launch_refit_t<true, 256>(a, host_local, threads, smem, stream);
  return launch_refit_t<false, 1>(a, nullptr, threads, smem, stream);
}

}  // namespace svo
