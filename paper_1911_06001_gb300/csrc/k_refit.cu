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
//     farthest image of a box corner.  Any sphere that holds every leaf culls
//     no hit; the tighter one culls more rays;
//  5. rebuild the cluster level of the sphere hierarchy: parts sorted by the
//     Morton code of their sphere centres, runs of 8 enclosed by one sphere
//     (the scene-level structure the paper proposes for many parts, Sec. V-E).
//
// GB300 issues FP64 at about two lanes per clock per SM, so one warp's FP64
// instruction occupies a sub-partition for ~64 clocks whatever its active
// lanes.  The kernel therefore (a) spreads the FP64 work of a part over
// three lanes (one matrix row each) and the parts over all eight warps, and
// (b) keeps FP64 for what must be exact -- compose, inverse, sphere centre
// and its local coordinates -- and computes the radii and norms in FP32 with
// upward-rounded error bounds, which only ever enlarge them.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <memory>
#include <mutex>

#include "svo_internal.h"

namespace svo {

namespace {

constexpr int kRefitThreads = 256;  // 8 warps: every FP64 sub-partition of the SM gets work
constexpr int kRefitWarps = kRefitThreads / 32;
constexpr int kQuadsPerPass = kRefitThreads / 4;  // parts handled at once (4 lanes each, 3 busy)
constexpr float kRelSlack = 9.5367431640625e-7f;   // 2^-20: covers FP32 rounding of the norms below

// Poses passed by value in the kernel parameters (no host-to-device copy),
// in size classes so that a small scene's launch carries a small parameter
// block (the whole block is fetched before the kernel starts).
template <int CAP>
struct InlinePoses {
  double local[CAP * 12];
};

__device__ __forceinline__ unsigned int spread10(unsigned int v) {
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Thread of the j-th item (part) of a pass.  A warp's FP64 instruction holds
// its sub-partition's FP64 pipe for the same time however few of its lanes
// are busy, so items fill one warp per sub-partition first (warps 0-3, one
// per sub-partition), eight lane groups deep, before warps 4-7 take items 32
// to 63: item j -> warp (j & 3) + 4 (j >> 5), lane group (j >> 2) & 7.  A
// 16-part scene then costs each sub-partition one warp's instructions, not
// two half-empty warps'.  Returns the item handled by thread t and the lane
// r (0..3) inside its group of four.
__device__ __forceinline__ int quad_item(int t, int &r) {
  static_assert(kRefitWarps == 8, "two warps per sub-partition");
  const int w = t >> 5, l = t & 31;
  r = l & 3;
  return 32 * (w >> 2) + 4 * (l >> 2) + (w & 3);
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

__device__ inline RefitSmem carve(unsigned char *base, int P, int NC, int L) {
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

// Upper bound of |x| for x = a - b evaluated in FP32.
__device__ __forceinline__ float abs_diff_up(float a, float b) {
  return fmaxf(fabsf(__fsub_ru(a, b)), fabsf(__fsub_rd(a, b)));
}

// Upper bound of sqrt(x^2 + y^2 + z^2) for non-negative x, y, z.
__device__ __forceinline__ float norm_up(float x, float y, float z) {
  return __fsqrt_ru(__fmaf_ru(x, x, __fmaf_ru(y, y, __fmul_ru(z, z))));
}

// The pose pipeline of one scene, run by one block.  local: where the local
// poses are read from; keep != nullptr: they are first copied to keep (the
// scene's device copy, kept in step with what is composed), and with
// read_keep the block then reads them back from there (a source in host
// memory is read once).
__device__ __forceinline__ void refit_scene(const RefitArgs &a, const double *local, double *keep, bool read_keep,
                                            unsigned char *refit_smem) {
  const int P = a.n_parts;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const RefitSmem sm = carve(refit_smem, P, a.n_clusters, a.n_levels);
  if (keep) {
    for (int k = tid; k < P * 12; k += kRefitThreads) keep[k] = local[k];
    if (read_keep) local = keep;  // visible to the block after the barrier below
  }
  // tree topology to shared memory (independent loads, one round trip)
  for (int i = tid; i < P; i += kRefitThreads) {
    sm.parent[i] = a.stat[i].parent;
    sm.lorder[i] = a.level_order[i];
  }
  for (int i = tid; i <= a.n_levels; i += kRefitThreads) sm.lstart[i] = a.level_start[i];
  __syncthreads();

  int r;  // lane inside the part's group of four: rows 0..2, lane 3 helps with the FP32 bounds
  const int q = quad_item(tid, r);
  const unsigned int qmask = 0xFu << (lane & ~3);

  // 1. compose, level by level (parents are on earlier levels); lane r
  //    computes row r of W_i = W_parent o L_i
  for (int L = 0; L < a.n_levels; ++L) {
    const int b = sm.lstart[L], e = sm.lstart[L + 1];
    for (int j = b + q; j < e; j += kQuadsPerPass) {
      if (r == 3) continue;
      const int i = sm.lorder[j];
      const int p = sm.parent[i];
      const double *Li = local + 12 * i;
      double out[4];
      if (p < 0) {
#pragma unroll
        for (int c = 0; c < 4; ++c) out[c] = Li[4 * r + c];
      } else {
        const double *Wp = sm.world + 12 * p + 4 * r;
        const double p0 = Wp[0], p1 = Wp[1], p2 = Wp[2], p3 = Wp[3];
        out[0] = p0 * Li[0] + p1 * Li[4] + p2 * Li[8];
        out[1] = p0 * Li[1] + p1 * Li[5] + p2 * Li[9];
        out[2] = p0 * Li[2] + p1 * Li[6] + p2 * Li[10];
        out[3] = p0 * Li[3] + p1 * Li[7] + p2 * Li[11] + p3;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) sm.world[12 * i + 4 * r + c] = out[c];
    }
    __syncthreads();
  }
  // change flags against the poses of the previous refit (bitwise; NaN-filled
  // at creation) and the device copy of the world poses, in one pass: one
  // global round trip for the whole scene instead of one per tree level
  for (int k = tid; k < 12 * P; k += kRefitThreads) {
    const double w = sm.world[k];
    if (__double_as_longlong(a.world[k]) != __double_as_longlong(w)) a.dirty[k / 12] = 1;
    a.world[k] = w;
  }

  // 2-4. per part: lane r < 3 inverts row r in FP64; all four lanes share the
  //      FP32 bounds (radius, norms) through quad shuffles
  float mn[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, mx[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  const int rr = r < 3 ? r : 2;  // lane 3 repeats row 2 (its FP64 results are not stored)
  for (int p = q; p < P; p += kQuadsPerPass) {
    const double *m = sm.world + 12 * p;
    const double A0 = m[0], A1 = m[1], A2 = m[2], A3 = m[4], A4 = m[5], A5 = m[6], A6 = m[8], A7 = m[9],
                 A8 = m[10];
    const double c00 = A4 * A8 - A5 * A7, c01 = A5 * A6 - A3 * A8, c02 = A3 * A7 - A4 * A6;
    const double det = A0 * c00 + A1 * c01 + A2 * c02;
    // row r of adj(A) = cofactors of column r of A
    const double P1 = rr == 0 ? A2 : (rr == 1 ? A0 : A1), Q1 = rr == 0 ? A7 : (rr == 1 ? A8 : A6);
    const double R1 = rr == 0 ? A1 : (rr == 1 ? A2 : A0), S1 = rr == 0 ? A8 : (rr == 1 ? A6 : A7);
    const double P2 = rr == 0 ? A1 : (rr == 1 ? A2 : A0), Q2 = rr == 0 ? A5 : (rr == 1 ? A3 : A4);
    const double R2 = rr == 0 ? A2 : (rr == 1 ? A0 : A1), S2 = rr == 0 ? A4 : (rr == 1 ? A5 : A3);
    const double e0 = rr == 0 ? c00 : (rr == 1 ? c01 : c02);
    const double e1 = P1 * Q1 - R1 * S1;
    const double e2 = P2 * Q2 - R2 * S2;
    bool ok = isfinite(det) && fabs(det) > 0.0;
    double iv[4] = {0.0, 0.0, 0.0, 0.0};
    if (ok) {
      const double rd = 1.0 / det;
      iv[0] = e0 * rd;
      iv[1] = e1 * rd;
      iv[2] = e2 * rd;
      iv[3] = -(iv[0] * m[3] + iv[1] * m[7] + iv[2] * m[11]);
#pragma unroll
      for (int k = 0; k < 4; ++k) ok = ok && isfinite(iv[k]);
    }
    ok = __all_sync(qmask, ok);
    if (!ok) {
#pragma unroll
      for (int k = 0; k < 4; ++k) iv[k] = 0.0;
      if (r == 0) atomicOr(a.err, kErrSingular);
    }
    if (r < 3) {
#pragma unroll
      for (int k = 0; k < 4; ++k) a.inv64[12 * p + 4 * r + k] = iv[k];
    }
    // sphere centre c = W (lo + hi) / 2 in FP64 (row r), its FP32 rounding,
    // and the local coordinates of that FP32 point (FP64, rounded once)
    const PartStatic &ps = a.stat[p];
    const float lo0 = ps.box_lo[0], lo1 = ps.box_lo[1], lo2 = ps.box_lo[2];
    const float hi0 = ps.box_hi[0], hi1 = ps.box_hi[1], hi2 = ps.box_hi[2];
    const double mid0 = 0.5 * ((double)lo0 + (double)hi0), mid1 = 0.5 * ((double)lo1 + (double)hi1),
                 mid2 = 0.5 * ((double)lo2 + (double)hi2);
    const double cr = m[4 * rr] * mid0 + m[4 * rr + 1] * mid1 + m[4 * rr + 2] * mid2 + m[4 * rr + 3];
    const float cfr = (float)cr;
    const float cfx = __shfl_sync(qmask, cfr, 0, 4), cfy = __shfl_sync(qmask, cfr, 1, 4),
                cfz = __shfl_sync(qmask, cfr, 2, 4);
    const float lcr = (float)(iv[0] * (double)cfx + iv[1] * (double)cfy + iv[2] * (double)cfz + iv[3]);
    const float f0 = (float)iv[0], f1 = (float)iv[1], f2 = (float)iv[2];
    if (r < 3) reinterpret_cast<float4 *>(&a.hot[p])[r] = make_float4(f0, f1, f2, lcr);
    // FP32 bounds, every sum of squares rounded up.  Box half extents and
    // the corner offsets +-e are exact in FP32 (multiples of 2^-depth).
    const bool row = r < 3;
    float rs = row ? __fadd_ru(__fadd_ru(fabsf(f0), fabsf(f1)), fabsf(f2)) : 0.f;  // row of |Ainv|
    const float ex0 = 0.5f * (hi0 - lo0), ex1 = 0.5f * (hi1 - lo1), ex2 = 0.5f * (hi2 - lo2);
    const float a0 = (float)m[4 * rr], a1 = (float)m[4 * rr + 1], a2 = (float)m[4 * rr + 2];
    const float u0 = a0 * ex0, u1 = a1 * ex1, u2 = a2 * ex2;
    float s[7];
    s[0] = u0 + u1 + u2;  // the four corner directions (the other four are their negatives)
    s[1] = u0 + u1 - u2;
    s[2] = u0 - u1 + u2;
    s[3] = u0 - u1 - u2;
    s[4] = fabsf(u0) + fabsf(u1) + fabsf(u2);  // |A| e: scale of every rounding error above
    s[5] = a0 + a1 + a2;                          // A (1,1,1): the leaf diagonal direction
    s[6] = (float)fabs(cr - (double)cfr);         // centre rounding
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      float v = row ? __fmul_ru(s[k], s[k]) : 0.f;
      v = __fadd_ru(v, __shfl_xor_sync(qmask, v, 1, 4));
      v = __fadd_ru(v, __shfl_xor_sync(qmask, v, 2, 4));
      s[k] = v;
    }
    rs = fmaxf(rs, __shfl_xor_sync(qmask, rs, 1, 4));
    rs = fmaxf(rs, __shfl_xor_sync(qmask, rs, 2, 4));
    if (r == 0) {
      // |A q - c| <= computed + rounding (<= 2^-20 |A| e) for every corner q,
      // plus the distance of the FP32 centre from the exact one
      const float rfl = __fsqrt_ru(fmaxf(fmaxf(s[0], s[1]), fmaxf(s[2], s[3])));
      const float rad = __fadd_ru(__fadd_ru(__fmul_ru(rfl, 1.0f + kRelSlack), __fmul_ru(__fsqrt_ru(s[4]), kRelSlack)),
                                  __fmul_ru(__fsqrt_ru(s[6]), 1.0f + kRelSlack));
      // a singular pose or an empty asset disables the sphere: no ray tests the part
      const float4 sph = make_float4(cfx, cfy, cfz, (ok && ps.n_nodes > 0) ? rad : -1.0f);
      reinterpret_cast<float4 *>(&a.hot[p])[3] = sph;
      sm.sph[p] = sph;
      PartAux x;
      x.nodes = ps.nodes;
      x.n_nodes = ps.n_nodes;
      x.depth = ps.depth;
      x.n_ainv = rs;
      x.hdiag = sqrtf(s[5]) * __int_as_float((127 - ps.depth) << 23);
      x.spare0 = 0.f;
      x.spare1 = 0.f;
      for (int k = 0; k < 3; ++k) {
        x.box_lo[k] = ps.box_lo[k];
        x.box_hi[k] = ps.box_hi[k];
      }
      x.pad[0] = x.pad[1] = 0.f;
      a.aux[p] = x;
      sm.na[p] = rs;
      mn[0] = fminf(mn[0], cfx);
      mn[1] = fminf(mn[1], cfy);
      mn[2] = fminf(mn[2], cfz);
      mx[0] = fmaxf(mx[0], cfx);
      mx[1] = fmaxf(mx[1], cfy);
      mx[2] = fmaxf(mx[2], cfz);
    }
  }
  // bounding box of the sphere centres: warp shuffles, then the eight warp
  // results through shared memory (min and max are exact in any order)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn[k] = fminf(mn[k], __shfl_xor_sync(0xffffffffu, mn[k], o));
      mx[k] = fmaxf(mx[k], __shfl_xor_sync(0xffffffffu, mx[k], o));
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      sm.red[k * kRefitWarps + (tid >> 5)] = mn[k];
      sm.red[(3 + k) * kRefitWarps + (tid >> 5)] = mx[k];
    }
  }
  __syncthreads();
  float bb[6];
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    float v = sm.red[k * kRefitWarps];
    for (int w = 1; w < kRefitWarps; ++w) v = k < 3 ? fminf(v, sm.red[k * kRefitWarps + w]) : fmaxf(v, sm.red[k * kRefitWarps + w]);
    bb[k] = v;
  }
  const float bx0 = bb[0], by0 = bb[1], bz0 = bb[2];
  const float bx1 = bb[3], by1 = bb[4], bz1 = bb[5];
  const float ex = fmaxf(bx1 - bx0, 1e-30f), ey = fmaxf(by1 - by0, 1e-30f), ez = fmaxf(bz1 - bz0, 1e-30f);
  // 5. Morton keys and a rank sort (P <= kMaxParts)
  for (int i = tid; i < P; i += kRefitThreads) {
    const float4 s = sm.sph[i];
    const unsigned int qx = (unsigned int)fminf(fmaxf((s.x - bx0) / ex * 1023.0f, 0.0f), 1023.0f);
    const unsigned int qy = (unsigned int)fminf(fmaxf((s.y - by0) / ey * 1023.0f, 0.0f), 1023.0f);
    const unsigned int qz = (unsigned int)fminf(fmaxf((s.z - bz0) / ez * 1023.0f, 0.0f), 1023.0f);
    const unsigned int mc = spread10(qx) | (spread10(qy) << 1) | (spread10(qz) << 2);
    sm.key[i] = ((unsigned long long)mc << 11) | (unsigned long long)i;
  }
  __syncthreads();
  for (int i = tid; i < P; i += kRefitThreads) {
    const unsigned long long k = sm.key[i];
    int rank = 0;
    for (int j = 0; j < P; ++j) rank += (sm.key[j] < k) ? 1 : 0;
    sm.ord[rank] = i;
    a.order[rank] = i;
  }
  __syncthreads();
  // clusters: a sphere around the member spheres, in FP32 rounded outward
  for (int cidx = tid; cidx < a.n_clusters; cidx += kRefitThreads) {
    const int first = cidx * kClusterSize;
    const int cnt = min(kClusterSize, P - first);
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    float na = 0.f;
    bool any = false;
    for (int k = 0; k < cnt; ++k) {
      const int p = sm.ord[first + k];
      const float4 s = sm.sph[p];
      if (s.w < 0.f) continue;
      any = true;
      lo[0] = fminf(lo[0], __fsub_rd(s.x, s.w));
      lo[1] = fminf(lo[1], __fsub_rd(s.y, s.w));
      lo[2] = fminf(lo[2], __fsub_rd(s.z, s.w));
      hi[0] = fmaxf(hi[0], __fadd_ru(s.x, s.w));
      hi[1] = fmaxf(hi[1], __fadd_ru(s.y, s.w));
      hi[2] = fmaxf(hi[2], __fadd_ru(s.z, s.w));
      na = fmaxf(na, sm.na[p]);
    }
    Cluster cl;
    if (any) {
      // any centre works: the radius is measured from it with upward rounding
      const float Cx = 0.5f * lo[0] + 0.5f * hi[0], Cy = 0.5f * lo[1] + 0.5f * hi[1], Cz = 0.5f * lo[2] + 0.5f * hi[2];
      float R = 0.f;
      for (int k = 0; k < cnt; ++k) {
        const float4 s = sm.sph[sm.ord[first + k]];
        if (s.w < 0.f) continue;
        R = fmaxf(R, __fadd_ru(norm_up(abs_diff_up(s.x, Cx), abs_diff_up(s.y, Cy), abs_diff_up(s.z, Cz)), s.w));
      }
      cl.sphere = make_float4(Cx, Cy, Cz, R);
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
      R = fmaxf(R, __fadd_ru(norm_up(abs_diff_up(s.x, Cx), abs_diff_up(s.y, Cy), abs_diff_up(s.z, Cz)), s.w));
    }
    *a.bound = make_float4(Cx, Cy, Cz, R);
  }
  // the scene grid, if any, no longer matches the spheres: the next grid
  // trace rebuilds it first
  if (a.grid != nullptr && tid == 0) a.grid->stale = 1;
}

template <bool INLINE, int CAP>
__global__ void __launch_bounds__(kRefitThreads) k_refit(RefitArgs a, const __grid_constant__ InlinePoses<CAP> poses) {
  extern __shared__ __align__(16) unsigned char refit_smem[];
  // inline poses: composed from the parameter block, and copied to the
  // scene's device copy on the way
  refit_scene(a, INLINE ? poses.local : a.local, INLINE ? const_cast<double *>(a.local) : nullptr, false, refit_smem);
}

// Many scenes in one launch, one block each (scene_refit_batch): block b
// refits B.a[b], reading its local poses from B.src[b] (device or mapped
// host memory) when that is set.
struct RefitBatch {
  RefitArgs a[kRefitBatch];
  const double *src[kRefitBatch];
  int32_t n;
};

__global__ void __launch_bounds__(kRefitThreads) k_refit_batch(const __grid_constant__ RefitBatch B) {
  extern __shared__ __align__(16) unsigned char refit_smem[];
  const int b = blockIdx.x;
  const RefitArgs &a = B.a[b];
  const double *src = B.src[b];
  refit_scene(a, src ? src : a.local, src ? const_cast<double *>(a.local) : nullptr, true, refit_smem);
}

template <bool INLINE, int CAP>
cudaError_t launch_refit_t(const RefitArgs &a, const double *host_local, size_t smem, cudaStream_t stream) {
  InlinePoses<CAP> p;
  if (INLINE)
    for (int k = 0; k < a.n_parts * 12; ++k) p.local[k] = host_local[k];
  cudaError_t e = cudaFuncSetAttribute(k_refit<INLINE, CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_refit<INLINE, CAP><<<1, kRefitThreads, smem, stream>>>(a, p);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_refit_batch(const RefitArgs *args, const double *const *src, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  if (n > kRefitBatch) return cudaErrorInvalidValue;
  // the parameter block (about 9 KB): one per host thread, allocated on its
  // first batched refit, so it stays off the caller's stack and no call
  // allocates it afresh
  thread_local std::unique_ptr<RefitBatch> block;
  if (!block) block.reset(new RefitBatch());
  RefitBatch &B = *block;
  size_t smem = 0;
  for (int i = 0; i < n; ++i) {
    B.a[i] = args[i];
    B.src[i] = src[i];
    const size_t m = refit_smem_bytes(args[i].n_parts, args[i].n_clusters, args[i].n_levels, kRefitThreads);
    smem = m > smem ? m : smem;
  }
  B.n = n;
  // the shared-memory attribute only ever grows: set it when this launch needs more (per device)
  constexpr int kMaxDevices = 64;
  static std::mutex mu;
  static size_t admitted[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  {
    std::lock_guard<std::mutex> g(mu);
    if (smem > admitted[dev]) {
      e = cudaFuncSetAttribute(k_refit_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      admitted[dev] = smem;
    }
  }
  k_refit_batch<<<n, kRefitThreads, smem, stream>>>(B);
  return cudaGetLastError();
}

cudaError_t launch_refit(const RefitArgs &a, const double *host_local, cudaStream_t stream) {
  static_assert(kInlinePoseParts == 256, "size classes below");
  const size_t smem = refit_smem_bytes(a.n_parts, a.n_clusters, a.n_levels, kRefitThreads);
  if (host_local && a.n_parts <= 16) return launch_refit_t<true, 16>(a, host_local, smem, stream);
  if (host_local && a.n_parts <= 64) return launch_refit_t<true, 64>(a, host_local, smem, stream);
  if (host_local && a.n_parts <= 256) return launch_refit_t<true, 256>(a, host_local, smem, stream);
  return launch_refit_t<false, 1>(a, nullptr, smem, stream);
}

}  // namespace svo
