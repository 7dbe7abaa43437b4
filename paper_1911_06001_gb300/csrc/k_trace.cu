// k_trace.cu -- ray casting against a scene of animated sparse voxel octrees.
//
// Per ray (Espe et al., Sec. III-IV):
//   * instance culling: conservative ray / bounding-sphere tests (Eq. 4 in its
//     general form, |d| != 1) against the cluster spheres, then the part
//     spheres of the clusters that are hit (warp vote skips a cluster no lane
//     needs);
//   * depth sorting: candidate parts are visited in increasing sphere entry t
//     and the walk stops once the best hit lies before the next entry
//     (Sec. IV-B);
//   * per candidate part: the ray is moved into the part's frame by the
//     inverse pose (Eq. 2-3; d is not renormalised, so t is shared by all
//     parts) and an iterative front-to-back octree descent runs over the
//     child-descriptor nodes;
//   * closest hit (t, part, voxel), ties broken by smaller part, then voxel.
//
// FP32 certification.  Every FP32 slab test runs on boxes inflated (and, at
// leaves, also deflated) by eta, a per (ray, part) bound on the position
// error of the FP32 local ray.  A leaf whose inflated box is hit is a
// candidate with entry bounds [lo, hi] (hi only if the deflated box is hit:
// "certain").  A ray is certified when the candidate with the smallest lo is
// certain, every other candidate's lo exceeds its hi, and its [lo, hi] is
// narrower than 2^-17 of its t; otherwise it is flagged and, with FP64_FIX,
// recomputed in FP64 by k_fix (whose arithmetic needs no certification).
//
// Traversal: children of a node are visited in the order their entry t
// increases.  With every direction component made non-negative by mirroring,
// the entry of child m is max(T0, max over axes in m of the mid-plane t), so
// the order follows from sorting the three mid-plane t values; a per-block
// table maps a child mask to that order.  A stack holds, per level, the
// parent's descriptor and the children still to visit.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>

#include "svo_internal.h"

namespace svo {

template <int NI>
struct TraceLaunchT {
  TraceItem items[NI];
  int32_t n_items;
  uint32_t flags;
  unsigned long long n_tiles;
  unsigned long long *tile_counter;
  unsigned long long *fix_list;
  unsigned int *fix_count;
  unsigned long long fix_capacity;
  svo_trace_stats *stats;
  unsigned int *err;
};

namespace {

constexpr float kU = 5.9604644775390625e-8f;   // 2^-24, FP32 unit roundoff
constexpr float kTau = 7.62939453125e-6f;      // 2^-17
constexpr int kCap = 8;                         // candidate parts per pass
constexpr int kSmemParts = 256;                 // parts staged in shared memory
constexpr int kBlock = 128;
constexpr int kRaysPerThread = 4;               // rays per thread per tile
constexpr int kTile = kBlock * kRaysPerThread;
constexpr unsigned long long kRayBits = 40;

struct Tables {
  uint8_t q[8][6][256];  // [mirror][perm][true child mask] -> mask in visiting order
  uint8_t k[8][6][8];    // [mirror][perm][q] -> true octant
};

__device__ __forceinline__ void perm_axes(int p, int &a0, int &a1, int &a2) {
  // p = 2*rank_x + (rank_y > rank_z)
  const int rx = p >> 1;
  const bool z_first = (p & 1) != 0;
  int r[3];
  r[0] = rx;
  const int lo = (rx == 0) ? 1 : 0, hi = (rx == 2) ? 1 : 2;
  r[1] = z_first ? hi : lo;
  r[2] = z_first ? lo : hi;
  a0 = (r[0] == 0) ? 0 : (r[1] == 0 ? 1 : 2);
  a1 = (r[0] == 1) ? 0 : (r[1] == 1 ? 1 : 2);
  a2 = (r[0] == 2) ? 0 : (r[1] == 2 ? 1 : 2);
}

__device__ void build_tables(Tables *t) {
  for (int e = threadIdx.x; e < 8 * 6 * 256; e += blockDim.x) {
    const int h = e & 255, p = (e >> 8) % 6, mir = (e >> 8) / 6;
    int a0, a1, a2;
    perm_axes(p, a0, a1, a2);
    unsigned int out = 0;
    for (int q = 0; q < 8; ++q) {
      const int m = ((q & 1) << a0) | (((q >> 1) & 1) << a1) | (((q >> 2) & 1) << a2);
      const int k = m ^ mir;
      out |= ((h >> k) & 1u) << q;
    }
    t->q[mir][p][h] = (uint8_t)out;
  }
  for (int e = threadIdx.x; e < 8 * 6 * 8; e += blockDim.x) {
    const int q = e & 7, p = (e >> 3) % 6, mir = (e >> 3) / 6;
    int a0, a1, a2;
    perm_axes(p, a0, a1, a2);
    const int m = ((q & 1) << a0) | (((q >> 1) & 1) << a1) | (((q >> 2) & 1) << a2);
    t->k[mir][p][q] = (uint8_t)(m ^ mir);
  }
}

template <typename R>
struct Num;
template <>
struct Num<float> {
  __device__ static float inf() { return __int_as_float(0x7f800000); }
  __device__ static float pow2neg(int l) { return __int_as_float((127 - l) << 23); }
  __device__ static float tiny() { return 1e-30f; }
  __device__ static float rcp(float x) { return __frcp_rn(x); }
};
template <>
struct Num<double> {
  __device__ static double inf() { return __longlong_as_double(0x7ff0000000000000ll); }
  __device__ static double pow2neg(int l) { return __longlong_as_double((long long)(1023 - l) << 52); }
  __device__ static double tiny() { return 1e-200; }
  __device__ static double rcp(double x) { return 1.0 / x; }
};

// t of the plane x_i = P along a mirrored axis with reciprocal direction inv
// and b = -o*inv.  FP32 uses one FMA (its rounding is part of the error bound
// behind eta); FP64 subtracts first so that the sign of P - o is exact, which
// decides slabs of direction components that are exactly zero.
template <typename R>
struct Slab;
template <>
struct Slab<float> {
  __device__ static float t(float P, float inv, float, float b) { return fmaf(P, inv, b); }
};
template <>
struct Slab<double> {
  __device__ static double t(double P, double inv, double o, double) { return (P - o) * inv; }
};

// FP32 per-ray state of the certified closest-hit search.
struct CertState {
  float lo1, hi1, te1;  // candidate with the smallest (lo, part, voxel)
  float lo2;            // smallest lo of all other candidates
  float hi_min;         // smallest hi of the certain candidates (prune bound)
  uint32_t part1;
  uint32_t cert1;
  unsigned long long vox1;
};

// FP64 per-ray state of the exact closest-hit search.
struct ExactState {
  double t;
  uint32_t part;
  unsigned long long vox;
};

__device__ __forceinline__ void offer(CertState &s, float lo, float hi, float te, bool cert, uint32_t part,
                                      unsigned long long vox) {
  if (cert) s.hi_min = fminf(s.hi_min, hi);
  const bool better = lo < s.lo1 || (lo == s.lo1 && (part < s.part1 || (part == s.part1 && vox < s.vox1)));
  if (better) {
    s.lo2 = fminf(s.lo2, s.lo1);
    s.lo1 = lo;
    s.hi1 = hi;
    s.te1 = te;
    s.part1 = part;
    s.vox1 = vox;
    s.cert1 = cert ? 1u : 0u;
  } else {
    s.lo2 = fminf(s.lo2, lo);
  }
}

__device__ __forceinline__ void offer(ExactState &s, double t, uint32_t part, unsigned long long vox) {
  if (t < s.t || (t == s.t && (part < s.part || (part == s.part && vox < s.vox)))) {
    s.t = t;
    s.part = part;
    s.vox = vox;
  }
}

__device__ __forceinline__ float prune_bound(const CertState &s, float tmax) { return fminf(tmax, s.hi_min); }
__device__ __forceinline__ double prune_bound(const ExactState &s, double tmax) { return fmin(tmax, s.t); }

struct Counters {
  uint32_t parts_tested, parts_entered, nodes, leaves, passes;
};

// Front-to-back descent of one part in its local frame.  (o, d): local ray;
// eta: inflation (0 for the exact FP64 search).  State S is CertState (R =
// float, certified) or ExactState (R = double).
template <typename R, typename S, bool STATS>
__device__ __forceinline__ void descend_part(const uint2 *__restrict__ nodes, uint32_t n_nodes, int D, R ox, R oy,
                                             R oz, R dx, R dy, R dz, R tmin, R tmax, R eta, uint32_t part,
                                             const Tables *__restrict__ tab, S &st, unsigned int &err,
                                             Counters &cnt) {
  if (n_nodes == 0) return;
  constexpr bool CERT = sizeof(R) == 4;
  uint32_t mir = 0;
  if (dx < R(0)) {
    ox = R(1) - ox;
    dx = -dx;
    mir |= 1u;
  }
  if (dy < R(0)) {
    oy = R(1) - oy;
    dy = -dy;
    mir |= 2u;
  }
  if (dz < R(0)) {
    oz = R(1) - oz;
    dz = -dz;
    mir |= 4u;
  }
  dx = dx > Num<R>::tiny() ? dx : Num<R>::tiny();
  dy = dy > Num<R>::tiny() ? dy : Num<R>::tiny();
  dz = dz > Num<R>::tiny() ? dz : Num<R>::tiny();
  const R ix = Num<R>::rcp(dx), iy = Num<R>::rcp(dy), iz = Num<R>::rcp(dz);
  const R bx = -(ox * ix), by = -(oy * iy), bz = -(oz * iz);
  // masks (true octant space) of the children lying in the far half along
  // each mirrored axis
  const uint32_t HX = (mir & 1u) ? 0x55u : 0xAAu;
  const uint32_t HY = (mir & 2u) ? 0x33u : 0xCCu;
  const uint32_t HZ = (mir & 4u) ? 0x0Fu : 0xF0u;
  const uint8_t *__restrict__ qt = &tab->q[mir][0][0];
  const uint8_t *__restrict__ kt = &tab->k[mir][0][0];
  const uint32_t side = 1u << D;

  uint2 stk[kMaxDepth];
  int level = 0;
  uint32_t px = 0, py = 0, pz = 0;
  uint2 desc = __ldg(&nodes[0]);
  if (STATS) ++cnt.nodes;
  bool down = true;
  for (;;) {
    if (down) {
      const R sz = Num<R>::pow2neg(level), h = sz * R(0.5);
      const R lx = R(px) * sz, ly = R(py) * sz, lz = R(pz) * sz;
      const R tl = prune_bound(st, tmax);
      const R Ax = Slab<R>::t(lx - eta, ix, ox, bx), Ay = Slab<R>::t(ly - eta, iy, oy, by), Az = Slab<R>::t(lz - eta, iz, oz, bz);
      const R Bx = Slab<R>::t((lx + h) - eta, ix, ox, bx), By = Slab<R>::t((ly + h) - eta, iy, oy, by), Bz = Slab<R>::t((lz + h) - eta, iz, oz, bz);
      const R Cx = CERT ? Slab<R>::t((lx + h) + eta, ix, ox, bx) : Bx;
      const R Cy = CERT ? Slab<R>::t((ly + h) + eta, iy, oy, by) : By;
      const R Cz = CERT ? Slab<R>::t((lz + h) + eta, iz, oz, bz) : Bz;
      const R Ex = Slab<R>::t((lx + sz) + eta, ix, ox, bx), Ey = Slab<R>::t((ly + sz) + eta, iy, oy, by), Ez = Slab<R>::t((lz + sz) + eta, iz, oz, bz);
      const R T0 = fmax(fmax(Ax, Ay), fmax(Az, tmin));
      const R T1 = fmin(fmin(Ex, Ey), fmin(Ez, tl));
      // child m (mirrored) is hit iff max(T0, B_i : i in m) <= min(T1, C_j : j not in m)
      uint32_t hit = (T0 <= T1) ? 0xFFu : 0u;
      hit &= (Bx <= T1) ? 0xFFu : ~HX;
      hit &= (By <= T1) ? 0xFFu : ~HY;
      hit &= (Bz <= T1) ? 0xFFu : ~HZ;
      hit &= (Cx >= T0) ? 0xFFu : HX;
      hit &= (Cy >= T0) ? 0xFFu : HY;
      hit &= (Cz >= T0) ? 0xFFu : HZ;
      hit &= (Bx <= Cy) ? 0xFFu : ~(HX & ~HY);
      hit &= (Bx <= Cz) ? 0xFFu : ~(HX & ~HZ);
      hit &= (By <= Cx) ? 0xFFu : ~(HY & ~HX);
      hit &= (By <= Cz) ? 0xFFu : ~(HY & ~HZ);
      hit &= (Bz <= Cx) ? 0xFFu : ~(HZ & ~HX);
      hit &= (Bz <= Cy) ? 0xFFu : ~(HZ & ~HY);
      const uint32_t cmask = desc.y & 0xFFu;
      hit &= cmask;
      if (hit == 0u) {
        down = false;
        continue;
      }
      const bool cxy = Bx <= By, cxz = Bx <= Bz, cyz = By <= Bz;
      const int rx = (cxy ? 0 : 1) + (cxz ? 0 : 1);
      const int ry = (cxy ? 1 : 0) + (cyz ? 0 : 1);
      const int rz = (cxz ? 1 : 0) + (cyz ? 1 : 0);
      const int p = 2 * rx + (ry > rz ? 1 : 0);
      uint32_t hq = qt[p * 256 + hit];
      if (level == D - 1) {
        // children are leaves: test them in visiting order
        while (hq) {
          const int q = __ffs(hq) - 1;
          hq &= hq - 1u;
          const uint32_t k = kt[p * 8 + q];
          const uint32_t m = k ^ mir;
          R lo = T0;
          if (m & 1u) lo = fmax(lo, Bx);
          if (m & 2u) lo = fmax(lo, By);
          if (m & 4u) lo = fmax(lo, Bz);
          if (lo > prune_bound(st, tmax)) break;  // later leaves start even later
          if (STATS) ++cnt.leaves;
          const uint32_t vx = 2u * px + (m & 1u), vy = 2u * py + ((m >> 1) & 1u), vz = 2u * pz + ((m >> 2) & 1u);
          const unsigned long long gx = (mir & 1u) ? (side - 1u - vx) : vx;
          const unsigned long long gy = (mir & 2u) ? (side - 1u - vy) : vy;
          const unsigned long long gz = (mir & 4u) ? (side - 1u - vz) : vz;
          const unsigned long long vox = gx | (gy << D) | (gz << (2 * D));
          if constexpr (CERT) {
            const R clx = (m & 1u) ? lx + h : lx, cly = (m & 2u) ? ly + h : ly, clz = (m & 4u) ? lz + h : lz;
            const R dlo = fmax(fmax(Slab<R>::t(clx + eta, ix, ox, bx), Slab<R>::t(cly + eta, iy, oy, by)), fmax(Slab<R>::t(clz + eta, iz, oz, bz), tmin));
            const R dhi = fmin(fmin(Slab<R>::t((clx + h) - eta, ix, ox, bx), Slab<R>::t((cly + h) - eta, iy, oy, by)),
                               fmin(Slab<R>::t((clz + h) - eta, iz, oz, bz), tmax));
            const R te = fmax(fmax(Slab<R>::t(clx, ix, ox, bx), Slab<R>::t(cly, iy, oy, by)), fmax(Slab<R>::t(clz, iz, oz, bz), tmin));
            const bool cert = dlo <= dhi;
            offer(st, lo, cert ? dlo : Num<R>::inf(), te, cert, part, vox);
          } else {
            offer(st, lo, part, vox);
          }
        }
        down = false;
        continue;
      }
      const int q = __ffs(hq) - 1;
      const uint32_t rest = hq & (hq - 1u);
      stk[level] = make_uint2(desc.x, cmask | (rest << 8) | ((uint32_t)p << 16));
      const uint32_t k = kt[p * 8 + q];
      const uint32_t idx = desc.x + __popc(cmask & ((1u << k) - 1u));
      if (idx >= n_nodes) {
        err |= kErrNodeIndex;
        return;
      }
      desc = __ldg(&nodes[idx]);
      if (STATS) ++cnt.nodes;
      const uint32_t m = k ^ mir;
      px = 2u * px + (m & 1u);
      py = 2u * py + ((m >> 1) & 1u);
      pz = 2u * pz + ((m >> 2) & 1u);
      ++level;
    } else {
      if (level == 0) return;
      --level;
      px >>= 1;
      py >>= 1;
      pz >>= 1;
      const uint2 e = stk[level];
      uint32_t rest = (e.y >> 8) & 0xFFu;
      if (rest == 0u) continue;
      const int q = __ffs(rest) - 1;
      rest &= rest - 1u;
      const int p = (int)(e.y >> 16);
      // entry of the next child: max(T0, mid-plane t of its highest-ranked axis)
      const R sz = Num<R>::pow2neg(level), h = sz * R(0.5);
      const R lx = R(px) * sz, ly = R(py) * sz, lz = R(pz) * sz;
      const R T0 = fmax(fmax(Slab<R>::t(lx - eta, ix, ox, bx), Slab<R>::t(ly - eta, iy, oy, by)), fmax(Slab<R>::t(lz - eta, iz, oz, bz), tmin));
      const int rank = 31 - __clz(q);
      int a0, a1, a2;
      perm_axes(p, a0, a1, a2);
      const int ax = rank == 0 ? a0 : (rank == 1 ? a1 : a2);
      const R Bsel = ax == 0 ? Slab<R>::t((lx + h) - eta, ix, ox, bx) : (ax == 1 ? Slab<R>::t((ly + h) - eta, iy, oy, by) : Slab<R>::t((lz + h) - eta, iz, oz, bz));
      const R en = fmax(T0, Bsel);
      if (en > prune_bound(st, tmax)) continue;  // this and all later siblings are too far
      stk[level].y = (e.y & ~0xFF00u) | (rest << 8);
      const uint32_t k = kt[p * 8 + q];
      const uint32_t cmask = e.y & 0xFFu;
      const uint32_t idx = e.x + __popc(cmask & ((1u << k) - 1u));
      if (idx >= n_nodes) {
        err |= kErrNodeIndex;
        return;
      }
      desc = __ldg(&nodes[idx]);
      if (STATS) ++cnt.nodes;
      const uint32_t m = k ^ mir;
      px = 2u * px + (m & 1u);
      py = 2u * py + ((m >> 1) & 1u);
      pz = 2u * pz + ((m >> 2) & 1u);
      ++level;
      down = true;
    }
  }
}

struct RayW {
  float ox, oy, oz, tmin, dx, dy, dz, tmax;
  float inv_dd;
  float onorm;  // ||o||_inf
};

// Conservative ray / sphere test: sphere (c, R) is hit by the segment.  Eq. 4
// with a direction of any length: l = c - o, tc = (l.d)/|d|^2, the squared
// distance of the centre to the line is |l - tc d|^2.
__device__ __forceinline__ bool sphere_test(const RayW &r, float lx, float ly, float lz, float R, float &tin) {
  const float tc = (lx * r.dx + ly * r.dy + lz * r.dz) * r.inv_dd;
  const float qx = fmaf(-tc, r.dx, lx), qy = fmaf(-tc, r.dy, ly), qz = fmaf(-tc, r.dz, lz);
  const float p2 = qx * qx + qy * qy + qz * qz;
  const float R2 = R * R;
  if (!(p2 <= R2)) return false;
  const float half = sqrtf((R2 - p2) * r.inv_dd);
  const float tout = tc + half;
  tin = tc - half;
  return tout >= r.tmin && tin <= r.tmax;
}

// Part test with the error slack of this ray; returns the eta for its descent.
__device__ __forceinline__ bool part_cull(const RayW &r, const PartHot &ph, const PartAux &pa, float &tin, float &eta) {
  const float4 s = ph.sphere;
  if (s.w < 0.f) return false;
  const float lx = s.x - r.ox, ly = s.y - r.oy, lz = s.z - r.oz;
  const float ln = fabsf(lx) + fabsf(ly) + fabsf(lz);
  eta = kU * (16.0f * fmaf(pa.n_ainv, r.onorm, pa.n_binv) + 8.0f * pa.n_ainv * (ln + 2.0f * s.w) + 8.0f);
  const float Rt = s.w * (1.0f + 9.5367431640625e-7f) + eta * pa.cull_scale + 16.0f * kU * (ln + s.w);
  return sphere_test(r, lx, ly, lz, Rt, tin);
}

__device__ __forceinline__ bool cluster_cull(const RayW &r, const Cluster &c) {
  const float4 s = c.sphere;
  if (s.w < 0.f) return false;
  const float lx = s.x - r.ox, ly = s.y - r.oy, lz = s.z - r.oz;
  const float ln = fabsf(lx) + fabsf(ly) + fabsf(lz);
  const float lm = ln + 1.7320508f * s.w;
  const float eta = kU * (16.0f * fmaf(c.aux.x, r.onorm, c.aux.y) + 8.0f * c.aux.x * (lm + 2.0f * s.w) + 8.0f);
  const float Rt = s.w * (1.0f + 9.5367431640625e-7f) + eta * c.aux.z + 16.0f * kU * (2.0f * ln + 3.7320508f * s.w);
  float tin;
  return sphere_test(r, lx, ly, lz, Rt, tin);
}

template <bool STATS>
__device__ __forceinline__ void trace_part_f32(const RayW &r, const PartHot &ph, const PartAux &pa, float eta,
                                               uint32_t part, const Tables *tab, CertState &st, unsigned int &err,
                                               Counters &cnt) {
  const float4 a = ph.r0, b = ph.r1, c = ph.r2;
  const float ox = fmaf(a.x, r.ox, fmaf(a.y, r.oy, fmaf(a.z, r.oz, a.w)));
  const float oy = fmaf(b.x, r.ox, fmaf(b.y, r.oy, fmaf(b.z, r.oz, b.w)));
  const float oz = fmaf(c.x, r.ox, fmaf(c.y, r.oy, fmaf(c.z, r.oz, c.w)));
  const float dx = fmaf(a.x, r.dx, fmaf(a.y, r.dy, a.z * r.dz));
  const float dy = fmaf(b.x, r.dx, fmaf(b.y, r.dy, b.z * r.dz));
  const float dz = fmaf(c.x, r.dx, fmaf(c.y, r.dy, c.z * r.dz));
  if (STATS) ++cnt.parts_entered;
  descend_part<float, CertState, STATS>(pa.nodes, pa.n_nodes, pa.depth, ox, oy, oz, dx, dy, dz, r.tmin, r.tmax,
                                        eta, part, tab, st, err, cnt);
}

// Insert (t, p) into the sorted register list (ct, cp); the displaced largest
// entry is returned in (t, p).
__device__ __forceinline__ void list_insert(float (&ct)[kCap], float (&ce)[kCap], int (&cp)[kCap], float &t,
                                            float &e, int &p) {
#pragma unroll
  for (int i = 0; i < kCap; ++i) {
    const bool sw = t < ct[i] || (t == ct[i] && p < cp[i]);
    const float t2 = sw ? ct[i] : t, e2 = sw ? ce[i] : e;
    const int p2 = sw ? cp[i] : p;
    ct[i] = sw ? t : ct[i];
    ce[i] = sw ? e : ce[i];
    cp[i] = sw ? p : cp[i];
    t = t2;
    e = e2;
    p = p2;
  }
}

template <bool STATS>
__device__ void trace_ray_f32(const RayW &r, bool active, uint32_t flags, int P, int NC,
                              const PartHot *__restrict__ hot, const PartAux *__restrict__ aux,
                              const Cluster *__restrict__ cl, const int32_t *__restrict__ order, const Tables *tab,
                              CertState &st, unsigned int &err, Counters &cnt) {
  st.lo1 = st.hi1 = st.te1 = st.lo2 = st.hi_min = Num<float>::inf();
  st.part1 = kMissPart;
  st.cert1 = 0;
  st.vox1 = kMissVoxel;
  const bool cull = (flags & SVO_TRACE_CULL) != 0;
  const bool sort = (flags & SVO_TRACE_SORT) != 0;
  if (cull && sort) {
    float last_t = -Num<float>::inf();
    int last_p = -1;
    for (;;) {
      float ct[kCap], ce[kCap];
      int cp[kCap];
#pragma unroll
      for (int i = 0; i < kCap; ++i) {
        ct[i] = Num<float>::inf();
        ce[i] = 0.f;
        cp[i] = 0x7fffffff;
      }
      float over_t = Num<float>::inf();  // smallest entry that did not fit the list
      if (STATS && active) ++cnt.passes;
      for (int c = 0; c < NC; ++c) {
        const Cluster cc = cl[c];
        const bool hc = active && cluster_cull(r, cc);
        if (__ballot_sync(__activemask(), hc) == 0u) continue;  // no lane needs this cluster
        if (!hc) continue;
        const uint32_t fc = __float_as_uint(cc.aux.w);
        const int first = (int)(fc & 0xFFFFu), count = (int)(fc >> 16);
        for (int k = 0; k < count; ++k) {
          const int p = order[first + k];
          float tin, eta;
          if (STATS) ++cnt.parts_tested;
          if (!part_cull(r, hot[p], aux[p], tin, eta)) continue;
          if (tin < last_t || (tin == last_t && p <= last_p)) continue;  // visited in an earlier pass
          float t = tin, e = eta;
          int pp = p;
          list_insert(ct, ce, cp, t, e, pp);
          over_t = fminf(over_t, t);
        }
      }
      // visit in order of sphere entry, stop once the best hit is nearer
      bool stopped = false;
      while (ct[0] != Num<float>::inf()) {
        const float tin = ct[0], eta = ce[0];
        const int p = cp[0];
#pragma unroll
        for (int i = 0; i < kCap - 1; ++i) {
          ct[i] = ct[i + 1];
          ce[i] = ce[i + 1];
          cp[i] = cp[i + 1];
        }
        ct[kCap - 1] = Num<float>::inf();
        if (tin > prune_bound(st, r.tmax)) {
          stopped = true;
          break;
        }
        trace_part_f32<STATS>(r, hot[p], aux[p], eta, (uint32_t)p, tab, st, err, cnt);
        last_t = tin;
        last_p = p;
      }
      if (stopped || !(over_t <= prune_bound(st, r.tmax))) break;
    }
  } else {
    for (int p = 0; p < P; ++p) {
      float tin, eta;
      if (STATS) ++cnt.parts_tested;
      const bool h = active && part_cull(r, hot[p], aux[p], tin, eta);
      if (cull && !h) continue;
      if (!active) continue;
      if (!h) {
        // plain trace of a part whose sphere is missed: still descend, with an
        // eta valid for any point of the ray near the part
        const float4 s = hot[p].sphere;
        const float ln = fabsf(s.x - r.ox) + fabsf(s.y - r.oy) + fabsf(s.z - r.oz);
        eta = kU * (16.0f * fmaf(aux[p].n_ainv, r.onorm, aux[p].n_binv) + 8.0f * aux[p].n_ainv * (ln + 2.0f * fabsf(s.w)) + 8.0f);
      }
      trace_part_f32<STATS>(r, hot[p], aux[p], eta, (uint32_t)p, tab, st, err, cnt);
    }
  }
}

template <int NI>
__device__ __forceinline__ int find_item(const TraceLaunchT<NI> &L, unsigned long long tile) {
  int lo = 0, hi = L.n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (L.items[mid].tile_begin <= tile)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void flush_stats(svo_trace_stats *st, const Counters &c, uint32_t rays, uint32_t flagged) {
  unsigned long long v[7] = {rays, flagged, c.parts_tested, c.parts_entered, c.nodes, c.leaves, c.passes};
#pragma unroll
  for (int i = 0; i < 7; ++i) {
    unsigned long long x = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    v[i] = x;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&st->rays, v[0]);
    atomicAdd(&st->flagged, v[1]);
    atomicAdd(&st->parts_tested, v[2]);
    atomicAdd(&st->parts_entered, v[3]);
    atomicAdd(&st->nodes_visited, v[4]);
    atomicAdd(&st->leaves_tested, v[5]);
    atomicAdd(&st->passes, v[6]);
  }
}

template <int NI, bool STATS>
__global__ void __launch_bounds__(kBlock) k_trace(const __grid_constant__ TraceLaunchT<NI> L) {
  extern __shared__ __align__(16) unsigned char smem[];
  Tables *tab = reinterpret_cast<Tables *>(smem);
  PartHot *sHot = reinterpret_cast<PartHot *>(smem + ((sizeof(Tables) + 15) & ~size_t(15)));
  PartAux *sAux = reinterpret_cast<PartAux *>(sHot + kSmemParts);
  Cluster *sCl = reinterpret_cast<Cluster *>(sAux + kSmemParts);
  int32_t *sOrd = reinterpret_cast<int32_t *>(sCl + kSmemParts / kClusterSize);
  __shared__ unsigned long long s_tile;
  build_tables(tab);
  const PartHot *cur = nullptr;
  unsigned int err = 0;
  Counters cnt = {0, 0, 0, 0, 0};
  uint32_t n_rays = 0, n_flag = 0;
  const int lane = threadIdx.x & 31;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = atomicAdd(L.tile_counter, 1ull);
    __syncthreads();
    const unsigned long long tile = s_tile;
    if (tile >= L.n_tiles) break;
    const int it = find_item(L, tile);
    const TraceItem &I = L.items[it];
    const int P = I.n_parts, NC = I.n_clusters;
    const bool staged = P <= kSmemParts;
    if (staged && I.hot != cur) {
      for (int i = threadIdx.x; i < P; i += kBlock) {
        sHot[i] = I.hot[i];
        sAux[i] = I.aux[i];
        sOrd[i] = I.order[i];
      }
      for (int i = threadIdx.x; i < NC; i += kBlock) sCl[i] = I.clusters[i];
      cur = I.hot;
      __syncthreads();
    }
    const PartHot *hot = staged ? sHot : I.hot;
    const PartAux *aux = staged ? sAux : I.aux;
    const Cluster *cls = staged ? sCl : I.clusters;
    const int32_t *ord = staged ? sOrd : I.order;
    const unsigned long long base = (tile - I.tile_begin) * (unsigned long long)kTile;
#pragma unroll 1
    for (int j = 0; j < kRaysPerThread; ++j) {
      const unsigned long long ray = base + (unsigned long long)(j * kBlock + threadIdx.x);
      bool active = ray < I.n;
      RayW r;
      if (active) {
        const float4 o = __ldcs(&I.rays[2 * ray]);
        const float4 d = __ldcs(&I.rays[2 * ray + 1]);
        r.ox = o.x;
        r.oy = o.y;
        r.oz = o.z;
        r.tmin = o.w;
        r.dx = d.x;
        r.dy = d.y;
        r.dz = d.z;
        r.tmax = d.w;
        const float dd = d.x * d.x + d.y * d.y + d.z * d.z;
        const bool finite = isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) &&
                            isfinite(d.z) && !isnan(o.w) && !isnan(d.w) && dd > 0.f && isfinite(dd);
        r.inv_dd = 1.0f / dd;
        r.onorm = fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fabsf(o.z));
        active = finite && (o.w <= d.w);
        if (STATS) ++n_rays;
      } else {
        r.ox = r.oy = r.oz = r.dx = r.dy = r.dz = 0.f;
        r.tmin = 0.f;
        r.tmax = -1.f;
        r.inv_dd = 0.f;
        r.onorm = 0.f;
      }
      CertState st;
      trace_ray_f32<STATS>(r, active, L.flags, P, NC, hot, aux, cls, ord, tab, st, err, cnt);
      bool flagged = false;
      if (ray < I.n) {
        float t = Num<float>::inf();
        uint32_t part = kMissPart;
        unsigned long long vox = kMissVoxel;
        if (st.part1 != kMissPart) {
          const bool certified = st.cert1 && st.lo2 > st.hi1 && (st.hi1 - st.lo1) <= kTau * st.lo1;
          flagged = !certified;
          t = fminf(fmaxf(st.te1, st.lo1), st.hi1);
          if (!st.cert1) t = st.te1;
          part = st.part1;
          vox = st.vox1;
        }
        uint4 hv;
        hv.x = __float_as_uint(t);
        hv.y = part;
        hv.z = (uint32_t)(vox & 0xFFFFFFFFull);
        hv.w = (uint32_t)(vox >> 32);
        __stcs(&I.hits[ray], hv);
        if (I.ray_flags) I.ray_flags[ray] = flagged ? SVO_RAY_UNCERTAIN : 0u;
        if (STATS && flagged) ++n_flag;
      }
      // compact flagged rays for the FP64 pass (one atomic per warp)
      if (L.flags & SVO_TRACE_FP64_FIX) {
        const unsigned int m = __ballot_sync(0xffffffffu, flagged);
        if (m) {
          const int leader = __ffs(m) - 1;
          unsigned int basei = 0;
          if (lane == leader) basei = atomicAdd(L.fix_count, (unsigned int)__popc(m));
          basei = __shfl_sync(0xffffffffu, basei, leader);
          if (flagged) {
            const unsigned long long slot = basei + __popc(m & ((1u << lane) - 1u));
            if (slot < L.fix_capacity)
              L.fix_list[slot] = ((unsigned long long)it << kRayBits) | ray;
            else
              err |= kErrFixOverflow;
          }
        }
      }
    }
  }
  if (STATS) flush_stats(L.stats, cnt, n_rays, n_flag);
  if (err) atomicOr(L.err, err);
}

// ------------------------------------------------------------- FP64 pass

__device__ __forceinline__ bool sphere_test64(double ox, double oy, double oz, double dx, double dy, double dz,
                                              double tmin, double tmax, float4 s, double &tin) {
  const double lx = s.x - ox, ly = s.y - oy, lz = s.z - oz;
  const double dd = dx * dx + dy * dy + dz * dz;
  const double tc = (lx * dx + ly * dy + lz * dz) / dd;
  const double qx = lx - tc * dx, qy = ly - tc * dy, qz = lz - tc * dz;
  const double p2 = qx * qx + qy * qy + qz * qz;
  const double R = (double)s.w * (1.0 + 1e-9) + 1e-12 * (fabs(lx) + fabs(ly) + fabs(lz) + (double)s.w);
  if (!(p2 <= R * R)) return false;
  const double half = sqrt((R * R - p2) / dd);
  tin = tc - half;
  return tc + half >= tmin && tin <= tmax;
}

template <int NI>
__global__ void __launch_bounds__(kBlock) k_fix(const __grid_constant__ TraceLaunchT<NI> L) {
  __shared__ Tables tab;
  build_tables(&tab);
  __syncthreads();
  unsigned int err = 0;
  Counters cnt = {0, 0, 0, 0, 0};
  const unsigned long long n = min((unsigned long long)*L.fix_count, L.fix_capacity);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long e = L.fix_list[i];
    const int it = (int)(e >> kRayBits);
    const unsigned long long ray = e & ((1ull << kRayBits) - 1ull);
    const TraceItem &I = L.items[it];
    const float4 o = I.rays[2 * ray], d = I.rays[2 * ray + 1];
    const double ox = o.x, oy = o.y, oz = o.z, dx = d.x, dy = d.y, dz = d.z, tmin = o.w, tmax = d.w;
    ExactState st;
    st.t = Num<double>::inf();
    st.part = kMissPart;
    st.vox = kMissVoxel;
    for (int p = 0; p < I.n_parts; ++p) {
      const float4 s = I.hot[p].sphere;
      if (s.w < 0.f) continue;
      double tin;
      if (!sphere_test64(ox, oy, oz, dx, dy, dz, tmin, tmax, s, tin)) continue;
      if (tin > st.t) continue;
      const double *m = I.inv64 + 12 * p;
      const double lx = m[0] * ox + m[1] * oy + m[2] * oz + m[3];
      const double ly = m[4] * ox + m[5] * oy + m[6] * oz + m[7];
      const double lz = m[8] * ox + m[9] * oy + m[10] * oz + m[11];
      const double ldx = m[0] * dx + m[1] * dy + m[2] * dz;
      const double ldy = m[4] * dx + m[5] * dy + m[6] * dz;
      const double ldz = m[8] * dx + m[9] * dy + m[10] * dz;
      const PartAux pa = I.aux[p];
      descend_part<double, ExactState, false>(pa.nodes, pa.n_nodes, pa.depth, lx, ly, lz, ldx, ldy, ldz, tmin, tmax,
                                              0.0, (uint32_t)p, &tab, st, err, cnt);
    }
    uint4 hv;
    hv.x = __float_as_uint((float)st.t);
    hv.y = st.part;
    hv.z = (uint32_t)(st.vox & 0xFFFFFFFFull);
    hv.w = (uint32_t)(st.vox >> 32);
    I.hits[ray] = hv;
    if (I.ray_flags) I.ray_flags[ray] = SVO_RAY_UNCERTAIN | SVO_RAY_FIXED;
  }
  if (L.stats) {
    // count fixed rays once per launch
    if (blockIdx.x == 0 && threadIdx.x == 0 && (L.flags & SVO_TRACE_STATS)) atomicAdd(&L.stats->fixed, n);
  }
  if (err) atomicOr(L.err, err);
}

size_t trace_smem_bytes() {
  return ((sizeof(Tables) + 15) & ~size_t(15)) + kSmemParts * (sizeof(PartHot) + sizeof(PartAux)) +
         (kSmemParts / kClusterSize) * sizeof(Cluster) + kSmemParts * sizeof(int32_t);
}

template <int NI>
cudaError_t launch_trace_t(const TraceLaunchT<NI> &L, int n_sm, cudaStream_t stream) {
  const size_t smem = trace_smem_bytes();
  const bool stats = (L.flags & SVO_TRACE_STATS) && L.stats;
  auto kern = stats ? k_trace<NI, true> : k_trace<NI, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBlock, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  unsigned long long grid = (unsigned long long)n_sm * per_sm;
  if (grid > L.n_tiles) grid = L.n_tiles;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned int)grid, kBlock, smem, stream>>>(L);
  return cudaGetLastError();
}

template <int NI>
cudaError_t launch_fix_t(const TraceLaunchT<NI> &L, int n_sm, cudaStream_t stream) {
  k_fix<NI><<<(unsigned int)(n_sm * 2), kBlock, 0, stream>>>(L);
  return cudaGetLastError();
}

template <int NI>
void fill_launch(const TraceLaunch &src, TraceLaunchT<NI> &dst) {
  for (int i = 0; i < src.n_items && i < NI; ++i) dst.items[i] = src.items[i];
  dst.n_items = src.n_items;
  dst.flags = src.flags;
  dst.n_tiles = src.n_tiles;
  dst.tile_counter = src.tile_counter;
  dst.fix_list = src.fix_list;
  dst.fix_count = src.fix_count;
  dst.fix_capacity = src.fix_capacity;
  dst.stats = src.stats;
  dst.err = src.err;
}

}  // namespace

unsigned long long trace_tile_rays() { return kTile; }

cudaError_t launch_trace(const TraceLaunch &L, int n_sm, cudaStream_t stream) {
  if (L.n_items <= 1) {
    TraceLaunchT<1> l1;
    fill_launch(L, l1);
    return launch_trace_t(l1, n_sm, stream);
  }
  TraceLaunchT<kMaxBatchItems> *p = new TraceLaunchT<kMaxBatchItems>();  // large: off the host stack
  fill_launch(L, *p);
  cudaError_t e = launch_trace_t(*p, n_sm, stream);
  delete p;
  return e;
}

cudaError_t launch_fix(const TraceLaunch &L, int n_sm, cudaStream_t stream) {
  if (L.n_items <= 1) {
    TraceLaunchT<1> l1;
    fill_launch(L, l1);
    return launch_fix_t(l1, n_sm, stream);
  }
  TraceLaunchT<kMaxBatchItems> *p = new TraceLaunchT<kMaxBatchItems>();
  fill_launch(L, *p);
  cudaError_t e = launch_fix_t(*p, n_sm, stream);
  delete p;
  return e;
}

}  // namespace svo
