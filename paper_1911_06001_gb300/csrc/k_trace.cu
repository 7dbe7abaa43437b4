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
// parent's descriptor, the children still to visit, the parent's entry T0 and
// the entry of the next child to visit, so that popping past a child that
// starts beyond the best hit is one load and one compare.
#include <cuda_runtime.h>

#include <cfloat>
#include <cmath>
#include <cstdint>
#include <memory>
#include <mutex>
#include <type_traits>
#include <vector>

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
  uint4 *fix_cand;                  // pool of stored leaves (winner, contenders or re-trace cap)
  unsigned long long cand_capacity; // pool entries
  unsigned int *cand_count;         // pool entries taken (zeroed before the launch)
  uint32_t *fix_off;                // per list slot: its first pool entry, or kNoCand
  svo_trace_stats *stats;
  unsigned int *err;
  int32_t one_scene;     // every item traces the same scene: stage its tables in shared memory
  int32_t stack_levels;  // traversal stack levels per thread (max asset depth - 1)
  int32_t mbox_words;    // grid walk: words of each thread's tested-part bitset (max parts / 32)
  int32_t block;         // threads per block of the trace kernel: 64, 128 or 256
  int32_t rays_per_lane; // rays per lane in a warp's tile (tile = 32 * rays_per_lane rays)
  const int2 *top;       // one_scene: per part (first, count) of its top-level nodes staged in shared memory
  int32_t top_nodes;     // staged nodes per block (0: none)
  int32_t top_levels;    // levels staged of every part
  QueueEntry *queue;                // SVO_TRACE_WAVEFRONT: the ray queue (item i from items[i].qbase)
  unsigned int *queue_count;        // SVO_TRACE_WAVEFRONT: entries queued per item
  unsigned long long *queue_tile;   // SVO_TRACE_WAVEFRONT: tile counter of the descent launch
};

namespace {

constexpr float kU = 5.9604644775390625e-8f;   // 2^-24, FP32 unit roundoff
constexpr float kTau = 7.62939453125e-6f;      // 2^-17
constexpr int kCap = 4;  // candidate parts per pass (4: 1.5-2% faster than 8, fewer live registers)
constexpr int kSmemParts = 256;                 // parts staged in shared memory
constexpr int kBlock = 128;  // block size of the FP64 pass; the trace kernel takes 64, 128 or 256
// Resident threads per SM the trace kernel's register allocation must allow
// (768 = 24 warps: at most 80 registers a thread, no spills).  Measured per
// frame:
//   * articulated figure: 0.353 ms at the compiler's own 163 registers (12
//     warps), 0.327 ms at 128 (16 warps), flat from 16 to 24 warps;
//   * incoherent rays against ~120 parts: 9% faster at 24 warps than at 16;
//   * 32 warps (64 registers) spill and lose.
// The counting (STATS) and hit-buffer (REUSE) builds keep 16 warps: they would
// spill at 80.
constexpr int kTraceThreadsPerSM = 768;

constexpr unsigned long long kRayBits = 40;
constexpr uint32_t kNoCand = 0xFFFFFFFFu;  // a list slot without stored leaves

struct Tables {
  uint8_t q[8][6][256];  // [mirror][perm][true child mask] -> mask in visiting order
  uint8_t k[8][6][8];    // [mirror][perm][q] -> true octant
};
constexpr size_t kTablesBytes = (sizeof(Tables) + 15) & ~size_t(15);

__host__ __device__ constexpr void perm_axes(int p, int &a0, int &a1, int &a2) {
  // p = 2*rank_x + (rank_y > rank_z)
  const int rx = p >> 1;
  const bool z_first = (p & 1) != 0;
  int r[3] = {rx, 0, 0};
  const int lo = (rx == 0) ? 1 : 0, hi = (rx == 2) ? 1 : 2;
  r[1] = z_first ? hi : lo;
  r[2] = z_first ? lo : hi;
  a0 = (r[0] == 0) ? 0 : (r[1] == 0 ? 1 : 2);
  a1 = (r[0] == 1) ? 0 : (r[1] == 1 ? 1 : 2);
  a2 = (r[0] == 2) ? 0 : (r[1] == 2 ? 1 : 2);
}

// perm_axes packed: bits [6p + 2r, 6p + 2r + 2) hold the axis of rank r under
// order p.
constexpr unsigned long long pack_axis_order() {
  unsigned long long v = 0;
  for (int p = 0; p < 6; ++p) {
    int a0 = 0, a1 = 0, a2 = 0;
    perm_axes(p, a0, a1, a2);
    v |= (unsigned long long)(a0 | (a1 << 2) | (a2 << 4)) << (6 * p);
  }
  return v;
}
constexpr unsigned long long kAxisOrder = pack_axis_order();
static_assert(kAxisOrder == 0x1894a1624ull, "axis order table");

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

// The tables are built once per device (svo_ctx_create) and copied into
// shared memory by every block.
__device__ __align__(16) Tables g_tables;

__global__ void k_init_tables() { build_tables(&g_tables); }

__device__ __forceinline__ void load_tables(Tables *t) {
  static_assert(sizeof(Tables) % 16 == 0, "Tables must be a whole number of 16-byte words");
  const uint4 *src = reinterpret_cast<const uint4 *>(&g_tables);
  uint4 *dst = reinterpret_cast<uint4 *>(t);
  for (int i = threadIdx.x; i < (int)(sizeof(Tables) / 16); i += blockDim.x) dst[i] = src[i];
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
// and b = -o*inv: one FMA, whose rounding is part of the error bound behind
// eta.
template <typename R>
struct Slab;
template <>
struct Slab<float> {
  __device__ static float t(float P, float inv, float, float b) { return fmaf(P, inv, b); }
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

// Closed-box entry of one leaf in FP64 (the definition the oracle follows,
// each slab quotient taken as a product with the reciprocal of the direction
// component): ray to the part frame with the FP64 inverse, slab test of the
// leaf cell's box; a zero direction component keeps the slab only if the
// origin lies in it.  Returns whether the leaf is hit and its candidate t.
__device__ __forceinline__ bool leaf_entry64(const double *__restrict__ m, int D, unsigned long long vox, float4 o,
                                             float4 d, double &t) {
  const double ox = o.x, oy = o.y, oz = o.z, dx = d.x, dy = d.y, dz = d.z;
  const double lo3[3] = {fma(m[0], ox, fma(m[1], oy, fma(m[2], oz, m[3]))),
                         fma(m[4], ox, fma(m[5], oy, fma(m[6], oz, m[7]))),
                         fma(m[8], ox, fma(m[9], oy, fma(m[10], oz, m[11])))};
  const double ld3[3] = {fma(m[0], dx, fma(m[1], dy, m[2] * dz)), fma(m[4], dx, fma(m[5], dy, m[6] * dz)),
                         fma(m[8], dx, fma(m[9], dy, m[10] * dz))};
  const unsigned long long mask = (1ull << D) - 1ull;
  const double s = Num<double>::pow2neg(D);
  double t0 = (double)o.w, t1 = (double)d.w;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double c = (double)((vox >> (k * D)) & mask);
    const double blo = c * s, bhi = (c + 1.0) * s;
    if (ld3[k] == 0.0) {
      if (lo3[k] < blo || lo3[k] > bhi) return false;
      continue;
    }
    // one reciprocal per axis instead of two divisions: FP64 issues at a few
    // lanes per clock, so this pass is bound by its FP64 instruction count
    // (the result differs from the quotient by at most an ulp or two)
    const double inv = 1.0 / ld3[k];
    double ta = (blo - lo3[k]) * inv, tb = (bhi - lo3[k]) * inv;
    if (ta > tb) {
      const double x = ta;
      ta = tb;
      tb = x;
    }
    t0 = fmax(t0, ta);
    t1 = fmin(t1, tb);
  }
  t = t0;
  return t0 <= t1;
}

// The FP64 pass for a ray whose contender list overflowed: the FP32 descent
// with inflated boxes (as in the certified pass, so no leaf the FP64 rule could
// hit is skipped), each leaf reached decided by leaf_entry64, and the
// lexicographic minimum kept in FP64.  Same result as an FP64 descent, at FP32
// speed for the interior nodes.
struct HybridState {
  ExactState ex;
  const double *inv64;  // the part's FP64 world->local rows
  float4 o, d;          // the ray as given (FP32)
};

__device__ __forceinline__ float rel_bound(const HybridState &s, float tmax_rel, float tshift) {
  return fminf(tmax_rel, __fsub_ru(__double2float_ru(s.ex.t), tshift));
}

// Leaves that may still be the closest hit: every candidate whose entry lower
// bound lo does not exceed hi_min (the best upper bound of a certainly hit
// leaf).  The true winner is always among them, so a flagged ray can be
// resolved by intersecting only these leaves in FP64.
struct Contenders {
  float lo[kContenders];
  uint32_t part[kContenders];
  unsigned long long vox[kContenders];
  int n;
  bool overflow;
};

__device__ __forceinline__ void keep_contender(Contenders &c, float hi_min, float lo, uint32_t part,
                                               unsigned long long vox) {
  if (!(lo <= hi_min)) return;
  if (c.n < kContenders) {
    c.lo[c.n] = lo;
    c.part[c.n] = part;
    c.vox[c.n] = vox;
    ++c.n;
    return;
  }
  for (int i = 0; i < kContenders; ++i) {
    if (!(c.lo[i] <= hi_min)) {  // no longer a contender: reuse its slot
      c.lo[i] = lo;
      c.part[i] = part;
      c.vox[i] = vox;
      return;
    }
  }
  c.overflow = true;
}

__device__ __forceinline__ void offer(CertState &s, Contenders &c, float lo, float hi, float te, bool cert,
                                      uint32_t part, unsigned long long vox) {
  if (cert) s.hi_min = fminf(s.hi_min, hi);
  keep_contender(c, s.hi_min, lo, part, vox);
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
// The same bound in a part's shifted parameter t_rel = t - tshift, rounded up
// so that pruning stays conservative.
__device__ __forceinline__ float rel_bound(const CertState &s, float tmax_rel, float tshift) {
  return fminf(tmax_rel, __fsub_ru(s.hi_min, tshift));
}

struct Counters {
  uint32_t parts_tested, parts_entered, nodes, leaves, passes;
  uint32_t f_winner, f_overlap, f_width, reused;
};

// Front-to-back descent of one part in its local frame, in FP32 with boxes
// inflated by eta.  (o, d): local ray whose parameter is t - tshift;
// tmin/tmax are in that shifted parameter.  State S is CertState (the
// certified search: leaves give entry bounds) or HybridState (the FP64 pass's
// re-trace: every leaf reached is decided by leaf_entry64).
// Node descriptor idx of a part: the first ntop come from the block's
// shared-memory copy of the part's top levels, the rest from global memory.
// Descriptor idx, a node of level `lev`, of a part.  The node array is
// breadth first, so the nodes of the top `top_levels` levels are its first
// ones; those come from the block's shared-memory copy at address `top`
// (32-bit shared address of the part's first staged node), the rest from
// global memory.
__device__ __forceinline__ uint2 node_at(const uint2 *__restrict__ nodes, uint32_t top, int top_levels, int lev,
                                         uint32_t idx) {
  if (top_levels > 0 && lev < top_levels) {  // folds away where top_levels is the constant 0
    uint2 v;
    asm("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(top + 8u * idx));
    return v;
  }
  return __ldg(&nodes[idx]);
}

// One part's front-to-back descent in progress: what the descent keeps
// between node visits (its stack lives in shared memory).  The local ray
// has every direction component made non-negative by mirroring (mir: the
// mirrored axes), with reciprocals (ix, iy, iz) and b = -o * (1/d).
template <typename R>
struct Descent {
  R ox, oy, oz, ix, iy, iz, bx, by, bz, tmin, tmax, eta, tshift;
  const uint2 *nodes;
  uint32_t n_nodes, part, top, mir;
  int D, top_levels, level;
  uint32_t px, py, pz;
  uint32_t live;  // bit l: the stack entry of level l still has a child that may hold the closest hit
  uint2 desc;     // the descriptor of the node visited next
};

// Starts a descent at the part's root (the caller has checked n_nodes > 0).
template <typename R, bool STATS>
__device__ __forceinline__ void descent_start(Descent<R> &s, const uint2 *__restrict__ nodes, uint32_t n_nodes,
                                              uint32_t top, int top_levels, int D, R ox, R oy, R oz, R dx, R dy,
                                              R dz, R tmin, R tmax, R eta, R tshift, uint32_t part, Counters &cnt) {
  static_assert(std::is_same<R, float>::value, "the stack stores FP32 entry parameters");
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
  s.ix = Num<R>::rcp(dx);
  s.iy = Num<R>::rcp(dy);
  s.iz = Num<R>::rcp(dz);
  s.bx = -(ox * s.ix);
  s.by = -(oy * s.iy);
  s.bz = -(oz * s.iz);
  s.ox = ox;
  s.oy = oy;
  s.oz = oz;
  s.tmin = tmin;
  s.tmax = tmax;
  s.eta = eta;
  s.tshift = tshift;
  s.nodes = nodes;
  s.n_nodes = n_nodes;
  s.part = part;
  s.top = top;
  s.mir = mir;
  s.D = D;
  s.top_levels = top_levels;
  s.level = 0;
  s.px = s.py = s.pz = 0;
  s.live = 0;
  s.desc = node_at(nodes, top, top_levels, 0, 0u);
  if (STATS) ++cnt.nodes;
}

// One node of a descent, in FP32 with boxes inflated by eta; (o, d) is the
// local ray whose parameter is t - tshift, tmin / tmax in that parameter.
// State S is CertState (the certified search: leaves give entry bounds) or
// HybridState (the FP64 pass's re-trace: every leaf reached is decided by
// leaf_entry64).  The node's child mask comes first, then a push and a step
// down, its leaves, or a pop: a pop goes straight to the deepest level that
// still has a child to visit, so levels with nothing left cost no step, and
// a lane that pops is at its next node in the same step as lanes that
// descend.  Returns false once the part is done.
template <typename R, typename S, bool STATS, int STRIDE>
__device__ __forceinline__ bool descent_step(Descent<R> &s, uint4 *__restrict__ stk, const Tables *__restrict__ tab,
                                             S &st, Contenders *con, unsigned int &err, Counters &cnt) {
  constexpr bool CERT = std::is_same<S, CertState>::value;
  constexpr bool HYBRID = std::is_same<S, HybridState>::value;
  constexpr bool INFLATE = sizeof(R) == 4;  // FP32 descents inflate boxes by eta
  const R ox = s.ox, oy = s.oy, oz = s.oz, ix = s.ix, iy = s.iy, iz = s.iz, bx = s.bx, by = s.by, bz = s.bz;
  const R tmin = s.tmin, tmax = s.tmax, eta = s.eta, tshift = s.tshift;
  const uint32_t mir = s.mir, part = s.part;
  const int D = s.D;
  // masks (true octant space) of the children lying in the far half along
  // each mirrored axis
  const uint32_t HX = (mir & 1u) ? 0x55u : 0xAAu;
  const uint32_t HY = (mir & 2u) ? 0x33u : 0xCCu;
  const uint32_t HZ = (mir & 4u) ? 0x0Fu : 0xF0u;
  const uint8_t *__restrict__ qt = &tab->q[mir][0][0];
  const uint8_t *__restrict__ kt = &tab->k[mir][0][0];
  int level = s.level;
  uint32_t px = s.px, py = s.py, pz = s.pz;
  uint32_t live = s.live;
  const uint2 desc = s.desc;
  {
    const R sz = Num<R>::pow2neg(level), h = sz * R(0.5);
    const R lx = R(px) * sz, ly = R(py) * sz, lz = R(pz) * sz;
    const R tl = rel_bound(st, tmax, tshift);
    const R Ax = Slab<R>::t(lx - eta, ix, ox, bx), Ay = Slab<R>::t(ly - eta, iy, oy, by), Az = Slab<R>::t(lz - eta, iz, oz, bz);
    const R Bx = Slab<R>::t((lx + h) - eta, ix, ox, bx), By = Slab<R>::t((ly + h) - eta, iy, oy, by), Bz = Slab<R>::t((lz + h) - eta, iz, oz, bz);
    const R Cx = INFLATE ? Slab<R>::t((lx + h) + eta, ix, ox, bx) : Bx;
    const R Cy = INFLATE ? Slab<R>::t((ly + h) + eta, iy, oy, by) : By;
    const R Cz = INFLATE ? Slab<R>::t((lz + h) + eta, iz, oz, bz) : Bz;
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
    if (hit != 0u) {
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
          if (lo > rel_bound(st, tmax, tshift)) break;  // later leaves start even later
          if (STATS) ++cnt.leaves;
          const uint32_t vx = 2u * px + (m & 1u), vy = 2u * py + ((m >> 1) & 1u), vz = 2u * pz + ((m >> 2) & 1u);
          const unsigned long long gx = (mir & 1u) ? (((1u << D) - 1u) ^ vx) : vx;
          const unsigned long long gy = (mir & 2u) ? (((1u << D) - 1u) ^ vy) : vy;
          const unsigned long long gz = (mir & 4u) ? (((1u << D) - 1u) ^ vz) : vz;
          const unsigned long long vox = gx | (gy << D) | (gz << (2 * D));
          if constexpr (CERT) {
            const R clx = (m & 1u) ? lx + h : lx, cly = (m & 2u) ? ly + h : ly, clz = (m & 4u) ? lz + h : lz;
            const R dlo = fmax(fmax(Slab<R>::t(clx + eta, ix, ox, bx), Slab<R>::t(cly + eta, iy, oy, by)), fmax(Slab<R>::t(clz + eta, iz, oz, bz), tmin));
            const R dhi = fmin(fmin(Slab<R>::t((clx + h) - eta, ix, ox, bx), Slab<R>::t((cly + h) - eta, iy, oy, by)),
                               fmin(Slab<R>::t((clz + h) - eta, iz, oz, bz), tmax));
            const R te = fmax(fmax(Slab<R>::t(clx, ix, ox, bx), Slab<R>::t(cly, iy, oy, by)), fmax(Slab<R>::t(clz, iz, oz, bz), tmin));
            const bool cert = dlo <= dhi;
            // back to the ray's own parameter, rounding the bounds outward
            offer(st, *con, __fadd_rd(tshift, lo), cert ? __fadd_ru(tshift, dlo) : Num<R>::inf(), tshift + te, cert,
                  part, vox);
          } else if constexpr (HYBRID) {
            double tq;
            if (leaf_entry64(st.inv64, D, vox, st.o, st.d, tq)) offer(st.ex, tq, part, vox);
          } else {
            static_assert(CERT || HYBRID, "descent_step: CertState or HybridState");
          }
        }
      } else {
        const int q = __ffs(hq) - 1;
        const uint32_t rest = hq & (hq - 1u);
        // the entry of the child visited after this one (if any), kept with the
        // node so that a pop past it needs no plane arithmetic
        R en = Num<R>::inf();
        if (rest) {
          const int ax = (int)((kAxisOrder >> (6 * p + 2 * (31 - __clz(__ffs(rest) - 1)))) & 3ull);
          en = fmax(T0, ax == 0 ? Bx : (ax == 1 ? By : Bz));
        }
        stk[level * STRIDE] = make_uint4(desc.x, cmask | (rest << 8) | ((uint32_t)p << 16), __float_as_uint(en),
                                         __float_as_uint(T0));
        live = rest ? (live | (1u << level)) : (live & ~(1u << level));
        const uint32_t k = kt[p * 8 + q];
        const uint32_t idx = desc.x + __popc(cmask & ((1u << k) - 1u));
        if (idx >= s.n_nodes) {
          err |= kErrNodeIndex;
          return false;
        }
        s.desc = node_at(s.nodes, s.top, s.top_levels, level + 1, idx);
        if (STATS) ++cnt.nodes;
        const uint32_t m = k ^ mir;
        s.px = 2u * px + (m & 1u);
        s.py = 2u * py + ((m >> 1) & 1u);
        s.pz = 2u * pz + ((m >> 2) & 1u);
        s.level = level + 1;
        s.live = live;
        return true;
      }
    }
  }
  for (;;) {  // pop to the deepest level above that still has a child to visit
    const uint32_t cand = live & ((1u << level) - 1u);
    if (cand == 0u) return false;
    const int up = level - (31 - __clz(cand));
    level -= up;
    px >>= up;
    py >>= up;
    pz >>= up;
    const uint4 e = stk[level * STRIDE];
    uint32_t rest = (e.y >> 8) & 0xFFu;
    // the next child's entry, max(T0, mid-plane t of its highest-ranked
    // axis), was stored when the node was pushed; past the bound, this and
    // all later siblings are too far for good (the bound only shrinks)
    if (__uint_as_float(e.z) > rel_bound(st, tmax, tshift)) {
      live &= ~(1u << level);
      continue;
    }
    const int q = __ffs(rest) - 1;
    rest &= rest - 1u;
    if (!rest) live &= ~(1u << level);
    const int p = (int)(e.y >> 16);
    R en = Num<R>::inf();
    if (rest) {  // the entry of the child after it
      const R sz = Num<R>::pow2neg(level), h = sz * R(0.5);
      const int ax = (int)((kAxisOrder >> (6 * p + 2 * (31 - __clz(__ffs(rest) - 1)))) & 3ull);
      const R Bsel = ax == 0   ? Slab<R>::t((R(px) * sz + h) - eta, ix, ox, bx)
                     : ax == 1 ? Slab<R>::t((R(py) * sz + h) - eta, iy, oy, by)
                               : Slab<R>::t((R(pz) * sz + h) - eta, iz, oz, bz);
      en = fmax(__uint_as_float(e.w), Bsel);
    }
    stk[level * STRIDE] = make_uint4(e.x, (e.y & ~0xFF00u) | (rest << 8), __float_as_uint(en), e.w);
    const uint32_t k = kt[p * 8 + q];
    const uint32_t cmask = e.y & 0xFFu;
    const uint32_t idx = e.x + __popc(cmask & ((1u << k) - 1u));
    if (idx >= s.n_nodes) {
      err |= kErrNodeIndex;
      return false;
    }
    s.desc = node_at(s.nodes, s.top, s.top_levels, level + 1, idx);
    if (STATS) ++cnt.nodes;
    const uint32_t m = k ^ mir;
    s.px = 2u * px + (m & 1u);
    s.py = 2u * py + ((m >> 1) & 1u);
    s.pz = 2u * pz + ((m >> 2) & 1u);
    s.level = level + 1;
    s.live = live;
    return true;
  }
}

struct RayW {
  float ox, oy, oz, tmin, dx, dy, dz, tmax;
  float inv_dd;
  float inv_len;  // 1/|d|
  float onorm;    // ||o||_inf
};

// Conservative ray / sphere test: sphere (c, R) is hit by the segment.  Eq. 4
// with a direction of any length: l = c - o, tc = (l.d)/|d|^2, the squared
// distance of the centre to the line is |l - tc d|^2.
__device__ __forceinline__ bool sphere_test(const RayW &r, float lx, float ly, float lz, float R, float &tin,
                                            float &tc) {
  tc = (lx * r.dx + ly * r.dy + lz * r.dz) * r.inv_dd;
  const float qx = fmaf(-tc, r.dx, lx), qy = fmaf(-tc, r.dy, ly), qz = fmaf(-tc, r.dz, lz);
  const float p2 = qx * qx + qy * qy + qz * qz;
  const float R2 = R * R;
  if (!(p2 <= R2)) return false;
  const float half = sqrtf((R2 - p2) * r.inv_dd);
  const float tout = tc + half;
  tin = tc - half;
  return tout >= r.tmin && tin <= r.tmax;
}

// Part test.  The part's cube lies in its exact bounding sphere, so a ray that
// truly meets the cube passes once the FP32 test's own rounding is covered
// (16 u (|l|_1 + r) of slack).  tref: the reference parameter for the part's
// descent -- the sphere entry (or the closest approach on a miss), not before
// tmin.
__device__ __forceinline__ bool part_cull(const RayW &r, const PartHot &ph, float &tin, float &tref) {
  const float4 s = ph.sphere;
  if (s.w < 0.f) return false;
  const float lx = s.x - r.ox, ly = s.y - r.oy, lz = s.z - r.oz;
  const float ln = fabsf(lx) + fabsf(ly) + fabsf(lz);
  const float Rt = s.w * (1.0f + 9.5367431640625e-7f) + 16.0f * kU * (ln + s.w);
  float tc;
  const bool hit = sphere_test(r, lx, ly, lz, Rt, tin, tc);
  tref = fmaxf(hit ? tin : tc, r.tmin);
  return hit;
}

__device__ __forceinline__ bool cluster_cull(const RayW &r, const Cluster &c) {
  const float4 s = c.sphere;
  if (s.w < 0.f) return false;
  const float lx = s.x - r.ox, ly = s.y - r.oy, lz = s.z - r.oz;
  const float ln = fabsf(lx) + fabsf(ly) + fabsf(lz);
  // covers every member test's slack 16 u (|l_m|_1 + r_m), |l_m|_1 <= |l|_1 + sqrt(3) R
  const float Rt = s.w * (1.0f + 9.5367431640625e-7f) + 48.0f * kU * (2.0f * ln + 3.8f * s.w);
  float tin, tc;
  return sphere_test(r, lx, ly, lz, Rt, tin, tc);
}

// Ray -> part frame (Eq. 3) and descent.  The origin is first moved along the
// ray to q = o + tref d (tref: sphere entry), and q is mapped relative to the
// sphere centre c, o' = Ainv (q - c) + c', with c' the FP64-accurate local
// coordinates of c: all FP32 arithmetic then works on numbers of order one.
// The descent's parameter is t - tref.  eta bounds the position error of the
// FP32 local ray over the part (in local units), doubled for safety:
//   q rounding            u ||Ainv||_inf ||q||_inf
//   q - c and Ainv (q-c)   5u ||Ainv||_inf ||q - c||_inf, c' rounding u |c'|
//   mirroring, slabs      u (4 |o'| + 3)
//   FP32 direction        4u ||Ainv||_inf (|c - q|_1 + r)
// stop: shared-memory address of the block's staged top-level nodes, of
// which each part has its top `top_levels` levels (pa.spare0 carries, as
// bits, the part's first staged node; 0 levels when nothing is staged).
// part_start sets up the descent (returns false when the part's box is
// missed, starts beyond the bound, or the part is empty); trace_part_f32
// runs it to the end.
template <bool STATS, typename S>
__device__ __forceinline__ bool part_start(const RayW &r, const PartHot &ph, const PartAux &pa, float tref,
                                           uint32_t part, uint32_t stop, int top_levels, const S &st,
                                           Descent<float> &ds, Counters &cnt) {
  const float4 a = ph.r0, b = ph.r1, c = ph.r2;
  const float4 s = ph.sphere;
  const float qx = fmaf(tref, r.dx, r.ox), qy = fmaf(tref, r.dy, r.oy), qz = fmaf(tref, r.dz, r.oz);
  const float vx = qx - s.x, vy = qy - s.y, vz = qz - s.z;
  const float ox = fmaf(a.x, vx, fmaf(a.y, vy, fmaf(a.z, vz, a.w)));
  const float oy = fmaf(b.x, vx, fmaf(b.y, vy, fmaf(b.z, vz, b.w)));
  const float oz = fmaf(c.x, vx, fmaf(c.y, vy, fmaf(c.z, vz, c.w)));
  const float dx = fmaf(a.x, r.dx, fmaf(a.y, r.dy, a.z * r.dz));
  const float dy = fmaf(b.x, r.dx, fmaf(b.y, r.dy, b.z * r.dz));
  const float dz = fmaf(c.x, r.dx, fmaf(c.y, r.dy, c.z * r.dz));
  const float qn = fmaxf(fmaxf(fabsf(qx), fabsf(qy)), fabsf(qz));
  const float vn = fmaxf(fmaxf(fabsf(vx), fabsf(vy)), fabsf(vz));
  const float v1 = fabsf(vx) + fabsf(vy) + fabsf(vz);
  const float on = fmaxf(fmaxf(fabsf(ox), fabsf(oy)), fabsf(oz));
  const float cn = fmaxf(fmaxf(fabsf(a.w), fabsf(b.w)), fabsf(c.w));
  const float eta =
      kU * (2.0f * pa.n_ainv * (qn + 5.0f * vn + 4.0f * (v1 + fabsf(s.w))) + 2.0f * cn + 8.0f * on + 6.0f) * 1.001f;
  float tmin_rel = __fsub_rd(r.tmin, tref), tmax_rel = __fsub_ru(r.tmax, tref);
  // Clip the segment to the part's occupied box, inflated by 2 eta: one eta
  // for the local ray's error, one for this slab arithmetic.  Every leaf lies
  // in the box, so a leaf's entry is never before the clipped start nor its
  // exit after the clipped end: no candidate and no entry value changes, the
  // nodes outside the box along the ray are never visited, and a part whose
  // box the ray misses is not descended at all.
  {
    const float o3[3] = {ox, oy, oz}, d3[3] = {dx, dy, dz};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float lo = pa.box_lo[k] - 2.0f * eta, hi = pa.box_hi[k] + 2.0f * eta;
      if (d3[k] == 0.f) {
        if (o3[k] < lo || o3[k] > hi) tmax_rel = -Num<float>::inf();
        continue;
      }
      const float inv = 1.0f / d3[k];
      float ta = (lo - o3[k]) * inv, tb = (hi - o3[k]) * inv;
      if (ta > tb) {
        const float x = ta;
        ta = tb;
        tb = x;
      }
      tmin_rel = fmaxf(tmin_rel, ta);
      tmax_rel = fminf(tmax_rel, tb);
    }
  }
  // nothing to do either when the box starts beyond the best certain hit so
  // far (the descent's own bound)
  if (!(tmin_rel <= tmax_rel) || tmin_rel > rel_bound(st, tmax_rel, tref)) return false;
  if (STATS) ++cnt.parts_entered;
  if (pa.n_nodes == 0) return false;
  descent_start<float, STATS>(ds, pa.nodes, pa.n_nodes, stop + 8u * __float_as_uint(pa.spare0), top_levels, pa.depth,
                              ox, oy, oz, dx, dy, dz, tmin_rel, tmax_rel, eta, tref, part, cnt);
  return true;
}

template <bool STATS, typename S = CertState, int STRIDE = kBlock>
__device__ __forceinline__ void trace_part_f32(const RayW &r, const PartHot &ph, const PartAux &pa, float tref,
                                               uint32_t part, const Tables *tab, uint32_t stop, int top_levels,
                                               uint4 *stk, S &st, Contenders *con, unsigned int &err,
                                               Counters &cnt) {
  Descent<float> ds;
  if (part_start<STATS, S>(r, ph, pa, tref, part, stop, top_levels, st, ds, cnt))
    while (descent_step<float, S, STATS, STRIDE>(ds, stk, tab, st, con, err, cnt)) {
    }
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

// Culling through the scene-level grid (Sec. V-E).  Each cell lists every
// part whose sphere box comes within m = 2^-10 cells of it.  The ray walks the
// cells it crosses front to back (a 3D DDA whose crossing parameters are
// computed afresh from each cell plane, (plane - o) * (1/d), three roundings
// each, increasing along the walk); for t in the parameter interval of a visited cell
// the exact ray point lies within the rounding error of that cell, and a ray
// is only walked when that error is below m/2 (else the function returns
// false for it and the ray takes the cluster level).  The intervals of the
// visited cells follow each other without gaps, so a part whose sphere the
// exact ray meets at some t in them is listed in a visited cell.  Each listed
// part is sphere-tested once (a bitset per thread); the walk ends after the
// first cell whose interval reaches past the bound, the segment or the box.
//
// Called by the whole warp (go: this lane's ray takes part).  Each round,
// every walking lane gathers up to kCap candidates from its cell's list, and
// then the lanes descend their candidates together, in order of entry, so
// that the warp runs the descents side by side as on the cluster level.
template <bool STATS, int BLOCK>
__device__ __forceinline__ bool grid_walk(const RayW &r, bool go, const SceneGrid &g,
                                          const int32_t *__restrict__ cstart, const int32_t *__restrict__ cparts,
                                          const PartHot *__restrict__ hot, const PartAux *__restrict__ aux,
                                          const Tables *tab, uint32_t stop, int top_levels, uint4 *stk, uint32_t *mbox,
                                          int mwords, CertState &st, Contenders &con, unsigned int &err,
                                          Counters &cnt) {
  const int G = g.G;
  const float o[3] = {r.ox, r.oy, r.oz}, d[3] = {r.dx, r.dy, r.dz};
  bool ok = true, walking = go;
  // the segment inside the grid box
  float t0 = r.tmin, t1 = r.tmax;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float blo = g.lo[a], bhi = fmaf((float)G, g.cs[a], g.lo[a]);
    if (d[a] == 0.f) {
      if (o[a] < blo || o[a] > bhi) t1 = -Num<float>::inf();
      continue;
    }
    float ta = (blo - o[a]) / d[a], tb = (bhi - o[a]) / d[a];
    // else a component too small for the walk's arithmetic (the crossings
    // below stay within a few roundings of these, so they stay finite)
    ok = ok && fabsf(ta) < 1e38f && fabsf(tb) < 1e38f;
    if (ta > tb) {
      const float x = ta;
      ta = tb;
      tb = x;
    }
    t0 = fmaxf(t0, ta);
    t1 = fminf(t1, tb);
  }
  // the rounding allowance: a few units of roundoff of the largest magnitudes
  // in the crossing and start-cell arithmetic, against m/2 = 2^-11 cells
  int cur[3], step[3];
  float rd[3], tn[3];  // 1/d; the crossing of the current cell's far plane per axis
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float mag = fabsf(o[a]) + fabsf(g.lo[a]) + (float)G * g.cs[a] + fabsf(t0 * d[a]);
    ok = ok && 8.0f * kU * mag <= g.cs[a] * 4.8828125e-4f;
    const float f = (fmaf(t0, d[a], o[a]) - g.lo[a]) * g.inv_cs[a];
    const int i = (int)floorf(fminf(fmaxf(f, 0.f), (float)G));
    cur[a] = i > G - 1 ? G - 1 : i;
    step[a] = d[a] > 0.f ? 1 : (d[a] < 0.f ? -1 : 0);
    rd[a] = d[a] != 0.f ? 1.0f / d[a] : 0.f;
    tn[a] = d[a] != 0.f ? (fmaf((float)(cur[a] + (step[a] > 0 ? 1 : 0)), g.cs[a], g.lo[a]) - o[a]) * rd[a]
                        : Num<float>::inf();
  }
  walking = walking && ok && t0 <= t1;  // t0 > t1: the segment misses every sphere box
  int k = 0, kend = 0;
  if (walking) {
    for (int w = 0; w < mwords; ++w) mbox[w * BLOCK] = 0u;
    const int c = cur[0] + G * (cur[1] + G * cur[2]);
    k = cstart[c];
    kend = cstart[c + 1];
  }
  while (__any_sync(0xffffffffu, walking)) {
    float ct[kCap], ce[kCap];
    int cp[kCap];
#pragma unroll
    for (int i = 0; i < kCap; ++i) {
      ct[i] = Num<float>::inf();
      ce[i] = 0.f;
      cp[i] = 0x7fffffff;
    }
    if (walking) {
      // gather: the next candidates of this cell, up to kCap
      int n = 0;
      while (k < kend && n < kCap) {
        const int p = cparts[k++];
        uint32_t *wp = mbox + (p >> 5) * BLOCK;
        const uint32_t bit = 1u << (p & 31), wv = *wp;
        if (wv & bit) continue;
        *wp = wv | bit;
        float tin, tref;
        if (STATS) ++cnt.parts_tested;
        if (!part_cull(r, hot[p], tin, tref)) continue;
        if (tin > prune_bound(st, r.tmax)) continue;  // the bound only shrinks: never needed
        int pp = p;
        list_insert(ct, ce, cp, tin, tref, pp);  // not full: nothing is pushed out
        ++n;
      }
    }
    // descend, the warp's lanes side by side (the list shifts down each step)
#pragma unroll 1
    for (int i = 0; i < kCap && __any_sync(0xffffffffu, ct[0] != Num<float>::inf()); ++i) {
      if (ct[0] != Num<float>::inf() && ct[0] <= prune_bound(st, r.tmax))
        trace_part_f32<STATS, CertState, BLOCK>(r, hot[cp[0]], aux[cp[0]], ce[0], (uint32_t)cp[0], tab, stop,
                                                top_levels, stk, st, &con, err, cnt);
#pragma unroll
      for (int j = 0; j < kCap - 1; ++j) {
        ct[j] = ct[j + 1];
        ce[j] = ce[j + 1];
        cp[j] = cp[j + 1];
      }
      ct[kCap - 1] = Num<float>::inf();
    }
    if (walking && k >= kend) {
      // the cell's exit: the nearest crossing of a far cell plane
      const int ax = tn[0] <= tn[1] ? (tn[0] <= tn[2] ? 0 : 2) : (tn[1] <= tn[2] ? 1 : 2);
      const float tx = fminf(fminf(tn[0], tn[1]), tn[2]);
      if (!(tx < t1) || tx > prune_bound(st, r.tmax)) {  // also: no axis moves (tx infinite)
        walking = false;
      } else {
        bool out = false;
#pragma unroll
        for (int a = 0; a < 3; ++a) {  // static indices keep the arrays in registers
          if (a != ax) continue;
          cur[a] += step[a];
          out = cur[a] < 0 || cur[a] > G - 1;
          tn[a] = (fmaf((float)(cur[a] + (step[a] > 0 ? 1 : 0)), g.cs[a], g.lo[a]) - o[a]) * rd[a];
        }
        if (out) {
          walking = false;
        } else {
          const int c = cur[0] + G * (cur[1] + G * cur[2]);
          k = cstart[c];
          kend = cstart[c + 1];
        }
      }
    }
  }
  return ok;
}

// One culling pass (Sec. IV-A/B): the ray against the cluster spheres, then
// against the part spheres of the clusters it meets; the first kCap
// candidates in order of sphere entry (entry t, descent reference parameter,
// part) that come after (last_t, last_p), the last part an earlier pass
// descended, and in over_t the smallest entry that did not fit the list.
// Called by the whole warp (need: this lane's ray takes part); NC must be
// the same on every lane.  Every lane that met a cluster tests all its
// members; with VOTE the others idle through them, and a cluster no lane
// met is skipped.  VOTE false: a lane alone (no warp vote; its warp's lanes
// may hold rays of different items), as the refilling descent launch calls
// it.
template <bool STATS, bool VOTE = true>
__device__ __forceinline__ void cull_pass(const RayW &r, bool need, int NC, const PartHot *__restrict__ hot,
                                          const Cluster *__restrict__ cl, const int32_t *__restrict__ order,
                                          float last_t, int last_p, float (&ct)[kCap], float (&ce)[kCap],
                                          int (&cp)[kCap], float &over_t, Counters &cnt) {
  for (int c = 0; c < NC; ++c) {
    const Cluster cc = cl[c];
    const bool hc = need && cluster_cull(r, cc);
    if (VOTE && __ballot_sync(0xffffffffu, hc) == 0u) continue;  // no lane needs this cluster
    if (hc) {
      const uint32_t fc = __float_as_uint(cc.aux.w);
      const int first = (int)(fc & 0xFFFFu), count = (int)(fc >> 16);
      for (int k = 0; k < count; ++k) {
        const int p = order[first + k];
        float tin, eta;
        if (STATS) ++cnt.parts_tested;
        if (!part_cull(r, hot[p], tin, eta)) continue;
        if (tin < last_t || (tin == last_t && p <= last_p)) continue;  // visited in an earlier pass
        float t = tin, e = eta;
        int pp = p;
        list_insert(ct, ce, cp, t, e, pp);
        over_t = fminf(over_t, t);
      }
    }
  }
}

// The first culling pass of the culling launch (the same candidates as
// cull_pass with nothing descended before), with the member tests packed
// over the warp's lanes across clusters.  Incoherent rays meet a cluster a
// few lanes at a time, and testing its members in place would leave most
// lanes idle.  So every (lane, cluster) pair of a cluster met by at most
// kInPlaceLanes lanes goes into the warp's ring in shared memory (owner
// lane, first | count << 16). Whenever four pairs wait, one round tests
// their 32 (pair, member) combinations: lane q takes member q & 7 of pair
// q >> 3 against its owner's ray (read by shuffles), and every hit goes back
// to the owner's list.  A cluster met by more lanes has its members tested
// in place.  The list keeps the kCap smallest (t, part) keys, and over_t the
// smallest t of the others, whatever the order of insertion, so the result
// is that of cull_pass.
constexpr int kPackRing = 64;      // ring slots per warp: a power of two above 3 + kInPlaceLanes
constexpr int kInPlaceLanes = 16;  // lanes above which a cluster's members are tested in place
static_assert(kClusterSize == 8 && kInPlaceLanes + 3 < kPackRing, "four pairs of eight members fill a round");

// One round: pairs ring[head .. head + n_pairs) (n_pairs <= 4), member
// lane & 7 of pair lane >> 3 on every lane.
template <bool STATS>
__device__ __forceinline__ void member_round(const RayW &r, const int2 *ring, int head, int n_pairs,
                                             const PartHot *__restrict__ hot, const int32_t *__restrict__ order,
                                             float (&ct)[kCap], float (&ce)[kCap], int (&cp)[kCap],
                                             float &over_t, Counters &cnt) {
  const int lane = threadIdx.x & 31;
  const int e = lane >> 3, k = lane & 7;
  int owner = lane;
  uint32_t fc = 0u;  // no pair: count 0
  if (e < n_pairs) {
    const int2 q = ring[(head + e) & (kPackRing - 1)];
    owner = q.x;
    fc = (uint32_t)q.y;
  }
  const bool valid = k < (int)(fc >> 16);
  RayW ro;
  ro.ox = __shfl_sync(0xffffffffu, r.ox, owner);
  ro.oy = __shfl_sync(0xffffffffu, r.oy, owner);
  ro.oz = __shfl_sync(0xffffffffu, r.oz, owner);
  ro.dx = __shfl_sync(0xffffffffu, r.dx, owner);
  ro.dy = __shfl_sync(0xffffffffu, r.dy, owner);
  ro.dz = __shfl_sync(0xffffffffu, r.dz, owner);
  ro.tmin = __shfl_sync(0xffffffffu, r.tmin, owner);
  ro.tmax = __shfl_sync(0xffffffffu, r.tmax, owner);
  ro.inv_dd = __shfl_sync(0xffffffffu, r.inv_dd, owner);
  ro.inv_len = 0.f;
  ro.onorm = 0.f;
  float tin = 0.f, tref = 0.f;
  int p = 0;
  bool hit = false;
  if (valid) {
    p = order[(int)(fc & 0xFFFFu) + k];
    if (STATS) ++cnt.parts_tested;
    hit = part_cull(ro, hot[p], tin, tref);
  }
  // hand each hit to its ray's lane (hits are rare: one round each)
  for (unsigned int hm = __ballot_sync(0xffffffffu, hit); hm != 0u; hm &= hm - 1u) {
    const int src = __ffs(hm) - 1;
    const int o = __shfl_sync(0xffffffffu, owner, src);
    float t = __shfl_sync(0xffffffffu, tin, src), te = __shfl_sync(0xffffffffu, tref, src);
    int pp = __shfl_sync(0xffffffffu, p, src);
    if (lane == o) {
      list_insert(ct, ce, cp, t, te, pp);
      over_t = fminf(over_t, t);
    }
  }
}

// ring: the warp's kPackRing slots.  Called by the whole warp.
template <bool STATS>
__device__ __forceinline__ void cull_first_packed(const RayW &r, bool need, int NC, const PartHot *__restrict__ hot,
                                                  const Cluster *__restrict__ cl,
                                                  const int32_t *__restrict__ order, int2 *ring, float (&ct)[kCap],
                                                  float (&ce)[kCap], int (&cp)[kCap], float &over_t,
                                                  Counters &cnt) {
  const int lane = threadIdx.x & 31;
  int head = 0, pending = 0;  // warp-uniform: the ring's first waiting pair and the number waiting
  for (int c = 0; c < NC; ++c) {
    const Cluster cc = cl[c];
    const bool hc = need && cluster_cull(r, cc);
    const unsigned int m = __ballot_sync(0xffffffffu, hc);
    if (m == 0u) continue;  // no lane needs this cluster
    const uint32_t fc = __float_as_uint(cc.aux.w);
    const int nl = __popc(m);
    if (nl > kInPlaceLanes) {
      if (hc) {
        const int first = (int)(fc & 0xFFFFu), count = (int)(fc >> 16);
        for (int k = 0; k < count; ++k) {
          const int p = order[first + k];
          float tin, eta;
          if (STATS) ++cnt.parts_tested;
          if (!part_cull(r, hot[p], tin, eta)) continue;
          float t = tin, e = eta;
          int pp = p;
          list_insert(ct, ce, cp, t, e, pp);
          over_t = fminf(over_t, t);
        }
      }
      continue;
    }
    __syncwarp();  // the last round's reads of the ring are done
    if (hc) ring[(head + pending + __popc(m & ((1u << lane) - 1u))) & (kPackRing - 1)] = make_int2(lane, (int)fc);
    __syncwarp();
    pending += nl;
    for (; pending >= 4; pending -= 4, head = (head + 4) & (kPackRing - 1))
      member_round<STATS>(r, ring, head, 4, hot, order, ct, ce, cp, over_t, cnt);
  }
  for (; pending > 0; pending -= 4, head = (head + 4) & (kPackRing - 1))  // the last pairs
    member_round<STATS>(r, ring, head, min(pending, 4), hot, order, ct, ce, cp, over_t, cnt);
}

template <bool STATS, int BLOCK, bool GRID>
__device__ void trace_ray_f32(const RayW &r, bool active, uint32_t flags, int P, int NC,
                              const PartHot *__restrict__ hot, const PartAux *__restrict__ aux,
                              const Cluster *__restrict__ cl, const int32_t *__restrict__ order, const Tables *tab,
                              uint32_t stop, int top_levels, uint4 *stk, CertState &st, Contenders &con,
                              unsigned int &err,
                              Counters &cnt,
                              bool reuse, uint32_t prev_part, const uint8_t *__restrict__ dirty, bool &reused,
                              const SceneGrid *__restrict__ grid, uint32_t *mbox, int mwords) {
  reused = false;
  st.lo1 = st.hi1 = st.te1 = st.lo2 = st.hi_min = Num<float>::inf();
  st.part1 = kMissPart;
  st.cert1 = 0;
  st.vox1 = kMissVoxel;
  con.n = 0;
  con.overflow = false;
  const bool cull = (flags & SVO_TRACE_CULL) != 0;
  const bool sort = (flags & SVO_TRACE_SORT) != 0;
  if (cull && sort) {
    // Passes are warp-uniform (every lane of the warp calls this function for
    // one ray each): a lane that needs no further pass takes part with
    // need = false, so every vote below runs with the full warp mask.
    float last_t = -Num<float>::inf();
    int last_p = -1;
    bool need = active;
    if (GRID && grid != nullptr && grid->valid != 0) {  // warp-uniform: one item per warp
      // a ray the walk cannot take safely goes on to the cluster level below
      const SceneGrid &g = *grid;
      const bool walked = grid_walk<STATS, BLOCK>(r, need, g, g.cell_start, g.cell_parts, hot, aux, tab, stop,
                                                  top_levels, stk, mbox, mwords, st, con, err, cnt);
      if (STATS && need && walked) ++cnt.passes;
      need = need && !walked;
    }
    while (__any_sync(0xffffffffu, need)) {
      float ct[kCap], ce[kCap];
      int cp[kCap];
#pragma unroll
      for (int i = 0; i < kCap; ++i) {
        ct[i] = Num<float>::inf();
        ce[i] = 0.f;
        cp[i] = 0x7fffffff;
      }
      float over_t = Num<float>::inf();  // smallest entry that did not fit the list
      if (STATS && need) ++cnt.passes;
      cull_pass<STATS>(r, need, NC, hot, cl, order, last_t, last_p, ct, ce, cp, over_t, cnt);
      // hit buffer reuse (Sec. IV-C, Fig. 5).  The paper reuses a pixel whose
      // ray meets one sphere, that of its unmoved previous part.  The same
      // holds whenever every part whose sphere the ray meets is unmoved and
      // so is the previous winner (or there was none): unmoved parts keep
      // their spheres and their closest leaves along the ray, so the
      // candidates are a subset of the previous ones, and they contain the
      // previous winner, whose sphere is still met.
      if (need && reuse && last_p < 0 && ct[0] != Num<float>::inf() && over_t == Num<float>::inf() &&
          (prev_part == kMissPart || (prev_part < (uint32_t)P && dirty[prev_part] == 0))) {
        bool clean = true;
#pragma unroll
        for (int i = 0; i < kCap; ++i)
          if (ct[i] != Num<float>::inf()) clean = clean && dirty[cp[i]] == 0;
        if (clean) {
          reused = true;
          need = false;
        }
      }
      if (need) {
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
          trace_part_f32<STATS, CertState, BLOCK>(r, hot[p], aux[p], eta, (uint32_t)p, tab, stop, top_levels, stk,
                                                  st, &con, err, cnt);
          last_t = tin;
          last_p = p;
        }
        // another pass only if some candidate did not fit the list and may still matter
        need = !stopped && over_t < Num<float>::inf() && over_t <= prune_bound(st, r.tmax);
      }
    }
  } else {
    for (int p = 0; p < P; ++p) {
      float tin, tref = r.tmin;
      if (!active) continue;
      if (STATS) ++cnt.parts_tested;
      const bool h = part_cull(r, hot[p], tin, tref);
      if (cull && !h) continue;
      // the plain trace descends every part, even one whose sphere is missed
      trace_part_f32<STATS, CertState, BLOCK>(r, hot[p], aux[p], tref, (uint32_t)p, tab, stop, top_levels, stk, st,
                                              &con, err, cnt);
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
  unsigned long long v[11] = {rays, flagged, c.parts_tested, c.parts_entered, c.nodes, c.leaves, c.passes,
                              c.f_winner, c.f_overlap, c.f_width, c.reused};
#pragma unroll
  for (int i = 0; i < 11; ++i) {
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
    atomicAdd(&st->flag_winner, v[7]);
    atomicAdd(&st->flag_overlap, v[8]);
    atomicAdd(&st->flag_width, v[9]);
    atomicAdd(&st->reused, v[10]);
  }
}

// The ray of `lane` in pass j of warp tile `tile` of item I: its index in the
// item's ray buffer (through the item's visiting order, if any); in_range is
// false past the item's end.  The tile of an image item is a block of
// 8 x 4*rays_per_lane pixels, claimed in the item's tile order (row by row
// without one).
template <int NI>
__device__ __forceinline__ unsigned long long tile_ray(const TraceLaunchT<NI> &L, const TraceItem &I,
                                                       unsigned long long tile, int j, int lane, bool &in_range) {
  const int rpl = L.rays_per_lane;
  const unsigned long long base = (tile - I.tile_begin) * (unsigned long long)(32 * rpl);
  unsigned long long slot_i = base + (unsigned long long)(j * 32 + lane);
  in_range = slot_i < I.n;
  if (I.tiles_x) {
    const uint32_t T = (uint32_t)(tile - I.tile_begin);
    uint32_t ty, tx;
    if (I.tile_order) {
      const uint32_t v = __ldg(&I.tile_order[T]);
      tx = v & 0xFFFFu;
      ty = v >> 16;
    } else {
      ty = T / I.tiles_x;
      tx = T - ty * I.tiles_x;
    }
    const uint32_t k = (uint32_t)(j * 32 + lane);
    const uint32_t x = tx * 8u + (k & 7u);
    const unsigned long long y = (unsigned long long)ty * (unsigned long long)(4 * rpl) + (k >> 3);
    slot_i = y * I.width + x;
    in_range = x < I.width && slot_i < I.n;
  }
  return (in_range && I.perm) ? (unsigned long long)I.perm[slot_i] : slot_i;
}

// Ray `ray` of item I (in_range false: an empty ray).  Returns whether it
// takes part: a ray needs a direction (Eq. 1) -- its largest component
// magnitude must lie in [2^-60, 2^60], so that |d|^2 is a normal FP32 number
// -- and origin, direction and bounds must be numbers, with tmin <= tmax;
// anything else is a miss.  Exact comparisons: the rule does not depend on
// rounding.
__device__ __forceinline__ bool load_ray(const TraceItem &I, unsigned long long ray, bool in_range, RayW &r) {
  bool active = in_range;
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
    const float dm = fmaxf(fmaxf(fabsf(d.x), fabsf(d.y)), fabsf(d.z));
    const bool finite = isfinite(o.x) && isfinite(o.y) && isfinite(o.z) && isfinite(d.x) && isfinite(d.y) &&
                        isfinite(d.z) && !isnan(o.w) && !isnan(d.w) && dm >= 0x1p-60f && dm <= 0x1p60f;
    r.inv_dd = __frcp_rn(dd);  // the correctly rounded 1 / dd
    r.inv_len = rsqrtf(dd);
    r.onorm = fmaxf(fmaxf(fabsf(o.x), fabsf(o.y)), fabsf(o.z));
    active = finite && (o.w <= d.w);
  } else {
    r.ox = r.oy = r.oz = r.dx = r.dy = r.dz = 0.f;
    r.tmin = 0.f;
    r.tmax = -1.f;
    r.inv_dd = 0.f;
    r.inv_len = 0.f;
    r.onorm = 0.f;
  }
  return active;
}

// The result of one ray, called by every lane of the warp (in_range false: a
// lane without a ray): the hit and its flags, and -- with FP64_FIX -- the
// ray's entry in the FP64 pass's list with the leaves that pass needs.
// LANE: a lane alone (its warp's other lanes are elsewhere in their work):
// its list slot and pool entries come from atomics of its own instead of
// one atomic per warp.
template <int NI, bool STATS, bool LANE = false>
__device__ __forceinline__ void finish_ray(const TraceLaunchT<NI> &L, const TraceItem &I, int it,
                                           unsigned long long ray, bool in_range, bool reused, const RayW &r,
                                           const PartAux *__restrict__ aux, const CertState &st,
                                           const Contenders &con, int lane, unsigned int &err, Counters &cnt,
                                           uint32_t &n_flag) {
  bool flagged = false, ids_ok = true;
  uint32_t tbound = 0;  // T_REFINED: the certified error exponent, biased (flag bits 8-15)
  if (in_range && reused) {
    if (I.ray_flags) I.ray_flags[ray] = SVO_RAY_REUSED;
    if (STATS) ++cnt.reused;
  } else if (in_range) {
    float t = Num<float>::inf();
    uint32_t part = kMissPart;
    unsigned long long vox = kMissVoxel;
    if (st.part1 != kMissPart) {
      // the reported t lies in [lo1, hi1]; its error is at most half the width
      const float scale = fmaxf(st.lo1, aux[st.part1].hdiag * r.inv_len);
      const bool w_ok = st.cert1 != 0u;
      const bool o_ok = st.lo2 > st.hi1;
      const bool t_ok = 0.5f * (st.hi1 - st.lo1) <= kTau * scale;
      ids_ok = w_ok && o_ok;
      flagged = !(ids_ok && t_ok);
      if (ids_ok && !t_ok && I.ray_flags) {
        // the written t and the exact one both lie in [lo1, hi1]: their
        // distance is at most 2^e scale with e = ceil(log2((hi1 - lo1) /
        // scale)), both operations rounded up
        const uint32_t bits = __float_as_uint(__fdiv_ru(__fsub_ru(st.hi1, st.lo1), scale));
        const int e = (int)(bits >> 23) - 127 + ((bits & 0x7FFFFFu) != 0u ? 1 : 0);
        tbound = (uint32_t)min(max(e + 128, 1), 255);
      }
      if (STATS) {
        cnt.f_winner += w_ok ? 0u : 1u;
        cnt.f_overlap += (w_ok && !o_ok) ? 1u : 0u;
        cnt.f_width += (ids_ok && !t_ok) ? 1u : 0u;
      }
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
    if (I.ray_flags)
      I.ray_flags[ray] = !ids_ok ? SVO_RAY_UNCERTAIN : (flagged ? (SVO_RAY_T_REFINED | (tbound << 8)) : 0u);
    if (STATS && !ids_ok) ++n_flag;
  }
  // compact flagged rays for the FP64 pass: one list slot each and, from
  // a pool, exactly the leaves the pass needs (one atomic per warp for
  // each): the winner alone when only t needs FP64, the contenders still
  // in play (lo <= hi_min) otherwise, or -- when the contender list
  // overflowed -- one entry carrying hi_min, where the full re-trace may
  // stop.  A ray the pool cannot hold is re-traced without that bound.
  if (L.flags & SVO_TRACE_FP64_FIX) {
    const unsigned int m = LANE ? (flagged ? 1u : 0u) : __ballot_sync(0xffffffffu, flagged);
    if (m) {
      unsigned int ncon = 0;  // contenders in play
      if (flagged && !ids_ok && !con.overflow)
        for (int q = 0; q < con.n; ++q) ncon += (con.lo[q] <= st.hi_min) ? 1u : 0u;
      const unsigned int need = !flagged ? 0u : (ids_ok || con.overflow || ncon == 0u) ? 1u : ncon;
      unsigned long long slot = 0, off = 0;
      if (LANE) {
        slot = atomicAdd(L.fix_count, 1u);
        off = atomicAdd(L.cand_count, need);
      } else {
        const int leader = __ffs(m) - 1;
        unsigned int incl = need;  // inclusive scan of the lanes' pool entries
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const unsigned int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const unsigned int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned int basei = 0, basep = 0;
        if (lane == leader) {
          basei = atomicAdd(L.fix_count, (unsigned int)__popc(m));
          basep = atomicAdd(L.cand_count, total);
        }
        basei = __shfl_sync(0xffffffffu, basei, leader);
        basep = __shfl_sync(0xffffffffu, basep, leader);
        slot = basei + __popc(m & ((1u << lane) - 1u));
        off = (unsigned long long)basep + (incl - need);
      }
      if (flagged) {
        if (slot < L.fix_capacity) {
          const bool stored = off + need <= L.cand_capacity;
          unsigned long long nc = 0;  // leaves listed; 0 = full FP64 re-trace
          if (stored) {
            if (ids_ok) {
              // ids certified, only t needs FP64: the winner alone
              L.fix_cand[off] = make_uint4(st.part1, (uint32_t)(st.vox1 & 0xFFFFFFFFull),
                                           (uint32_t)(st.vox1 >> 32), __float_as_uint(st.lo1));
              nc = 1;
            } else if (!con.overflow && ncon > 0u) {
              for (int q = 0; q < con.n; ++q) {
                if (!(con.lo[q] <= st.hi_min)) continue;
                L.fix_cand[off + nc] = make_uint4(con.part[q], (uint32_t)(con.vox[q] & 0xFFFFFFFFull),
                                                  (uint32_t)(con.vox[q] >> 32), __float_as_uint(con.lo[q]));
                ++nc;
              }
            } else {
              // the re-trace may stop at hi_min, an upper bound (rounded up) of the winner's t
              L.fix_cand[off] = make_uint4(0u, 0u, 0u, __float_as_uint(st.hi_min));
            }
          }
          L.fix_off[slot] = stored ? (uint32_t)off : kNoCand;
          const unsigned long long t_only = ids_ok ? 1ull : 0ull;  // ids certain, t needs FP64
          L.fix_list[slot] = (nc << 48) | (t_only << 47) | ((unsigned long long)it << kRayBits) | ray;
        } else {
          err |= kErrFixOverflow;
        }
      }
    }
  }

}

// REUSE: hit buffer reuse compiled in (a separate instantiation, so that the
// common kernel carries none of its registers or tests).
// GRID: the scene-level grid walk compiled in (likewise).
// TOP: the top levels of every part staged in shared memory (a separate
// instantiation: the staged-node base is one more live register, which the
// common kernel does not carry).
template <int NI, bool STATS, int BLOCK, bool REUSE, bool GRID, bool TOP = false>
__global__ void __launch_bounds__(BLOCK, (STATS || REUSE || GRID ? 512 : kTraceThreadsPerSM) / BLOCK) k_trace(const __grid_constant__ TraceLaunchT<NI> L) {
  extern __shared__ __align__(16) unsigned char smem[];
  // [tables | traversal stacks, level-major | staged part tables]
  Tables *tab = reinterpret_cast<Tables *>(smem);
  uint4 *sStack = reinterpret_cast<uint4 *>(smem + kTablesBytes) + threadIdx.x;
  const int sp = L.one_scene ? L.items[0].n_parts : 0;
  const int sc = L.one_scene ? L.items[0].n_clusters : 0;
  PartHot *sHot = reinterpret_cast<PartHot *>(smem + kTablesBytes + (size_t)L.stack_levels * BLOCK * sizeof(uint4));
  PartAux *sAux = reinterpret_cast<PartAux *>(sHot + sp);
  Cluster *sCl = reinterpret_cast<Cluster *>(sAux + sp);
  int32_t *sOrd = reinterpret_cast<int32_t *>(sCl + sc);
  uint2 *sTop = reinterpret_cast<uint2 *>(sOrd + sp + (sp & 1));  // 8-byte aligned: sOrd starts so
  const int ntop_all = (TOP && L.one_scene) ? L.top_nodes : 0;
  uint32_t *sMbox = reinterpret_cast<uint32_t *>(sTop + ntop_all) + threadIdx.x;  // word-major, stride BLOCK
  const uint32_t sTopAddr = (uint32_t)__cvta_generic_to_shared(sTop);
  load_tables(tab);
  if (L.one_scene) {
    const TraceItem &I0 = L.items[0];
    for (int i = threadIdx.x; i < I0.n_parts; i += BLOCK) {
      sHot[i] = I0.hot[i];
      PartAux a = I0.aux[i];
      if (ntop_all > 0) {
        const int2 t = L.top[i];
        a.spare0 = __uint_as_float((uint32_t)t.x);
        a.spare1 = __uint_as_float((uint32_t)t.y);  // count (the kernel needs only the first)
      }
      sAux[i] = a;
      sOrd[i] = I0.order[i];
    }
    for (int i = threadIdx.x; i < I0.n_clusters; i += BLOCK) sCl[i] = I0.clusters[i];
    // every part's top levels: breadth first, they are the first nodes of its array
    for (int p = 0; p < I0.n_parts && ntop_all > 0; ++p) {
      const int2 t = L.top[p];
      const uint2 *src = I0.aux[p].nodes;
      for (int k = threadIdx.x; k < t.y; k += BLOCK) sTop[t.x + k] = __ldg(&src[k]);
    }
  }
  __syncthreads();  // the only block barrier: warps then take tiles independently
  unsigned int err = 0;
  Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t n_rays = 0, n_flag = 0;
  const int lane = threadIdx.x & 31;
  for (;;) {
    unsigned long long tile = 0;
    if (lane == 0) tile = atomicAdd(L.tile_counter, 1ull);
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile >= L.n_tiles) break;
    const int it = find_item(L, tile);
    const TraceItem &I = L.items[it];
    const int P = I.n_parts, NC = I.n_clusters;
    const bool staged = L.one_scene != 0;
    const PartHot *hot = staged ? sHot : I.hot;
    const PartAux *aux = staged ? sAux : I.aux;
    const Cluster *cls = staged ? sCl : I.clusters;
    const int32_t *ord = staged ? sOrd : I.order;
    const int rpl = L.rays_per_lane;
#pragma unroll 1
    for (int j = 0; j < rpl; ++j) {
      bool in_range = false;
      const unsigned long long ray = tile_ray(L, I, tile, j, lane, in_range);
      RayW r;
      const bool active = load_ray(I, ray, in_range, r);
      if (STATS && in_range) ++n_rays;
      CertState st;
      Contenders con;
      const bool reuse = REUSE && active;
      const uint32_t prev_part = reuse ? reinterpret_cast<const uint32_t *>(&I.hits[ray])[1] : kMissPart;
      bool reused;
      trace_ray_f32<STATS, BLOCK, GRID>(r, active, L.flags, P, NC, hot, aux, cls, ord, tab, sTopAddr,
                                        (TOP && ntop_all > 0) ? L.top_levels : 0, sStack, st, con,
                                        err, cnt, reuse, prev_part, I.dirty, reused, GRID ? I.grid : nullptr,
                                        sMbox, L.mbox_words);
      finish_ray<NI, STATS>(L, I, it, ray, in_range, reused, r, aux, st, con, lane, err, cnt, n_flag);
    }
  }
  if (STATS) flush_stats(L.stats, cnt, n_rays, n_flag);
  if (err) atomicOr(L.err, err);
}

// The culling launch of SVO_TRACE_WAVEFRONT.  Its warps take the trace's
// tiles of rays statically (a warp's tiles are its index plus multiples of
// the warp count: the work per ray varies little, and no counter is
// contended), run each ray's first culling pass (Sec. IV-A/B) and either
// write its miss -- no part sphere met: the result the trace would write --
// or queue it with its candidates in its item's region of the queue (one
// atomic per warp).  The descent launch traces the queued rays from there.
template <int NI, bool STATS, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK) k_cull(const __grid_constant__ TraceLaunchT<NI> L) {
  extern __shared__ __align__(16) unsigned char smem[];
  // [per-warp rings of member-test pairs | staged part spheres | clusters | part order of a one-scene launch]
  const int sp = L.one_scene ? L.items[0].n_parts : 0;
  const int sc = L.one_scene ? L.items[0].n_clusters : 0;
  int2 *ring = reinterpret_cast<int2 *>(smem) + (threadIdx.x >> 5) * kPackRing;
  PartHot *sHot = reinterpret_cast<PartHot *>(smem + (BLOCK / 32) * kPackRing * sizeof(int2));
  Cluster *sCl = reinterpret_cast<Cluster *>(sHot + sp);
  int32_t *sOrd = reinterpret_cast<int32_t *>(sCl + sc);
  if (L.one_scene) {
    const TraceItem &I0 = L.items[0];
    for (int i = threadIdx.x; i < I0.n_parts; i += BLOCK) {
      sHot[i] = I0.hot[i];
      sOrd[i] = I0.order[i];
    }
    for (int i = threadIdx.x; i < I0.n_clusters; i += BLOCK) sCl[i] = I0.clusters[i];
  }
  __syncthreads();
  Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t n_rays = 0;
  const int lane = threadIdx.x & 31;
  const unsigned long long n_warps = (unsigned long long)gridDim.x * (BLOCK / 32);
  for (unsigned long long tile = (unsigned long long)blockIdx.x * (BLOCK / 32) + (threadIdx.x >> 5);
       tile < L.n_tiles; tile += n_warps) {
    const int it = find_item(L, tile);
    const TraceItem &I = L.items[it];
    const bool staged = L.one_scene != 0;
    const PartHot *hot = staged ? sHot : I.hot;
    const Cluster *cls = staged ? sCl : I.clusters;
    const int32_t *ord = staged ? sOrd : I.order;
#pragma unroll 1
    for (int j = 0; j < L.rays_per_lane; ++j) {
      bool in_range;
      const unsigned long long ray = tile_ray(L, I, tile, j, lane, in_range);
      RayW r;
      const bool active = load_ray(I, ray, in_range, r);
      if (STATS && in_range) ++n_rays;
      float ct[kCap], ce[kCap];
      int cp[kCap];
#pragma unroll
      for (int i = 0; i < kCap; ++i) {
        ct[i] = Num<float>::inf();
        ce[i] = 0.f;
        cp[i] = 0x7fffffff;
      }
      float over_t = Num<float>::inf();
      if (STATS && active) ++cnt.passes;
      cull_first_packed<STATS>(r, active, I.n_clusters, hot, cls, ord, ring, ct, ce, cp, over_t, cnt);
      // over_t is set only by a full list, so an empty list means no candidate at all
      const bool queued = active && ct[0] != Num<float>::inf();
      if (in_range && !queued) {
        __stcs(&I.hits[ray], make_uint4(0x7f800000u, kMissPart, 0xFFFFFFFFu, 0xFFFFFFFFu));
        if (I.ray_flags) I.ray_flags[ray] = 0u;
      }
      const unsigned int m = __ballot_sync(0xffffffffu, queued);
      if (m) {
        const int leader = __ffs(m) - 1;
        unsigned int base = 0;
        if (lane == leader) base = atomicAdd(&L.queue_count[it], (unsigned int)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (queued) {
          QueueEntry *q = L.queue + I.qbase + base + (unsigned int)__popc(m & ((1u << lane) - 1u));
          q->id = make_uint4((uint32_t)ray, (uint32_t)(ray >> 32), __float_as_uint(over_t), 0u);
          q->ct = make_float4(ct[0], ct[1], ct[2], ct[3]);
          q->ce = make_float4(ce[0], ce[1], ce[2], ce[3]);
          q->cp = make_int4(cp[0], cp[1], cp[2], cp[3]);
        }
      }
    }
  }
  if (STATS) flush_stats(L.stats, cnt, n_rays, 0u);
}

// The descent launch of SVO_TRACE_WAVEFRONT.  Every lane works through the
// queued rays on its own: when its part's descent ends it goes on to the
// ray's next candidate, a further culling pass, or the ray's result and the
// next queued ray, while the other lanes of its warp carry on with their
// own descents.  A warp thus stays full until the queue runs dry, instead
// of waiting for the longest of a tile's 32 descents (incoherent rays into
// assets of different depths descend for very different lengths).  Each
// step of the loop: lanes that need a ray take the next entries of the
// warp's claimed run (32 entries claimed with one atomic), lanes between
// parts set up their next part, and every lane in a descent takes one node.
// The arithmetic is that of the fused kernel: part_start, descent_step,
// cull_pass and finish_ray, so results are the same bit for bit.
constexpr int kRefillLanes = 16;  // lanes that wait before the warp serves them

template <int NI, bool STATS, int BLOCK>
__global__ void __launch_bounds__(BLOCK, 512 / BLOCK) k_descend(const __grid_constant__ TraceLaunchT<NI> L) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned long long sQE[NI + 1];  // first entry of each item in the flat order of all queued rays
  // [tables | traversal stacks, level-major | staged part tables]
  Tables *tab = reinterpret_cast<Tables *>(smem);
  uint4 *sStack = reinterpret_cast<uint4 *>(smem + kTablesBytes) + threadIdx.x;
  const int sp = L.one_scene ? L.items[0].n_parts : 0;
  const int sc = L.one_scene ? L.items[0].n_clusters : 0;
  PartHot *sHot = reinterpret_cast<PartHot *>(smem + kTablesBytes + (size_t)L.stack_levels * BLOCK * sizeof(uint4));
  PartAux *sAux = reinterpret_cast<PartAux *>(sHot + sp);
  Cluster *sCl = reinterpret_cast<Cluster *>(sAux + sp);
  int32_t *sOrd = reinterpret_cast<int32_t *>(sCl + sc);
  load_tables(tab);
  if (L.one_scene) {
    const TraceItem &I0 = L.items[0];
    for (int i = threadIdx.x; i < I0.n_parts; i += BLOCK) {
      sHot[i] = I0.hot[i];
      sAux[i] = I0.aux[i];
      sOrd[i] = I0.order[i];
    }
    for (int i = threadIdx.x; i < I0.n_clusters; i += BLOCK) sCl[i] = I0.clusters[i];
  }
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int i = 0; i < L.n_items; ++i) {
      sQE[i] = acc;
      acc += min((unsigned long long)L.queue_count[i], L.items[i].n);
    }
    sQE[L.n_items] = acc;
  }
  __syncthreads();  // the only block barrier
  const unsigned long long total = sQE[L.n_items];
  const bool staged = L.one_scene != 0;
  unsigned int err = 0;
  Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  uint32_t n_flag = 0;
  const int lane = threadIdx.x & 31;
  enum { kNeedRay = 0, kBetween = 1, kDescending = 2, kDone = 3 };
  int state = kNeedRay;
  int it = 0;
  unsigned long long ray = 0;
  RayW r;
  CertState st;
  Contenders con;
  float ct[kCap], ce[kCap];
  int cp[kCap];
  float over_t = 0.f, last_t = 0.f;
  int last_p = -1;
  bool stopped = false;
  Descent<float> ds;
  unsigned long long wnext = 0, wend = 0;  // the warp's claimed run of entries (warp-uniform)
  for (;;) {
    // lanes waiting for work are served together, once enough of them wait
    // (or no lane is descending): the set-up of a part and the result of a
    // ray then run for many lanes at a time
    const unsigned int waiting = __ballot_sync(0xffffffffu, state == kNeedRay || state == kBetween);
    const bool serve = __popc(waiting) >= kRefillLanes || !__any_sync(0xffffffffu, state == kDescending);
    // lanes that need a ray take the next entries of the warp's run
    unsigned int want = serve ? __ballot_sync(0xffffffffu, state == kNeedRay) : 0u;
    while (want) {
      if (wnext >= wend) {
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(L.queue_tile, 32ull);
        b = __shfl_sync(0xffffffffu, b, 0);
        wnext = b;
        wend = b + 32ull < total ? b + 32ull : total;
        if (wnext >= total) {
          if (want & (1u << lane)) state = kDone;  // the queue is empty
          break;
        }
      }
      const unsigned int take = min((unsigned int)__popc(want), (unsigned int)(wend - wnext));
      const unsigned int rank = __popc(want & ((1u << lane) - 1u));
      if ((want & (1u << lane)) && rank < take) {
        const unsigned long long g = wnext + rank;
        int lo = 0, hi = L.n_items - 1;  // the item holding flat entry g
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (sQE[mid] <= g)
            lo = mid;
          else
            hi = mid - 1;
        }
        it = lo;
        const TraceItem &I = L.items[it];
        const QueueEntry *q = L.queue + I.qbase + (g - sQE[it]);
        const uint4 id = q->id;
        ray = (unsigned long long)id.x | ((unsigned long long)id.y << 32);
        over_t = __uint_as_float(id.z);
        const float4 a = q->ct, b = q->ce;
        const int4 c = q->cp;
        static_assert(kCap == 4, "a queued ray carries four candidates");
        ct[0] = a.x, ct[1] = a.y, ct[2] = a.z, ct[3] = a.w;
        ce[0] = b.x, ce[1] = b.y, ce[2] = b.z, ce[3] = b.w;
        cp[0] = c.x, cp[1] = c.y, cp[2] = c.z, cp[3] = c.w;
        load_ray(I, ray, true, r);  // a queued ray is a ray: the culling launch checked it
        st.lo1 = st.hi1 = st.te1 = st.lo2 = st.hi_min = Num<float>::inf();
        st.part1 = kMissPart;
        st.cert1 = 0;
        st.vox1 = kMissVoxel;
        con.n = 0;
        con.overflow = false;
        last_t = -Num<float>::inf();
        last_p = -1;
        stopped = false;
        state = kBetween;
      }
      // warp-uniform bookkeeping of the run and of the lanes still waiting
      unsigned int served = 0u, w = want;
      for (unsigned int k = 0; k < take; ++k) {
        served |= w & (0u - w);  // lowest waiting lane
        w &= w - 1u;
      }
      want &= ~served;
      wnext += take;
    }
    // lanes between parts: the next candidate, a further culling pass, or the ray's result
    while (serve && state == kBetween) {
      const TraceItem &I = L.items[it];
      const PartHot *hot = staged ? sHot : I.hot;
      const PartAux *aux = staged ? sAux : I.aux;
      if (ct[0] != Num<float>::inf()) {
        const float tin = ct[0], tref = ce[0];
        const int p = cp[0];
#pragma unroll
        for (int i = 0; i < kCap - 1; ++i) {
          ct[i] = ct[i + 1];
          ce[i] = ce[i + 1];
          cp[i] = cp[i + 1];
        }
        ct[kCap - 1] = Num<float>::inf();
        if (tin > prune_bound(st, r.tmax)) {  // this and every later candidate start beyond the best hit
          stopped = true;
#pragma unroll
          for (int i = 0; i < kCap; ++i) ct[i] = Num<float>::inf();
          continue;
        }
        last_t = tin;
        last_p = p;
        if (part_start<STATS, CertState>(r, hot[p], aux[p], tref, (uint32_t)p, 0u, 0, st, ds, cnt)) state = kDescending;
        continue;
      }
      if (!stopped && over_t < Num<float>::inf() && over_t <= prune_bound(st, r.tmax)) {
        // some candidate did not fit the list and may still matter: another pass
#pragma unroll
        for (int i = 0; i < kCap; ++i) {
          ct[i] = Num<float>::inf();
          ce[i] = 0.f;
          cp[i] = 0x7fffffff;
        }
        over_t = Num<float>::inf();
        if (STATS) ++cnt.passes;
        cull_pass<STATS, false>(r, true, I.n_clusters, hot, staged ? sCl : I.clusters, staged ? sOrd : I.order,
                                       last_t, last_p, ct, ce, cp, over_t, cnt);
        continue;
      }
      finish_ray<NI, STATS, true>(L, I, it, ray, true, false, r, aux, st, con, lane, err, cnt, n_flag);
      state = kNeedRay;
    }
    if (__all_sync(0xffffffffu, state == kDone)) break;
    if (state == kDescending && !descent_step<float, CertState, STATS, BLOCK>(ds, sStack, tab, st, &con, err, cnt))
      state = kBetween;
  }
  if (STATS) flush_stats(L.stats, cnt, 0u, n_flag);
  if (err) atomicOr(L.err, err);
}

// ------------------------------------------------------------- FP64 pass

// Lexicographic minimum of (t, part, voxel) across the warp (every lane
// returns it).
__device__ __forceinline__ void warp_min(ExactState &s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ExactState x;
    x.t = __shfl_xor_sync(0xffffffffu, s.t, o);
    x.part = __shfl_xor_sync(0xffffffffu, s.part, o);
    x.vox = __shfl_xor_sync(0xffffffffu, s.vox, o);
    offer(s, x.t, x.part, x.vox);
  }
}

__device__ __forceinline__ void write_fixed(const TraceItem &I, unsigned long long ray, const ExactState &st,
                                            uint32_t why) {
  uint4 hv;
  hv.x = __float_as_uint((float)st.t);
  hv.y = st.part;
  hv.z = (uint32_t)(st.vox & 0xFFFFFFFFull);
  hv.w = (uint32_t)(st.vox >> 32);
  I.hits[ray] = hv;
  if (I.ray_flags) I.ray_flags[ray] = why | SVO_RAY_FIXED;
}

// Lexicographic minimum of (t, part, voxel) across each aligned group of 8
// lanes (every lane of the group returns it).
__device__ __forceinline__ void group_min8(ExactState &s) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) {
    ExactState x;
    x.t = __shfl_xor_sync(0xffffffffu, s.t, o);
    x.part = __shfl_xor_sync(0xffffffffu, s.part, o);
    x.vox = __shfl_xor_sync(0xffffffffu, s.vox, o);
    offer(s, x.t, x.part, x.vox);
  }
}

// The FP64 pass for a flagged ray without a contender list (the list
// overflowed), called by the whole warp (i: its list index, e: its entry).
// The warp re-traces the ray, lane q taking parts q, q + 32, ...; each lane
// keeps the exact minimum over its parts, the warp's best hit so far prunes
// whole parts, and a warp reduction gives the overall minimum.  The segment
// ends at the FP32 pass's certain upper bound of the winner's t where one was
// stored: the winner (and every leaf tied with it) starts no later, so no
// candidate is lost and the leaves beyond it are never tested in FP64.
template <int NI>
__device__ void overflow_retrace(const TraceLaunchT<NI> &L, unsigned long long i, unsigned long long e,
                                 const Tables *tab, unsigned int &err, Counters &cnt) {
  const int lane = threadIdx.x & 31;
  const uint32_t why = ((e >> 47) & 1ull) ? SVO_RAY_T_REFINED : SVO_RAY_UNCERTAIN;
  const int it = (int)((e >> kRayBits) & 0x7Fu);
  const unsigned long long ray = e & ((1ull << kRayBits) - 1ull);
  const TraceItem &I = L.items[it];
  const float4 o = I.rays[2 * ray], d = I.rays[2 * ray + 1];
  const uint32_t off = L.fix_off[i];
  const float tcap = off != kNoCand ? __uint_as_float(L.fix_cand[off].w) : Num<float>::inf();
  RayW r;
  r.ox = o.x;
  r.oy = o.y;
  r.oz = o.z;
  r.tmin = o.w;
  r.dx = d.x;
  r.dy = d.y;
  r.dz = d.z;
  r.tmax = fminf(d.w, tcap);
  r.inv_dd = 1.0f / (d.x * d.x + d.y * d.y + d.z * d.z);
  r.inv_len = 0.f;
  r.onorm = 0.f;
  HybridState hs;
  hs.ex.t = Num<double>::inf();
  hs.ex.part = kMissPart;
  hs.ex.vox = kMissVoxel;
  hs.o = o;
  hs.d = make_float4(d.x, d.y, d.z, r.tmax);
  uint4 stk_local[kMaxDepth];
  double best = Num<double>::inf();  // the warp's best hit t after each round
  for (int base = 0; base < I.n_parts; base += 32) {
    const int p = base + lane;
    if (p < I.n_parts) {
      float tin, tref;
      if (part_cull(r, I.hot[p], tin, tref) && !(tin > __double2float_ru(fmin(best, hs.ex.t)))) {
        hs.inv64 = I.inv64 + 12 * p;
        trace_part_f32<false, HybridState, 1>(r, I.hot[p], I.aux[p], tref, (uint32_t)p, tab, 0u, 0, stk_local, hs,
                                              nullptr, err, cnt);
      }
    }
    double bb = hs.ex.t;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) bb = fmin(bb, __shfl_xor_sync(0xffffffffu, bb, off));
    best = bb;
  }
  warp_min(hs.ex);
  if (lane == 0) write_fixed(I, ray, hs.ex, why);
}

// Re-intersects the rays the FP32 pass flagged, in FP64 and without
// certification:
//   * with a contender list (the leaves that may still be the closest hit),
//     lane q of the ray's 8-lane group intersects contender q with the exact
//     closed-box rule and a group reduction keeps the lexicographic minimum
//     of (t, part, voxel);
//   * without one (the contender list overflowed, or the leaf pool was
//     full), the warp re-traces the ray, the parts dealt over the lanes: the
//     FP32 descent with inflated boxes, every leaf reached decided in FP64.
// GB300 issues FP64 at 2 lanes per clock per SM, so spreading a ray's
// contenders over lanes (instead of one lane looping over them) cuts the
// pass's latency by the contender count.  Groups of four list entries are
// dealt round-robin over the warps so that a short list still spreads over
// the whole GPU.
template <int NI>
__global__ void __launch_bounds__(kBlock) k_fix(const __grid_constant__ TraceLaunchT<NI> L) {
  // the rare re-traces read the order tables from global memory (L1/L2), so
  // blocks start without staging them
  const Tables *tab = &g_tables;
  unsigned int err = 0;
  Counters cnt = {0, 0, 0, 0, 0, 0, 0, 0};
  const unsigned long long n = min((unsigned long long)*L.fix_count, L.fix_capacity);
  const int lane = threadIdx.x & 31;
  const unsigned long long n_warps = (unsigned long long)gridDim.x * (blockDim.x / 32);
  const unsigned long long warp = blockIdx.x + (unsigned long long)gridDim.x * (threadIdx.x >> 5);
  // Four list entries per warp, one group of 8 lanes each (at most 16
  // contenders per entry, two per lane): FP64 issues at a few lanes per clock
  // and a warp instruction holds the pipe whatever its active lanes, so
  // packing entries cuts the pipe time per entry.  Entries without contenders
  // are re-traced afterwards by the whole warp, one at a time.
  static_assert(kContenders <= 16, "8-lane groups, two contenders per lane at most");
  const int sub = lane >> 3, sl = lane & 7;
  if (n > 8ull * n_warps) {
    // A long list (more than two rounds of four entries per warp): runs of 32
    // entries per warp.  An entry with one stored leaf (every t refinement)
    // takes one lane, so 32 of them share each FP64 instruction; entries with
    // a contender list go four at a time in 8-lane groups; entries without
    // one get the whole warp.  A short list keeps four entries per warp
    // (below), which spreads it over more warps.
    for (unsigned long long i0 = 32 * warp; i0 < n; i0 += 32 * n_warps) {
      const unsigned long long i = i0 + (unsigned long long)lane;
      const bool have = i < n;
      const unsigned long long e = have ? L.fix_list[i] : 0ull;
      const int nc = (int)(e >> 48);
      if (have && nc == 1) {
        const int it = (int)((e >> kRayBits) & 0x7Fu);
        const unsigned long long ray = e & ((1ull << kRayBits) - 1ull);
        const TraceItem &I = L.items[it];
        const float4 o = I.rays[2 * ray], d = I.rays[2 * ray + 1];
        const uint4 cv = L.fix_cand[L.fix_off[i]];
        const uint32_t p = cv.x;
        const unsigned long long vox = (unsigned long long)cv.y | ((unsigned long long)cv.z << 32);
        ExactState st;
        st.t = Num<double>::inf();
        st.part = kMissPart;
        st.vox = kMissVoxel;
        double tq;
        if (leaf_entry64(I.inv64 + 12 * p, I.aux[p].depth, vox, o, d, tq)) offer(st, tq, p, vox);
        write_fixed(I, ray, st, ((e >> 47) & 1ull) ? SVO_RAY_T_REFINED : SVO_RAY_UNCERTAIN);
      }
      for (unsigned int multi = __ballot_sync(0xffffffffu, have && nc >= 2); multi != 0u;) {
        // the next four such entries, one 8-lane group each
        int src = -1;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const int s = multi ? __ffs(multi) - 1 : -1;
          if (g == sub) src = s;
          if (multi) multi &= multi - 1u;
        }
        const unsigned long long ee = __shfl_sync(0xffffffffu, e, src < 0 ? 0 : src);
        const int ncg = src >= 0 ? (int)(ee >> 48) : 0;
        const int it = (int)((ee >> kRayBits) & 0x7Fu);
        const unsigned long long ray = ee & ((1ull << kRayBits) - 1ull);
        ExactState st;
        st.t = Num<double>::inf();
        st.part = kMissPart;
        st.vox = kMissVoxel;
        if (sl < ncg) {
          const TraceItem &I = L.items[it];
          const float4 o = I.rays[2 * ray], d = I.rays[2 * ray + 1];
          const uint32_t off = L.fix_off[i0 + (unsigned long long)src];
          for (int q = sl; q < ncg; q += 8) {
            const uint4 cv = L.fix_cand[off + q];
            const uint32_t p = cv.x;
            const unsigned long long vox = (unsigned long long)cv.y | ((unsigned long long)cv.z << 32);
            double tq;
            if (leaf_entry64(I.inv64 + 12 * p, I.aux[p].depth, vox, o, d, tq)) offer(st, tq, p, vox);
          }
        }
        group_min8(st);
        if (ncg > 0 && sl == 0)
          write_fixed(L.items[it], ray, st, ((ee >> 47) & 1ull) ? SVO_RAY_T_REFINED : SVO_RAY_UNCERTAIN);
      }
      for (unsigned int pending = __ballot_sync(0xffffffffu, have && nc == 0); pending != 0u; pending &= pending - 1u) {
        const int src = __ffs(pending) - 1;
        overflow_retrace(L, i0 + (unsigned long long)src, __shfl_sync(0xffffffffu, e, src), tab, err, cnt);
      }
    }
  } else
  for (unsigned long long i0 = 4 * warp; i0 < n; i0 += 4 * n_warps) {
    const unsigned long long i = i0 + (unsigned long long)sub;
    const bool have = i < n;
    const unsigned long long e = have ? L.fix_list[i] : 0ull;
    const int nc = (int)(e >> 48);
    {
      // the FP32 pass narrowed the ray to nc contender leaves: lane q of the
      // group takes contenders q and q + 8
      ExactState st;
      st.t = Num<double>::inf();
      st.part = kMissPart;
      st.vox = kMissVoxel;
      const int it = (int)((e >> kRayBits) & 0x7Fu);
      const unsigned long long ray = e & ((1ull << kRayBits) - 1ull);
      if (have && sl < nc) {
        const TraceItem &I = L.items[it];
        const float4 o = I.rays[2 * ray], d = I.rays[2 * ray + 1];
        const uint32_t off = L.fix_off[i];
        for (int q = sl; q < nc; q += 8) {
          const uint4 cv = L.fix_cand[off + q];
          const uint32_t p = cv.x;
          const unsigned long long vox = (unsigned long long)cv.y | ((unsigned long long)cv.z << 32);
          double tq;
          if (leaf_entry64(I.inv64 + 12 * p, I.aux[p].depth, vox, o, d, tq)) offer(st, tq, p, vox);
        }
      }
      group_min8(st);
      if (have && nc > 0 && sl == 0)
        write_fixed(L.items[it], ray, st, ((e >> 47) & 1ull) ? SVO_RAY_T_REFINED : SVO_RAY_UNCERTAIN);
    }
    unsigned int pending = __ballot_sync(0xffffffffu, have && nc == 0 && sl == 0);
    while (pending) {
      const int src = __ffs(pending) - 1;
      pending &= pending - 1u;
      const unsigned long long ie = i0 + (unsigned long long)(src >> 3);
      const unsigned long long ee = __shfl_sync(0xffffffffu, e, src);
      overflow_retrace(L, ie, ee, tab, err, cnt);
    }
  }
  // count fixed rays once per launch
  if (L.stats && blockIdx.x == 0 && threadIdx.x == 0 && (L.flags & SVO_TRACE_STATS)) atomicAdd(&L.stats->fixed, n);
  if (err) atomicOr(L.err, err);
}

size_t trace_smem_bytes(int stack_levels, int parts, int clusters, int block, int mbox_words, int top_nodes) {
  return kTablesBytes + (size_t)stack_levels * block * sizeof(uint4) + parts * (sizeof(PartHot) + sizeof(PartAux)) +
         clusters * sizeof(Cluster) + (parts + (parts & 1)) * sizeof(int32_t) + (size_t)top_nodes * sizeof(uint2) +
         (size_t)mbox_words * block * sizeof(uint32_t);
}

// Resident blocks per SM of a trace kernel at a dynamic shared-memory size.
// The attribute that admits the size and the occupancy are host calls of a
// few microseconds each, so they are made once per (device, kernel, size); the
// attribute only ever grows, so a size admitted once stays admitted.
struct OccEntry {
  const void *fn;
  int dev;
  size_t smem;
  int per_sm;
};
struct AttrEntry {
  const void *fn;
  int dev;
  size_t smem_max;
};
std::mutex g_occ_mu;
std::vector<OccEntry> g_occ;
std::vector<AttrEntry> g_attr;

template <typename K>
cudaError_t blocks_per_sm(K kern, int block, size_t smem, int &per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const void *fn = reinterpret_cast<const void *>(kern);
  std::lock_guard<std::mutex> g(g_occ_mu);
  for (const OccEntry &x : g_occ)
    if (x.fn == fn && x.dev == dev && x.smem == smem) {
      per_sm = x.per_sm;
      return cudaSuccess;
    }
  AttrEntry *a = nullptr;
  for (AttrEntry &x : g_attr)
    if (x.fn == fn && x.dev == dev) a = &x;
  if (!a || a->smem_max < smem) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (a)
      a->smem_max = smem;
    else
      g_attr.push_back({fn, dev, smem});
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, block, smem);
  if (e != cudaSuccess) return e;
  g_occ.push_back({fn, dev, smem, per_sm});
  return cudaSuccess;
}

template <int NI, int BLOCK>
cudaError_t launch_trace_b(const TraceLaunchT<NI> &L, int n_sm, cudaStream_t stream) {
  const bool stats = (L.flags & SVO_TRACE_STATS) && L.stats;
  const bool reuse = (L.flags & SVO_TRACE_REUSE) != 0;
  bool walk = (L.flags & SVO_TRACE_GRID) != 0 && !reuse;
  if (walk) {
    bool any = false;
    for (int i = 0; i < L.n_items; ++i) any = any || L.items[i].grid != nullptr;
    walk = any;
  }
  if (L.flags & SVO_TRACE_WAVEFRONT) {
    // the culling launch, then the descent launch over the queued rays (the
    // host has checked CULL | SORT without REUSE or GRID)
    const int parts = L.one_scene ? L.items[0].n_parts : 0, clusters = L.one_scene ? L.items[0].n_clusters : 0;
    const size_t csmem = (size_t)(BLOCK / 32) * kPackRing * sizeof(int2) +
                         (size_t)parts * (sizeof(PartHot) + sizeof(int32_t)) + (size_t)clusters * sizeof(Cluster);
    auto ck = stats ? k_cull<NI, true, BLOCK> : k_cull<NI, false, BLOCK>;
    int per_sm = 0;
    cudaError_t e = blocks_per_sm(ck, BLOCK, csmem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    unsigned long long grid = (unsigned long long)n_sm * per_sm;
    const unsigned long long need = (L.n_tiles + BLOCK / 32 - 1) / (BLOCK / 32);
    if (grid > need) grid = need;
    if (grid == 0) return cudaSuccess;
    ck<<<(unsigned int)grid, BLOCK, csmem, stream>>>(L);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the number of queued rays is known on the device only: a full persistent grid
    const size_t smem = trace_smem_bytes(L.stack_levels, parts, clusters, BLOCK, 0, 0);
    auto kq = stats ? k_descend<NI, true, BLOCK> : k_descend<NI, false, BLOCK>;
    e = blocks_per_sm(kq, BLOCK, smem, per_sm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    kq<<<(unsigned int)(n_sm * per_sm), BLOCK, smem, stream>>>(L);
    return cudaGetLastError();
  }
  // the staged top levels only in the common kernel (counting, reuse and grid traces give the same
  // results without them)
  const bool top = L.one_scene && L.top_nodes > 0 && !stats && !reuse && !walk;
  const size_t smem = trace_smem_bytes(L.stack_levels, L.one_scene ? L.items[0].n_parts : 0,
                                       L.one_scene ? L.items[0].n_clusters : 0, BLOCK, walk ? L.mbox_words : 0,
                                       top ? L.top_nodes : 0);
  auto kern = walk ? (stats ? k_trace<NI, true, BLOCK, false, true> : k_trace<NI, false, BLOCK, false, true>)
              : stats ? (reuse ? k_trace<NI, true, BLOCK, true, false> : k_trace<NI, true, BLOCK, false, false>)
              : reuse ? k_trace<NI, false, BLOCK, true, false>
              : top   ? k_trace<NI, false, BLOCK, false, false, true>
                      : k_trace<NI, false, BLOCK, false, false>;
  int per_sm = 0;
  const cudaError_t e = blocks_per_sm(kern, BLOCK, smem, per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  // one warp per tile: no more blocks than the tiles can keep busy
  unsigned long long grid = (unsigned long long)n_sm * per_sm;
  const unsigned long long need = (L.n_tiles + BLOCK / 32 - 1) / (BLOCK / 32);
  if (grid > need) grid = need;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned int)grid, BLOCK, smem, stream>>>(L);
  return cudaGetLastError();
}

template <int NI>
cudaError_t launch_trace_t(const TraceLaunchT<NI> &L, int n_sm, cudaStream_t stream) {
  if (L.block == 64) return launch_trace_b<NI, 64>(L, n_sm, stream);
  if (L.block == 256) return launch_trace_b<NI, 256>(L, n_sm, stream);
  return launch_trace_b<NI, 128>(L, n_sm, stream);
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
  dst.fix_cand = src.fix_cand;
  dst.cand_capacity = src.cand_capacity;
  dst.cand_count = src.cand_count;
  dst.fix_off = src.fix_off;
  bool one = true;
  for (int i = 1; i < src.n_items && i < NI; ++i) one = one && src.items[i].hot == src.items[0].hot;
  dst.one_scene = one && src.items[0].n_parts <= kSmemParts ? 1 : 0;
  int lv = 1;
  for (int i = 0; i < src.n_items && i < NI; ++i) lv = src.items[i].max_depth - 1 > lv ? src.items[i].max_depth - 1 : lv;
  dst.stack_levels = lv;
  int mp = 0;
  for (int i = 0; i < src.n_items && i < NI; ++i) mp = src.items[i].n_parts > mp ? src.items[i].n_parts : mp;
  dst.mbox_words = (mp + 31) / 32;
  dst.stats = src.stats;
  dst.err = src.err;
  dst.block = src.block;
  dst.rays_per_lane = src.rays_per_lane < 1 ? 1 : src.rays_per_lane;
  dst.top = src.top;
  dst.top_nodes = (dst.one_scene && src.top) ? src.top_nodes : 0;
  dst.top_levels = dst.top_nodes > 0 ? src.top_levels : 0;
  dst.queue = src.queue;
  dst.queue_count = src.queue_count;
  dst.queue_tile = src.queue_tile;
}

}  // namespace

cudaError_t init_trace_tables(cudaStream_t stream) {
  k_init_tables<<<1, 256, 0, stream>>>();
  return cudaGetLastError();
}

// The kernel parameter block of a batch (about 16 KB): one per host thread,
// allocated on its first batch, so it stays off the caller's stack and off
// the heap of later calls.
TraceLaunchT<kMaxBatchItems> &batch_params() {
  thread_local std::unique_ptr<TraceLaunchT<kMaxBatchItems>> p;
  if (!p) p.reset(new TraceLaunchT<kMaxBatchItems>());
  return *p;
}

cudaError_t launch_trace(const TraceLaunch &L, int n_sm, cudaStream_t stream) {
  if (L.n_items <= 1) {
    TraceLaunchT<1> l1;
    fill_launch(L, l1);
    return launch_trace_t(l1, n_sm, stream);
  }
  TraceLaunchT<kMaxBatchItems> &p = batch_params();
  fill_launch(L, p);
  return launch_trace_t(p, n_sm, stream);
}

cudaError_t launch_fix(const TraceLaunch &L, int n_sm, cudaStream_t stream) {
  if (L.n_items <= 1) {
    TraceLaunchT<1> l1;
    fill_launch(L, l1);
    return launch_fix_t(l1, n_sm, stream);
  }
  TraceLaunchT<kMaxBatchItems> &p = batch_params();
  fill_launch(L, p);
  return launch_fix_t(p, n_sm, stream);
}

}  // namespace svo
