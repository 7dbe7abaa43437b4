// k_grid.cu -- the scene-level grid over the part spheres (the larger
// structure the paper suggests for scenes of many parts, Sec. V-E).
//
// Built on demand: every refit marks a scene's grid stale, and a trace with
// SVO_TRACE_GRID first launches k_build_grid, whose block for that scene
// rebuilds the grid only if it is stale.  Scenes never traced with the grid
// pay one store per refit.  The staleness lives on the device, so the rule
// holds for any mix of eager launches and CUDA-graph replays.
//
// One block per scene: the spheres' box (block reduction), per-cell counts
// (shared-memory atomics), an exclusive scan, the fill, and a sort of each
// cell's list into increasing part order (results do not depend on the order
// of the atomics).
#include <cuda_runtime.h>

#include <cfloat>

#include "svo_internal.h"

namespace svo {

namespace {

constexpr int kGridThreads = 256;
constexpr float kU32 = 5.9604644775390625e-8f;  // 2^-24

// Cell range of a sphere box along one axis: every cell within 2^-10 cells of
// the box (the walk's rounding allowance), plus 2^-12 cells for the rounding
// of the index itself (at most 2^-13 cells while the grid is valid).
__device__ __forceinline__ void cell_range(float c, float r, float lo, float inv, int G, int &i0, int &i1) {
  constexpr float kPad = 9.765625e-4f + 2.44140625e-4f;  // 2^-10 + 2^-12
  const float f0 = (__fsub_rd(c, r) - lo) * inv - kPad, f1 = (__fadd_ru(c, r) - lo) * inv + kPad;
  i0 = (int)floorf(fmaxf(f0, 0.f));
  i1 = (int)floorf(fminf(f1, (float)G - 0.5f));
  i0 = i0 < 0 ? 0 : (i0 > G - 1 ? G - 1 : i0);
  i1 = i1 < i0 ? i0 : (i1 > G - 1 ? G - 1 : i1);
}

__global__ void __launch_bounds__(kGridThreads) k_build_grid(const __grid_constant__ GridLaunch L) {
  const GridJob job = L.jobs[blockIdx.x];
  SceneGrid *grid = job.grid;
  if (grid->stale == 0) return;  // block-uniform
  const int tid = threadIdx.x, P = job.n_parts, G = grid->G, NC3 = G * G * G;
  int32_t *cell_start = grid->cell_start;
  int32_t *cell_parts = grid->cell_parts;
  extern __shared__ __align__(16) unsigned char smem[];
  float *red = reinterpret_cast<float *>(smem);                          // 6 x threads
  int32_t *gcnt = reinterpret_cast<int32_t *>(red + 6 * kGridThreads);  // G^3 + 1
  __shared__ int wsum[kGridThreads / 32];

  // the enabled spheres' box, rounded outward
  float bl[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, bh[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
  for (int i = tid; i < P; i += kGridThreads) {
    const float4 s = job.hot[i].sphere;
    if (s.w < 0.f) continue;
    bl[0] = fminf(bl[0], __fsub_rd(s.x, s.w));
    bl[1] = fminf(bl[1], __fsub_rd(s.y, s.w));
    bl[2] = fminf(bl[2], __fsub_rd(s.z, s.w));
    bh[0] = fmaxf(bh[0], __fadd_ru(s.x, s.w));
    bh[1] = fmaxf(bh[1], __fadd_ru(s.y, s.w));
    bh[2] = fmaxf(bh[2], __fadd_ru(s.z, s.w));
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    red[k * kGridThreads + tid] = bl[k];
    red[(3 + k) * kGridThreads + tid] = bh[k];
  }
  __syncthreads();
  for (int w = kGridThreads / 2; w > 0; w >>= 1) {
    if (tid < w) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float *lo = red + k * kGridThreads, *hi = red + (3 + k) * kGridThreads;
        lo[tid] = fminf(lo[tid], lo[tid + w]);
        hi[tid] = fmaxf(hi[tid], hi[tid + w]);
      }
    }
    __syncthreads();
  }
  // grid box: the spheres' box widened by m = 2^-10 of a cell on each side,
  // so that every sphere box lies at least m inside it
  float lo[3], cs[3], inv[3];
  bool any = true, exact = true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float l0 = red[k * kGridThreads], h0 = red[(3 + k) * kGridThreads];
    any = any && h0 >= l0;
    const float m = fmaxf(__fmul_ru(__fdiv_ru(__fsub_ru(h0, l0), (float)G), 9.765625e-4f), 1e-30f);
    lo[k] = __fsub_rd(l0, m);
    cs[k] = fmaxf(__fdiv_ru(__fsub_ru(__fadd_ru(h0, m), lo[k]), (float)G), 1e-30f);  // lo + G cs covers h0 + m
    inv[k] = 1.0f / cs[k];
    // the walk's and the lists' rounding stays below 2^-13 cells only for a
    // grid not too far from the origin relative to its cell size
    exact = exact && 16.0f * kU32 * (fabsf(lo[k]) + (float)G * cs[k]) <= cs[k] * 2.44140625e-4f;
  }
  any = any && exact;
  for (int c = tid; c <= NC3; c += kGridThreads) gcnt[c] = 0;
  __syncthreads();
  for (int i = tid; i < P && any; i += kGridThreads) {
    const float4 s = job.hot[i].sphere;
    if (s.w < 0.f) continue;
    int x0, x1, y0, y1, z0, z1;
    cell_range(s.x, s.w, lo[0], inv[0], G, x0, x1);
    cell_range(s.y, s.w, lo[1], inv[1], G, y0, y1);
    cell_range(s.z, s.w, lo[2], inv[2], G, z0, z1);
    for (int z = z0; z <= z1; ++z)
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) atomicAdd(&gcnt[x + G * (y + G * z)], 1);
  }
  __syncthreads();
  {  // exclusive scan of the counts: per-thread chunks, then warp and block offsets
    const int chunk = (NC3 + kGridThreads - 1) / kGridThreads;
    const int c0 = min(tid * chunk, NC3), c1 = min(c0 + chunk, NC3);
    int sum = 0;
    for (int c = c0; c < c1; ++c) sum += gcnt[c];
    const int lane = tid & 31, warp = tid >> 5;
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < warp; ++w) base += wsum[w];
    int run = base + incl - sum;
    for (int c = c0; c < c1; ++c) {
      const int n = gcnt[c];
      gcnt[c] = run;
      cell_start[c] = run;
      run += n;
    }
    if (tid == kGridThreads - 1) {
      gcnt[NC3] = run;
      cell_start[NC3] = run;
    }
  }
  __syncthreads();
  const bool fits = any && gcnt[NC3] <= grid->cap;
  for (int i = tid; i < P && fits; i += kGridThreads) {
    const float4 s = job.hot[i].sphere;
    if (s.w < 0.f) continue;
    int x0, x1, y0, y1, z0, z1;
    cell_range(s.x, s.w, lo[0], inv[0], G, x0, x1);
    cell_range(s.y, s.w, lo[1], inv[1], G, y0, y1);
    cell_range(s.z, s.w, lo[2], inv[2], G, z0, z1);
    for (int z = z0; z <= z1; ++z)
      for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) cell_parts[atomicAdd(&gcnt[x + G * (y + G * z)], 1)] = i;
  }
  __syncthreads();
  // deterministic order inside each cell: increasing part id
  for (int c = tid; c < NC3 && fits; c += kGridThreads) {
    const int b = cell_start[c], e = cell_start[c + 1];
    for (int i = b + 1; i < e; ++i) {
      const int v = cell_parts[i];
      int j = i - 1;
      while (j >= b && cell_parts[j] > v) {
        cell_parts[j + 1] = cell_parts[j];
        --j;
      }
      cell_parts[j + 1] = v;
    }
  }
  if (tid == 0) {
    for (int k = 0; k < 3; ++k) {
      grid->lo[k] = lo[k];
      grid->cs[k] = cs[k];
      grid->inv_cs[k] = inv[k];
    }
    grid->valid = fits ? 1 : 0;
    grid->stale = 0;
  }
}

}  // namespace

size_t grid_smem_bytes(int G) { return (6 * kGridThreads + (size_t)G * G * G + 1) * sizeof(float); }

cudaError_t launch_grid(const GridLaunch &L, cudaStream_t stream) {
  if (L.n_jobs <= 0) return cudaSuccess;
  int gmax = 0;
  for (int i = 0; i < L.n_jobs; ++i) gmax = L.jobs[i].G > gmax ? L.jobs[i].G : gmax;
  const size_t smem = grid_smem_bytes(gmax);
  cudaError_t e = cudaFuncSetAttribute(k_build_grid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_build_grid<<<(unsigned int)L.n_jobs, kGridThreads, smem, stream>>>(L);
  return cudaGetLastError();
}

}  // namespace svo
