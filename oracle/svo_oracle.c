/*
 * svo_oracle.c -- plain, slow, FP64 CPU reference for ray casting against a
 * scene of animated sparse voxel octrees (Espe, Gjermundnes, Hendseth,
 * "Efficient Animation of Sparse Voxel Octrees for Real-Time Ray Tracing").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: it exists so that tests, the smoke check and the benchmark's
 * CPU-baseline leg can check the CUDA library against an independent
 * definition.  It shares no code, header, table or helper with the library.
 *
 * What it computes (the definition the GPU path must reproduce):
 *
 *   Scene (Sec. III): every part p is a static SVO (an asset) with a pose.
 *   The pose of a part relative to its parent is an affine map L_p; the world
 *   pose is W_p = W_parent(p) o L_p (the transform tree is a reading of the
 *   paper's one-transform-per-SVO model; a root part has W_p = L_p).
 *
 *   Ray (Eq. 1): R(t) = r_o + t r_d, restricted to tmin <= t <= tmax.
 *
 *   Ray to local frame (Eq. 2-3): instead of moving the voxels the ray is moved
 *   by the inverse pose, r_o' = W^-1 r_o, r_d' = W^-1 r_d (for a rigid pose
 *   W^-1 is the transposed rotation and the negated translation).  The
 *   direction is not renormalised, so t means the same point in world and
 *   local space and hits of different parts compare directly.
 *
 *   Asset local frame: the unit cube [0,1]^3 with the octree origin at a
 *   corner (Fig. 2); a leaf cell (x,y,z) of a depth-D asset is the closed box
 *   [x,y,z]/2^D .. [x+1,y+1,z+1]/2^D.  Its voxel id is x | y<<D | z<<2D.
 *
 *   Candidate: a leaf whose closed box meets the ray segment; its t is the
 *   entry parameter max(slab entry, tmin).  The closest hit (Sec. IV-B) is the
 *   lexicographic minimum of (t, part, voxel) over all candidates of all
 *   parts; a miss is t = +inf, part = 0xFFFFFFFF, voxel = UINT64_MAX.
 *   "second" is the smallest t among the other candidates (used to recognise
 *   near ties).
 *
 * Two independent evaluations of that definition are provided:
 *   mode 0  brute force: every leaf of every part is slab-tested;
 *   mode 1  recursive descent over the oracle's own octree (the sorted list of
 *           the leaves' Morton codes; a node of level l is the run of codes
 *           that share their top 3l bits).  A child is entered only if its
 *           closed box meets [tmin, min(tmax, second)] along the ray.
 * Neither culls by bounding spheres: culling and depth sorting (Sec. IV-A/B)
 * only save work and must not change this result.
 *
 * Also here: the per-frame pose pipeline in FP64 (compose, invert, part
 * bounding sphere) and the ray-sphere test of Eq. 4 in its general form, so
 * tests can pin them and compare the library's per-frame outputs.
 */
#include <math.h>
#include <pthread.h>
#include <stdatomic.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_MISS_PART 0xFFFFFFFFu
#define ORACLE_MISS_VOXEL 0xFFFFFFFFFFFFFFFFull

/* ------------------------------------------------------------ poses (Eq. 3) */

/* 3x4 row-major affine [A | b]: y = A x + b. */
static void affine_mul(const double *p, const double *q, double *out) {
  /* out = p o q : out.A = p.A q.A, out.b = p.A q.b + p.b */
  double r[12];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += p[i * 4 + k] * q[k * 4 + j];
      r[i * 4 + j] = s;
    }
    double s = p[i * 4 + 3];
    for (int k = 0; k < 3; ++k) s += p[i * 4 + k] * q[k * 4 + 3];
    r[i * 4 + 3] = s;
  }
  memcpy(out, r, sizeof(r));
}

/* World pose of every part: W_i = W_parent(i) o L_i, parents first.
 * Returns 0, or -1 if some parent index is not smaller than its child's. */
int oracle_compose(int n_parts, const int32_t *parent, const double *local, double *world) {
  for (int i = 0; i < n_parts; ++i) {
    int p = parent[i];
    if (p >= i) return -1;
    if (p < 0)
      memcpy(world + 12 * i, local + 12 * i, 12 * sizeof(double));
    else
      affine_mul(world + 12 * p, local + 12 * i, world + 12 * i);
  }
  return 0;
}

/* Inverse affine: A^-1 = adj(A)/det(A), b' = -A^-1 b.  Returns 0, -1 if singular. */
int oracle_invert(int n_parts, const double *world, double *inv) {
  for (int p = 0; p < n_parts; ++p) {
    const double *m = world + 12 * p;
    double a = m[0], b = m[1], c = m[2];
    double d = m[4], e = m[5], f = m[6];
    double g = m[8], h = m[9], k = m[10];
    double c00 = e * k - f * h, c01 = f * g - d * k, c02 = d * h - e * g;
    double det = a * c00 + b * c01 + c * c02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return -1;
    double adj[9] = {
        c00, c * h - b * k, b * f - c * e,
        c01, a * k - c * g, c * d - a * f,
        c02, b * g - a * h, a * e - b * d,
    };
    double *o = inv + 12 * p;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) o[i * 4 + j] = adj[i * 3 + j] / det;
    for (int i = 0; i < 3; ++i)
      o[i * 4 + 3] = -(o[i * 4 + 0] * m[3] + o[i * 4 + 1] * m[7] + o[i * 4 + 2] * m[11]);
  }
  return 0;
}

/* Bounding sphere of a part (Sec. IV-A) around the local box [lo, hi] of
 * its content (box6 = lo[3], hi[3] per part; NULL = the unit cube):
 * centre = image of the box centre, radius = largest distance from it to the
 * image of a box corner.  Any box that holds every occupied leaf gives a
 * sphere that culls no hit. */
void oracle_part_sphere(int n_parts, const double *world, const double *box6, double *sphere4) {
  for (int p = 0; p < n_parts; ++p) {
    const double *m = world + 12 * p;
    const double lo[3] = {box6 ? box6[6 * p] : 0.0, box6 ? box6[6 * p + 1] : 0.0, box6 ? box6[6 * p + 2] : 0.0};
    const double hi[3] = {box6 ? box6[6 * p + 3] : 1.0, box6 ? box6[6 * p + 4] : 1.0, box6 ? box6[6 * p + 5] : 1.0};
    double mid[3], c[3], r2 = 0.0;
    for (int i = 0; i < 3; ++i) mid[i] = 0.5 * (lo[i] + hi[i]);
    for (int i = 0; i < 3; ++i) c[i] = m[i * 4] * mid[0] + m[i * 4 + 1] * mid[1] + m[i * 4 + 2] * mid[2] + m[i * 4 + 3];
    for (int corner = 0; corner < 8; ++corner) {
      double q[3] = {(corner & 1) ? hi[0] : lo[0], ((corner >> 1) & 1) ? hi[1] : lo[1],
                     ((corner >> 2) & 1) ? hi[2] : lo[2]};
      double s = 0.0;
      for (int i = 0; i < 3; ++i) {
        double v = m[i * 4] * q[0] + m[i * 4 + 1] * q[1] + m[i * 4 + 2] * q[2] + m[i * 4 + 3] - c[i];
        s += v * v;
      }
      if (s > r2) r2 = s;
    }
    sphere4[4 * p + 0] = c[0];
    sphere4[4 * p + 1] = c[1];
    sphere4[4 * p + 2] = c[2];
    sphere4[4 * p + 3] = sqrt(r2);
  }
}

/* Ray-sphere test of Eq. 4 for a direction of any length: l = s_c - r_o,
 * squared distance from the centre to the line d^2 = l.l - (l.r_d)^2 / |r_d|^2.
 * The sphere is hit iff d^2 <= r^2 and its far intersection lies at t >= 0
 * (the prose case of a ray pointing away from the SVO).  On a hit, *t_in and
 * *t_out are the entry and exit parameters (t_in clamped below at 0). */
int oracle_ray_sphere(const double *o, const double *d, const double *sphere4, double *t_in, double *t_out) {
  double l[3] = {sphere4[0] - o[0], sphere4[1] - o[1], sphere4[2] - o[2]};
  double ll = l[0] * l[0] + l[1] * l[1] + l[2] * l[2];
  double ld = l[0] * d[0] + l[1] * d[1] + l[2] * d[2];
  double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  double r = sphere4[3];
  if (!(dd > 0.0)) return 0;
  double dist2 = ll - ld * ld / dd;
  if (dist2 > r * r) return 0;
  double half = sqrt((r * r - dist2) / dd);
  double tc = ld / dd;
  if (tc + half < 0.0) return 0;
  *t_in = tc - half > 0.0 ? tc - half : 0.0;
  *t_out = tc + half;
  return 1;
}

/* ---------------------------------------------------------- the oracle octree */

typedef struct {
  int depth;
  int64_t n;
  uint64_t *morton; /* sorted Morton codes (x in bit 3k, y in 3k+1, z in 3k+2) */
} oracle_asset;

static uint64_t morton_of(uint64_t x, uint64_t y, uint64_t z, int depth) {
  uint64_t m = 0;
  for (int k = 0; k < depth; ++k) {
    m |= ((x >> k) & 1ull) << (3 * k);
    m |= ((y >> k) & 1ull) << (3 * k + 1);
    m |= ((z >> k) & 1ull) << (3 * k + 2);
  }
  return m;
}

static void cell_of_morton(uint64_t m, int levels, uint64_t *x, uint64_t *y, uint64_t *z) {
  uint64_t a = 0, b = 0, c = 0;
  for (int k = 0; k < levels; ++k) {
    a |= ((m >> (3 * k)) & 1ull) << k;
    b |= ((m >> (3 * k + 1)) & 1ull) << k;
    c |= ((m >> (3 * k + 2)) & 1ull) << k;
  }
  *x = a;
  *y = b;
  *z = c;
}

static int cmp_u64(const void *a, const void *b) {
  uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Build the oracle's octree from a leaf list (voxel ids x | y<<D | z<<2D).
 * Duplicates are removed.  Returns NULL on bad input. */
void *oracle_asset_new(int depth, int64_t n, const uint64_t *leaf_ids) {
  if (depth < 1 || depth > 21 || n < 0) return NULL;
  oracle_asset *a = (oracle_asset *)calloc(1, sizeof(oracle_asset));
  if (!a) return NULL;
  a->depth = depth;
  a->morton = (uint64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint64_t));
  if (!a->morton) {
    free(a);
    return NULL;
  }
  uint64_t mask = (1ull << depth) - 1ull;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t v = leaf_ids[i];
    a->morton[i] = morton_of(v & mask, (v >> depth) & mask, (v >> (2 * depth)) & mask, depth);
  }
  qsort(a->morton, (size_t)n, sizeof(uint64_t), cmp_u64);
  int64_t w = 0;
  for (int64_t i = 0; i < n; ++i)
    if (w == 0 || a->morton[i] != a->morton[w - 1]) a->morton[w++] = a->morton[i];
  a->n = w;
  return a;
}

void oracle_asset_free(void *p) {
  oracle_asset *a = (oracle_asset *)p;
  if (!a) return;
  free(a->morton);
  free(a);
}

int64_t oracle_asset_leaves(const void *p) { return ((const oracle_asset *)p)->n; }

/* --------------------------------------------------------------- slab test */

/* Closed box [lo, hi] against the ray segment t in [t_lo, t_hi].
 * A zero direction component keeps the slab unbounded if the origin lies in
 * it, and empties it otherwise.  Returns 1 and the clamped entry / exit. */
static int slab(const double o[3], const double d[3], const double lo[3], const double hi[3], double t_lo,
                double t_hi, double *t0, double *t1) {
  double a = t_lo, b = t_hi;
  for (int i = 0; i < 3; ++i) {
    if (d[i] == 0.0) {
      if (o[i] < lo[i] || o[i] > hi[i]) return 0;
      continue;
    }
    double ta = (lo[i] - o[i]) / d[i];
    double tb = (hi[i] - o[i]) / d[i];
    if (ta > tb) {
      double s = ta;
      ta = tb;
      tb = s;
    }
    if (ta > a) a = ta;
    if (tb < b) b = tb;
  }
  if (!(a <= b)) return 0;
  *t0 = a;
  *t1 = b;
  return 1;
}

int oracle_slab(const double *o, const double *d, const double *lo, const double *hi, double t_lo, double t_hi,
                double *t01) {
  return slab(o, d, lo, hi, t_lo, t_hi, &t01[0], &t01[1]);
}

/* ------------------------------------------------------------- trace state */

typedef struct {
  double t, second;
  uint32_t part;
  uint64_t voxel;
} best_hit;

static void best_init(best_hit *b) {
  b->t = INFINITY;
  b->second = INFINITY;
  b->part = ORACLE_MISS_PART;
  b->voxel = ORACLE_MISS_VOXEL;
}

/* Offer one candidate (t, part, voxel); each (part, voxel) is offered once. */
static void best_offer(best_hit *b, double t, uint32_t part, uint64_t voxel) {
  int better = t < b->t || (t == b->t && (part < b->part || (part == b->part && voxel < b->voxel)));
  if (better) {
    if (b->t < b->second) b->second = b->t;
    b->t = t;
    b->part = part;
    b->voxel = voxel;
  } else if (t < b->second) {
    b->second = t;
  }
}

static uint64_t voxel_id(uint64_t x, uint64_t y, uint64_t z, int depth) {
  return x | (y << depth) | (z << (2 * depth));
}

/* mode 0: every leaf of the part. */
static void trace_brute(const oracle_asset *a, uint32_t part, const double o[3], const double d[3], double tmin,
                        double tmax, best_hit *b) {
  double s = ldexp(1.0, -a->depth);
  for (int64_t i = 0; i < a->n; ++i) {
    uint64_t x, y, z;
    cell_of_morton(a->morton[i], a->depth, &x, &y, &z);
    double lo[3] = {x * s, y * s, z * s};
    double hi[3] = {(x + 1) * s, (y + 1) * s, (z + 1) * s};
    double t0, t1;
    if (slab(o, d, lo, hi, tmin, tmax, &t0, &t1)) best_offer(b, t0, part, voxel_id(x, y, z, a->depth));
  }
}

/* First index in [lo, hi) whose code is >= key. */
static int64_t lower_bound(const uint64_t *v, int64_t lo, int64_t hi, uint64_t key) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (v[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

typedef struct {
  const oracle_asset *a;
  uint32_t part;
  double o[3], d[3], tmin, tmax;
  best_hit *b;
} descent_ctx;

/* Node of level `level` = codes in [lo, hi) sharing the prefix `prefix` (the
 * code's top 3*level bits).  Its box is cell (x,y,z) of the level-`level` grid. */
static void descend(const descent_ctx *c, int level, uint64_t prefix, int64_t lo, int64_t hi) {
  const oracle_asset *a = c->a;
  uint64_t x, y, z;
  cell_of_morton(prefix, level, &x, &y, &z);
  if (level == a->depth) {
    double s = ldexp(1.0, -a->depth);
    double blo[3] = {x * s, y * s, z * s};
    double bhi[3] = {(x + 1) * s, (y + 1) * s, (z + 1) * s};
    double t0, t1;
    if (slab(c->o, c->d, blo, bhi, c->tmin, c->tmax, &t0, &t1)) best_offer(c->b, t0, c->part, voxel_id(x, y, z, a->depth));
    return;
  }
  /* children: the 8 runs split by the next 3-bit digit; visit them nearest first */
  int shift = 3 * (a->depth - level - 1);
  int64_t start[9];
  for (int k = 0; k < 8; ++k) start[k] = lower_bound(a->morton, lo, hi, ((prefix << 3) | (uint64_t)k) << shift);
  start[8] = hi;
  double cs = ldexp(1.0, -(level + 1));
  int order[8], n_ord = 0;
  double entry[8];
  for (int k = 0; k < 8; ++k) {
    if (start[k] == start[k + 1]) continue;
    uint64_t cx = 2 * x + (k & 1), cy = 2 * y + ((k >> 1) & 1), cz = 2 * z + ((k >> 2) & 1);
    double blo[3] = {cx * cs, cy * cs, cz * cs};
    double bhi[3] = {(cx + 1) * cs, (cy + 1) * cs, (cz + 1) * cs};
    double bound = c->tmax < c->b->second ? c->tmax : c->b->second;
    double t0, t1;
    if (!slab(c->o, c->d, blo, bhi, c->tmin, bound, &t0, &t1)) continue;
    int j = n_ord++;
    while (j > 0 && entry[j - 1] > t0) {
      entry[j] = entry[j - 1];
      order[j] = order[j - 1];
      --j;
    }
    entry[j] = t0;
    order[j] = k;
  }
  for (int j = 0; j < n_ord; ++j) {
    double bound = c->tmax < c->b->second ? c->tmax : c->b->second;
    if (entry[j] > bound) break; /* later children start even further */
    int k = order[j];
    descend(c, level + 1, (prefix << 3) | (uint64_t)k, start[k], start[k + 1]);
  }
}

static void trace_descent(const oracle_asset *a, uint32_t part, const double o[3], const double d[3], double tmin,
                          double tmax, best_hit *b) {
  if (a->n == 0) return;
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, t0, t1;
  if (!slab(o, d, lo, hi, tmin, tmax < b->second ? tmax : b->second, &t0, &t1)) return;
  descent_ctx c = {a, part, {o[0], o[1], o[2]}, {d[0], d[1], d[2]}, tmin, tmax, b};
  descend(&c, 0, 0, 0, a->n);
}

/* ------------------------------------------------------------- the tracer */

typedef struct {
  int n_parts;
  const oracle_asset *const *assets; /* per part */
  const double *inv;                 /* per part 3x4 world -> local */
  int64_t n_rays;
  const double *rays; /* 8 per ray: ox oy oz tmin dx dy dz tmax */
  double *out_t, *out_second;
  uint32_t *out_part;
  uint64_t *out_voxel;
  int mode;
  atomic_llong next;
} trace_job;

/* Which inputs are rays (Eq. 1: an origin, a direction, t in [tmin, tmax]).
 * The paper's rays always have a direction; this reading makes it a rule:
 * the largest direction component magnitude must lie in [2^-60, 2^60] (the
 * zero vector has none, and the bounds keep |d|^2 a normal FP32 number for
 * every such direction), origin and direction must be finite, and neither
 * bound may be NaN.  Anything else meets nothing and is reported as a miss.
 * Every test is an exact comparison, so any implementation applies it alike. */
static int ray_valid(const double *ray) {
  for (int i = 0; i < 3; ++i)
    if (!isfinite(ray[i]) || !isfinite(ray[4 + i])) return 0;
  if (isnan(ray[3]) || isnan(ray[7])) return 0;
  double m = fabs(ray[4]);
  if (fabs(ray[5]) > m) m = fabs(ray[5]);
  if (fabs(ray[6]) > m) m = fabs(ray[6]);
  return m >= ldexp(1.0, -60) && m <= ldexp(1.0, 60);
}

int oracle_ray_valid(const double *ray8) { return ray_valid(ray8); }

static void trace_one(const trace_job *j, int64_t r) {
  const double *ray = j->rays + 8 * r;
  best_hit b;
  best_init(&b);
  for (int p = 0; p < j->n_parts && ray_valid(ray); ++p) {
    const double *m = j->inv + 12 * p;
    double o[3], d[3];
    for (int i = 0; i < 3; ++i) {
      o[i] = m[i * 4] * ray[0] + m[i * 4 + 1] * ray[1] + m[i * 4 + 2] * ray[2] + m[i * 4 + 3];
      d[i] = m[i * 4] * ray[4] + m[i * 4 + 1] * ray[5] + m[i * 4 + 2] * ray[6];
    }
    if (j->mode == 0)
      trace_brute(j->assets[p], (uint32_t)p, o, d, ray[3], ray[7], &b);
    else
      trace_descent(j->assets[p], (uint32_t)p, o, d, ray[3], ray[7], &b);
  }
  j->out_t[r] = b.t;
  j->out_second[r] = b.second;
  j->out_part[r] = b.part;
  j->out_voxel[r] = b.voxel;
}

static void *trace_worker(void *arg) {
  trace_job *j = (trace_job *)arg;
  const int64_t chunk = 64;
  for (;;) {
    int64_t s = atomic_fetch_add(&j->next, chunk);
    if (s >= j->n_rays) break;
    int64_t e = s + chunk < j->n_rays ? s + chunk : j->n_rays;
    for (int64_t r = s; r < e; ++r) trace_one(j, r);
  }
  return NULL;
}

/* Trace n_rays rays against n_parts parts.  part_assets[p] is the oracle asset
 * of part p, inv the FP64 world->local pose of each part (oracle_invert).
 * mode 0 = brute force, 1 = descent.  Uses n_threads POSIX threads. */
int oracle_trace(int n_parts, void *const *part_assets, const double *inv, int64_t n_rays, const double *rays,
                 double *out_t, uint32_t *out_part, uint64_t *out_voxel, double *out_second, int mode,
                 int n_threads) {
  if (n_parts < 0 || n_rays < 0 || (mode != 0 && mode != 1)) return -1;
  trace_job job;
  job.n_parts = n_parts;
  job.assets = (const oracle_asset *const *)part_assets;
  job.inv = inv;
  job.n_rays = n_rays;
  job.rays = rays;
  job.out_t = out_t;
  job.out_second = out_second;
  job.out_part = out_part;
  job.out_voxel = out_voxel;
  job.mode = mode;
  atomic_init(&job.next, 0);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  int started = 0;
  for (int i = 1; i < n_threads; ++i)
    if (pthread_create(&th[started], NULL, trace_worker, &job) == 0) ++started;
  trace_worker(&job);
  for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
  return 0;
}
