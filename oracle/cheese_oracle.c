/*
 * cheese_oracle.c -- plain, slow, single-threaded CPU restatement of the
 * Cheesemap grid index and its two queries (arXiv 2502.11602, Section 3).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code, header or
 * constant with the CUDA library, and the CUDA library never calls it.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off matters: the sphere predicate is defined without fused
 * multiply-add, and gcc on aarch64 contracts a*b+c by default.
 *
 * Layout conventions (all arrays owned by the caller unless stated):
 *   points and queries: AoS double [n][3] (x, y, z), original order.
 *   indices returned are original point indices (0-based int32).
 *
 * What each function follows:
 *   bbox            -- Section 3.1 (corners p-, p+ of the cloud).
 *   grid size n_a   -- Section 3.2, Eq. grid-size: floor((p+ - p-)/s) + 1.
 *   voxel of point  -- Section 3.2, Eq. chs-point-to-idcs, 0-based.
 *   global index g  -- Section 3.3.1, Eqs. indices-to-global-2D / -3D.
 *   dense flavour   -- Section 3.3.1 (array over all voxels).
 *   sparse flavour  -- Section 3.3.2 (map keyed by g over non-empty voxels;
 *                      here a sorted key array searched by bisection).
 *   mixed flavour   -- Section 3.3.3 (z slices, each dense iff at least 80 %
 *                      of its voxels are non-empty; 2D = one slice).
 *   kernel search   -- Algorithm 1 (bounding box -> voxel range -> scan);
 *                      kernels: sphere, cube, and the vertical cylinder
 *                      (xy only, z unbounded) of Section 2.
 *   k-NN            -- Algorithm 2 (growing radius + taboo box, Section 3.5).
 *   brute force     -- the definition of both result sets (Section 2).
 *
 * Predicates (the fixed reading of Section 2 / 3.4):
 *   dx = fl(p_x - c_x), likewise dy, dz (IEEE binary64, round to nearest)
 *   sphere: d2 = fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) <= r2, r2 = fl(r*r)
 *   cube:   max(fl(dx*dx), fl(dy*dy), fl(dz*dz)) <= r2
 *   k-NN:   the first min(k, N) points under the order (d2, original index).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OG_DENSE 0
#define OG_SPARSE 1
#define OG_MIXED 2
#define OG_SPHERE 0
#define OG_CUBE 1
#define OG_CYLINDER 2
#define OG_GROW_MONOTONE 0
#define OG_GROW_DENSITY 1
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* predicates                                                                */
/* ------------------------------------------------------------------------ */

/* Squared Euclidean distance in the fixed evaluation order (no contraction). */
double og_d2(const double* p, const double* c) {
  double dx = p[0] - c[0];
  double dy = p[1] - c[1];
  double dz = p[2] - c[2];
  double sxy = dx * dx + dy * dy;
  return sxy + dz * dz;
}

/* Cube (L-infinity) predicate value: the largest per-axis squared offset. */
double og_cube2(const double* p, const double* c) {
  double dx = p[0] - c[0];
  double dy = p[1] - c[1];
  double dz = p[2] - c[2];
  double ax = dx * dx, ay = dy * dy, az = dz * dz;
  double m = ax > ay ? ax : ay;
  return m > az ? m : az;
}

/* Vertical cylinder (the xy-only kernel of Section 2): squared horizontal
   distance, z ignored, same evaluation order as the sphere's first terms. */
double og_cyl2(const double* p, const double* c) {
  double dx = p[0] - c[0];
  double dy = p[1] - c[1];
  return dx * dx + dy * dy;
}

static int og_inside(const double* p, const double* c, double r2, int kernel) {
  if (kernel == OG_CUBE) return og_cube2(p, c) <= r2;
  if (kernel == OG_CYLINDER) return og_cyl2(p, c) <= r2;
  return og_d2(p, c) <= r2;
}

/* ------------------------------------------------------------------------ */
/* grid geometry: Sections 3.1 and 3.2                                       */
/* ------------------------------------------------------------------------ */

/* Bounding box corners p-, p+ (Section 3.1).  n must be > 0. */
void og_bbox(const double* xyz, int64_t n, double* lo, double* hi) {
  for (int a = 0; a < 3; ++a) { lo[a] = xyz[a]; hi[a] = xyz[a]; }
  for (int64_t i = 1; i < n; ++i)
    for (int a = 0; a < 3; ++a) {
      double v = xyz[3 * i + a];
      if (v < lo[a]) lo[a] = v;
      if (v > hi[a]) hi[a] = v;
    }
}

/* Eq. grid-size: n_a = floor((p+_a - p-_a) / s_a) + 1. */
int64_t og_grid_size(double lo, double hi, double s) {
  return (int64_t)floor((hi - lo) / s) + 1;
}

/* Eq. chs-point-to-idcs (0-based): floor((p_a - p-_a) / s_a). */
int64_t og_voxel_coord(double p, double lo, double s) {
  return (int64_t)floor((p - lo) / s);
}

/* ------------------------------------------------------------------------ */
/* the index                                                                 */
/* ------------------------------------------------------------------------ */

typedef struct {
  int dense;          /* 1: table over every voxel of the slice; 0: sorted keys */
  int64_t ncells;     /* voxels in the slice                                    */
  int64_t npts;       /* points in the slice                                    */
  int64_t* ids;       /* [npts] point ids grouped by voxel, ascending per voxel */
  int64_t* vstart;    /* dense:  [ncells+1] start of each voxel in ids          */
  int64_t nkeys;      /* sparse: number of non-empty voxels in the slice        */
  int64_t* keys;      /* sparse: [nkeys] sorted slice-local voxel numbers       */
  int64_t* kstart;    /* sparse: [nkeys+1] start of each stored voxel in ids    */
} og_slice;

typedef struct {
  int dim, flavor;
  int64_t n;
  double lo[3], hi[3], s[3];
  int64_t nc[3];      /* n_x, n_y, n_z (n_z = 1 in 2D)                          */
  int64_t ncell;      /* total voxels of the grid G                             */
  const double* xyz;  /* borrowed: caller keeps the points alive                */
  int64_t nonempty;
  int64_t nslices;
  og_slice* slices;
} og_index;

/* Global index of a voxel, Eqs. indices-to-global-2D / -3D. */
static int64_t og_global(const og_index* ix, int64_t i, int64_t j, int64_t k) {
  if (ix->dim == 2) return i * ix->nc[1] + j;
  return i * (ix->nc[1] * ix->nc[2]) + j * ix->nc[2] + k;
}

/* Slice of a global index and the voxel's number inside that slice.  One
   slice: the slice-local number is g itself.  3D mixed: slice = k, and the
   local number is i*n_y + j. */
static void og_slice_of(const og_index* ix, int64_t g, int64_t* sl, int64_t* local) {
  if (ix->nslices == 1) { *sl = 0; *local = g; return; }
  *sl = g % ix->nc[2];
  *local = g / ix->nc[2];
}

typedef struct { int64_t key, id; } og_pair;

static int og_pair_cmp(const void* a, const void* b) {
  const og_pair* x = (const og_pair*)a;
  const og_pair* y = (const og_pair*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

void og_free(og_index* ix);

/*
 * Build the index.  cell_xy is the voxel size in x and y, cell_z in z (the
 * footnote of Section 3.2 allows a different size per axis; for the mixed
 * flavour cell_z is the slice thickness s_z of Section 3.3.3).
 * Returns NULL on invalid arguments or allocation failure.
 */
og_index* og_build(const double* xyz, int64_t n, double cell_xy, double cell_z,
                   int dim, int flavor) {
  if (n <= 0 || !(cell_xy > 0) || !(cell_z > 0) || (dim != 2 && dim != 3) ||
      flavor < OG_DENSE || flavor > OG_MIXED)
    return NULL;
  og_index* ix = (og_index*)calloc(1, sizeof(og_index));
  if (!ix) return NULL;
  ix->dim = dim; ix->flavor = flavor; ix->n = n; ix->xyz = xyz;
  ix->s[0] = cell_xy; ix->s[1] = cell_xy; ix->s[2] = cell_z;
  og_bbox(xyz, n, ix->lo, ix->hi);
  for (int a = 0; a < 3; ++a) ix->nc[a] = og_grid_size(ix->lo[a], ix->hi[a], ix->s[a]);
  if (dim == 2) ix->nc[2] = 1;
  ix->ncell = ix->nc[0] * ix->nc[1] * ix->nc[2];

  /* key every point (Eq. chs-point-to-idcs, then the global index), then
     group by key with ties in ascending point id */
  og_pair* pr = (og_pair*)malloc(sizeof(og_pair) * (size_t)n);
  if (!pr) { og_free(ix); return NULL; }
  for (int64_t p = 0; p < n; ++p) {
    const double* q = xyz + 3 * p;
    int64_t i = og_voxel_coord(q[0], ix->lo[0], ix->s[0]);
    int64_t j = og_voxel_coord(q[1], ix->lo[1], ix->s[1]);
    int64_t k = dim == 3 ? og_voxel_coord(q[2], ix->lo[2], ix->s[2]) : 0;
    pr[p].key = og_global(ix, i, j, k);
    pr[p].id = p;
  }
  qsort(pr, (size_t)n, sizeof(og_pair), og_pair_cmp);

  /* slices: the whole grid is one slice for dense and sparse, and for 2D
     mixed; 3D mixed has one slice per z layer (Section 3.3.3). */
  int64_t nsl = (flavor == OG_MIXED && dim == 3) ? ix->nc[2] : 1;
  ix->nslices = nsl;
  ix->slices = (og_slice*)calloc((size_t)nsl, sizeof(og_slice));
  int64_t* ne = (int64_t*)calloc((size_t)nsl, sizeof(int64_t));
  if (!ix->slices || !ne) { free(ne); free(pr); og_free(ix); return NULL; }

  /* points and non-empty voxels per slice */
  for (int64_t p = 0; p < n; ++p) {
    int64_t sl, local;
    og_slice_of(ix, pr[p].key, &sl, &local);
    ix->slices[sl].npts++;
    if (p == 0 || pr[p].key != pr[p - 1].key) { ne[sl]++; ix->nonempty++; }
  }
  int64_t cells_per_slice = ix->ncell / nsl;
  for (int64_t sl = 0; sl < nsl; ++sl) {
    og_slice* S = &ix->slices[sl];
    S->ncells = cells_per_slice;
    if (flavor == OG_DENSE) S->dense = 1;
    else if (flavor == OG_SPARSE) S->dense = 0;
    else S->dense = (5 * ne[sl] >= 4 * cells_per_slice); /* the 80 % rule */
    S->ids = (int64_t*)malloc(sizeof(int64_t) * (size_t)(S->npts + 1));
    if (S->dense) {
      S->vstart = (int64_t*)calloc((size_t)cells_per_slice + 1, sizeof(int64_t));
    } else {
      S->keys = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne[sl] + 1));
      S->kstart = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ne[sl] + 1));
    }
    if (!S->ids || (S->dense && !S->vstart) || (!S->dense && (!S->keys || !S->kstart))) {
      free(ne); free(pr); og_free(ix); return NULL;
    }
    S->npts = 0; /* reused as a fill cursor below */
  }
  free(ne);

  /* fill each slice: the grouped order visits the voxels of every slice in
     ascending slice-local number, so appending keeps each list grouped */
  for (int64_t p = 0; p < n;) {
    int64_t key = pr[p].key, e = p;
    while (e < n && pr[e].key == key) ++e;
    int64_t sl, local;
    og_slice_of(ix, key, &sl, &local);
    og_slice* S = &ix->slices[sl];
    if (S->dense) {
      S->vstart[local + 1] = e - p; /* count; turned into starts below */
    } else {
      S->keys[S->nkeys] = local;
      S->kstart[S->nkeys] = S->npts;
      S->nkeys++;
    }
    for (int64_t t = p; t < e; ++t) S->ids[S->npts++] = pr[t].id;
    p = e;
  }
  for (int64_t sl = 0; sl < nsl; ++sl) {
    og_slice* S = &ix->slices[sl];
    if (S->dense) {
      for (int64_t c = 0; c < S->ncells; ++c) S->vstart[c + 1] += S->vstart[c];
    } else {
      S->kstart[S->nkeys] = S->npts;
    }
  }
  free(pr);
  return ix;
}

void og_free(og_index* ix) {
  if (!ix) return;
  if (ix->slices) {
    for (int64_t s = 0; s < ix->nslices; ++s) {
      free(ix->slices[s].ids);
      free(ix->slices[s].vstart);
      free(ix->slices[s].keys);
      free(ix->slices[s].kstart);
    }
    free(ix->slices);
  }
  free(ix);
}

/*
 * Points of voxel (i, j, k): returns the count and sets *ids to their
 * original ids (ascending).  Returns 0 for an empty or absent voxel: the
 * existence check of Algorithm 1, which dense slices skip (Section 3.5).
 */
static int64_t og_voxel_points(const og_index* ix, int64_t i, int64_t j, int64_t k,
                               const int64_t** ids) {
  int64_t sl, local;
  og_slice_of(ix, og_global(ix, i, j, k), &sl, &local);
  const og_slice* S = &ix->slices[sl];
  if (S->dense) {
    *ids = S->ids + S->vstart[local];
    return S->vstart[local + 1] - S->vstart[local];
  }
  /* sparse: bisection over the sorted keys of the slice */
  int64_t a = 0, b = S->nkeys;
  while (a < b) {
    int64_t m = a + (b - a) / 2;
    if (S->keys[m] < local) a = m + 1; else b = m;
  }
  if (a == S->nkeys || S->keys[a] != local) return 0;
  *ids = S->ids + S->kstart[a];
  return S->kstart[a + 1] - S->kstart[a];
}

/* ------------------------------------------------------------------------ */
/* index introspection (tests)                                               */
/* ------------------------------------------------------------------------ */

void og_info(const og_index* ix, int64_t* nc /*[3]*/, double* lo /*[3]*/, double* hi /*[3]*/,
             int64_t* ncell, int64_t* nonempty, int64_t* nslices) {
  for (int a = 0; a < 3; ++a) { nc[a] = ix->nc[a]; lo[a] = ix->lo[a]; hi[a] = ix->hi[a]; }
  *ncell = ix->ncell; *nonempty = ix->nonempty; *nslices = ix->nslices;
}

/* 1 if slice sl is stored dense. */
int og_slice_dense(const og_index* ix, int64_t sl) { return ix->slices[sl].dense; }

/* Number of points stored in voxel (i, j, k); -1 when the voxel is outside G. */
int64_t og_voxel_count(const og_index* ix, int64_t i, int64_t j, int64_t k) {
  if (i < 0 || j < 0 || k < 0 || i >= ix->nc[0] || j >= ix->nc[1] || k >= ix->nc[2]) return -1;
  const int64_t* ids;
  return og_voxel_points(ix, i, j, k, &ids);
}

/* 1 if the sparse table of the voxel's slice holds voxel (i,j,k) as a key
   (dense slices hold every voxel: always 1). */
int og_voxel_stored(const og_index* ix, int64_t i, int64_t j, int64_t k) {
  int64_t sl, local;
  og_slice_of(ix, og_global(ix, i, j, k), &sl, &local);
  const og_slice* S = &ix->slices[sl];
  if (S->dense) return 1;
  for (int64_t t = 0; t < S->nkeys; ++t) if (S->keys[t] == local) return 1;
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: kernel-based search                                          */
/* ------------------------------------------------------------------------ */

static int og_cmp_i64(const void* a, const void* b) {
  int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* Voxel range [*a, *b] along axis `ax` covering [c - r, c + r]: the voxel
   coordinate of each bounding-box corner (Eq. chs-point-to-idcs), widened by
   one voxel on each side so that the rounding of the keys can never hide a
   point, then clamped to the grid.  Returns 0 if the range is empty. */
static int og_axis_range(const og_index* ix, int ax, double c, double r,
                         int64_t* a, int64_t* b) {
  double lo = floor((c - r - ix->lo[ax]) / ix->s[ax]) - 1.0;
  double hi = floor((c + r - ix->lo[ax]) / ix->s[ax]) + 1.0;
  if (hi < 0 || lo > (double)(ix->nc[ax] - 1)) return 0;
  *a = lo < 0 ? 0 : (int64_t)lo;
  *b = hi > (double)(ix->nc[ax] - 1) ? ix->nc[ax] - 1 : (int64_t)hi;
  return 1;
}

/*
 * Algorithm 1 for one query: collect the ids of all indexed points inside
 * the kernel centred at c, ascending.  out must hold N entries (or NULL to
 * count only).  Returns the number of neighbours.
 */
int64_t og_kernel_search(const og_index* ix, const double* c, double r, int kernel,
                         int64_t* out) {
  double r2 = r * r;
  int64_t i0, i1, j0, j1, k0 = 0, k1 = 0;
  if (!og_axis_range(ix, 0, c[0], r, &i0, &i1)) return 0;
  if (!og_axis_range(ix, 1, c[1], r, &j0, &j1)) return 0;
  if (ix->dim == 3) {
    if (kernel == OG_CYLINDER) {  /* unbounded in z: every slice */
      k0 = 0;
      k1 = ix->nc[2] - 1;
    } else if (!og_axis_range(ix, 2, c[2], r, &k0, &k1)) {
      return 0;
    }
  }
  int64_t cnt = 0;
  for (int64_t i = i0; i <= i1; ++i)
    for (int64_t j = j0; j <= j1; ++j)
      for (int64_t k = k0; k <= k1; ++k) {
        const int64_t* ids;
        int64_t m = og_voxel_points(ix, i, j, k, &ids);
        for (int64_t t = 0; t < m; ++t) {
          const double* p = ix->xyz + 3 * ids[t];
          if (og_inside(p, c, r2, kernel)) {
            if (out) out[cnt] = ids[t];
            ++cnt;
          }
        }
      }
  if (out) qsort(out, (size_t)cnt, sizeof(int64_t), og_cmp_i64);
  return cnt;
}

/* Counts for a batch of queries (AoS [nq][3]). */
void og_radius_count(const og_index* ix, const double* q, int64_t nq, double r, int kernel,
                     int64_t* counts) {
  for (int64_t t = 0; t < nq; ++t) counts[t] = og_kernel_search(ix, q + 3 * t, r, kernel, NULL);
}

/* CSR for a batch: offsets[nq+1] must already hold the exclusive prefix sum
   of the counts; indices[offsets[nq]] receives the rows (int32 ids). */
void og_radius_fill(const og_index* ix, const double* q, int64_t nq, double r, int kernel,
                    const int64_t* offsets, int32_t* indices) {
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)ix->n);
  if (!tmp) return;
  for (int64_t t = 0; t < nq; ++t) {
    int64_t m = og_kernel_search(ix, q + 3 * t, r, kernel, tmp);
    for (int64_t u = 0; u < m; ++u) indices[offsets[t] + u] = (int32_t)tmp[u];
  }
  free(tmp);
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: k-NN with a growing radius and a taboo box                   */
/* ------------------------------------------------------------------------ */

typedef struct { double d2; int64_t id; } og_cand;

static int og_cand_cmp(const void* a, const void* b) {
  const og_cand* x = (const og_cand*)a;
  const og_cand* y = (const og_cand*)b;
  if (x->d2 != y->d2) return x->d2 < y->d2 ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}

/*
 * Algorithm 2 for one query.  Writes min(k, N) ids ordered by (d2, id) into
 * idx[0..k) and their d2 into d2o; remaining slots get id -1 and d2 = +inf.
 *
 * Steps, in the order of Algorithm 2:
 *  - r starts at the distance from c to the nearest wall of its voxel
 *    (the initial-radius formula of Section 3.4.2, over the indexed axes);
 *  - each iteration visits the voxels of the bounding box of B(c, r) that are
 *    outside the taboo box T (stored as an index box, Section 3.5) and adds
 *    their points to the candidate set;
 *  - P^ = candidates with d(p, c) <= r, compared as d2 <= fl(r*r);
 *  - the loop ends when |P^| >= k or T covers G; otherwise r grows.
 * Growth (policy):
 *  OG_GROW_MONOTONE  r + s, s the smallest voxel side (the first phase of
 *                    Section 3.4.2, used throughout);
 *  OG_GROW_DENSITY   Algorithm 2's second phase: with P^ non-empty, the
 *                    density rho = |P^| / ((4/3) pi r^3) of the ball gives
 *                    the radius whose ball holds k points at that density,
 *                    r = (3 k / (4 pi rho))^(1/3) (the paper prints this
 *                    step without the 3 / (4 pi) of the ball volume, and once
 *                    with rho and k swapped; the reading here keeps the
 *                    ball's volume, which the density's own definition uses);
 *                    with P^ empty, or |P^| the same as in the previous
 *                    iteration (the density did not change), r + s.
 * The policy changes only the sequence of radii, never the result: the loop
 * stops only when every point within r has been collected and at least k of
 * them are within r.  When T covers G with |P^| < k, every point is a
 * candidate and the k nearest candidates are returned (N < k: all N).
 * *visited (if non-NULL) receives |T|, the number of voxels of the final
 * taboo box (Section 3.5: the voxels the search explored).
 */
void og_knn_one_policy(const og_index* ix, const double* c, int64_t k, int policy, int32_t* idx,
                       double* d2o, int64_t* visited) {
  int64_t n = ix->n;
  og_cand* cand = (og_cand*)malloc(sizeof(og_cand) * (size_t)n);
  if (!cand) return;
  int64_t ncand = 0;

  /* voxel of c, clamped to the grid (queries may lie outside the bbox) */
  int64_t v[3] = {0, 0, 0};
  int nax = ix->dim;
  for (int a = 0; a < nax; ++a) {
    double t = floor((c[a] - ix->lo[a]) / ix->s[a]);
    if (t < 0) t = 0;
    if (t > (double)(ix->nc[a] - 1)) t = (double)(ix->nc[a] - 1);
    v[a] = (int64_t)t;
  }
  /* initial radius: nearest wall of the voxel of c */
  double r = INFINITY;
  for (int a = 0; a < nax; ++a) {
    double wlo = ix->lo[a] + (double)v[a] * ix->s[a];
    double whi = wlo + ix->s[a];
    double d0 = fabs(c[a] - wlo), d1 = fabs(c[a] - whi);
    if (d0 < r) r = d0;
    if (d1 < r) r = d1;
  }
  double s_min = ix->s[0] < ix->s[1] ? ix->s[0] : ix->s[1];
  if (nax == 3 && ix->s[2] < s_min) s_min = ix->s[2];

  int have_T = 0;
  int64_t T0[3] = {0, 0, 0}, T1[3] = {-1, -1, -1};
  int64_t inside = 0, inside_prev = -1;
  for (;;) {
    int64_t b0[3] = {0, 0, 0}, b1[3] = {0, 0, 0};
    int empty = 0;
    for (int a = 0; a < nax; ++a)
      if (!og_axis_range(ix, a, c[a], r, &b0[a], &b1[a])) empty = 1;
    if (!empty) {
      for (int64_t i = b0[0]; i <= b1[0]; ++i)
        for (int64_t j = b0[1]; j <= b1[1]; ++j)
          for (int64_t kk = b0[2]; kk <= b1[2]; ++kk) {
            if (have_T && i >= T0[0] && i <= T1[0] && j >= T0[1] && j <= T1[1] &&
                kk >= T0[2] && kk <= T1[2])
              continue; /* taboo: already visited */
            const int64_t* ids;
            int64_t m = og_voxel_points(ix, i, j, kk, &ids);
            for (int64_t t = 0; t < m; ++t) {
              cand[ncand].id = ids[t];
              cand[ncand].d2 = og_d2(ix->xyz + 3 * ids[t], c);
              ++ncand;
            }
          }
      /* the visited region is now the union of the old and new boxes; both
         are boxes containing the query's clamped voxel neighbourhood and the
         new one contains the old one (r only grows), so T = new box */
      for (int a = 0; a < 3; ++a) { T0[a] = b0[a]; T1[a] = b1[a]; }
      have_T = 1;
    }
    double r2 = r * r;
    inside = 0;
    for (int64_t t = 0; t < ncand; ++t) inside += cand[t].d2 <= r2;
    int covers = have_T;
    for (int a = 0; a < nax; ++a)
      if (T0[a] != 0 || T1[a] != ix->nc[a] - 1) covers = 0;
    if (inside >= k || covers) break;
    if (policy == OG_GROW_DENSITY && inside > 0 && inside != inside_prev) {
      double rho = (double)inside / ((4.0 / 3.0) * M_PI * r * r * r);
      r = cbrt(3.0 * (double)k / (4.0 * M_PI * rho));
    } else {
      r = r + s_min;
    }
    inside_prev = inside;
  }
  if (visited) {
    int64_t v = 1;
    for (int a = 0; a < 3; ++a) v *= have_T ? (T1[a] - T0[a] + 1) : 0;
    *visited = v;
  }
  qsort(cand, (size_t)ncand, sizeof(og_cand), og_cand_cmp);
  for (int64_t t = 0; t < k; ++t) {
    if (t < ncand) { idx[t] = (int32_t)cand[t].id; d2o[t] = cand[t].d2; }
    else { idx[t] = -1; d2o[t] = INFINITY; }
  }
  free(cand);
}

void og_knn_one(const og_index* ix, const double* c, int64_t k, int32_t* idx, double* d2o) {
  og_knn_one_policy(ix, c, k, OG_GROW_MONOTONE, idx, d2o, NULL);
}

void og_knn(const og_index* ix, const double* q, int64_t nq, int64_t k, int32_t* idx, double* d2) {
  for (int64_t t = 0; t < nq; ++t) og_knn_one(ix, q + 3 * t, k, idx + k * t, d2 + k * t);
}

/* ------------------------------------------------------------------------ */
/* brute force: the definition of both result sets                           */
/* ------------------------------------------------------------------------ */

int64_t og_brute_radius_one(const double* xyz, int64_t n, const double* c, double r,
                            int kernel, int64_t* out) {
  double r2 = r * r;
  int64_t cnt = 0;
  for (int64_t p = 0; p < n; ++p)
    if (og_inside(xyz + 3 * p, c, r2, kernel)) { if (out) out[cnt] = p; ++cnt; }
  return cnt;
}

void og_brute_knn_one(const double* xyz, int64_t n, const double* c, int64_t k,
                      int32_t* idx, double* d2o) {
  og_cand* cand = (og_cand*)malloc(sizeof(og_cand) * (size_t)n);
  if (!cand) return;
  for (int64_t p = 0; p < n; ++p) { cand[p].id = p; cand[p].d2 = og_d2(xyz + 3 * p, c); }
  qsort(cand, (size_t)n, sizeof(og_cand), og_cand_cmp);
  for (int64_t t = 0; t < k; ++t) {
    if (t < n) { idx[t] = (int32_t)cand[t].id; d2o[t] = cand[t].d2; }
    else { idx[t] = -1; d2o[t] = INFINITY; }
  }
  free(cand);
}

/* ------------------------------------------------------------------------ */
/* multi-threaded drivers: the per-query code above, split by query range    */
/* ------------------------------------------------------------------------ */

typedef struct {
  const og_index* ix; const double* q; int64_t q0, q1; double r; int kernel; int64_t k;
  int64_t* counts; const int64_t* offsets; int32_t* indices; int32_t* kidx; double* kd2;
  int mode; int policy; int64_t* visited;
} og_job;

static void* og_worker(void* arg) {
  og_job* jb = (og_job*)arg;
  if (jb->mode == 0) {
    for (int64_t t = jb->q0; t < jb->q1; ++t)
      jb->counts[t] = og_kernel_search(jb->ix, jb->q + 3 * t, jb->r, jb->kernel, NULL);
  } else if (jb->mode == 1) {
    int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * (size_t)jb->ix->n);
    if (!tmp) return NULL;
    for (int64_t t = jb->q0; t < jb->q1; ++t) {
      int64_t m = og_kernel_search(jb->ix, jb->q + 3 * t, jb->r, jb->kernel, tmp);
      for (int64_t u = 0; u < m; ++u) jb->indices[jb->offsets[t] + u] = (int32_t)tmp[u];
    }
    free(tmp);
  } else {
    for (int64_t t = jb->q0; t < jb->q1; ++t)
      og_knn_one_policy(jb->ix, jb->q + 3 * t, jb->k, jb->policy, jb->kidx + jb->k * t, jb->kd2 + jb->k * t,
                        jb->visited ? jb->visited + t : NULL);
  }
  return NULL;
}

static void og_run(og_job base, int64_t nq, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  og_job jobs[256];
  int started = 0;
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = base;
    jobs[t].q0 = nq * t / nthreads;
    jobs[t].q1 = nq * (t + 1) / nthreads;
    if (nthreads == 1 || pthread_create(&th[t], NULL, og_worker, &jobs[t]) != 0) {
      og_worker(&jobs[t]);
      th[t] = 0;
    } else {
      ++started;
    }
  }
  for (int t = 0; t < nthreads; ++t) if (th[t]) pthread_join(th[t], NULL);
  (void)started;
}

void og_radius_count_mt(const og_index* ix, const double* q, int64_t nq, double r, int kernel,
                        int64_t* counts, int nthreads) {
  og_job b; memset(&b, 0, sizeof b);
  b.ix = ix; b.q = q; b.r = r; b.kernel = kernel; b.counts = counts; b.mode = 0;
  og_run(b, nq, nthreads);
}

void og_radius_fill_mt(const og_index* ix, const double* q, int64_t nq, double r, int kernel,
                       const int64_t* offsets, int32_t* indices, int nthreads) {
  og_job b; memset(&b, 0, sizeof b);
  b.ix = ix; b.q = q; b.r = r; b.kernel = kernel; b.offsets = offsets; b.indices = indices;
  b.mode = 1;
  og_run(b, nq, nthreads);
}

void og_knn_mt(const og_index* ix, const double* q, int64_t nq, int64_t k, int32_t* idx,
               double* d2, int nthreads) {
  og_job b; memset(&b, 0, sizeof b);
  b.ix = ix; b.q = q; b.k = k; b.kidx = idx; b.kd2 = d2; b.mode = 2;
  og_run(b, nq, nthreads);
}

/* k-NN under a growth policy, with the voxels each search visited. */
void og_knn_policy_mt(const og_index* ix, const double* q, int64_t nq, int64_t k, int policy, int32_t* idx,
                      double* d2, int64_t* visited, int nthreads) {
  og_job b; memset(&b, 0, sizeof b);
  b.ix = ix; b.q = q; b.k = k; b.kidx = idx; b.kd2 = d2; b.mode = 2; b.policy = policy; b.visited = visited;
  og_run(b, nq, nthreads);
}
