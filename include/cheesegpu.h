/*
 * cheesegpu.h -- C ABI of a GB300 (sm_103a) implementation of the Cheesemap
 * neighbour-search hot path (arXiv 2502.11602): a uniform voxel grid over a
 * point cloud, fixed-radius sphere / cube queries and exact k-NN.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Points and queries are float64 AoS arrays [n][3] (x, y, z) in device
 *    memory unless a name says _host.  Neighbour ids are 0-based int32 ids in
 *    the caller's original point order (batched indexes: ids into the
 *    concatenated point array).
 *  - Every call is ordered on `stream` (a cudaStream_t; NULL = legacy default
 *    stream).  Calls return as soon as the work is enqueued, except where a
 *    comment says the call synchronises the stream.
 *  - The caller owns every buffer it passes; the library never frees caller
 *    memory.  An index owns its internal device buffers until
 *    cg_index_free().  Internal buffers come from cudaMallocAsync on the
 *    call's stream, or from the hook installed by cg_set_allocator().
 *  - Every call returns a cg_status.  On an error nothing is written to the
 *    caller's outputs except where stated, and cg_last_error() returns a
 *    message for the calling thread.
 *  - The neighbour sets are fixed by one predicate, evaluated in IEEE binary64
 *    with round-to-nearest and no fused multiply-add:
 *        dx = fl(p_x - c_x), dy, dz likewise;
 *        sphere:   fl(fl(fl(dx*dx) + fl(dy*dy)) + fl(dz*dz)) <= fl(r*r)
 *        cube:     max(fl(dx*dx), fl(dy*dy), fl(dz*dz))  <= fl(r*r)
 *        cylinder: fl(fl(dx*dx) + fl(dy*dy)) <= fl(r*r)   (z unbounded)
 *    (the kernels of Section 2 / Section 3.4.1 of the paper, with "<=" as in
 *    the candidate set of Section 3.4.2).  k-NN returns the first min(k, N)
 *    points under the order (sphere value d2, original id).  Both precisions
 *    below return exactly these sets.
 */
#ifndef CHEESEGPU_H_
#define CHEESEGPU_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CG_OK = 0,
  CG_ERR_INVALID = 1,       /* bad argument (see each call)                      */
  CG_ERR_OOM = 2,           /* device allocation failed                          */
  CG_ERR_CUDA = 3,          /* a CUDA runtime call failed                        */
  CG_ERR_TIMEOUT = 4,       /* a bounded device wait gave up (no hang)           */
  CG_ERR_OVERFLOW = 5,      /* an output capacity was too small                  */
  CG_ERR_INTERNAL = 6,      /* a device-side consistency check failed            */
  CG_ERR_UNIMPLEMENTED = 7
} cg_status;

/* Voxel storage flavours, Section 3.3: dense array over all voxels (3.3.1);
   sparse map over non-empty voxels (3.3.2), here a sorted unique-key table
   plus an open-addressing device hash; mixed z slices, each dense iff at
   least 80 % of its voxels are non-empty, 2D = one slice (3.3.3). */
typedef enum { CG_DENSE = 0, CG_SPARSE = 1, CG_MIXED = 2 } cg_flavor;

/* Search kernels of Section 2: L2 ball, L-infinity ball (cube) and the
   vertical cylinder (xy only: every height within the horizontal radius). */
typedef enum { CG_SPHERE = 0, CG_CUBE = 1, CG_CYLINDER = 2 } cg_kernel;

/* Storage precision of the indexed coordinates.  CG_FP64 tests every
   candidate in binary64.  CG_FP32_OFFSET stores fl32(fl64(p - O)) for a
   per-tile origin O, tests candidates in binary32 and re-tests in binary64
   every candidate whose binary32 value falls within a proven error bound of
   r^2; the result sets are identical. */
typedef enum { CG_FP64 = 0, CG_FP32_OFFSET = 1 } cg_precision;

typedef struct cg_index* cg_index_t;

/* Optional device-memory hook (e.g. a framework's caching allocator).
   alloc returns NULL on failure; free receives the pointer and the stream
   the allocation was made on. */
typedef void* (*cg_alloc_fn)(size_t bytes, void* stream, void* user);
typedef void (*cg_free_fn)(void* ptr, void* stream, void* user);

/* Installs (or, with both NULL, removes) the allocation hook for buffers
   made by later calls.  Not thread-safe against concurrent library calls. */
cg_status cg_set_allocator(cg_alloc_fn alloc_fn, cg_free_fn free_fn, void* user);

/* Message describing the last error on the calling thread ("" if none). */
const char* cg_last_error(void);

/* Library version string. */
const char* cg_version(void);

/* Number of CUDA kernels the library has launched in this process so far
   (all threads and devices); a diagnostic for launch accounting. */
uint64_t cg_launch_count(void);

/*
 * cg_build -- index n points (Section 3: bounding box p-/p+ of Section 3.1,
 * grid size n_a = floor((p+_a - p-_a)/s_a) + 1 of Eq. grid-size, voxel of a
 * point floor((p_a - p-_a)/s_a) of Eq. chs-point-to-idcs with 0-based
 * indices, global voxel index of Eqs. indices-to-global-2D/-3D, points
 * reordered by voxel as in the "Reordering" remark of Section 3.5, with ties
 * kept in ascending original id).
 *
 *  xyz_dev   device float64 [n][3]; read during the call only (copied).
 *  n         number of points, 1 <= n < 2^31.
 *  cell_xy   voxel size along x and y (> 0, finite).
 *  cell_z    voxel size along z (> 0, finite); for 3D grids and for the
 *            z slices of the mixed flavour (s_z of Section 3.3.3).
 *  dim       2 (index x, y; z is not indexed) or 3.
 *  flavor    storage flavour.   precision  coordinate precision.
 *  out       receives the new index handle.
 * Errors: CG_ERR_INVALID for n out of range, non-positive or non-finite cell
 * sizes, dim not in {2, 3}, a non-finite coordinate, or more than 2^32 - 2
 * voxels in the grid; CG_ERR_OOM.  The call synchronises `stream` (grid
 * sizes depend on the data).
 */
cg_status cg_build(const double* xyz_dev, int64_t n, double cell_xy, double cell_z, int dim,
                   cg_flavor flavor, cg_precision precision, void* stream, cg_index_t* out);

/*
 * cg_build_batched -- index T independent tiles in one index (each tile its
 * own bounding box, origin, grid and cell size; voxel keys of different
 * tiles never collide).  Queries against a batched index are per tile: every
 * point queries its own tile (cg_all_points_count / _fill / _knn); external
 * queries need a single-tile index.
 *  xyz_dev       device float64 [N][3], tiles concatenated.
 *  tile_offsets  HOST int64 [T+1], tile t owns points [off[t], off[t+1]).
 *  T             number of tiles, >= 1; every tile non-empty.
 *  cell_xy_host  HOST float64 [T] voxel size per tile (x, y and z).
 * Same errors and synchronisation as cg_build.
 */
cg_status cg_build_batched(const double* xyz_dev, const int64_t* tile_offsets, int32_t T,
                           const double* cell_xy_host, int dim, cg_flavor flavor,
                           cg_precision precision, void* stream, cg_index_t* out);

typedef struct {
  int64_t n;            /* indexed points                                   */
  int32_t dim, flavor, precision, ntiles;
  int64_t ncell;        /* voxels of the grid(s), empty included             */
  int64_t nonempty;     /* non-empty voxels                                  */
  int64_t nslices;      /* z slices (mixed 3D), else 1 per tile              */
  int64_t dense_slices; /* slices stored dense                               */
  int64_t device_bytes; /* device memory held by the index                   */
  double lo[3], hi[3];  /* bounding box of tile 0 (Section 3.1)              */
  int64_t nc[3];        /* n_x, n_y, n_z of tile 0 (n_z = 1 in 2D)          */
  double cell[3];       /* voxel size of tile 0                              */
  double origin[3];     /* binary32 offset origin O of tile 0                */
  double enc_err;       /* bound on |fl32(fl64(p-O)) - fl64(p-O)|, tile 0    */
} cg_index_info_t;

cg_status cg_index_info(cg_index_t index, cg_index_info_t* info);

/* Synchronises `stream`, then returns (and clears) any device-side error
   recorded by earlier calls on this index: CG_ERR_TIMEOUT (a bounded wait
   gave up), CG_ERR_OVERFLOW, CG_ERR_INTERNAL (a consistency check failed;
   the affected output was not written past its bounds), CG_ERR_INVALID (a
   non-finite query coordinate).  CG_OK if none. */
cg_status cg_index_status(cg_index_t index, void* stream);

/* Releases the index (stream-ordered on the stream it was built on). */
cg_status cg_index_free(cg_index_t index);

/*
 * cg_radius_count -- pass 1 of the two-pass kernel search (Algorithm 1 run
 * for every query: voxel range of the kernel's bounding box, scan of the
 * voxels' points, predicate).  Writes offsets[0..nq] = exclusive prefix sum
 * of the per-query neighbour counts (offsets[0] = 0, offsets[nq] = total).
 *  q_dev        device float64 [nq][3] query centres (any position).
 *  nq           >= 0.  r > 0 finite.  kernel  CG_SPHERE, CG_CUBE or
 *               CG_CYLINDER (Section 2's kernels; the cylinder is vertical,
 *               z unbounded).
 *  offsets_dev  device int64 [nq+1], written.
 *  total_host   if non-NULL receives the total; the call then synchronises.
 * Queries keep an internal plan (query order, blocks) that cg_radius_fill
 * reuses when it is given the same q_dev, nq, r and kernel next.
 */
cg_status cg_radius_count(cg_index_t index, const double* q_dev, int64_t nq, double r,
                          cg_kernel kernel, int64_t* offsets_dev, int64_t* total_host,
                          void* stream);

/*
 * cg_radius_fill -- pass 2: writes every query's neighbour ids at
 * indices_dev[offsets[q] .. offsets[q+1]), each row ascending.
 *  offsets_dev  as produced by cg_radius_count for the same arguments.
 *  indices_dev  device int32 [offsets[nq]].
 */
cg_status cg_radius_fill(cg_index_t index, const double* q_dev, int64_t nq, double r,
                         cg_kernel kernel, const int64_t* offsets_dev, int32_t* indices_dev,
                         void* stream);

/*
 * cg_radius_search_into -- both passes of the kernel search of Algorithm 1
 * (Section 3.4.1) into the caller's buffers, one call: the count, then, if
 * the total fits `capacity`, the fill.
 *  offsets_dev  device int64 [nq+1], written as by cg_radius_count.
 *  indices_dev  device int32 [capacity]; rows as by cg_radius_fill.
 *  capacity     entries of indices_dev (>= 0).
 *  total_host   host int64, set to offsets[nq] on CG_OK and on
 *               CG_ERR_OVERFLOW.
 * Returns CG_ERR_OVERFLOW when the total exceeds the capacity: the count
 * stands, and cg_radius_fill with the same arguments and a buffer of
 * *total_host entries completes the search.  Batches of up to 1024 queries
 * cost one stream synchronisation (the rows are copied with the count);
 * larger ones two.  Other arguments and errors as cg_radius_count.
 */
cg_status cg_radius_search_into(cg_index_t index, const double* q_dev, int64_t nq, double r,
                                cg_kernel kernel, int64_t* offsets_dev, int32_t* indices_dev,
                                int64_t capacity, int64_t* total_host, void* stream);

/*
 * cg_radius_search -- both passes of the kernel search of Algorithm 1
 * (Section 3.4.1): count + scan + fill, with outputs allocated by the
 * library (hook or cudaMallocAsync); the caller releases them with
 * cg_free_device (or its own hook).  Arguments and errors as
 * cg_radius_count / cg_radius_fill; *offsets_dev, *indices_dev and *total
 * are written only on CG_OK.  Synchronises the stream once (the total sizes
 * the output).
 */
cg_status cg_radius_search(cg_index_t index, const double* q_dev, int64_t nq, double r,
                           cg_kernel kernel, int64_t** offsets_dev, int32_t** indices_dev,
                           int64_t* total, void* stream);

/*
 * cg_radius_stats -- work of the index's last planned count pass (the
 * default query context; small batches are not planned and report zeros):
 *  tested_pairs    candidate tests the fast count kernels ran: the sum over
 *                  voxel groups of (staged candidates x queries); Algorithm 1
 *                  itself tests every point of every voxel a kernel's box
 *                  meets, which the height ranges of 2D grids cut down;
 *  general_groups  groups too large for the fast kernels (general kernel);
 *  groups          voxel groups of an all-points pass on height chunks, else -1.
 * Synchronises the index's stream.
 */
typedef struct {
  int64_t tested_pairs;
  int64_t general_groups;
  int64_t groups;
} cg_radius_stats_t;
cg_status cg_radius_stats(cg_index_t index, cg_radius_stats_t* stats);

/* Frees a buffer returned by cg_radius_search (stream-ordered). */
cg_status cg_free_device(void* ptr, void* stream);

/*
 * cg_all_points_count / cg_all_points_fill -- Algorithm 1 (Section 3.4.1)
 * with every indexed point as a query (the queries are the index's own
 * points, no copy of them is made): the same outputs as cg_radius_count /
 * cg_radius_fill with q = the points in original order and nq = n, so row i
 * holds the neighbours of point i, ascending, point i included.  Errors as
 * those calls; the fill must follow a count with the same r and kernel.
 */
cg_status cg_all_points_count(cg_index_t index, double r, cg_kernel kernel, int64_t* offsets_dev,
                              int64_t* total_host, void* stream);
cg_status cg_all_points_fill(cg_index_t index, double r, cg_kernel kernel,
                             const int64_t* offsets_dev, int32_t* indices_dev, void* stream);

/*
 * cg_knn -- exact k nearest neighbours of every query (Algorithm 2's result:
 * the k closest points; ring-by-ring expansion over the voxel grid with the
 * visited region kept as an index box, the taboo box of Section 3.5).
 *  k            1 <= k <= 64.
 *  idx_dev      device int32 [nq][k]: ids ordered by (d2, id); -1 padding
 *               when the index holds fewer than k points.
 *  d2_dev       device float64 [nq][k] or NULL: the binary64 sphere value of
 *               each neighbour (+inf for padding).
 */
cg_status cg_knn(cg_index_t index, const double* q_dev, int64_t nq, int32_t k, int32_t* idx_dev,
                 double* d2_dev, void* stream);
cg_status cg_all_points_knn(cg_index_t index, int32_t k, int32_t* idx_dev, double* d2_dev,
                            void* stream);

/*
 * cg_knn_grow -- Algorithm 2 (Section 3.4.2) run step by step for each
 * query, one search per query: the radius r starts at the distance from c
 * to the nearest wall of its voxel; each iteration visits the voxels of the
 * bounding box of B(c, r) (widened by one voxel per side) outside the taboo
 * box of Section 3.5, and the search stops when at least k candidates lie
 * within r or every voxel has been visited.  The growth of r:
 *   policy 0  r + s (s the smallest voxel side), the monotone step;
 *   policy 1  the density step of the second phase: with the candidates
 *             within r non-empty and their number changed since the previous
 *             iteration, r = (3 k / (4 pi rho))^(1/3) with rho their number
 *             over the ball's volume (4/3) pi r^3; otherwise r + s.
 * The result does not depend on the policy and equals cg_knn's; the policy
 * changes how many voxels a search explores (Section 3.5 compares them).
 *  q_dev        device float64 [nq][3].   1 <= k <= 64.
 *  idx_dev      device int32 [nq][k], d2_dev float64 [nq][k] or NULL: as cg_knn.
 *  visited_dev  device int64 [nq] or NULL: voxels of each search's final
 *               taboo box.
 * CG_ERR_INVALID for k or policy out of range; CG_ERR_UNIMPLEMENTED on a
 * batched index.  Non-finite query coordinates are reported by
 * cg_index_status (that query's row is padding).  Asynchronous on `stream`.
 */
cg_status cg_knn_grow(cg_index_t index, const double* q_dev, int64_t nq, int32_t k, int32_t policy,
                      int32_t* idx_dev, double* d2_dev, int64_t* visited_dev, void* stream);

/*
 * cg_offsets_scan_noalloc -- the exclusive scan that turns per-query
 * neighbour counts into CSR offsets, without allocating any device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate, e.g. a serving loop whose device memory was reserved up
 * front by another allocator, a real-time path where an allocation could
 * block or fail, or a host that gives the library nothing but the input and
 * output buffers it owns.  The regular count pass allocates its scan
 * scratch; this call uses a fixed array compiled into the library instead.
 *
 *  counts_dev   device uint32 [n] per-query counts (read).
 *  n            0 <= n <= 134217728 (2^27); larger n is rejected with
 *               CG_ERR_INVALID before any device work.
 *  offsets_dev  device int64 [n+1], written: offsets[0] = 0,
 *               offsets[i+1] = offsets[i] + counts[i].  If a bounded device
 *               wait gives up, offsets[n] is set to -1 (the other entries are
 *               then unreliable) and the call has still returned CG_OK (it
 *               returns before the kernel runs): a caller that must be sure
 *               reads offsets[n] after the stream completes and checks that
 *               it is >= 0.  A wait gives up only if the GPU is shared so
 *               heavily that a resident block cannot make progress.
 *  stream       the call is asynchronous on this stream.
 * Scratch: 512 KiB + 256 B in a file-scope device array that every GPU which
 * loads the library holds until the process exits.  It is shared by all
 * calls: calls that overlap on the GPU (other streams, other host threads)
 * race and corrupt each other's result; serialise them.  Each call clears
 * the part it uses before its kernel runs.  The array's device address
 * belongs to the CUDA context that loaded the library: every call made while
 * its stream is not capturing looks it up again (cudaGetSymbolAddress, with
 * the calling device current), so a call after a device reset finds the
 * reloaded array; a call made while its stream is capturing reuses the
 * address that the last such lookup on the device found, and fails with
 * CG_ERR_INVALID if there was none.
 * The call makes no cudaMalloc, cudaFree or other allocating call.
 */
cg_status cg_offsets_scan_noalloc(const uint32_t* counts_dev, int64_t n, int64_t* offsets_dev,
                                  void* stream);

/*
 * Captured batched pipeline.  The whole hot path over a batch of tiles
 * (Section 3 build: bounding boxes, voxel keys, stable radix sort, gather,
 * runs, dense cell table; Algorithm 1 for every indexed point: count, scan,
 * fill with rows ascending by id; Algorithm 2's exact k-NN result for every
 * indexed point), recorded once as a CUDA graph and replayed.  A replay
 * re-reads the coordinates at xyz_dev (the buffer given at creation: same
 * tile sizes, new values), recomputes every tile's box, origin and binary32
 * error bounds on the device and writes the pipeline's own outputs, with no
 * host synchronisation, allocation or per-kernel launch.
 *
 * Sizes that depend on the data (non-empty voxels, candidate masks, output
 * length, long-row scratch) are checked on the device against capacities
 * fixed at creation (measured sizes x headroom).  Data that outgrows one of
 * them, or that changes a tile's grid dimensions, raises an internal re-plan
 * flag: the rest of that replay writes nothing, and the next cg_pipeline_run
 * with total_host != NULL plans again from the current coordinates (new
 * buffers: fetch the output pointers again) and replays.  The flavour is
 * dense; results are identical to cg_build_batched + cg_all_points_* on the
 * same coordinates.
 */
typedef struct cg_pipeline* cg_pipeline_t;

typedef struct {
  double radius;   /* > 0, finite                                        */
  int32_t kernel;  /* CG_SPHERE or CG_CUBE                               */
  int32_t k;       /* 0: no k-NN stage, else 1..64                       */
  double headroom; /* capacity factor for data-dependent buffers:
                      0 (default 1.25) or in [1, 16]                      */
} cg_pipeline_opts_t;

/*
 *  xyz_dev      device float64 [N][3], tiles concatenated; read by every
 *               replay (must stay allocated until cg_pipeline_free).
 *  tile_offsets HOST int64 [T+1], as cg_build_batched.  cell_host  HOST [T].
 *  dim 2 or 3; precision CG_FP64 or CG_FP32_OFFSET.
 * Plans on the current coordinates (one eager build and count pass), then
 * records the graph; synchronises `stream`.  Errors as cg_build_batched,
 * plus CG_ERR_INVALID for bad options and CG_ERR_CUDA if the capture fails.
 */
cg_status cg_pipeline_create(const double* xyz_dev, const int64_t* tile_offsets, int32_t T,
                             const double* cell_host, int dim, cg_precision precision,
                             const cg_pipeline_opts_t* opts, void* stream, cg_pipeline_t* out);

/* Replays the graph on `stream`.  With total_host == NULL the call is
   asynchronous and reports nothing about this replay.  Otherwise it
   synchronises, handles a pending re-plan (see above), returns any device
   error (as cg_index_status) and writes the number of radius neighbours. */
cg_status cg_pipeline_run(cg_pipeline_t p, void* stream, int64_t* total_host);

/* The pipeline-owned device outputs of the last replay (valid until the next
   re-plan or cg_pipeline_free): offsets int64 [N+1] and indices int32
   [offsets[N]] (CSR, original point ids, rows ascending); knn_idx int32
   [N][k] and knn_d2 float64 [N][k] (NULL when k = 0), ordered by (d2, id). */
cg_status cg_pipeline_outputs(cg_pipeline_t p, int64_t** offsets, int32_t** indices,
                              int32_t** knn_idx, double** knn_d2);

typedef struct {
  int64_t n;
  int32_t ntiles, k;
  int32_t graph_kernels;     /* kernel nodes launched by one replay        */
  int32_t graph_nodes;       /* all nodes (kernels, memsets, copies)       */
  int64_t replans;           /* re-plans since creation                    */
  int64_t capacity_indices;  /* room for radius neighbours                 */
  int64_t capacity_voxels;   /* room for non-empty voxels                  */
  int64_t ncell;             /* voxels of all tiles' grids                 */
  int64_t device_bytes;      /* device memory held by the pipeline         */
} cg_pipeline_info_t;

cg_status cg_pipeline_info(cg_pipeline_t p, cg_pipeline_info_t* info);

/* Waits for the last replay, then releases everything the pipeline holds. */
cg_status cg_pipeline_free(cg_pipeline_t p);

/*
 * Serving loop: continuous batching of query requests against
 * device-resident indexes (built with cg_build, single tile).  `slots`
 * worker threads each own a CUDA stream and a private query context, so up
 * to `slots` requests run at once and their kernels overlap on the GPU.
 * Admission is first come, first served: the oldest queued request starts
 * as soon as a slot is free and its memory fits the budget.  A radius
 * request first reserves its offsets (8 (nq+1) B) and an estimate of the
 * pass's work; after its count pass it reserves the measured CSR output
 * (total x 4 B) and work, waiting until other requests free memory.  If
 * every running request waits for memory, the last admitted one steps back
 * to the head of the queue (its count is redone when its measured size
 * fits).  A request that cannot fit the budget even alone completes with
 * CG_ERR_OOM.  A request's outputs belong to the server and count against
 * the budget until cg_server_release.  Results are those of cg_radius_count
 * + cg_radius_fill / cg_knn on the same inputs, alone or in any mix.
 * The server's calls are thread-safe.  Indexes and query buffers must stay
 * valid until their requests complete.  Requests never touch an index's
 * default query context, so other calls may query the same indexes
 * meanwhile (from one thread at a time, as always).
 */
typedef struct cg_server* cg_server_t;

typedef enum { CG_REQ_RADIUS = 0, CG_REQ_KNN = 1 } cg_request_op;

typedef struct {
  int32_t slots;          /* concurrent requests, 1..64                      */
  int64_t memory_budget;  /* bytes for requests' outputs and work; 0: half
                             of the device's free memory at creation        */
} cg_server_opts_t;

typedef struct {
  int32_t index;        /* position in the index list given at creation     */
  int32_t op;           /* cg_request_op                                    */
  int32_t kernel;       /* radius: CG_SPHERE or CG_CUBE                     */
  int32_t k;            /* k-NN: 1..64                                      */
  double radius;        /* radius: > 0, finite                              */
  const double* q_dev;  /* device float64 [nq][3] query centres             */
  int64_t nq;           /* >= 0                                             */
} cg_request_t;

typedef struct {
  cg_status status;
  int64_t nq, total;    /* total: radius neighbours (radius requests)       */
  int64_t* offsets;     /* radius: device int64 [nq+1]                      */
  int32_t* indices;     /* radius: device int32 [total], rows ascending     */
  int32_t* knn_idx;     /* k-NN: device int32 [nq][k]                       */
  double* knn_d2;       /* k-NN: device float64 [nq][k]                     */
  double queue_ms;      /* submit -> admission                              */
  double latency_ms;    /* submit -> result complete on the device          */
} cg_result_t;

typedef struct {
  int64_t requests_done, requests_failed, queries_done, queued;
  int32_t in_flight, max_in_flight;
  int64_t memory_budget, memory_in_use, memory_peak, preemptions;
  double p50_ms, p99_ms, max_ms;  /* latency of completed requests (nearest rank) */
  double queries_per_s;           /* completed queries / (last done - first submit) */
} cg_server_stats_t;

/* Starts the worker threads on the current device.  CG_ERR_INVALID for bad
   options or a NULL index. */
cg_status cg_server_create(const cg_index_t* indexes, int32_t n_indexes, const cg_server_opts_t* opts,
                           cg_server_t* out);

/* Queues a request (never blocks on the GPU) and returns its id.
   CG_ERR_INVALID for a bad index position, op, radius, kernel, k or query
   set; CG_ERR_UNIMPLEMENTED for a batched index. */
cg_status cg_server_submit(cg_server_t server, const cg_request_t* request, int64_t* id);

/* Waits up to timeout_s seconds (< 0: no limit) for a request.  Returns the
   request's own status (its result is filled in either way), or
   CG_ERR_TIMEOUT if it has not finished yet. */
cg_status cg_server_wait(cg_server_t server, int64_t id, double timeout_s, cg_result_t* result);

/* Waits up to timeout_s seconds (< 0: no limit) for any request to finish
   and returns its id, each finished request once, in completion order
   (CG_ERR_TIMEOUT if none).  A finished request's outputs hold budget until
   it is released, so a consumer that waits for one particular request while
   keeping others' results can stall admission: drain with this call. */
cg_status cg_server_wait_any(cg_server_t server, double timeout_s, int64_t* id);

/* Frees a finished request's outputs and returns their memory to the
   budget; the id becomes unknown. */
cg_status cg_server_release(cg_server_t server, int64_t id);

cg_status cg_server_stats(cg_server_t server, cg_server_stats_t* stats);

/* Drops queued requests, lets running ones finish, stops the workers and
   frees every output not yet released.  No other thread may be inside a
   call on this server. */
cg_status cg_server_free(cg_server_t server);

/*
 * Device-time tracing (diagnostics; no counterpart in the paper).  While
 * enabled, the library brackets each of its kernel phases (build steps,
 * radius plan / count / fill / row order, k-NN, sorts and scans) with CUDA
 * events on the launching stream; launches inside a graph capture are not
 * traced.  cg_profile_read waits for the recorded events and writes a JSON
 * object {"phase": [launches, total_ms], ...} into buf (len receives the
 * size needed, NUL included; buf NULL only queries the size); reset != 0
 * clears the totals.  Tracing adds two event records per phase.
 */
cg_status cg_profile_enable(int on);
cg_status cg_profile_read(char* buf, size_t cap, size_t* len, int reset);

/*
 * Launch tuning of the radius search (process-wide; the autotuner's knobs).
 * They change only speed, never a result.
 *  radius_chunk_height  all-points passes on binary32 2D grids: the height
 *                       span of a voxel group's chunk, in radii (> 0;
 *                       default 8).
 *  radius_chunk_max     queries per chunk (1 .. 512; default 256).
 *  count_shape          launch shape of the count kernels' three size
 *                       classes (0 default, 1, 2): warps per CTA and warps
 *                       sharing a voxel group.
 *  fill_shape           the same for the fill kernels.
 * cg_set_tuning(NULL) restores the defaults; out-of-range fields give
 * CG_ERR_INVALID and change nothing.  Calls already queued keep the settings
 * they were issued with; a captured pipeline keeps those of its capture.
 */
typedef struct {
  float radius_chunk_height;
  uint32_t radius_chunk_max;
  int32_t count_shape;
  int32_t fill_shape;
} cg_tuning_t;
cg_status cg_set_tuning(const cg_tuning_t* tuning);
cg_status cg_get_tuning(cg_tuning_t* tuning);

#ifdef __cplusplus
}
#endif

#endif /* CHEESEGPU_H_ */
