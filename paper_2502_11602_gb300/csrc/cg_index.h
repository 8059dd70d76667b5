// cg_index.h -- host-side index object and device-memory helpers (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "cg_internal.cuh"

namespace cg {

// Device allocation through the installed hook, else cudaMallocAsync.
void* dev_alloc(size_t bytes, cudaStream_t st);
void dev_free(void* p, cudaStream_t st);

// Thread-local last-error message.
void set_error(const std::string& msg);
cg_status fail(cg_status s, const std::string& msg);
cg_status cuda_fail(cudaError_t e, const char* what);

// Scoped list of device buffers owned by an object.
struct DevBufs {
  std::vector<void*> ptrs;
  size_t bytes = 0;
  void* get(size_t b, cudaStream_t st) {
    if (b == 0) b = 16;
    void* p = dev_alloc(b, st);
    if (p) { ptrs.push_back(p); bytes += b; }
    return p;
  }
  void release(cudaStream_t st) {
    for (void* p : ptrs) dev_free(p, st);
    ptrs.clear();
    bytes = 0;
  }
};

struct Thresholds;
struct BlockPlan;

// Cached plan of an external query set (query order, blocks, records).
struct QueryPlan {
  const double* q = nullptr;
  int64_t nq = -1;
  uint64_t version = 0;          // bumps each time a plan is (re)built
  uint64_t nblocks_host_version = ~0ull;
  DevBufs bufs;
  uint32_t nblocks = 0;          // host copy (valid when versions match)
  uint32_t* nblocks_dev = nullptr;  // [16]: [0] blocks, [4] max |query offset| bits
  uint32_t* blk_beg = nullptr;   // [nblocks+1] block start in query order
  uint32_t* blk_key = nullptr;   // [nblocks] voxel key of the block (clamped)
  float4* qrec = nullptr;        // [nq] sorted: x~, y~, z~, query id bits
  double4_32a* qrec64 = nullptr;     // [nq] sorted: x, y, z, query id bits (binary64 path)
};

// State of a radius count pass kept for the matching fill pass.
struct RadiusState {
  DevBufs bufs;
  bool valid = false, all_points = false, stats_known = false;
  const double* q = nullptr;
  int64_t nq = 0;
  double r = 0;
  int kernel = 0;
  uint64_t plan_version = 0;
  uint32_t* counts = nullptr;      // [nq] per query id
  uint32_t* heavy_list = nullptr;  // rows assembled from several sorted runs
  uint32_t* heavy_soff = nullptr;  // scratch offsets of long rows
  uint32_t* ctrs = nullptr;        // [64] counters (see cg_query.cu)
  Thresholds* thr = nullptr;
  void* scan_scratch = nullptr;
  uint32_t heavy_count = 0;
  uint64_t heavy_scratch = 0;
  char thr_host[64];
  // fast kernels: per-group plans, mask / id layouts and the large groups
  struct BlockPlan* plans = nullptr;
  uint32_t *msize = nullptr, *isize = nullptr;
  int64_t *moff = nullptr, *idoff = nullptr;  // exclusive scans of msize / isize (64-bit)
  uint32_t *masks = nullptr, *ids = nullptr, *big_list = nullptr;
  uint32_t big_n = 0;
  int64_t mtot = 0, itot = 0;  // mask words / staged ids of the last count
  // all-points groups cut into height chunks (height-sorted columns)
  uint32_t *zbeg = nullptr, *zkey = nullptr;
  uint32_t znb = 0;
  bool small = false;  // the count took the small-batch path (so does the fill)
  // the small-batch path's workspace, allocated once for kSmallBatch queries
  // and kept until the context is released: counts, sizes, sorted rows
  // (kSmallRowCap entries per query)
  DevBufs small_bufs;
  uint32_t *small_counts = nullptr, *small_stats = nullptr;
  int32_t* small_rows = nullptr;
  // search-into calls: the small count also copies the rows into the
  // caller's buffer (when they fit its capacity) before its one sync
  int32_t* direct_out = nullptr;
  int64_t direct_cap = 0;
  bool direct_done = false;
};

// Mutable state of queries against an index: the external query plan, the
// radius pass carried from count to fill, and the device status word the
// kernels report into.  An index has one default context; concurrent users
// of one index (the serving loop's slots) each bring their own.
struct QueryCtx {
  QueryPlan plan;
  RadiusState radius;
  uint32_t* status = nullptr;
  void release(cudaStream_t st) {
    plan.bufs.release(st);
    radius.bufs.release(st);
    radius.small_bufs.release(st);
    plan = QueryPlan();
    radius = RadiusState();
  }
};

// Workspace of a replayed radius pass: every data-dependent buffer sized
// once with headroom; kernels flag ST_REPLAN when new data outgrows them.
struct RadiusWork {
  DevBufs bufs;
  uint32_t *counts = nullptr, *heavy_list = nullptr, *heavy_soff = nullptr, *ctrs = nullptr;
  Thresholds* thr = nullptr;
  void *scan_scr = nullptr, *plan_scr = nullptr;
  struct BlockPlan* plans = nullptr;
  uint32_t *msize = nullptr, *isize = nullptr;
  int64_t *moff = nullptr, *idoff = nullptr;
  uint32_t *masks = nullptr, *ids = nullptr, *big_list = nullptr;
  int32_t* row_scratch = nullptr;
  uint32_t cap_nb = 0;
  int64_t cap_m = 0, cap_i = 0;
  uint64_t cap_scr = 0;
  int64_t cap_out = 0;
};

// Workspace of a replayed k-NN pass.
struct KnnWork {
  DevBufs bufs;
  uint32_t *slow = nullptr, *ctrs = nullptr, *bslot = nullptr;
  float* br2 = nullptr;
  Thresholds* thr = nullptr;
};

// Workspace of a replayed (graph-captured) build.
struct BuildWork {
  DevBufs bufs;
  uint32_t *keys = nullptr, *skeys = nullptr, *flag = nullptr, *rank = nullptr, *cnt = nullptr;
  void *sort_scr = nullptr, *scan_scr = nullptr;
  unsigned long long* bb = nullptr;
  int64_t* toff = nullptr;
  uint32_t *ukeys = nullptr, *ustart = nullptr;  // [cap_keys], [cap_keys + 1]
  const uint32_t* nkeys_dev = nullptr;           // non-empty voxels of the last replay
  uint32_t cap_keys = 0;
  int bits = 0;
  uint32_t* zlong = nullptr;  // [cap_keys + 1]: long runs of the height sort, then their count
};

}  // namespace cg

struct cg_index {
  int dim = 2, flavor = 0, precision = 0, ntiles = 1;
  int64_t n = 0;
  cudaStream_t stream = nullptr;
  std::vector<cg::Tile> tiles_host;
  cg::DevBufs bufs;
  cg::Tile* tiles = nullptr;
  float4* pts32 = nullptr;
  float4* pts32z = nullptr;      // binary32 2D grids: every voxel run sorted by height
  uint32_t* sidz = nullptr;      // [n] original id of every position of pts32z
  double4_32a* pts64s = nullptr;
  double* xyz64 = nullptr;
  uint32_t* ukeys = nullptr;
  uint32_t* ustart = nullptr;
  uint32_t* sid = nullptr;       // [n] original id of every sorted position
  uint32_t nkeys = 0;
  uint32_t* cstart = nullptr;
  unsigned long long* hash = nullptr;
  uint32_t hash_mask = 0;
  uint8_t* slice_dense = nullptr;
  uint32_t* slice_tab_off = nullptr;
  uint2* mtab = nullptr;
  int64_t ncell = 0, nslices = 0, dense_slices = 0;
  uint32_t* status = nullptr;    // device status word (ST_* bits)
  uint32_t* scratch_u32 = nullptr;  // small device scratch
  double enc_err0 = 0;
  cg::QueryCtx ctx;  // default query context (status = the index's word)
  int max_pts_per_voxel = 0;

  cg::IndexView view() const {
    cg::IndexView v;
    v.tiles = tiles;
    v.ntiles = ntiles;
    v.dim = dim;
    v.flavor = flavor;
    v.precision = precision;
    v.n = (uint32_t)n;
    v.nkeys = nkeys;
    v.pts32 = pts32;
    v.pts32z = pts32z;
    v.pts64s = pts64s;
    v.sid = sid;
    v.xyz64 = xyz64;
    v.ukeys = ukeys;
    v.ustart = ustart;
    v.cstart = cstart;
    v.hash = hash;
    v.hash_mask = hash_mask;
    v.slice_dense = slice_dense;
    v.slice_tab_off = slice_tab_off;
    v.mtab = mtab;
    return v;
  }
};

namespace cg {
// Reads and clears the device status word (synchronises the stream).
cg_status check_status(cg_index* ix, cudaStream_t st);
cg_status check_status_word(uint32_t* status, cudaStream_t st);
// The error a status word `w` already read back stands for (clears the
// device word on an error).
cg_status status_verdict(uint32_t w, uint32_t* status, cudaStream_t st);
cg_status prepare_queries(cg_index* ix, QueryCtx& C, const double* q, int64_t nq, bool reuse, cudaStream_t st);
cg_status make_zchunks(cg_index* ix, float dz, uint32_t qmax, DevBufs& bufs, uint32_t* status, cudaStream_t st,
                       uint32_t** cbeg, uint32_t** ckey, uint32_t* nchunks);
cg_status radius_pass(cg_index* ix, QueryCtx& C, bool all_points, const double* q, int64_t nq, double r,
                      int kernel, bool fill, int64_t* offsets, int32_t* out, int64_t* total_host,
                      cudaStream_t st);
// Count and fill into the caller's buffer of `cap` entries (cg_query.cu):
// CG_ERR_OVERFLOW with *total_host set when the rows do not fit (the count
// stands; a fill with a larger buffer completes the search).
cg_status radius_search_into(cg_index* ix, QueryCtx& C, const double* q, int64_t nq, double r, int kernel,
                             int64_t* offsets, int32_t* out, int64_t cap, int64_t* total_host, cudaStream_t st);
cg_status knn_pass(cg_index* ix, QueryCtx& C, bool all_points, const double* q, int64_t nq, int k, int32_t* idx,
                   double* d2, cudaStream_t st);
// Algorithm 2 step by step under a growth policy (0 monotone, 1 density),
// with the voxels each search visited (cg_knn.cu).
cg_status knn_grow_pass(cg_index* ix, const double* q, int64_t nq, int k, int policy, int32_t* idx, double* d2,
                        int64_t* visited, cudaStream_t st, uint32_t* status = nullptr);
cg_status build_work_alloc(cg_index* ix, BuildWork& w, cudaStream_t st);
cg_status build_replay(cg_index* ix, BuildWork& w, const double* xyz, cudaStream_t st);
cg_status radius_work_alloc(cg_index* ix, RadiusWork& w, uint32_t cap_nb, double headroom, int64_t total,
                            cudaStream_t st);
cg_status radius_replay(cg_index* ix, RadiusWork& w, const uint32_t* nkeys_dev, double r, int kernel,
                        int64_t* offsets, int32_t* out, cudaStream_t st);
cg_status knn_work_alloc(cg_index* ix, KnnWork& w, cudaStream_t st);
cg_status knn_replay(cg_index* ix, KnnWork& w, const uint32_t* nkeys_dev, uint32_t cap_nb, int k, int32_t* idx,
                     double* d2, cudaStream_t st);
}  // namespace cg
