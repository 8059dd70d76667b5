// cg_internal.cuh -- shared structures and device helpers of the cheesegpu
// library (not part of the public C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/cheesegpu.h"

namespace cg {

// --------------------------------------------------------------------------
// Per-tile grid description, resident in device memory.  A plain index has
// one tile; a batched index has one per tile, with disjoint key ranges.
// --------------------------------------------------------------------------
struct Tile {
  double lo[3];       // p- (Section 3.1)
  double hi[3];       // p+
  double s[3];        // voxel size per axis (footnote of Section 3.2)
  double origin[3];   // O: origin of the binary32 offsets
  int32_t n[3];       // n_x, n_y, n_z (Eq. grid-size); n_z = 1 in 2D
  uint32_t key_base;  // first global voxel key of the tile
  uint32_t pt_base;   // first point (concatenated order) of the tile
  uint32_t pt_count;  // points of the tile
  uint32_t slice_base;// first z slice id of the tile (mixed flavour)
  uint32_t nslices;   // z slices of the tile (mixed 3D: n_z, else 1)
  float D[3];         // fl32(O - p-): cell coordinate offset of the origin
  float inv_sf[3];    // fl32(1 / s)
  float eta;          // cell-unit padding for ranges computed in binary32
  float enc_err;      // bound on |x~ - (p - O)| per axis (metres)
  float pad_[2];
};

// Device status word bits (read by the host after a sync).
enum : uint32_t {
  ST_NONFINITE = 1u,   // a coordinate was NaN / inf
  ST_TIMEOUT = 2u,     // a bounded spin gave up: the whole pass is void (every
                       // kernel of it, on every forked stream), the host fails it
  ST_OVERFLOW = 4u,    // an output capacity was exceeded
  ST_INTERNAL = 8u,    // a consistency check failed
  ST_KNN_SLOW = 16u,   // some k-NN queries need the slow path (not an error)
  ST_REPLAN = 32u,     // a captured pipeline no longer fits its data: skip, re-plan
};

// Kernels of a captured pipeline stop at once when the pipeline has been
// invalidated earlier in the same run (sizes or capacities changed).
__device__ __forceinline__ bool replan_pending(const uint32_t* status) {
  return status != nullptr && (*((volatile const uint32_t*)status) & ST_REPLAN) != 0u;
}

// Spin bound for decoupled look-back and work queues: about a second at
// most on a GB300 before the wait is abandoned with ST_TIMEOUT.
constexpr uint32_t kSpinLimit = 1u << 24;

// Counts kernel launches made by the library (host side, diagnostics).
void note_launch(int n = 1);

// Fork / join of independent kernels of one pass onto extra streams (one
// set per host thread and device), so that they overlap on the GPU: every
// branch starts after the work already on the origin stream, and the origin
// continues only after every branch.  Works inside a stream capture (the
// branches become parallel graph nodes).  Branch kMax - 1 runs at the
// device's highest stream priority.
struct Fork {
  static constexpr int kMax = 4;
  Fork(cudaStream_t origin, int branches);
  cudaStream_t operator[](int i) const { return i == 0 ? origin_ : aux_[i - 1]; }
  void join();
  ~Fork() { join(); }
  Fork(const Fork&) = delete;
  Fork& operator=(const Fork&) = delete;

 private:
  cudaStream_t origin_;
  cudaStream_t aux_[kMax - 1];
  cudaEvent_t join_[kMax - 1];
  int n_ = 1;
  bool joined_ = false;
};

// Device-time tracing of the library's kernels (off unless enabled through
// cg_profile_enable): a scope records CUDA events around the launches it
// encloses on their stream; nothing is recorded while a stream is being
// captured into a graph.
struct ProfScope {
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;
  const char* name = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr;
};

// Small host <-> device transfers that do not use the copy engines.  A copy
// engine serves its queue in order, so a 4-byte cudaMemcpyAsync readback
// issued on one stream waits behind every bulk copy in the same direction
// that any stream of the process has in flight (a 2.7 GB result download
// holds it ~14 ms).  Here a kernel moves the bytes through mapped pinned
// host memory, which the SMs reach directly; the staging buffers belong to
// the calling host thread.
//
// HostRead: queue device -> host reads with get(); sync() launches one
// copy kernel for all of them on `st`, synchronizes `st` and stores the
// bytes at the host addresses.  Not usable while `st` is being captured.
class HostRead {
 public:
  void get(void* host, const void* dev, size_t bytes);
  cudaError_t sync(cudaStream_t st);

 private:
  static constexpr int kMax = 8;
  void* host_[kMax];
  const void* dev_[kMax];
  size_t bytes_[kMax];
  int n_ = 0;
};

// Host -> device: stages `bytes` from `host` and copies them into `dev` on
// `st` with a kernel.  `host` may be reused on return; the copy is ordered
// on `st` like a cudaMemcpyAsync.  Not usable while `st` is being captured.
cudaError_t host_put(void* dev, const void* host, size_t bytes, cudaStream_t st);

// Device -> device copy by a kernel on `st` (HBM bandwidth, no copy engine).
cudaError_t dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t st);

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Monotone map of a double to uint64 (for atomic min / max).
__device__ __forceinline__ unsigned long long dbl_to_ord(double d) {
  unsigned long long u = (unsigned long long)__double_as_longlong(d);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__host__ __device__ __forceinline__ double ord_to_dbl(unsigned long long u) {
  u = (u >> 63) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u;
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)u);
#else
  double d;
  __builtin_memcpy(&d, &u, 8);
  return d;
#endif
}

// 64-bit finaliser (MurmurHash3 fmix64) for the open-addressing table.
__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

constexpr unsigned long long kHashEmpty = ~0ull;

// Looks up a voxel key in the open-addressing table (linear probing; the
// slot stores key << 32 | row).  Returns the row of the sorted unique-key
// table, or -1.
__device__ __forceinline__ int hash_find(const unsigned long long* __restrict__ table,
                                         uint32_t mask, uint32_t key) {
  uint32_t h = (uint32_t)fmix64(key) & mask;
  for (uint32_t probe = 0; probe <= mask; ++probe) {
    unsigned long long e = __ldg(table + h);
    if (e == kHashEmpty) return -1;
    if ((uint32_t)(e >> 32) == key) return (int)(uint32_t)e;
    h = (h + 1) & mask;
  }
  return -1;
}

// --------------------------------------------------------------------------
// Device view of an index, passed by value to kernels.
// --------------------------------------------------------------------------
struct IndexView {
  const Tile* tiles;
  int32_t ntiles;
  int32_t dim;
  int32_t flavor;
  int32_t precision;
  uint32_t n;              // points
  uint32_t nkeys;          // non-empty voxels (runs)
  const float4* pts32;     // [n] sorted: x~, y~, z~, id bits (binary32 path)
  const float4* pts32z;    // [n] the same runs, each sorted by z~ (binary32 2D grids), or null
  const double4_32a* pts64s;   // [n] sorted: x, y, z, id bits (binary64 path)
  const double* xyz64;     // [n][3] original order (exact rechecks)
  const uint32_t* sid;     // [n] original id of every sorted position
  const uint32_t* ukeys;   // [nkeys] sorted unique voxel keys
  const uint32_t* ustart;  // [nkeys+1] start of each run in sorted order
  const uint32_t* cstart;  // dense: [ncell+1]
  const unsigned long long* hash;  // sparse / mixed: open addressing table
  uint32_t hash_mask;
  const uint8_t* slice_dense;      // mixed: [total slices]
  const uint32_t* slice_tab_off;   // mixed: [total slices] offset into mtab
  const uint2* mtab;               // mixed: (start, end) per voxel of dense slices
};

// Tile owning a global voxel key (binary search over key_base).
__device__ __forceinline__ int tile_of_key(const Tile* tiles, int ntiles, uint32_t key) {
  int a = 0, b = ntiles - 1;
  while (a < b) {
    int m = (a + b + 1) >> 1;
    if (tiles[m].key_base <= key) a = m; else b = m - 1;
  }
  return a;
}

// Tile owning a point id of the concatenated input (binary search over pt_base).
__device__ __forceinline__ int tile_of_id(const Tile* tiles, int ntiles, uint32_t id) {
  int a = 0, b = ntiles - 1;
  while (a < b) {
    int m = (a + b + 1) >> 1;
    if (tiles[m].pt_base <= id) a = m; else b = m - 1;
  }
  return a;
}

// (start, end) of the sorted points of voxel `key` (end == start if empty).
__device__ __forceinline__ uint2 voxel_span(const IndexView& ix, const Tile& t, uint32_t key) {
  if (ix.flavor == CG_DENSE) return make_uint2(__ldg(ix.cstart + key), __ldg(ix.cstart + key + 1));
  if (ix.flavor == CG_MIXED) {
    uint32_t g = key - t.key_base;
    uint32_t sl = (ix.dim == 3) ? (g % (uint32_t)t.n[2]) : 0u;
    uint32_t gs = t.slice_base + sl;
    if (__ldg(ix.slice_dense + gs)) {
      uint32_t local = (ix.dim == 3) ? g / (uint32_t)t.n[2] : g;
      uint2 v = ix.mtab[__ldg(ix.slice_tab_off + gs) + local];
      return v;
    }
  }
  int row = hash_find(ix.hash, ix.hash_mask, key);
  if (row < 0) return make_uint2(0u, 0u);
  return make_uint2(__ldg(ix.ustart + row), __ldg(ix.ustart + row + 1));
}

// Contiguous sorted span of the consecutive voxel keys [k0, k1] (one row of
// a 2D grid or one (i, j) column of a 3D grid): keys are consecutive, so
// their points are contiguous in the sorted order.
__device__ __forceinline__ uint2 row_span(const IndexView& ix, const Tile& t, uint32_t k0,
                                          uint32_t k1) {
  if (ix.flavor == CG_DENSE) return make_uint2(__ldg(ix.cstart + k0), __ldg(ix.cstart + k1 + 1));
  uint32_t s = 0, e = 0;
  bool found = false;
  for (uint32_t k = k0; k <= k1; ++k) {
    uint2 v = voxel_span(ix, t, k);
    if (v.y > v.x) {
      if (!found) { s = v.x; found = true; }
      e = v.y;
    }
  }
  return found ? make_uint2(s, e) : make_uint2(0u, 0u);
}

}  // namespace cg
