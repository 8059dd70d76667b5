// cg_build.cu -- grid index build on the GPU (Section 3 of arXiv 2502.11602).
//
// Steps (each a kernel, all ordered on one stream):
//   B0  bounding box p-, p+ per tile (Section 3.1) and grid size per axis,
//       n_a = floor((p+_a - p-_a) / s_a) + 1 (Eq. grid-size), on the host
//       from the reduced box (one stream sync: the grid size sizes the tables);
//   B1  voxel key of every point: floor(fl64(fl64(p_a - p-_a) / s_a)) per
//       axis (Eq. chs-point-to-idcs, 0-based), global index i*n_y + j or
//       i*n_y*n_z + j*n_z + k (Eqs. indices-to-global-2D/-3D), plus the
//       tile's first key;
//   B3  stable LSD radix sort of (key, point id) (the reordering remark of
//       Section 3.5; ties in ascending id);
//   B4  gather of the sorted records (binary32 offsets fl32(fl64(p - O)) with
//       the id, or binary64 coordinates with the id), the sorted unique-key
//       table (runs), and the voxel tables of the flavour: dense start array
//       via an exclusive scan of voxel counts (Section 3.3.1); sparse hash
//       over the non-empty voxels (Section 3.3.2); mixed per-slice choice by
//       the 80 % rule with dense slice tables (Section 3.3.3).
#include <math.h>

#include <algorithm>
#include <vector>

#include "cg_index.h"
#include "cg_query.cuh"
#include "cg_sort.cuh"

namespace cg {
namespace {

constexpr int kThreads = 256;

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

__device__ __forceinline__ int tile_of_point(const Tile* tiles, int ntiles, uint32_t p) {
  int a = 0, b = ntiles - 1;
  while (a < b) {
    int m = (a + b + 1) >> 1;
    if (tiles[m].pt_base <= p) a = m; else b = m - 1;
  }
  return a;
}

// --- B0: bounding box ------------------------------------------------------

// bb[t*6 + a] = min ord, bb[t*6 + 3 + a] = max ord
__global__ void bbox_init_kernel(unsigned long long* bb, int ntiles) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < ntiles * 6) bb[i] = (i % 6) < 3 ? ~0ull : 0ull;
}

constexpr int kBoxItems = 8;

// Coordinates are reduced as their order-preserving 64-bit images
// (dbl_to_ord): integer minima and maxima run on the ALU pipe, binary64
// ones would run on the narrow FP64 pipe.
__device__ __forceinline__ unsigned long long ord_bits(unsigned long long u) {
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ bool finite_bits(unsigned long long u) { return ((u >> 52) & 0x7ffull) != 0x7ffull; }

// Block-wide min / max of the running box, merged into tile t's entry.
__device__ __forceinline__ void bbox_flush(unsigned long long (&mn)[3], unsigned long long (&mx)[3], int t,
                                           unsigned long long* bb, unsigned long long (*s_red)[kThreads / 32]) {
  for (int a = 0; a < 3; ++a) {
    for (int o = 16; o > 0; o >>= 1) {
      mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
      mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
    }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 3; ++a) { s_red[a][w] = mn[a]; s_red[3 + a][w] = mx[a]; }
  __syncthreads();
  if (threadIdx.x < 6) {
    const int a = threadIdx.x;
    unsigned long long r = s_red[a][0];
    for (int k = 1; k < kThreads / 32; ++k) r = a < 3 ? min(r, s_red[a][k]) : max(r, s_red[a][k]);
    if (a < 3) atomicMin(bb + 6 * t + a, r);
    else atomicMax(bb + 6 * t + a, r);
  }
  __syncthreads();
  for (int a = 0; a < 3; ++a) { mn[a] = ~0ull; mx[a] = 0ull; }
}

// Persistent grid over chunks of kThreads * kBoxItems points: a block keeps
// one running box while its chunks stay in one tile and merges it into the
// tile's entry when the tile changes and at the end; a chunk that straddles
// tiles merges point by point.
__global__ void __launch_bounds__(kThreads) bbox_kernel(const double* __restrict__ xyz, int64_t n,
                                                        const int64_t* __restrict__ toff,
                                                        int ntiles, unsigned long long* bb,
                                                        uint32_t* status) {
  __shared__ unsigned long long s_red[6][kThreads / 32];
  __shared__ int s_t0, s_t1;
  constexpr int64_t kChunk = (int64_t)kThreads * kBoxItems;
  const int64_t nchunks = (n + kChunk - 1) / kChunk;
  const unsigned long long* __restrict__ xb = reinterpret_cast<const unsigned long long*>(xyz);
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  int cur = -1;  // tile of the running box (block-uniform)
  bool bad = false;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t base = c * kChunk;
    const int64_t last = min(base + kChunk, n) - 1;
    if (threadIdx.x == 0) {
      // tiles of the first and last point of this chunk
      int a = 0, b = ntiles - 1;
      while (a < b) { int m = (a + b + 1) >> 1; if (toff[m] <= base) a = m; else b = m - 1; }
      s_t0 = a;
      a = 0; b = ntiles - 1;
      while (a < b) { int m = (a + b + 1) >> 1; if (toff[m] <= last) a = m; else b = m - 1; }
      s_t1 = a;
    }
    __syncthreads();
    const int t0 = s_t0, t1 = s_t1;
    __syncthreads();  // s_t0 / s_t1 are rewritten for the next chunk
    const bool uniform = t0 == t1;
    if (uniform && t0 != cur) {
      if (cur >= 0) bbox_flush(mn, mx, cur, bb, s_red);
      cur = t0;
    }
    // every load of the thread first (all in flight), then the reductions
    unsigned long long v[kBoxItems][3];
#pragma unroll
    for (int j = 0; j < kBoxItems; ++j) {
      const int64_t p = base + (int64_t)j * kThreads + threadIdx.x;
#pragma unroll
      for (int a = 0; a < 3; ++a) v[j][a] = p < n ? __ldg(xb + 3 * p + a) : 0ull;
    }
#pragma unroll
    for (int j = 0; j < kBoxItems; ++j) {
      const int64_t p = base + (int64_t)j * kThreads + threadIdx.x;
      if (p >= n) break;
      bad |= !(finite_bits(v[j][0]) && finite_bits(v[j][1]) && finite_bits(v[j][2]));
      if (uniform) {
        for (int a = 0; a < 3; ++a) {
          const unsigned long long o = ord_bits(v[j][a]);
          mn[a] = min(mn[a], o);
          mx[a] = max(mx[a], o);
        }
      } else {
        int a = t0, b = t1;
        while (a < b) { int m = (a + b + 1) >> 1; if (toff[m] <= p) a = m; else b = m - 1; }
        for (int ax = 0; ax < 3; ++ax) {
          atomicMin(bb + 6 * a + ax, ord_bits(v[j][ax]));
          atomicMax(bb + 6 * a + 3 + ax, ord_bits(v[j][ax]));
        }
      }
    }
  }
  if (bad) atomicOr(status, ST_NONFINITE);
  if (cur >= 0) bbox_flush(mn, mx, cur, bb, s_red);
}

// Grid of bbox_kernel: a few resident blocks per SM.
unsigned bbox_grid(int64_t n) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  const int64_t chunks = (n + (int64_t)kThreads * kBoxItems - 1) / ((int64_t)kThreads * kBoxItems);
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(chunks, 4 * (int64_t)sms));
}

// --- B1: keys --------------------------------------------------------------

// floor(fl64(d / s)) without a binary64 division in the common case: a
// binary32 estimate decides whenever it is farther than its error bound
// from an integer; otherwise the exact binary64 quotient is taken.
__device__ __forceinline__ int voxel_floor(double d, double s, float inv_sf) {
  float qf = __fmul_rn(__double2float_rn(d), inv_sf);
  float fl = floorf(qf);
  float margin = __fmaf_rn(fabsf(qf), 4.0e-7f, 1.0e-6f);
  if (fabsf(qf) < 4194304.0f && __fsub_rn(qf, fl) > margin && __fsub_rn(__fadd_rn(fl, 1.0f), qf) > margin)
    return (int)fl;
  return (int)floor(__ddiv_rn(d, s));
}

__global__ void __launch_bounds__(kThreads) key_kernel(const double* __restrict__ xyz, int64_t n,
                                                       const Tile* __restrict__ tiles, int ntiles,
                                                       int dim, uint32_t* __restrict__ keys) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
       p += (int64_t)gridDim.x * blockDim.x) {
    const Tile& t = tiles[ntiles == 1 ? 0 : tile_of_point(tiles, ntiles, (uint32_t)p)];
    int c[3];
    for (int a = 0; a < dim; ++a) {
      double d = __dsub_rn(xyz[3 * p + a], t.lo[a]);
      int v = voxel_floor(d, t.s[a], t.inv_sf[a]);
      c[a] = min(max(v, 0), t.n[a] - 1);  // indexed points are in range by construction
    }
    uint32_t g = dim == 2 ? (uint32_t)c[0] * (uint32_t)t.n[1] + (uint32_t)c[1]
                          : ((uint32_t)c[0] * (uint32_t)t.n[1] + (uint32_t)c[1]) * (uint32_t)t.n[2] +
                                (uint32_t)c[2];
    keys[p] = t.key_base + g;
  }
}

// --- B4: gather, runs, tables -----------------------------------------------

__global__ void __launch_bounds__(kThreads) gather_kernel(
    const double* __restrict__ xyz, int64_t n, const uint32_t* __restrict__ perm,
    const uint32_t* __restrict__ skeys, const Tile* __restrict__ tiles, int ntiles,
    float4* __restrict__ pts32, double4_32a* __restrict__ pts64s) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t id = perm[i];
    double x = xyz[3 * (size_t)id], y = xyz[3 * (size_t)id + 1], z = xyz[3 * (size_t)id + 2];
    if (pts32) {
      const Tile& t = tiles[ntiles == 1 ? 0 : tile_of_key(tiles, ntiles, skeys[i])];
      float4 r;
      r.x = __double2float_rn(__dsub_rn(x, t.origin[0]));
      r.y = __double2float_rn(__dsub_rn(y, t.origin[1]));
      r.z = __double2float_rn(__dsub_rn(z, t.origin[2]));
      r.w = __uint_as_float(id);
      pts32[i] = r;
    }
    if (pts64s) pts64s[i] = make_double4_32a(x, y, z, __longlong_as_double((long long)id));
  }
}

__global__ void run_flag_kernel(const uint32_t* __restrict__ skeys, int64_t n,
                                uint32_t* __restrict__ flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || skeys[i] != skeys[i - 1]) ? 1u : 0u;
}

// runs: ukeys[r] = key, ustart[r] = first sorted position; ustart[m] = n
__global__ void run_emit_kernel(const uint32_t* __restrict__ skeys, int64_t n,
                                const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                                uint32_t* __restrict__ ukeys, uint32_t* __restrict__ ustart, uint32_t cap) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (flag[i]) {
      uint32_t r = rank[i];
      if (r < cap) {  // a replay whose data grew more runs is flagged, never overruns
        ukeys[r] = skeys[i];
        ustart[r] = (uint32_t)i;
      }
    }
    if (i == n - 1 && rank[n] <= cap) ustart[rank[n]] = (uint32_t)n;
  }
}

// --- replay support -------------------------------------------------------

// Recomputes every tile's box, origin and error bounds from the reduced
// bounding boxes (the host formulas of build_index, in binary64 without
// contraction); a grid size that differs from the captured one flags a
// re-plan instead of changing the key layout.
__global__ void tiles_refresh_kernel(Tile* tiles, int ntiles, const unsigned long long* __restrict__ bb, int dim,
                                     uint32_t* status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  Tile& T = tiles[t];
  double M = 0.0, ext = 0.0;
  int64_t nmax = 1;
  bool same = true;
  for (int a = 0; a < 3; ++a) {
    const double lo = ord_to_dbl(bb[6 * t + a]), hi = ord_to_dbl(bb[6 * t + 3 + a]);
    const double w = __dsub_rn(hi, lo);
    int64_t na = (int64_t)floor(__ddiv_rn(w, T.s[a])) + 1;
    if (dim == 2 && a == 2) na = 1;
    same &= na == (int64_t)T.n[a];
    nmax = max(nmax, na);
    T.lo[a] = lo;
    T.hi[a] = hi;
    const double o = __dadd_rn(lo, __dmul_rn(0.5, w));
    T.origin[a] = o;
    M = fmax(M, fmax(fabs(__dsub_rn(hi, o)), fabs(__dsub_rn(o, lo))));
    T.D[a] = __double2float_rn(__dsub_rn(o, lo));
    ext = fmax(ext, w);
  }
  M = __dmul_rn(M, 1.0 + 1e-12);
  const double enc = __dadd_rn(__dmul_rn(ldexp(M, -24), 1.0 + 1e-6), ldexp(M, -52));
  T.enc_err = __double2float_ru(enc);
  const double smin = fmin(T.s[0], fmin(T.s[1], T.s[2]));
  T.eta = __double2float_ru(4.0 * ((enc + ldexp(3.0 * ext + 2.0 * M, -24)) / smin + ldexp((double)nmax + 2.0, -22)) + 1e-6);
  if (!same) atomicOr(status, ST_REPLAN);
}

__global__ void voxel_count_dev_kernel(const uint32_t* __restrict__ ukeys, const uint32_t* __restrict__ ustart,
                                       const uint32_t* __restrict__ m_dev, uint32_t cap, uint32_t* __restrict__ cnt) {
  const uint32_t m = min(*m_dev, cap);
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
    cnt[ukeys[r]] = ustart[r + 1] - ustart[r];
}

__global__ void voxel_count_kernel(const uint32_t* __restrict__ ukeys,
                                   const uint32_t* __restrict__ ustart, uint32_t m,
                                   uint32_t* __restrict__ cnt) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
    cnt[ukeys[r]] = ustart[r + 1] - ustart[r];
}

__global__ void max_run_kernel(const uint32_t* __restrict__ ustart, uint32_t m, uint32_t* out) {
  uint32_t best = 0;
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
    best = max(best, ustart[r + 1] - ustart[r]);
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, best);
}

__global__ void hash_insert_kernel(const uint32_t* __restrict__ ukeys, uint32_t m,
                                   unsigned long long* table, uint32_t mask, uint32_t* status) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    uint32_t key = ukeys[r];
    unsigned long long e = ((unsigned long long)key << 32) | r;
    uint32_t h = (uint32_t)fmix64(key) & mask;
    bool done = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
      unsigned long long prev = atomicCAS(table + h, kHashEmpty, e);
      if (prev == kHashEmpty) { done = true; break; }
      h = (h + 1) & mask;
    }
    if (!done) atomicOr(status, ST_INTERNAL);
  }
}

// mixed: non-empty voxels per (tile, slice)
__global__ void slice_count_kernel(const uint32_t* __restrict__ ukeys, uint32_t m,
                                   const Tile* __restrict__ tiles, int ntiles, int dim,
                                   uint32_t* __restrict__ ne) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    uint32_t key = ukeys[r];
    const Tile& t = tiles[ntiles == 1 ? 0 : tile_of_key(tiles, ntiles, key)];
    uint32_t g = key - t.key_base;
    uint32_t sl = dim == 3 ? g % (uint32_t)t.n[2] : 0u;
    atomicAdd(ne + t.slice_base + sl, 1u);
  }
}

__global__ void mixed_fill_kernel(const uint32_t* __restrict__ ukeys,
                                  const uint32_t* __restrict__ ustart, uint32_t m,
                                  const Tile* __restrict__ tiles, int ntiles, int dim,
                                  const uint8_t* __restrict__ sdense,
                                  const uint32_t* __restrict__ soff, uint2* __restrict__ mtab) {
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
    uint32_t key = ukeys[r];
    const Tile& t = tiles[ntiles == 1 ? 0 : tile_of_key(tiles, ntiles, key)];
    uint32_t g = key - t.key_base;
    uint32_t sl = dim == 3 ? g % (uint32_t)t.n[2] : 0u;
    uint32_t gs = t.slice_base + sl;
    if (sdense[gs]) {
      uint32_t local = dim == 3 ? g / (uint32_t)t.n[2] : g;
      mtab[soff[gs] + local] = make_uint2(ustart[r], ustart[r + 1]);
    }
  }
}

uint32_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return (uint32_t)p;
}

}  // namespace

cg_status build_index(const double* xyz, int64_t n, const int64_t* toff_host, int ntiles,
                      const double* cell_xy, const double* cell_z, int dim, int flavor,
                      int precision, cudaStream_t st, cg_index** out) {
  cudaError_t e;
  cg_index* ix = new cg_index();
  ix->dim = dim;
  ix->flavor = flavor;
  ix->precision = precision;
  ix->ntiles = ntiles;
  ix->n = n;
  ix->stream = st;
  DevBufs tmp;
  auto bail = [&](cg_status s, const std::string& m) {
    tmp.release(st);
    ix->bufs.release(st);
    delete ix;
    return fail(s, m);
  };
#define CG_ALLOC(dst, T, count, owner)                                       \
  do {                                                                       \
    dst = (T*)(owner).get(sizeof(T) * (size_t)(count), st);                  \
    if (!dst) return bail(CG_ERR_OOM, "device allocation failed (" #dst ")"); \
  } while (0)
#define CG_CUDA(call)                                                             \
  do {                                                                            \
    e = (call);                                                                   \
    if (e != cudaSuccess) return bail(CG_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e)); \
  } while (0)

  CG_ALLOC(ix->status, uint32_t, 64, ix->bufs);
  ix->ctx.status = ix->status;
  ix->scratch_u32 = ix->status + 16;
  CG_CUDA(cudaMemsetAsync(ix->status, 0, 64 * 4, st));

  // B0: bounding boxes
  int64_t* toff_dev;
  unsigned long long* bb;
  CG_ALLOC(toff_dev, int64_t, ntiles + 1, tmp);
  CG_ALLOC(bb, unsigned long long, 6 * ntiles, tmp);
  CG_CUDA(host_put(toff_dev, toff_host, sizeof(int64_t) * (ntiles + 1), st));
  bbox_init_kernel<<<(6 * ntiles + 255) / 256, 256, 0, st>>>(bb, ntiles); note_launch();
  {
    ProfScope prof("build_bbox", st);
    bbox_kernel<<<bbox_grid(n), kThreads, 0, st>>>(xyz, n, toff_dev, ntiles, bb, ix->status); note_launch();
  }
  CG_CUDA(cudaGetLastError());
  std::vector<unsigned long long> bbh(6 * ntiles);
  uint32_t st_word = 0;
  HostRead rd;
  rd.get(bbh.data(), bb, 8 * 6 * ntiles);
  rd.get(&st_word, ix->status, 4);
  CG_CUDA(rd.sync(st));
  if (st_word & ST_NONFINITE) return bail(CG_ERR_INVALID, "non-finite point coordinate");

  // grid of every tile (host, binary64; Eq. grid-size)
  ix->tiles_host.resize(ntiles);
  uint64_t key_base = 0, slice_base = 0;
  for (int t = 0; t < ntiles; ++t) {
    Tile& T = ix->tiles_host[t];
    memset(&T, 0, sizeof(Tile));
    double s[3] = {cell_xy[t], cell_xy[t], cell_z[t]};
    double M = 0;
    int64_t nmax = 1;
    for (int a = 0; a < 3; ++a) {
      T.lo[a] = ord_to_dbl(bbh[6 * t + a]);
      T.hi[a] = ord_to_dbl(bbh[6 * t + 3 + a]);
      T.s[a] = s[a];
      int64_t na = (int64_t)floor((T.hi[a] - T.lo[a]) / s[a]) + 1;
      if (dim == 2 && a == 2) na = 1;
      if (na < 1 || na > (int64_t)0x7fffffff) return bail(CG_ERR_INVALID, "grid axis too large");
      T.n[a] = (int32_t)na;
      nmax = std::max(nmax, na);
      T.origin[a] = T.lo[a] + 0.5 * (T.hi[a] - T.lo[a]);
      M = std::max(M, std::max(fabs(T.hi[a] - T.origin[a]), fabs(T.origin[a] - T.lo[a])));
      T.D[a] = (float)(T.origin[a] - T.lo[a]);
      T.inv_sf[a] = (float)(1.0 / s[a]);
    }
    M *= 1.0 + 1e-12;
    // |fl32(a) - a| <= 2^-24 |a| for |a| <= M, plus the binary64 rounding of p - O
    T.enc_err = (float)(ldexp(M, -24) * (1.0 + 1e-6) + ldexp(M, -52));
    // padding (voxel units) of binary32 voxel coordinates u = (x~ + D) / s:
    // encode error, rounding of D, of the sum and of the product, and of the
    // binary64 key itself; a factor 4 of headroom
    double smin = std::min(s[0], std::min(s[1], s[2]));
    double ext = 0;
    for (int a = 0; a < 3; ++a) ext = std::max(ext, T.hi[a] - T.lo[a]);
    T.eta = (float)(4.0 * ((T.enc_err + ldexp(3.0 * ext + 2.0 * M, -24)) / smin +
                           ldexp((double)nmax + 2.0, -22)) + 1e-6);
    uint64_t cells = (uint64_t)T.n[0] * (uint64_t)T.n[1] * (uint64_t)T.n[2];
    T.key_base = (uint32_t)key_base;
    key_base += cells;
    if (key_base > 0xfffffffdull) return bail(CG_ERR_INVALID, "more than 2^32-2 voxels in the grid");
    T.pt_base = (uint32_t)toff_host[t];
    T.pt_count = (uint32_t)(toff_host[t + 1] - toff_host[t]);
    T.nslices = (flavor == CG_MIXED && dim == 3) ? (uint32_t)T.n[2] : 1u;
    T.slice_base = (uint32_t)slice_base;
    slice_base += T.nslices;
  }
  ix->ncell = (int64_t)key_base;
  ix->nslices = (int64_t)slice_base;
  ix->enc_err0 = ix->tiles_host[0].enc_err;
  CG_ALLOC(ix->tiles, Tile, ntiles, ix->bufs);
  CG_CUDA(host_put(ix->tiles, ix->tiles_host.data(), sizeof(Tile) * ntiles, st));

  // B1: keys
  uint32_t *keys, *skeys, *perm;
  CG_ALLOC(keys, uint32_t, n, tmp);
  CG_ALLOC(skeys, uint32_t, n, tmp);
  CG_ALLOC(perm, uint32_t, n, ix->bufs);  // kept: original id of every sorted position
  ix->sid = perm;
  {
    ProfScope prof("build_keys", st);
    key_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(xyz, n, ix->tiles, ntiles, dim, keys); note_launch();
  }
  CG_CUDA(cudaGetLastError());

  // B3: stable radix sort of (key, id)
  int bits = 0;
  while (bits < 32 && ((uint64_t)1 << bits) < key_base) ++bits;
  void* sort_scratch;
  CG_ALLOC(sort_scratch, char, radix_sort_scratch_bytes(n), tmp);
  {
    ProfScope prof("build_sort", st);
    CG_CUDA(radix_sort_pairs(keys, n, bits, skeys, perm, sort_scratch, ix->status, st));
  }

  // B4: records and the exact binary64 copy in original order
  CG_ALLOC(ix->xyz64, double, 3 * n, ix->bufs);
  CG_CUDA(dev_copy(ix->xyz64, xyz, sizeof(double) * 3 * n, st));
  if (precision == CG_FP32_OFFSET) CG_ALLOC(ix->pts32, float4, n, ix->bufs);
  else CG_ALLOC(ix->pts64s, double4_32a, n, ix->bufs);
  {
    ProfScope prof("build_gather", st);
    gather_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(xyz, n, perm, skeys, ix->tiles, ntiles,
                                                               ix->pts32, ix->pts64s); note_launch();
  }
  CG_CUDA(cudaGetLastError());

  // runs of equal keys: the sorted unique-key table
  uint32_t *flag, *rank;
  CG_ALLOC(flag, uint32_t, n, tmp);
  CG_ALLOC(rank, uint32_t, n + 1, tmp);
  void* scan_scratch;
  CG_ALLOC(scan_scratch, char, scan_scratch_bytes(std::max<int64_t>(n, key_base + 1)), tmp);
  {
    ProfScope prof("build_runs", st);
    run_flag_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(skeys, n, flag); note_launch();
    CG_CUDA(exclusive_scan_u32_u32(flag, rank, n, scan_scratch, ix->status, st));
  }
  uint32_t m = 0;
  rd.get(&m, rank + n, 4);
  CG_CUDA(rd.sync(st));
  ix->nkeys = m;
  CG_ALLOC(ix->ukeys, uint32_t, m, ix->bufs);
  CG_ALLOC(ix->ustart, uint32_t, m + 1, ix->bufs);
  run_emit_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(skeys, n, flag, rank, ix->ukeys, ix->ustart, m); note_launch();
  CG_CUDA(cudaGetLastError());
  CG_CUDA(cudaMemsetAsync(ix->scratch_u32, 0, 4, st));
  max_run_kernel<<<grid_for(m, kThreads, 152 * 4), kThreads, 0, st>>>(ix->ustart, m, ix->scratch_u32); note_launch();
  if (precision == CG_FP32_OFFSET && dim == 2) {
    // every voxel run again, sorted by height (the radius kernels' z windows)
    uint32_t* zlong;
    CG_ALLOC(ix->pts32z, float4, n, ix->bufs);
    CG_ALLOC(ix->sidz, uint32_t, n, ix->bufs);
    CG_ALLOC(zlong, uint32_t, m + 1, tmp);
    CG_CUDA(launch_zsort(ix->pts32, ix->pts32z, ix->sidz, ix->ustart, m, nullptr, (uint32_t)n, zlong, zlong + m,
                         ix->status, st));
  }

  if (flavor == CG_DENSE) {
    uint32_t* cnt;
    CG_ALLOC(cnt, uint32_t, key_base, tmp);
    CG_ALLOC(ix->cstart, uint32_t, key_base + 1, ix->bufs);
    ProfScope prof("build_cells", st);
    CG_CUDA(cudaMemsetAsync(cnt, 0, 4 * key_base, st));
    voxel_count_kernel<<<grid_for(m, kThreads), kThreads, 0, st>>>(ix->ukeys, ix->ustart, m, cnt); note_launch();
    CG_CUDA(exclusive_scan_u32_u32(cnt, ix->cstart, (int64_t)key_base, scan_scratch, ix->status, st));
    ix->dense_slices = ntiles;
  } else {
    uint32_t cap = next_pow2(std::max<uint64_t>(64, 2ull * m));
    ix->hash_mask = cap - 1;
    CG_ALLOC(ix->hash, unsigned long long, cap, ix->bufs);
    CG_CUDA(cudaMemsetAsync(ix->hash, 0xff, 8ull * cap, st));
    hash_insert_kernel<<<grid_for(m, kThreads), kThreads, 0, st>>>(ix->ukeys, m, ix->hash, ix->hash_mask,
                                                                   ix->status); note_launch();
    CG_CUDA(cudaGetLastError());
    if (flavor == CG_MIXED) {
      uint32_t* ne;
      CG_ALLOC(ne, uint32_t, slice_base, tmp);
      CG_CUDA(cudaMemsetAsync(ne, 0, 4 * slice_base, st));
      slice_count_kernel<<<grid_for(m, kThreads), kThreads, 0, st>>>(ix->ukeys, m, ix->tiles, ntiles, dim, ne); note_launch();
      std::vector<uint32_t> neh(slice_base);
      rd.get(neh.data(), ne, 4 * slice_base);
      CG_CUDA(rd.sync(st));
      std::vector<uint8_t> dense(slice_base);
      std::vector<uint32_t> off(slice_base);
      uint64_t tab = 0;
      for (int t = 0; t < ntiles; ++t) {
        const Tile& T = ix->tiles_host[t];
        uint64_t per = (uint64_t)T.n[0] * T.n[1] * T.n[2] / T.nslices;
        for (uint32_t sl = 0; sl < T.nslices; ++sl) {
          uint32_t gs = T.slice_base + sl;
          dense[gs] = (5ull * neh[gs] >= 4ull * per) ? 1 : 0;  // the 80 % rule
          off[gs] = (uint32_t)tab;
          if (dense[gs]) { tab += per; ix->dense_slices++; }
        }
      }
      if (tab > 0xffffffffull) return bail(CG_ERR_INVALID, "mixed dense slices too large");
      CG_ALLOC(ix->slice_dense, uint8_t, slice_base, ix->bufs);
      CG_ALLOC(ix->slice_tab_off, uint32_t, slice_base, ix->bufs);
      CG_ALLOC(ix->mtab, uint2, std::max<uint64_t>(tab, 1), ix->bufs);
      CG_CUDA(host_put(ix->slice_dense, dense.data(), slice_base, st));
      CG_CUDA(host_put(ix->slice_tab_off, off.data(), 4 * slice_base, st));
      CG_CUDA(cudaMemsetAsync(ix->mtab, 0, 8 * std::max<uint64_t>(tab, 1), st));
      mixed_fill_kernel<<<grid_for(m, kThreads), kThreads, 0, st>>>(ix->ukeys, ix->ustart, m, ix->tiles,
                                                                    ntiles, dim, ix->slice_dense,
                                                                    ix->slice_tab_off, ix->mtab); note_launch();
      CG_CUDA(cudaGetLastError());
    }
  }
  uint32_t maxrun = 0;
  rd.get(&maxrun, ix->scratch_u32, 4);
  rd.get(&st_word, ix->status, 4);
  tmp.release(st);
  CG_CUDA(rd.sync(st));
  ix->max_pts_per_voxel = (int)maxrun;
  if (st_word & ST_TIMEOUT) return bail(CG_ERR_TIMEOUT, "device wait bound reached during build");
  if (st_word & ST_INTERNAL) return bail(CG_ERR_INTERNAL, "hash table insertion failed");
  *out = ix;
  return CG_OK;
#undef CG_ALLOC
#undef CG_CUDA
}


// Buffers a replayed build needs besides the index's own (kept for the
// lifetime of a captured pipeline).
cg_status build_work_alloc(cg_index* ix, BuildWork& w, cudaStream_t st) {
  const int64_t n = ix->n;
  w.keys = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.skeys = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.flag = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.rank = (uint32_t*)w.bufs.get(4 * (size_t)(n + 1), st);
  w.cnt = (uint32_t*)w.bufs.get(4 * (size_t)std::max<int64_t>(ix->ncell, 1), st);
  w.sort_scr = w.bufs.get(radix_sort_scratch_bytes(n), st);
  w.scan_scr = w.bufs.get(scan_scratch_bytes(std::max<int64_t>(n, ix->ncell + 1)), st);
  w.bb = (unsigned long long*)w.bufs.get(8 * 6 * (size_t)ix->ntiles, st);
  w.toff = (int64_t*)w.bufs.get(8 * (size_t)(ix->ntiles + 1), st);
  // voxel runs: room for every possible non-empty voxel, so that new data
  // of the same tile sizes never needs a larger table
  w.cap_keys = (uint32_t)std::min<int64_t>(n, ix->ncell);
  w.ukeys = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_keys, st);
  w.ustart = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_keys + 4, st);
  if (ix->pts32z) w.zlong = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_keys + 4, st);
  if (!w.keys || !w.skeys || !w.flag || !w.rank || !w.cnt || !w.sort_scr || !w.scan_scr || !w.bb || !w.toff ||
      !w.ukeys || !w.ustart || (ix->pts32z && !w.zlong))
    return fail(CG_ERR_OOM, "device allocation failed (pipeline build work)");
  std::vector<int64_t> toff(ix->ntiles + 1);
  for (int t = 0; t < ix->ntiles; ++t) toff[t] = ix->tiles_host[t].pt_base;
  toff[ix->ntiles] = n;
  cudaError_t e = host_put(w.toff, toff.data(), 8 * toff.size(), st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline build work");
  int bits = 0;
  while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)ix->ncell) ++bits;
  w.bits = bits;
  w.nkeys_dev = w.rank + n;
  // the index now reads its runs from the pipeline's tables
  ix->ukeys = w.ukeys;
  ix->ustart = w.ustart;
  return CG_OK;
}

// The dense build again, into the index's existing buffers, with no host
// synchronisation and no allocation (so it can be captured in a graph).
cg_status build_replay(cg_index* ix, BuildWork& w, const double* xyz, cudaStream_t st) {
  if (ix->flavor != CG_DENSE) return fail(CG_ERR_UNIMPLEMENTED, "pipeline replay needs the dense flavour");
  const int64_t n = ix->n;
  const int T = ix->ntiles;
  cudaError_t e;
  bbox_init_kernel<<<(6 * T + 255) / 256, 256, 0, st>>>(w.bb, T); note_launch();
  {
    bbox_kernel<<<bbox_grid(n), kThreads, 0, st>>>(xyz, n, w.toff, T, w.bb, ix->status); note_launch();
  }
  tiles_refresh_kernel<<<(T + 127) / 128, 128, 0, st>>>(ix->tiles, T, w.bb, ix->dim, ix->status); note_launch();
  key_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(xyz, n, ix->tiles, T, ix->dim, w.keys); note_launch();
  e = radix_sort_pairs(w.keys, n, w.bits, w.skeys, ix->sid, w.sort_scr, ix->status, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay sort");
  gather_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(xyz, n, ix->sid, w.skeys, ix->tiles, T, ix->pts32,
                                                             ix->pts64s); note_launch();
  if (ix->xyz64 != xyz) {  // a pipeline reads the caller's buffer in place
    e = dev_copy(ix->xyz64, xyz, sizeof(double) * 3 * n, st);
    if (e != cudaSuccess) return cuda_fail(e, "replay copy");
  }
  run_flag_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(w.skeys, n, w.flag); note_launch();
  e = exclusive_scan_u32_u32(w.flag, w.rank, n, w.scan_scr, ix->status, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay scan");
  run_emit_kernel<<<grid_for(n, kThreads), kThreads, 0, st>>>(w.skeys, n, w.flag, w.rank, ix->ukeys, ix->ustart,
                                                               w.cap_keys); note_launch();
  if (ix->pts32z) {
    e = launch_zsort(ix->pts32, ix->pts32z, ix->sidz, ix->ustart, w.cap_keys, w.nkeys_dev, (uint32_t)n, w.zlong,
                     w.zlong + w.cap_keys, ix->status, st);
    if (e != cudaSuccess) return cuda_fail(e, "replay height sort");
  }
  e = cudaMemsetAsync(w.cnt, 0, 4 * (size_t)ix->ncell, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay memset");
  voxel_count_dev_kernel<<<grid_for(w.cap_keys, kThreads), kThreads, 0, st>>>(ix->ukeys, ix->ustart, w.nkeys_dev,
                                                                              w.cap_keys, w.cnt); note_launch();
  e = exclusive_scan_u32_u32(w.cnt, ix->cstart, ix->ncell, w.scan_scr, ix->status, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay cell starts");
  return CG_OK;
}

}  // namespace cg
