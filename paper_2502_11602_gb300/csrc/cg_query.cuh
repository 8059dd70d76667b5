// cg_query.cuh -- query-side structures shared by the radius and k-NN
// kernels (internal).
#pragma once
#include <math.h>

#include "cg_index.h"

namespace cg {

// Decision thresholds of the binary32 path (see make_thresholds).
struct Thresholds {
  double r2;      // fl64(r * r)
  float s_lo;     // sphere: binary32 value <= s_lo  -> inside for sure
  float s_hi;     // sphere: binary32 value >  s_hi  -> outside for sure
  float c_lo;     // cube, per axis
  float c_hi;
  float r_f;      // r rounded up to binary32
  float e_q;      // encode error bound of the queries used here
  float pad_[2];
};

namespace {
__host__ __device__ inline float f_down(double x) {
#ifdef __CUDA_ARCH__
  return __double2float_rd(x);
#else
  float f = (float)x;
  if ((double)f > x) f = nextafterf(f, -INFINITY);
  return f;
#endif
}
__host__ __device__ inline float f_up(double x) {
#ifdef __CUDA_ARCH__
  return __double2float_ru(x);
#else
  float f = (float)x;
  if ((double)f < x) f = nextafterf(f, INFINITY);
  return f;
#endif
}
}  // namespace

// Binary32 offset test, error model.  Per axis the binary32 difference
// dxf = fl32(x~_p - x~_c) and the exact dx = fl64(p - c) satisfy
//   |dxf - dx| <= alpha + beta |dx|,  alpha = (e_p + e_q)(1 + u),
//   beta = (u + U)(1 + 2U),  u = 2^-24, U = 2^-53,
// where e_p, e_q bound |x~ - (x - O)| (binary32 rounding of the offset plus
// the binary64 rounding of x - O).  With S = sum dx^2 and Sf = sum dxf^2:
//   |Sf - S| <= c1 sqrt(S) + c0 + c2 S,  c1 = 2 alpha (1 + beta) sqrt(3),
//   c0 = 3 alpha^2, c2 = 2 beta + beta^2 (Cauchy-Schwarz on the three axes).
// The binary32 value d2f is within 3.0000002 u Sf of Sf (three roundings) and
// the binary64 value d2 within 3.0000001 U S of S.  Hence
//   d2f <= T_lo  =>  d2 <= r2     T_lo = (S_in (1 - c2) - c1 sqrt(S_in) - c0)(1 - 3.0000002u)
//   d2f >  T_hi  =>  d2 >  r2     T_hi = (S_mx (1 + c2) + c1 sqrt(S_mx) + c0)(1 + 3.0000002u)
// with S_in = r2 (1 - 4U), S_mx = r2 (1 + 4U); the margins are doubled for
// headroom.  The cube uses the same argument on each axis alone.
inline __host__ __device__ Thresholds make_thresholds(double r, double e_p, double e_q) {
  const double u = 5.9604644775390625e-08;   // 2^-24
  const double U = 1.1102230246251565e-16;   // 2^-53
  Thresholds t;
  t.r2 = r * r;
  const double r2 = t.r2;
  const double alpha = (e_p + e_q) * (1.0 + u);
  const double beta = (u + U) * (1.0 + 2.0 * U);
  const double c1 = 2.0 * alpha * (1.0 + beta) * 1.7320508075688774;
  const double c0 = 3.0 * alpha * alpha;
  const double c2 = 2.0 * beta + beta * beta;
  const double s_in = r2 * (1.0 - 4.0 * U);
  const double s_mx = r2 * (1.0 + 4.0 * U);
  double t_lo = (s_in * (1.0 - c2) - c1 * sqrt(s_in) - c0) * (1.0 - 3.0000002 * u);
  double t_hi = (s_mx * (1.0 + c2) + c1 * sqrt(s_mx) + c0) * (1.0 + 3.0000002 * u);
  t_lo = r2 - 2.0 * (r2 - t_lo);
  t_hi = r2 + 2.0 * (t_hi - r2);
  t.s_lo = t_lo > 0 ? f_down(t_lo) : -1.0f;
  t.s_hi = f_up(t_hi);
  // cube: one axis, |dx| <= r (1 + U) when fl64(dx^2) <= r2
  const double rin = sqrt(r2 * (1.0 - 2.0 * U)) * (1.0 - beta) - alpha;
  double c_lo = rin > 0 ? (1.0 - 1.0000001 * u) * rin * rin : -1.0;
  const double rmx = sqrt(r2 * (1.0 + 2.0 * U)) * (1.0 + beta) + alpha;
  double c_hi = (1.0 + 1.0000001 * u) * rmx * rmx;
  c_lo = r2 - 2.0 * (r2 - c_lo);
  c_hi = r2 + 2.0 * (c_hi - r2);
  t.c_lo = c_lo > 0 ? f_down(c_lo) : -1.0f;
  t.c_hi = f_up(c_hi);
  t.r_f = f_up(r);
  t.e_q = f_up(e_q);
  t.pad_[0] = t.pad_[1] = 0.f;
  return t;
}


// Queries of one call, in block order.
struct QuerySet {
  int all_points;              // queries are the indexed points
  uint32_t nq;
  uint32_t nblocks;
  const uint32_t* blk_beg;     // [nblocks+1] block start in query order
  const uint32_t* blk_key;     // [nblocks] voxel key of the block
  const float4* qrec;          // [nq] x~, y~, z~, id bits (binary32)
  const double4_32a* qrec64;       // [nq] x, y, z, id bits (binary64)
  const double* q64;           // [nq][3] original order, exact coordinates
  const uint32_t* blk_list = nullptr;    // optional subset of blocks to process
  const uint32_t* blk_list_n = nullptr;  // its length (device)
  // replayed pipelines: the true block count lives on the device and
  // nblocks is only its capacity
  const uint32_t* nblocks_dev = nullptr;
};

__device__ __forceinline__ uint32_t qs_nblocks(const QuerySet& qs) {
  return qs.nblocks_dev ? min(*qs.nblocks_dev, qs.nblocks) : qs.nblocks;
}

// Voxel runs up to this length are kept sorted by height in pts32z; longer
// runs keep id order there (searched whole by the z-window kernels).
constexpr uint32_t kZsortMax = 2048;

// Per voxel group: what the fast radius kernels need (see cg_radius2.cu).
constexpr int kPlanSpans = 32;  // non-empty voxel runs per group
struct BlockPlan {
  uint32_t q0, nq;       // queries [q0, q0 + nq) in query order
  uint32_t K;            // staged candidates (sum of span lengths)
  uint16_t nsp, W;       // spans, 32-bit mask words per query
  uint32_t heavy;        // 1: handled by the general CTA kernel
  uint32_t pad_[3];
  uint32_t start[kPlanSpans];
  uint32_t len[kPlanSpans];
};

// Fast radius kernels (cg_radius2.cu).
// zw: candidates come from the height-sorted columns, each column restricted
// to the group's height range widened by the kernel's half height and pad.
cudaError_t launch_radius_plan(int prec, int kern, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                               BlockPlan* plans, uint32_t* msize, uint32_t* isize, uint32_t* big_list,
                               uint32_t* big_n, const uint32_t* status, cudaStream_t st, bool zw = false,
                               unsigned long long* pairs = nullptr);
cudaError_t launch_radius_count2(int prec, int kern, const IndexView& iv, const QuerySet& qs,
                                 const Thresholds* thr, const BlockPlan* plans, const int64_t* moff,
                                 const int64_t* idoff, uint32_t* counts, uint32_t* masks, uint32_t* ids,
                                 unsigned* work, uint32_t* status, cudaStream_t st);
cudaError_t launch_radius_fill2(int prec, const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                const int64_t* moff, const int64_t* idoff, const uint32_t* masks,
                                const uint32_t* ids, const int64_t* offsets, int32_t* out, unsigned* work,
                                const uint32_t* status, cudaStream_t st);

// Binary32 records: warp-per-group count and fill for the two size classes.
cudaError_t launch_radius_count32(int kern, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                                  const BlockPlan* plans, const int64_t* moff, const int64_t* idoff,
                                  uint32_t* counts, uint32_t* masks, uint32_t* ids, unsigned* work,
                                  uint32_t* status, const cudaStream_t* sts, bool zspan = false);
cudaError_t launch_radius_fill32(const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                 const int64_t* moff, const int64_t* idoff, const uint32_t* masks,
                                 const uint32_t* ids, const int64_t* offsets, int32_t* out, unsigned* work,
                                 const uint32_t* status, const cudaStream_t* sts);

// Height order of the voxel columns and the height chunks of all-points
// radius passes (cg_zwin.cu): chunks span at most kRadiusChunkDz x r in
// height and hold at most kRadiusChunkMax queries (the fastest of 2, 4, 8
// and 16 x r and 128 - 512 queries on the 12M ALS tile at r = 1 m).
constexpr float kRadiusChunkDz = 8.0f;
constexpr uint32_t kRadiusChunkMax = 256;

// The process-wide launch tuning (cg_set_tuning; defaults above and shape 0).
cg_tuning_t default_tuning();
cg_tuning_t current_tuning();
void set_tuning(const cg_tuning_t& t);
// Height sort of every voxel run of `in` into `out` and the ids into
// `sid_out` (runs [ustart[i], ustart[i+1]) for i < min(*ndev, cap), or < cap
// when ndev is null; n points).
cudaError_t launch_zsort(const float4* in, float4* out, uint32_t* sid_out, const uint32_t* ustart, uint32_t cap,
                         const uint32_t* ndev, uint32_t n, uint32_t* long_list, uint32_t* long_n,
                         const uint32_t* status, cudaStream_t st);
// Chunks per run (cnt[nruns]), then, with coff = exclusive scan of cnt,
// every chunk's first position (cbeg[total + 1], cbeg[total] = n) and key.
cudaError_t launch_zchunk_count(const float4* pz, const uint32_t* ustart, uint32_t nruns, float dz, uint32_t qmax,
                                uint32_t* cnt, cudaStream_t st);
cudaError_t launch_zchunk_emit(const float4* pz, const uint32_t* ustart, const uint32_t* ukeys, uint32_t nruns,
                               float dz, uint32_t qmax, const uint32_t* coff, uint32_t* cbeg, uint32_t* ckey,
                               uint32_t n, cudaStream_t st);
// Whether a radius pass on this index and kernel uses the height-sorted
// columns (binary32 2D grids; sphere and cube, whose kernels are bounded in z).
inline bool zw_applies(const cg_index* ix, int kern) {
  return ix->pts32z != nullptr && ix->precision == CG_FP32_OFFSET && ix->dim == 2 &&
         (kern == CG_SPHERE || kern == CG_CUBE);
}

// Small query batches (cg_small.cu): one block per query, no plan.  Calls of
// up to kSmallBatch external queries take this path when their rows are at
// most kSmallRowCap long (checked by the count, which also writes the rows
// to a scratch buffer of kSmallRowCap entries per query; the fill copies).
constexpr int64_t kSmallBatch = 1024;
constexpr int kSmallRowCap = 2048;
// results the small count's last block copies itself (larger ones: a copy
// kernel, one block per query)
constexpr int64_t kSmallDirectMax = 4096;
constexpr uint32_t kSmallDirectQueries = 32;
cudaError_t launch_small_count(const IndexView& iv, const Tile& T, int kern, const double* q, uint32_t nq, double r,
                               uint32_t* counts, int32_t* rows, int64_t* offsets, uint32_t* stats,
                               uint32_t* status, unsigned long long* host_out, int32_t* direct_out,
                               int64_t direct_cap, cudaStream_t st);
cudaError_t launch_small_fill(const int32_t* rows, uint32_t nq, const int64_t* offsets, int32_t* out,
                              uint32_t* status, cudaStream_t st, int64_t cap = -1, const uint32_t* skip = nullptr);

QuerySet query_set(cg_index* ix, const double* q, int64_t nq, bool all_points);

// The sorted points of a voxel box [lo, hi] (one contiguous span per grid
// row of a 2D grid, per (i, j) column of a 3D grid), visited by a whole
// block of kBoxThreads threads: the spans of up to kBoxThreads rows or
// columns are looked up at once, then every thread takes candidates
// threadIdx.x, + kBoxThreads, ... of their concatenation, so that all the
// loads of a box are in flight together.  f(t, valid) is called by every
// thread the same number of times (valid false past the end), t the sorted
// position; s_start / s_off are kBoxThreads + 1 words of shared memory.
constexpr int kBoxThreads = 256;
template <class F>
__device__ __forceinline__ void for_each_in_box(const IndexView& ix, const Tile& T, const int* lo, const int* hi,
                                                uint32_t* s_start, uint32_t* s_off, F f) {
  const int nax = ix.dim;
  const int ni = hi[0] - lo[0] + 1, nj = hi[1] - lo[1] + 1;
  const int nsp = nax == 2 ? ni : ni * nj;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int b0 = 0; b0 < nsp; b0 += kBoxThreads) {
    const int nb = min(kBoxThreads, nsp - b0);
    __syncthreads();  // the previous batch's spans are no longer read
    uint32_t len = 0;
    if ((int)threadIdx.x < nb) {
      const int sidx = b0 + (int)threadIdx.x;
      uint32_t k0, k1;
      if (nax == 2) {
        const uint32_t row = (uint32_t)(lo[0] + sidx) * (uint32_t)T.n[1];
        k0 = T.key_base + row + (uint32_t)lo[1];
        k1 = T.key_base + row + (uint32_t)hi[1];
      } else {
        const int i = lo[0] + sidx / nj, j = lo[1] + sidx % nj;
        const uint32_t col = ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
        k0 = T.key_base + col + (uint32_t)lo[2];
        k1 = T.key_base + col + (uint32_t)hi[2];
      }
      const uint2 sp = row_span(ix, T, k0, k1);
      s_start[threadIdx.x] = sp.x;
      len = sp.y - sp.x;
    }
    // exclusive scan of the lengths over the block (s_off[nb] = total)
    uint32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_off[kBoxThreads - 1 - warp] = incl;  // warp totals, parked at the end
    __syncthreads();
    uint32_t wbase = 0, total = 0;
    for (uint32_t w = 0; w < kBoxThreads / 32; ++w) {
      const uint32_t x = s_off[kBoxThreads - 1 - w];
      wbase += w < warp ? x : 0u;
      total += x;
    }
    __syncthreads();
    if ((int)threadIdx.x < nb) s_off[threadIdx.x] = wbase + incl - len;
    if (threadIdx.x == 0) s_off[nb] = total;
    __syncthreads();
    for (uint32_t c0 = 0; c0 < total; c0 += kBoxThreads) {
      const uint32_t c = c0 + threadIdx.x;
      const bool valid = c < total;
      uint32_t t = 0;
      if (valid) {
        int a = 0, b = nb - 1;  // the span holding candidate c
        while (a < b) {
          const int m = (a + b + 1) >> 1;
          if (s_off[m] <= c) a = m;
          else b = m - 1;
        }
        t = s_start[a] + (c - s_off[a]);
      }
      f(t, valid);
    }
  }
}

}  // namespace cg
