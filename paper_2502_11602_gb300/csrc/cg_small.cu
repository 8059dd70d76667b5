// cg_small.cu -- radius search for small query batches: one block per query,
// no query plan.
//
// The regular path groups the queries by voxel (a sort of the queries, a plan
// per group, several host reads of sizes) so that a group's candidates are
// staged once for all of its queries.  For a call of a few hundred queries
// that set-up costs far more than the search.  Here a block of SW warps takes
// one query (its warps split the candidates, so that many loads are in
// flight) and runs Algorithm 1 for it as stated: the voxel range of the
// kernel's bounding box (widened by one voxel on each side, so that the
// rounding of the voxel keys can never hide a point), every point of those
// voxels tested with the exact binary64 predicate.  A voxel row (2D) or
// column (3D) of consecutive keys is one contiguous run of sorted points.
//
//   count  per query, the number of points inside; then one block scans the
//          counts into offsets and records the largest row.
//   fill   per query, the ids of the points inside, gathered in shared
//          memory, sorted ascending (bitonic, the whole block) and written
//          out; rows longer than the shared buffer are refused on the host
//          (the caller then takes the regular path).
#include <math.h>

#include <algorithm>

#include "cg_f32x2.cuh"
#include "cg_query.cuh"

namespace cg {
namespace {

constexpr int SW = 4;  // warps per block

// The voxel range of the kernel's box on axis a, from binary64 (the
// oracle's formula); false when it misses the grid.
__device__ __forceinline__ bool small_range(const Tile& T, int a, double c, double r, int& lo, int& hi) {
  const double l = floor(__ddiv_rn(__dsub_rn(__dsub_rn(c, r), T.lo[a]), T.s[a])) - 1.0;
  const double h = floor(__ddiv_rn(__dsub_rn(__dadd_rn(c, r), T.lo[a]), T.s[a])) + 1.0;
  if (h < 0.0 || l > (double)(T.n[a] - 1)) return false;
  lo = l < 0.0 ? 0 : (int)l;
  hi = h > (double)(T.n[a] - 1) ? T.n[a] - 1 : (int)h;
  return true;
}

// Calls f(t0, t1) for every contiguous run of sorted points the kernel of
// query c can reach (warp-uniform); returns false if a coordinate is not
// finite.
template <int KERN, class F>
__device__ __forceinline__ bool small_runs(const IndexView& ix, const double* c, double r, F f) {
  const Tile& T = ix.tiles[0];
  const double cx[3] = {__ldg(c), __ldg(c + 1), __ldg(c + 2)};
  if (!(isfinite(cx[0]) && isfinite(cx[1]) && isfinite(cx[2]))) return false;
  int lo[3], hi[3];
  for (int a = 0; a < 2; ++a)
    if (!small_range(T, a, cx[a], r, lo[a], hi[a])) return true;
  if (ix.dim == 3) {
    if (KERN == CG_CYLINDER) {  // z unbounded: every slice of the columns
      lo[2] = 0;
      hi[2] = T.n[2] - 1;
    } else if (!small_range(T, 2, cx[2], r, lo[2], hi[2])) {
      return true;
    }
  }
  for (int i = lo[0]; i <= hi[0]; ++i) {
    if (ix.dim == 2) {
      const uint32_t row = T.key_base + (uint32_t)i * (uint32_t)T.n[1];
      const uint2 sp = row_span(ix, T, row + (uint32_t)lo[1], row + (uint32_t)hi[1]);
      if (sp.y > sp.x) f(sp.x, sp.y);
    } else {
      for (int j = lo[1]; j <= hi[1]; ++j) {
        const uint32_t col = T.key_base + ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
        const uint2 sp = row_span(ix, T, col + (uint32_t)lo[2], col + (uint32_t)hi[2]);
        if (sp.y > sp.x) f(sp.x, sp.y);
      }
    }
  }
  return true;
}

__device__ __forceinline__ uint32_t small_id(const IndexView& ix, uint32_t t) {
  return ix.precision == CG_FP32_OFFSET ? __float_as_uint(__ldg(&ix.pts32[t].w))
                                        : (uint32_t)__double_as_longlong(ix.pts64s[t].w);
}

template <int KERN>
__global__ void __launch_bounds__(SW * 32) small_count_kernel(IndexView ix, const double* __restrict__ q, uint32_t nq,
                                                              double r, uint32_t* __restrict__ counts,
                                                              uint32_t* status) {
  __shared__ uint32_t wsum[SW];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  const uint32_t e = blockIdx.x;
  if (e >= nq) return;
  const double* c = q + 3 * (size_t)e;
  const double r2 = __dmul_rn(r, r);
  uint32_t cnt = 0;
  const bool ok = small_runs<KERN>(ix, c, r, [&](uint32_t t0, uint32_t t1) {
    for (uint32_t t = t0 + threadIdx.x; t < t1; t += SW * 32)
      cnt += exact_in<KERN>(ix.xyz64 + 3 * (size_t)small_id(ix, t), c, r2) ? 1u : 0u;
  });
  cnt = __reduce_add_sync(0xffffffffu, cnt);
  if (lane == 0) wsum[w] = cnt;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t tot = 0;
    for (int i = 0; i < SW; ++i) tot += wsum[i];
    counts[e] = ok ? tot : 0u;
    if (!ok) atomicOr(status, ST_NONFINITE);
  }
}

// One block: offsets = exclusive scan of counts (offsets[nq] = total), and
// stats[0] = the largest count.
__global__ void __launch_bounds__(1024) small_scan_kernel(const uint32_t* __restrict__ counts, uint32_t nq,
                                                          int64_t* __restrict__ offsets, uint32_t* stats) {
  __shared__ unsigned long long warp_sum[32];
  __shared__ uint32_t warp_max[32];
  const uint32_t t = threadIdx.x, lane = t & 31u, w = t >> 5;
  const uint32_t v = t < nq ? counts[t] : 0u;
  unsigned long long incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  const uint32_t m = __reduce_max_sync(0xffffffffu, v);
  if (lane == 31) {
    warp_sum[w] = incl;
    warp_max[w] = m;
  }
  __syncthreads();
  if (w == 0) {
    const unsigned long long s = warp_sum[lane];
    unsigned long long inc2 = s;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc2, o);
      if (lane >= (uint32_t)o) inc2 += y;
    }
    warp_sum[lane] = inc2 - s;
    const uint32_t mm = __reduce_max_sync(0xffffffffu, warp_max[lane]);
    if (lane == 0) stats[0] = mm;
  }
  __syncthreads();
  const unsigned long long ex = warp_sum[w] + incl - v;
  if (t < nq) offsets[t] = (int64_t)ex;
  if (t == nq - 1) offsets[nq] = (int64_t)(ex + v);
}

template <int KERN, int CAP>
__global__ void __launch_bounds__(SW * 32) small_fill_kernel(IndexView ix, const double* __restrict__ q, uint32_t nq,
                                                             double r, const int64_t* __restrict__ offsets,
                                                             int32_t* __restrict__ out, uint32_t* status) {
  __shared__ uint32_t B[CAP];
  __shared__ uint32_t nhit;
  const uint32_t e = blockIdx.x;
  if (e >= nq) return;
  const double* c = q + 3 * (size_t)e;
  const double r2 = __dmul_rn(r, r);
  if (threadIdx.x == 0) nhit = 0;
  __syncthreads();
  small_runs<KERN>(ix, c, r, [&](uint32_t t0, uint32_t t1) {
    for (uint32_t t = t0 + threadIdx.x; t < t1; t += SW * 32) {
      const uint32_t id = small_id(ix, t);
      if (exact_in<KERN>(ix.xyz64 + 3 * (size_t)id, c, r2)) {
        const uint32_t at = atomicAdd(&nhit, 1u);
        if (at < (uint32_t)CAP) B[at] = id;
      }
    }
  });
  __syncthreads();
  const uint32_t n = nhit;
  const int64_t o0 = offsets[e];
  if ((int64_t)n != offsets[e + 1] - o0 || n > (uint32_t)CAP) {  // count and fill disagree, or too long
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  uint32_t n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (uint32_t i = n + threadIdx.x; i < n2; i += SW * 32) B[i] = 0xffffffffu;
  __syncthreads();
  for (uint32_t k = 2; k <= n2; k <<= 1)  // bitonic sort of the row, ascending
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < n2; i += SW * 32) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const uint32_t a = B[i], b = B[l];
          if (((i & k) == 0) ? a > b : a < b) {
            B[i] = b;
            B[l] = a;
          }
        }
      }
      __syncthreads();
    }
  for (uint32_t i = threadIdx.x; i < n; i += SW * 32) out[o0 + i] = (int32_t)B[i];
}

}  // namespace

// ------------------------------------------------------------------ host

cudaError_t launch_small_count(const IndexView& iv, int kern, const double* q, uint32_t nq, double r,
                               uint32_t* counts, int64_t* offsets, uint32_t* stats, uint32_t* status,
                               cudaStream_t st) {
  const int grid = (int)nq;  // a block per query
  ProfScope prof("radius_small_count", st);
  if (kern == CG_SPHERE) small_count_kernel<CG_SPHERE><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, counts, status);
  else if (kern == CG_CUBE) small_count_kernel<CG_CUBE><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, counts, status);
  else small_count_kernel<CG_CYLINDER><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, counts, status);
  note_launch();
  small_scan_kernel<<<1, 1024, 0, st>>>(counts, nq, offsets, stats);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_small_fill(const IndexView& iv, int kern, const double* q, uint32_t nq, double r,
                              const int64_t* offsets, int32_t* out, uint32_t* status, cudaStream_t st) {
  const int grid = (int)nq;  // a block per query
  ProfScope prof("radius_small_fill", st);
  if (kern == CG_SPHERE)
    small_fill_kernel<CG_SPHERE, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, offsets, out, status);
  else if (kern == CG_CUBE)
    small_fill_kernel<CG_CUBE, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, offsets, out, status);
  else
    small_fill_kernel<CG_CYLINDER, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, offsets, out, status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cg
