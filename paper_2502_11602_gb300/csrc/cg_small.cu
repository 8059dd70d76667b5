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
// voxels tested.  A voxel row (2D) or column (3D) of consecutive keys is one
// contiguous run of sorted points.  A candidate costs one load of its sorted
// record: binary32 offsets are screened with the thresholds of the regular
// path (computed per query from the query's own encode bound) and only the
// band between them is decided on the exact binary64 coordinates; binary64
// records are decided on the record itself.
//
//   count  per query, the ids of the points inside gathered in shared
//          memory, sorted ascending (bitonic, the whole block), written to a
//          scratch row of kSmallRowCap entries, and their number; the last
//          block to finish scans the numbers into offsets and records the
//          largest row (rows longer than the scratch row are refused on the
//          host, and the caller then takes the regular path).
//   fill   copies each scratch row to its place in the CSR output.
#include <math.h>

#include <algorithm>

#include "cg_f32x2.cuh"
#include "cg_query.cuh"

namespace cg {
namespace {

constexpr int SW = kBoxThreads / 32;  // warps per block

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

// The voxel box of query c's kernel (Algorithm 1's range, widened by one
// voxel); false when a coordinate is not finite, an empty box (lo > hi)
// when it misses the grid.
template <int KERN>
__device__ __forceinline__ bool small_box(const IndexView& ix, const double* cx, double r, int* lo, int* hi) {
  const Tile& T = ix.tiles[0];
  if (!(isfinite(cx[0]) && isfinite(cx[1]) && isfinite(cx[2]))) return false;
  lo[2] = 0;
  hi[2] = T.n[2] - 1;
  for (int a = 0; a < 2; ++a)
    if (!small_range(T, a, cx[a], r, lo[a], hi[a])) {
      lo[0] = 1;
      hi[0] = 0;
      return true;
    }
  if (ix.dim == 3 && KERN != CG_CYLINDER && !small_range(T, 2, cx[2], r, lo[2], hi[2])) {
    lo[0] = 1;
    hi[0] = 0;
  }
  return true;  // the cylinder is unbounded in z: every slice of the columns
}

// One query's screen: its binary32 offsets in the index's frame and the
// decision thresholds for its encode bound (the regular path's formulas,
// with the query set reduced to this query).  The host passes thresholds
// made for every query offset up to m_host (the tile's extent plus the
// radius); a query farther out makes its own (binary64, one thread).
struct SmallQuery {
  float4 qf;      // x~, y~, z~ of the query
  Thresholds thr;
};

__device__ __forceinline__ void small_query(const Tile& T, const double* cx, double r, const Thresholds& thr_host,
                                            float m_host, SmallQuery& S) {
  const float x = __double2float_rn(__dsub_rn(cx[0], T.origin[0]));
  const float y = __double2float_rn(__dsub_rn(cx[1], T.origin[1]));
  const float z = __double2float_rn(__dsub_rn(cx[2], T.origin[2]));
  S.qf = make_float4(x, y, z, 0.f);
  const float mf = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
  if (mf <= m_host) {
    S.thr = thr_host;
  } else {
    const double m = (double)mf;
    const double e_q = ldexp(m, -24) * (1.0 + 1e-6) + ldexp(m, -52) + 1e-30;
    S.thr = make_thresholds(r, (double)T.enc_err, e_q);
  }
}

// The voxel box of the kernel around a binary32 query (its ball's range with
// the proven pad of the binary32 voxel coordinates, the k-NN bounded
// search's formula); lo > hi when it misses the grid.  The cylinder is
// unbounded in z (every slice of the columns).
template <int KERN>
__device__ __forceinline__ void small_box_f(const IndexView& ix, const float4& q, const Thresholds& thr, int* lo,
                                            int* hi) {
  const Tile& T = ix.tiles[0];
  const float qa[3] = {q.x, q.y, q.z};
  const int nax = (ix.dim == 3 && KERN != CG_CYLINDER) ? 3 : 2;
  lo[2] = 0;
  hi[2] = T.n[2] - 1;
  for (int a = 0; a < nax; ++a) {
    const float u = __fmul_rn(__fadd_rn(qa[a], T.D[a]), T.inv_sf[a]);
    const float rr = __fmul_ru(__fmul_ru(thr.r_f, T.inv_sf[a]), 1.0000005f);
    float pad = __fadd_ru(__fadd_ru(rr, T.eta), __fmul_ru(__fadd_ru(fabsf(u), fabsf(qa[a]) * T.inv_sf[a]), 3.0e-7f));
    pad = __fadd_ru(pad, __fmul_ru(thr.e_q, T.inv_sf[a]));
    const float ul = fminf(fmaxf(__fsub_rd(u, pad), -1.0e9f), 1.0e9f);
    const float uh = fminf(fmaxf(__fadd_ru(u, pad), -1.0e9f), 1.0e9f);
    lo[a] = max((int)floorf(ul), 0);
    hi[a] = min((int)floorf(uh), T.n[a] - 1);
    if (lo[a] > hi[a]) {
      lo[0] = 1;
      hi[0] = 0;
      return;
    }
  }
}

// Is sorted record t inside the kernel around the query?  Binary32 records:
// the screen, then binary64 in the band; binary64 records: exact.
template <int KERN>
__device__ __forceinline__ bool small_in(const IndexView& ix, uint32_t t, const SmallQuery& S, const double* c,
                                         uint32_t& id) {
  if (ix.precision == CG_FP32_OFFSET) {
    const float4 p = __ldg(&ix.pts32[t]);
    id = __float_as_uint(p.w);
    const float dx = __fsub_rn(p.x, S.qf.x), dy = __fsub_rn(p.y, S.qf.y), dz = __fsub_rn(p.z, S.qf.z);
    float v, lo, hi;
    if (KERN == CG_CUBE) {
      v = fmaxf(fmaxf(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      lo = S.thr.c_lo;
      hi = S.thr.c_hi;
    } else {
      v = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
      if (KERN == CG_SPHERE) v = __fmaf_rn(dz, dz, v);
      lo = S.thr.s_lo;  // the cylinder's two-term value: the sphere's band bounds it
      hi = S.thr.s_hi;
    }
    if (v <= lo) return true;
    if (v > hi) return false;
    return exact_in<KERN>(ix.xyz64 + 3 * (size_t)id, c, S.thr.r2);
  }
  const double4_32a p = ix.pts64s[t];
  id = (uint32_t)__double_as_longlong(p.w);
  const double4_32a cc = make_double4_32a(__ldg(c), __ldg(c + 1), __ldg(c + 2), 0.0);
  return exact_in4<KERN>(p, cc, S.thr.r2);
}

// Count + gather: block e takes query e; its ids inside (at most CAP kept),
// sorted ascending, go to rows[e * CAP ...]; counts[e] = their number.
template <int KERN, int CAP>
__global__ void __launch_bounds__(SW * 32) small_count_kernel(IndexView ix, const double* __restrict__ q, uint32_t nq,
                                                              double r, const Thresholds thr_host, float m_host,
                                                              uint32_t* __restrict__ counts,
                                                              int32_t* __restrict__ rows, int64_t* __restrict__ offsets,
                                                              uint32_t* stats, uint32_t* status,
                                                              unsigned long long* host_out,
                                                              int32_t* __restrict__ direct_out, int64_t direct_cap) {
  __shared__ uint32_t B[CAP];
  __shared__ uint32_t s_start[kBoxThreads + 1], s_off[kBoxThreads + 1];
  __shared__ uint32_t nhit;
  __shared__ int s_box[7];  // lo[3], hi[3], coordinates finite
  __shared__ unsigned long long s_wsum[SW];
  __shared__ uint32_t s_wmax[SW];
  __shared__ SmallQuery S;
  const uint32_t e = blockIdx.x;
  if (e >= nq) return;
  const double* c = q + 3 * (size_t)e;
  if (threadIdx.x == 0) {  // set-up on one thread (the binary64 pipe is narrow)
    nhit = 0;
    const double cx[3] = {__ldg(c), __ldg(c + 1), __ldg(c + 2)};
    int l0[3] = {1, 1, 1}, h0[3] = {0, 0, 0};
    const bool fin = isfinite(cx[0]) && isfinite(cx[1]) && isfinite(cx[2]);
    if (fin) {
      small_query(ix.tiles[0], cx, r, thr_host, m_host, S);
      if (ix.precision == CG_FP32_OFFSET) small_box_f<KERN>(ix, S.qf, S.thr, l0, h0);
      else small_box<KERN>(ix, cx, r, l0, h0);
    }
    s_box[6] = fin ? 1 : 0;
    for (int a = 0; a < 3; ++a) {
      s_box[a] = l0[a];
      s_box[3 + a] = h0[a];
    }
  }
  __syncthreads();
  const SmallQuery Q = S;
  const int lo[3] = {s_box[0], s_box[1], s_box[2]}, hi[3] = {s_box[3], s_box[4], s_box[5]};
  const bool ok = s_box[6] != 0;
  if (ok && lo[0] <= hi[0])
    for_each_in_box(ix, ix.tiles[0], lo, hi, s_start, s_off, [&](uint32_t t, bool valid) {
      uint32_t id = 0;
      const bool in = valid && small_in<KERN>(ix, t, Q, c, id);
      const unsigned bm = __ballot_sync(0xffffffffu, in);
      uint32_t base = 0;
      if ((threadIdx.x & 31u) == 0 && bm) base = atomicAdd(&nhit, (uint32_t)__popc(bm));
      base = __shfl_sync(0xffffffffu, base, 0) + __popc(bm & lanemask_lt());
      if (in && base < (uint32_t)CAP) B[base] = id;
    });
  __syncthreads();
  const uint32_t n = ok ? nhit : 0u;
  if (threadIdx.x == 0) {
    counts[e] = n;
    if (!ok) atomicOr(status, ST_NONFINITE);
  }
  const uint32_t nsort = n > (uint32_t)CAP ? 0u : n;  // a longer row is refused on the host
  uint32_t n2 = 1;
  while (n2 < nsort) n2 <<= 1;
  if (nsort == 0) n2 = 0;
  for (uint32_t i = nsort + threadIdx.x; i < n2; i += SW * 32) B[i] = 0xffffffffu;
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
  int32_t* row = rows + (size_t)e * CAP;
  for (uint32_t i = threadIdx.x; i < nsort; i += SW * 32) row[i] = (int32_t)B[i];
  // the last block to finish scans the counts into offsets (offsets[nq] =
  // total) and records the largest count in stats[0]; the finish counter
  // stats[8] is zero before the launch and is left zero
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) nhit = atomicAdd(&stats[8], 1u) == nq - 1u ? 1u : 0u;
  __syncthreads();
  if (nhit == 0u) return;
  __threadfence();
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  uint32_t v[4], mx = 0;
  unsigned long long run = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t t = 4u * threadIdx.x + (uint32_t)i;
    v[i] = t < nq ? __ldcg(counts + t) : 0u;
    run += v[i];
    mx = max(mx, v[i]);
  }
  unsigned long long incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  mx = __reduce_max_sync(0xffffffffu, mx);
  if (lane == 31) {
    s_wsum[w] = incl;
    s_wmax[w] = mx;
  }
  __syncthreads();
  unsigned long long off = incl - run, tot = 0;
  uint32_t mall = 0;
  for (uint32_t i = 0; i < (uint32_t)SW; ++i) {
    off += i < w ? s_wsum[i] : 0ull;
    tot += s_wsum[i];
    mall = max(mall, s_wmax[i]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t t = 4u * threadIdx.x + (uint32_t)i;
    if (t < nq) offsets[t] = (int64_t)off;
    off += v[i];
  }
  if (threadIdx.x == 0) {
    offsets[nq] = (int64_t)tot;
    stats[0] = mall;
    stats[8] = 0u;
  }
  // a search-into call with a small result: this block also copies the rows
  // into the caller's buffer (no copy launch); host_out[3] says it did
  const bool copy = direct_out != nullptr && tot <= (unsigned long long)direct_cap &&
                    tot <= (unsigned long long)kSmallDirectMax && nq <= kSmallDirectQueries && mall <= (uint32_t)CAP;
  if (copy) {
    __syncthreads();  // offsets written
    for (uint32_t i = w; i < nq; i += SW) {  // a warp per row
      const int64_t o0 = offsets[i], len = offsets[i + 1] - o0;
      const int32_t* row = rows + (size_t)i * CAP;
      for (int64_t j = lane; j < len; j += 32) direct_out[o0 + j] = __ldcg(row + j);
    }
  }
  if (threadIdx.x == 0) stats[9] = copy ? 1u : 0u;  // a copy kernel behind it then does nothing
  if (threadIdx.x == 0 && host_out) {  // for the host, read after a stream sync
    host_out[0] = tot;
    host_out[1] = mall;
    host_out[2] = *((volatile uint32_t*)status);
    host_out[3] = copy ? 1ull : 0ull;
    __threadfence_system();
  }
}

// Block e copies scratch row e to its place in the CSR output.  cap >= 0
// (a copy issued with the count, before the host has seen the sizes):
// rows past cap entries, or longer than the scratch row, are skipped
// without a flag (the host redoes them); cap < 0: every row must fit.
template <int CAP>
__global__ void __launch_bounds__(SW * 32) small_copy_kernel(const int32_t* __restrict__ rows, uint32_t nq,
                                                             const int64_t* __restrict__ offsets,
                                                             int32_t* __restrict__ out, uint32_t* status,
                                                             int64_t cap, const uint32_t* skip) {
  const uint32_t e = blockIdx.x;
  if (e >= nq || (skip && *skip)) return;
  const int64_t o0 = offsets[e], n = offsets[e + 1] - o0;
  if (cap >= 0 && (n > CAP || o0 + n > cap)) return;
  if (n < 0 || n > CAP) {  // offsets not from this count
    if (threadIdx.x == 0) atomicOr(status, ST_INTERNAL);
    return;
  }
  const int32_t* row = rows + (size_t)e * CAP;
  for (int64_t i = threadIdx.x; i < n; i += SW * 32) out[o0 + i] = row[i];
}

}  // namespace

// ------------------------------------------------------------------ host

cudaError_t launch_small_count(const IndexView& iv, const Tile& T, int kern, const double* q, uint32_t nq, double r,
                               uint32_t* counts, int32_t* rows, int64_t* offsets, uint32_t* stats,
                               uint32_t* status, unsigned long long* host_out, int32_t* direct_out,
                               int64_t direct_cap, cudaStream_t st) {
  const int grid = (int)nq;  // a block per query
  // thresholds for query offsets up to the tile's extent plus the radius
  double m = 0.0;
  for (int a = 0; a < 3; ++a)
    m = std::max(m, std::max(std::fabs(T.lo[a] - T.origin[a]), std::fabs(T.hi[a] - T.origin[a])));
  const float m_host = (float)(m + r + 1.0);
  const double mq = (double)m_host;
  const Thresholds thr = make_thresholds(r, (double)T.enc_err, std::ldexp(mq, -24) * (1.0 + 1e-6) + std::ldexp(mq, -52) + 1e-30);
  ProfScope prof("radius_small_count", st);
  if (kern == CG_SPHERE)
    small_count_kernel<CG_SPHERE, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, thr, m_host, counts, rows, offsets, stats, status, host_out,
                                                                       direct_out, direct_cap);
  else if (kern == CG_CUBE)
    small_count_kernel<CG_CUBE, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, thr, m_host, counts, rows, offsets, stats, status, host_out,
                                                                       direct_out, direct_cap);
  else
    small_count_kernel<CG_CYLINDER, kSmallRowCap><<<grid, SW * 32, 0, st>>>(iv, q, nq, r, thr, m_host, counts, rows, offsets, stats, status, host_out,
                                                                       direct_out, direct_cap);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_small_fill(const int32_t* rows, uint32_t nq, const int64_t* offsets, int32_t* out,
                              uint32_t* status, cudaStream_t st, int64_t cap, const uint32_t* skip) {
  ProfScope prof("radius_small_fill", st);
  small_copy_kernel<kSmallRowCap><<<(int)nq, SW * 32, 0, st>>>(rows, nq, offsets, out, status, cap, skip);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cg
