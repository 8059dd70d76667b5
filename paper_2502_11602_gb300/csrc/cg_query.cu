// cg_query.cu -- fixed-radius kernel search on the GPU (Algorithm 1 of
// arXiv 2502.11602, run for a whole batch of queries in two passes).
//
// Blocked formulation.  Queries are grouped by the voxel that contains them
// (for "every point is a query" the groups are the index's own voxel runs).
// A CTA takes one group: it computes the union of the group's voxel ranges
// (the bounding box of each kernel mapped through Eq. chs-point-to-idcs,
// widened by a proven rounding pad), turns every row of that range (2D: one
// x row; 3D: one (x, y) column) into ONE contiguous span of the sorted points
// (consecutive global indices, Eqs. indices-to-global), stages the spans'
// records in shared memory, and tests every query of the group against every
// staged candidate (the point scan and is_inside of Algorithm 1).
//
//   count pass: per-query counts (no order needed)
//   fill pass : the staged records are first sorted by original id in shared
//               memory, so each query's hits come out ascending; one warp per
//               query writes them with a ballot compaction (coalesced rows).
//
// Precision.  Binary64 records are tested exactly.  Binary32 offset records
// are tested in binary32 and a candidate whose binary32 value lies within
// the proven band [s_lo, s_hi] of r^2 is re-tested with the exact binary64
// predicate on the original coordinates, so both give the same sets.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <string.h>

#include <algorithm>
#include <mutex>

#include "cg_query.cuh"
#include "cg_sort.cuh"

namespace cg {

namespace {

constexpr int RT = 256;         // threads per CTA
constexpr int RW = RT / 32;     // warps per CTA
constexpr int QB = 128;         // queries per sub-block
constexpr int MAX_SPANS = 256;  // spans staged per group of rows

template <int PREC> struct RecT;
template <> struct RecT<1> { using T = float4; static constexpr int KMAX = 4096; };
template <> struct RecT<0> { using T = double4_32a; static constexpr int KMAX = 2048; };

__device__ __forceinline__ uint32_t rec_id(const float4& r) { return __float_as_uint(r.w); }
__device__ __forceinline__ uint32_t rec_id(const double4_32a& r) {
  return (uint32_t)__double_as_longlong(r.w);
}
__device__ __forceinline__ float4 rec_sentinel(float4*) {
  return make_float4(0.f, 0.f, 0.f, __uint_as_float(0xffffffffu));
}
__device__ __forceinline__ double4_32a rec_sentinel(double4_32a*) {
  return make_double4_32a(0.0, 0.0, 0.0, __longlong_as_double(0xffffffffll));
}

// exact predicate on the original binary64 coordinates (no contraction)
template <int KERN>
__device__ __forceinline__ bool exact_inside(const double* __restrict__ p,
                                             const double* __restrict__ c, double r2) {
  double dx = __dsub_rn(__ldg(p), __ldg(c));
  double dy = __dsub_rn(__ldg(p + 1), __ldg(c + 1));
  double dz = __dsub_rn(__ldg(p + 2), __ldg(c + 2));
  if (KERN == CG_SPHERE) {
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= r2;
  }
  if (KERN == CG_CYLINDER) return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
  double m = fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return m <= r2;
}

template <int KERN>
__device__ __forceinline__ bool exact_inside4(const double4_32a& p, const double4_32a& c, double r2) {
  double dx = __dsub_rn(p.x, c.x);
  double dy = __dsub_rn(p.y, c.y);
  double dz = __dsub_rn(p.z, c.z);
  if (KERN == CG_SPHERE) {
    double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return d2 <= r2;
  }
  if (KERN == CG_CYLINDER) return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
  double m = fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  return m <= r2;
}

// binary32 screen; returns 1 inside, 0 outside, 2 undecided
template <int KERN>
__device__ __forceinline__ int screen32(const float4& c, const float4& q, const Thresholds& t) {
  float dx = __fsub_rn(c.x, q.x);
  float dy = __fsub_rn(c.y, q.y);
  float dz = __fsub_rn(c.z, q.z);
  float v;
  float lo, hi;
  if (KERN == CG_SPHERE) {
    v = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    lo = t.s_lo; hi = t.s_hi;
  } else if (KERN == CG_CYLINDER) {  // two terms: the sphere's band bounds it
    v = __fmaf_rn(dy, dy, __fmul_rn(dx, dx));
    lo = t.s_lo; hi = t.s_hi;
  } else {
    v = fmaxf(fmaxf(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    lo = t.c_lo; hi = t.c_hi;
  }
  if (v <= lo) return 1;
  if (v <= hi) return 2;
  return 0;
}

template <class R>
__device__ void bitonic_sort_by_id(R* a, int P) {
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
        int lo = 2 * j * (i / j) + (i % j);
        int hi = lo + j;
        bool asc = (lo & k) == 0;
        R x = a[lo], y = a[hi];
        if ((rec_id(x) > rec_id(y)) == asc) { a[lo] = y; a[hi] = x; }
      }
      __syncthreads();
    }
}

// Voxel coordinate u = (x - p-) / s of a query record, in binary32.
__device__ __forceinline__ float rec_u(const float4& q, const Tile& T, int a) {
  float x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__fadd_rn(x, T.D[a]), T.inv_sf[a]);
}
__device__ __forceinline__ float rec_u(const double4_32a& q, const Tile& T, int a) {
  double x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__double2float_rn(__dsub_rn(x, T.lo[a])), T.inv_sf[a]);
}
__device__ __forceinline__ float rec_abs_off(const float4& q, int a) {
  return fabsf(a == 0 ? q.x : (a == 1 ? q.y : q.z));
}
__device__ __forceinline__ float rec_abs_off(const double4_32a&, int) { return 0.f; }

struct HeavyOut {
  uint32_t* list;        // [cap] (query id, or id | 0x80000000 for rows needing scratch)
  uint32_t* count;       // number of entries
  unsigned long long* scratch_total;  // total scratch elements for long rows
  uint32_t* scratch_off; // [cap] scratch offset of each entry
  uint32_t* max_len;
  uint32_t cap;
};

constexpr uint32_t kSmemSortCap = 8192;  // rows up to this length sort in shared memory

template <int PREC, int KERN, bool FILL>
__global__ void __launch_bounds__(RT) radius_kernel(IndexView ix, QuerySet qs,
                                                    const Thresholds* __restrict__ thr_p,
                                                    uint32_t* __restrict__ counts,
                                                    const int64_t* __restrict__ offsets,
                                                    int32_t* __restrict__ out, HeavyOut heavy,
                                                    unsigned* work_ctr, uint32_t* status) {
  if (replan_pending(status)) return;
  using R = typename RecT<PREC>::T;
  constexpr int KMAX = RecT<PREC>::KMAX;
  extern __shared__ __align__(32) unsigned char smem[];
  R* rec = reinterpret_cast<R*>(smem);
  R* qr = rec + KMAX;
  long long* q_pos = reinterpret_cast<long long*>(qr + QB);
  uint32_t* q_cnt = reinterpret_cast<uint32_t*>(q_pos + QB);
  uint32_t* s_start = q_cnt + QB;
  uint32_t* s_off = s_start + MAX_SPANS;  // [MAX_SPANS + 1]
  __shared__ int s_lo[3], s_hi[3];
  __shared__ uint32_t s_blk;

  const Thresholds thr = *thr_p;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32)
                                        : reinterpret_cast<const R*>(ix.pts64s);
  const R* __restrict__ qsrc = qs.all_points ? pts
                                             : (PREC == 1 ? reinterpret_cast<const R*>(qs.qrec)
                                                          : reinterpret_cast<const R*>(qs.qrec64));
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;

  for (;;) {
    if (threadIdx.x == 0) s_blk = atomicAdd(work_ctr, 1u);
    __syncthreads();
    const uint32_t wi = s_blk;
    uint32_t b;
    if (qs.blk_list) {  // only the listed blocks (groups too large for the fast kernels)
      if (wi >= *qs.blk_list_n) break;
      b = qs.blk_list[wi];
    } else {
      if (wi >= qs_nblocks(qs)) break;
      b = wi;
    }
    const uint32_t qb0 = qs.blk_beg[b], qb1 = qs.blk_beg[b + 1];
    const uint32_t bkey = qs.blk_key[b];
    const int ti = ix.ntiles == 1 ? 0 : tile_of_key(ix.tiles, ix.ntiles, bkey);
    const Tile& T = ix.tiles[ti];
    const int dim = ix.dim;
    const int dimr = (KERN == CG_CYLINDER && dim == 3) ? 2 : dim;  // the cylinder spans every z slice

    for (uint32_t q0 = qb0; q0 < qb1; q0 += QB) {
      const int nqb = (int)min((uint32_t)QB, qb1 - q0);
      if (threadIdx.x < 3) { s_lo[threadIdx.x] = INT_MAX; s_hi[threadIdx.x] = INT_MIN; }
      __syncthreads();
      // queries of the sub-block and the union of their voxel ranges
      {
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
        for (int t = threadIdx.x; t < nqb; t += RT) {
          R q = qsrc[q0 + t];
          qr[t] = q;
          q_cnt[t] = 0;
          if (FILL) q_pos[t] = offsets[rec_id(q)];
          for (int a = 0; a < dimr; ++a) {
            float u = rec_u(q, T, a);
            float rr = __fmul_ru(__fmul_ru(thr.r_f, T.inv_sf[a]), 1.0000005f);
            float pad = __fadd_ru(__fadd_ru(rr, T.eta),
                                  __fmul_ru(__fadd_ru(fabsf(u), rec_abs_off(q, a) * T.inv_sf[a]), 3.0e-7f));
            pad = __fadd_ru(pad, __fmul_ru(thr.e_q, T.inv_sf[a]));
            float ul = fminf(fmaxf(__fsub_rd(u, pad), -1.0e9f), 1.0e9f);
            float uh = fminf(fmaxf(__fadd_ru(u, pad), -1.0e9f), 1.0e9f);
            lo[a] = min(lo[a], (int)floorf(ul));
            hi[a] = max(hi[a], (int)floorf(uh));
          }
        }
        for (int a = 0; a < dimr; ++a) {
          for (int o = 16; o > 0; o >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
          }
          if (lane == 0) { atomicMin(&s_lo[a], lo[a]); atomicMax(&s_hi[a], hi[a]); }
        }
      }
      __syncthreads();
      int lo[3], hi[3];
      bool empty = false;
      for (int a = 0; a < 3; ++a) {
        if (a < dimr) {
          lo[a] = max(s_lo[a], 0);
          hi[a] = min(s_hi[a], T.n[a] - 1);
          empty |= lo[a] > hi[a];
        } else {
          lo[a] = 0;
          hi[a] = T.n[a] - 1;
        }
      }
      int nchunks = 0;
      if (!empty) {
        const int ni = hi[0] - lo[0] + 1, nj = hi[1] - lo[1] + 1;
        const int nsp_total = dim == 2 ? ni : ni * nj;
        for (int sg = 0; sg < nsp_total; sg += MAX_SPANS) {
          const int nsp = min(MAX_SPANS, nsp_total - sg);
          for (int s = threadIdx.x; s < nsp; s += RT) {
            int id = sg + s;
            uint32_t k0, k1;
            if (dim == 2) {
              uint32_t row = (uint32_t)(lo[0] + id) * (uint32_t)T.n[1];
              k0 = T.key_base + row + (uint32_t)lo[1];
              k1 = T.key_base + row + (uint32_t)hi[1];
            } else {
              int i = lo[0] + id / nj, j = lo[1] + id % nj;
              uint32_t col = ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
              k0 = T.key_base + col + (uint32_t)lo[2];
              k1 = T.key_base + col + (uint32_t)hi[2];
            }
            uint2 sp = row_span(ix, T, k0, k1);
            s_start[s] = sp.x;
            s_off[s] = sp.y - sp.x;
          }
          __syncthreads();
          if (warp == 0) {  // exclusive scan of the span lengths (nsp <= 256)
            uint32_t v[MAX_SPANS / 32];
            uint32_t run = 0;
#pragma unroll
            for (int k = 0; k < MAX_SPANS / 32; ++k) {
              int s = lane * (MAX_SPANS / 32) + k;
              uint32_t x = s < nsp ? s_off[s] : 0u;
              v[k] = run;
              run += x;
            }
            uint32_t incl = run;
            for (int o = 1; o < 32; o <<= 1) {
              uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
              if (lane >= (unsigned)o) incl += y;
            }
            uint32_t base = incl - run;
#pragma unroll
            for (int k = 0; k < MAX_SPANS / 32; ++k) {
              int s = lane * (MAX_SPANS / 32) + k;
              if (s < nsp) s_off[s] = base + v[k];
            }
            if (lane == 31) s_off[nsp] = incl;
          }
          __syncthreads();
          const uint32_t ktot = s_off[nsp];
          for (uint32_t c0 = 0; c0 < ktot; c0 += KMAX) {
            const int K = (int)min((uint32_t)KMAX, ktot - c0);
            for (int t = threadIdx.x; t < K; t += RT) {
              uint32_t g = c0 + (uint32_t)t;
              int a = 0, bb = nsp - 1;  // last span with s_off <= g
              while (a < bb) {
                int m = (a + bb + 1) >> 1;
                if (s_off[m] <= g) a = m; else bb = m - 1;
              }
              rec[t] = pts[s_start[a] + (g - s_off[a])];
            }
            if (FILL) {
              int P = 32;
              while (P < K) P <<= 1;
              for (int t = K + threadIdx.x; t < P; t += RT) rec[t] = rec_sentinel((R*)nullptr);
              __syncthreads();
              bitonic_sort_by_id(rec, P);
            } else {
              __syncthreads();
            }
            // test: one warp per query, one lane per candidate
            for (int qi = warp; qi < nqb; qi += RW) {
              const R q = qr[qi];
              const uint32_t qid = rec_id(q);
              uint32_t cnt = 0;
              long long pos = FILL ? q_pos[qi] : 0;
              const long long lim = FILL ? offsets[qid + 1] : 0;
              for (int j0 = 0; j0 < K; j0 += 32) {
                const int j = j0 + (int)lane;
                bool in = false;
                uint32_t cid = 0;
                if (j < K) {
                  const R c = rec[j];
                  cid = rec_id(c);
                  if constexpr (PREC == 1) {
                    int sres = screen32<KERN>(c, q, thr);
                    in = sres == 1;
                    if (sres == 2) in = exact_inside<KERN>(ix.xyz64 + 3 * (size_t)cid, q64 + 3 * (size_t)qid, thr.r2);
                  } else {
                    in = exact_inside4<KERN>(c, q, thr.r2);
                  }
                }
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (FILL) {
                  if (in) {
                    const long long w = pos + __popc(m & lanemask_lt());
                    if (w < lim) out[w] = (int32_t)cid;   // never past the row
                    else atomicOr(status, ST_INTERNAL);
                  }
                  pos += __popc(m);
                } else {
                  cnt += __popc(m);
                }
              }
              if (lane == 0) {
                if (FILL) q_pos[qi] = pos; else q_cnt[qi] += cnt;
              }
            }
            __syncthreads();
            ++nchunks;
          }
        }
      }
      // results of the sub-block
      for (int t = threadIdx.x; t < nqb; t += RT) {
        const uint32_t qid = rec_id(qr[t]);
        if (!FILL) {
          const uint32_t c = q_cnt[t];
          counts[qid] = c;
          if (nchunks > 1 && c > 1) {  // rows made of several sorted runs
            uint32_t slot = atomicAdd(heavy.count, 1u);
            if (slot < heavy.cap) {
              uint32_t tag = 0, soff = 0;
              if (c > kSmemSortCap) {
                tag = 0x80000000u;
                soff = (uint32_t)atomicAdd(heavy.scratch_total, (unsigned long long)c);
              }
              heavy.list[slot] = qid | tag;
              heavy.scratch_off[slot] = soff;
              atomicMax(heavy.max_len, c);
            } else {
              atomicOr(status, ST_OVERFLOW);
            }
          }
        } else if (q_pos[t] != offsets[qid + 1]) {
          atomicOr(status, ST_INTERNAL);  // fill disagrees with the count pass
        }
      }
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------- row sort

// Sorts the rows listed by the count pass (rows assembled from several
// sorted runs).  Short rows: bitonic sort in shared memory.  Long rows:
// shared-memory sorted tiles, then pairwise merges through a scratch buffer
// (merge path), ping-ponging until one run remains.
__global__ void __launch_bounds__(512) row_sort_kernel(const uint32_t* __restrict__ list,
                                                       const uint32_t* __restrict__ scratch_off,
                                                       const uint32_t* __restrict__ count_p,
                                                       uint32_t cap, const int64_t* __restrict__ off,
                                                       int32_t* __restrict__ out,
                                                       int32_t* __restrict__ scratch, const uint32_t* status) {
  if (replan_pending(status)) return;
  extern __shared__ int32_t sbuf[];  // kSmemSortCap entries
  uint32_t cnt = min(*count_p, cap);
  for (uint32_t e = blockIdx.x; e < cnt; e += gridDim.x) {
    const uint32_t ent = list[e];
    const uint32_t qid = ent & 0x7fffffffu;
    int32_t* row = out + off[qid];
    const int64_t L = off[qid + 1] - off[qid];
    // sort tiles of kSmemSortCap in shared memory
    for (int64_t t0 = 0; t0 < L; t0 += kSmemSortCap) {
      const int n = (int)(L - t0 < (int64_t)kSmemSortCap ? L - t0 : (int64_t)kSmemSortCap);
      int P = 1;
      while (P < n) P <<= 1;
      for (int i = threadIdx.x; i < P; i += blockDim.x) sbuf[i] = i < n ? row[t0 + i] : INT_MAX;
      __syncthreads();
      for (int k = 2; k <= P; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
          for (int i = threadIdx.x; i < P / 2; i += blockDim.x) {
            int lo = 2 * j * (i / j) + (i % j), hi = lo + j;
            bool asc = (lo & k) == 0;
            int32_t x = sbuf[lo], y = sbuf[hi];
            if ((x > y) == asc) { sbuf[lo] = y; sbuf[hi] = x; }
          }
          __syncthreads();
        }
      for (int i = threadIdx.x; i < n; i += blockDim.x) row[t0 + i] = sbuf[i];
      __syncthreads();
    }
    if (L <= (int64_t)kSmemSortCap) continue;
    // merge passes
    int32_t* src = row;
    int32_t* dst = scratch + scratch_off[e];
    for (int64_t w = kSmemSortCap; w < L; w <<= 1) {
      for (int64_t a0 = 0; a0 < L; a0 += 2 * w) {
        const int64_t a1 = min(a0 + w, L), b1 = min(a0 + 2 * w, L);
        const int64_t na = a1 - a0, nb = b1 - a1, tot = na + nb;
        const int64_t per = (tot + blockDim.x - 1) / blockDim.x;
        const int64_t d0 = min((int64_t)threadIdx.x * per, tot);
        const int64_t d1 = min(d0 + per, tot);
        // merge path: split of diagonal d0
        int64_t lo = max((int64_t)0, d0 - nb), hi = min(d0, na);
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          if (src[a0 + mid] <= src[a1 + d0 - 1 - mid]) lo = mid + 1; else hi = mid;
        }
        int64_t ia = lo, ib = d0 - lo;
        for (int64_t d = d0; d < d1; ++d) {
          bool take_a = ib >= nb || (ia < na && src[a0 + ia] <= src[a1 + ib]);
          dst[a0 + d] = take_a ? src[a0 + ia++] : src[a1 + ib++];
        }
      }
      __syncthreads();
      int32_t* t = src; src = dst; dst = t;
    }
    if (src != row)
      for (int64_t i = threadIdx.x; i < L; i += blockDim.x) row[i] = src[i];
    __syncthreads();
  }
}

// ---------------------------------------------------------- external queries

__global__ void query_key_kernel(const double* __restrict__ q, int64_t nq, const Tile* __restrict__ tiles,
                                 int dim, uint32_t* __restrict__ keys, uint32_t* maxoff_bits,
                                 uint32_t* status) {
  const Tile& T = tiles[0];
  float mx = 0.f;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nq;
       p += (int64_t)gridDim.x * blockDim.x) {
    int c[3] = {0, 0, 0};
    bool bad = false;
    for (int a = 0; a < 3; ++a) {
      double x = q[3 * p + a];
      if (!isfinite(x)) { bad = true; continue; }
      mx = fmaxf(mx, fabsf(__double2float_ru(__dsub_rn(x, T.origin[a]))));
      if (a < dim) {
        double d = __dsub_rn(x, T.lo[a]);
        double v = floor(__ddiv_rn(d, T.s[a]));
        v = fmin(fmax(v, 0.0), (double)(T.n[a] - 1));
        c[a] = (int)v;
      }
    }
    if (bad) atomicOr(status, ST_NONFINITE);
    uint32_t g = dim == 2 ? (uint32_t)c[0] * (uint32_t)T.n[1] + (uint32_t)c[1]
                          : ((uint32_t)c[0] * (uint32_t)T.n[1] + (uint32_t)c[1]) * (uint32_t)T.n[2] + (uint32_t)c[2];
    keys[p] = T.key_base + g;
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxoff_bits, __float_as_uint(mx));
}

__global__ void query_gather_kernel(const double* __restrict__ q, int64_t nq,
                                    const uint32_t* __restrict__ perm, const Tile* __restrict__ tiles,
                                    float4* __restrict__ qrec, double4_32a* __restrict__ qrec64) {
  const Tile& T = tiles[0];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t id = perm[i];
    double x = q[3 * (size_t)id], y = q[3 * (size_t)id + 1], z = q[3 * (size_t)id + 2];
    if (qrec)
      qrec[i] = make_float4(__double2float_rn(__dsub_rn(x, T.origin[0])),
                            __double2float_rn(__dsub_rn(y, T.origin[1])),
                            __double2float_rn(__dsub_rn(z, T.origin[2])), __uint_as_float(id));
    if (qrec64) qrec64[i] = make_double4_32a(x, y, z, __longlong_as_double((long long)id));
  }
}

__global__ void qrun_flag_kernel(const uint32_t* __restrict__ skeys, int64_t n, uint32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = (i == 0 || skeys[i] != skeys[i - 1]) ? 1u : 0u;
}

__global__ void qrun_emit_kernel(const uint32_t* __restrict__ skeys, int64_t n,
                                 const uint32_t* __restrict__ flag, const uint32_t* __restrict__ rank,
                                 uint32_t* __restrict__ bkey, uint32_t* __restrict__ bbeg,
                                 uint32_t* nblocks) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (flag[i]) { bkey[rank[i]] = skeys[i]; bbeg[rank[i]] = (uint32_t)i; }
    if (i == n - 1) { bbeg[rank[n]] = (uint32_t)n; *nblocks = rank[n]; }
  }
}

__global__ void thresholds_kernel(Thresholds* out, double r, double e_p, const uint32_t* maxoff_bits) {
  // the query encode bound from the largest query offset magnitude
  double m = (double)__uint_as_float(*maxoff_bits);
  double e_q = ldexp(m, -24) * (1.0 + 1e-6) + ldexp(m, -52) + 1e-30;
  *out = make_thresholds(r, e_p, e_q);
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

template <int PREC>
size_t radius_smem() {
  using R = typename RecT<PREC>::T;
  return sizeof(R) * (RecT<PREC>::KMAX + QB) + sizeof(long long) * QB + 4 * QB + 4 * (2 * MAX_SPANS + 1);
}

// all-points thresholds of a replayed pass, from the refreshed tiles
__global__ void replay_thresholds_kernel(Thresholds* out, const Tile* __restrict__ tiles, int ntiles, double r) {
  float e = 0.f;
  for (int t = threadIdx.x; t < ntiles; t += 32) e = fmaxf(e, tiles[t].enc_err);
  for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (threadIdx.x == 0) *out = make_thresholds(r, (double)e, (double)e);
}

// capacity checks of a replayed pass: new data that outgrows a buffer
// stops the rest of the run (every later kernel tests ST_REPLAN first)
__global__ void replay_check_plan_kernel(const int64_t* __restrict__ moff_end, int64_t cap_m,
                                         const int64_t* __restrict__ idoff_end, int64_t cap_i, uint32_t* status) {
  if (*moff_end > cap_m || *idoff_end > cap_i) atomicOr(status, ST_REPLAN);
}
__global__ void replay_check_out_kernel(const int64_t* __restrict__ total, int64_t cap_out,
                                        const unsigned long long* __restrict__ scratch_total, uint64_t cap_scr,
                                        uint32_t* status) {
  if (*total > cap_out || *scratch_total > cap_scr) atomicOr(status, ST_REPLAN);
}

}  // namespace

// -------------------------------------------------------------- host side

// reuse: keep the plan of the same query buffer (a fill after its count);
// every other call plans again, as the buffer's contents may have changed.
cg_status prepare_queries(cg_index* ix, QueryCtx& C, const double* q, int64_t nq, bool reuse, cudaStream_t st) {
  QueryPlan& P = C.plan;
  if (reuse && P.q == q && P.nq == nq && P.nblocks_dev) return CG_OK;
  P.bufs.release(st);
  P.q = q;
  P.nq = nq;
  P.version++;
  DevBufs tmp;
  auto bail = [&](cg_status s, const std::string& m) {
    tmp.release(st);
    P.bufs.release(st);
    P.q = nullptr;
    P.nq = -1;
    P.nblocks_dev = nullptr;
    return fail(s, m);
  };
  const int64_t n = std::max<int64_t>(nq, 1);
  uint32_t *keys = (uint32_t*)tmp.get(4 * n, st), *skeys = (uint32_t*)tmp.get(4 * n, st),
           *perm = (uint32_t*)tmp.get(4 * n, st), *flag = (uint32_t*)tmp.get(4 * n, st),
           *rank = (uint32_t*)tmp.get(4 * (n + 1), st);
  void* sort_scratch = tmp.get(radix_sort_scratch_bytes(n), st);
  void* scan_scratch = tmp.get(scan_scratch_bytes(n), st);
  P.blk_beg = (uint32_t*)P.bufs.get(4 * (n + 1), st);
  P.blk_key = (uint32_t*)P.bufs.get(4 * n, st);
  P.nblocks_dev = (uint32_t*)P.bufs.get(64, st);
  if (ix->precision == CG_FP32_OFFSET) P.qrec = (float4*)P.bufs.get(16 * n, st);
  else P.qrec64 = (double4_32a*)P.bufs.get(32 * n, st);
  if (!keys || !skeys || !perm || !flag || !rank || !sort_scratch || !scan_scratch || !P.blk_beg ||
      !P.blk_key || !P.nblocks_dev || (!P.qrec && !P.qrec64))
    return bail(CG_ERR_OOM, "device allocation failed (query plan)");
  cudaError_t e = cudaMemsetAsync(P.nblocks_dev, 0, 64, st);
  ProfScope prof("query_plan", st);
  if (nq > 0) {
    query_key_kernel<<<grid_for(nq, 256), 256, 0, st>>>(q, nq, ix->tiles, ix->dim, keys,
                                                         P.nblocks_dev + 4, C.status); note_launch();
    const Tile& T = ix->tiles_host[0];
    int bits = 0;
    uint64_t kmax = (uint64_t)T.key_base + (uint64_t)T.n[0] * T.n[1] * T.n[2];
    while (bits < 32 && ((uint64_t)1 << bits) < kmax) ++bits;
    if (e == cudaSuccess) e = radix_sort_pairs(keys, nq, bits, skeys, perm, sort_scratch, C.status, st);
    query_gather_kernel<<<grid_for(nq, 256), 256, 0, st>>>(q, nq, perm, ix->tiles, P.qrec, P.qrec64); note_launch();
    qrun_flag_kernel<<<grid_for(nq, 256), 256, 0, st>>>(skeys, nq, flag); note_launch();
    if (e == cudaSuccess) e = exclusive_scan_u32_u32(flag, rank, nq, scan_scratch, C.status, st);
    qrun_emit_kernel<<<grid_for(nq, 256), 256, 0, st>>>(skeys, nq, flag, rank, P.blk_key, P.blk_beg,
                                                        P.nblocks_dev); note_launch();
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  tmp.release(st);
  if (e != cudaSuccess) return bail(CG_ERR_CUDA, std::string("query plan: ") + cudaGetErrorString(e));
  return CG_OK;
}

namespace {

struct RadiusLaunch {
  IndexView iv;
  QuerySet qs;
  const Thresholds* thr;
};

template <int PREC, int KERN, bool FILL>
cudaError_t launch_radius(const RadiusLaunch& L, uint32_t* counts, const int64_t* offsets, int32_t* out,
                          const HeavyOut& heavy, unsigned* work_ctr, uint32_t* status, int grid,
                          cudaStream_t st) {
  auto kern = radius_kernel<PREC, KERN, FILL>;
  const size_t smem = radius_smem<PREC>();
  static const bool configured = [&] {  // once per process, thread-safe
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return true;
  }();
  (void)configured;
  ProfScope prof(FILL ? "radius_v1_fill" : "radius_v1_count", st);
  kern<<<grid, RT, smem, st>>>(L.iv, L.qs, L.thr, counts, offsets, out, heavy, work_ctr, status); note_launch();
  return cudaGetLastError();
}

template <bool FILL>
cudaError_t dispatch_radius(int prec, int kern, const RadiusLaunch& L, uint32_t* counts,
                            const int64_t* offsets, int32_t* out, const HeavyOut& heavy,
                            unsigned* work_ctr, uint32_t* status, int grid, cudaStream_t st) {
  if (prec == CG_FP32_OFFSET) {
    if (kern == CG_SPHERE)
      return launch_radius<1, CG_SPHERE, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
    if (kern == CG_CYLINDER)
      return launch_radius<1, CG_CYLINDER, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
    return launch_radius<1, CG_CUBE, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
  }
  if (kern == CG_SPHERE)
    return launch_radius<0, CG_SPHERE, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
  if (kern == CG_CYLINDER)
    return launch_radius<0, CG_CYLINDER, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
  return launch_radius<0, CG_CUBE, FILL>(L, counts, offsets, out, heavy, work_ctr, status, grid, st);
}

int radius_grid(int prec) {
  static const int sms = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 152;
  }();
  size_t smem = prec == CG_FP32_OFFSET ? radius_smem<1>() : radius_smem<0>();
  int per_sm = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
  return sms * per_sm;
}

}  // namespace

namespace {
std::mutex g_tuning_mutex;
cg_tuning_t g_tuning = {kRadiusChunkDz, kRadiusChunkMax, 0, 0};
}  // namespace

cg_tuning_t default_tuning() { return cg_tuning_t{kRadiusChunkDz, kRadiusChunkMax, 0, 0}; }
cg_tuning_t current_tuning() {
  std::lock_guard<std::mutex> lock(g_tuning_mutex);
  return g_tuning;
}
void set_tuning(const cg_tuning_t& t) {
  std::lock_guard<std::mutex> lock(g_tuning_mutex);
  g_tuning = t;
}

// All-points voxel groups cut into height chunks (see cg_zwin.cu): the
// chunk table lives in `bufs`; one host read of the chunk count.
cg_status make_zchunks(cg_index* ix, float dz, uint32_t qmax, DevBufs& bufs, uint32_t* status, cudaStream_t st,
                       uint32_t** cbeg, uint32_t** ckey, uint32_t* nchunks) {
  const uint32_t nruns = ix->nkeys;
  uint32_t* cnt = (uint32_t*)bufs.get(4 * (size_t)std::max<uint32_t>(nruns, 1), st);
  uint32_t* coff = (uint32_t*)bufs.get(4 * ((size_t)nruns + 1), st);
  void* scr = bufs.get(scan_scratch_bytes(std::max<uint32_t>(nruns, 1)), st);
  if (!cnt || !coff || !scr) return fail(CG_ERR_OOM, "device allocation failed (height chunks)");
  cudaError_t e = launch_zchunk_count(ix->pts32z, ix->ustart, nruns, dz, qmax, cnt, st);
  if (e == cudaSuccess) e = exclusive_scan_u32_u32(cnt, coff, nruns, scr, status, st);
  uint32_t nch = 0;
  HostRead rd;
  rd.get(&nch, coff + nruns, 4);
  if (e == cudaSuccess) e = rd.sync(st);
  if (e != cudaSuccess) return cuda_fail(e, "height chunks");
  uint32_t* b = (uint32_t*)bufs.get(4 * ((size_t)nch + 1), st);
  uint32_t* k = (uint32_t*)bufs.get(4 * (size_t)std::max<uint32_t>(nch, 1), st);
  if (!b || !k) return fail(CG_ERR_OOM, "device allocation failed (height chunks)");
  e = launch_zchunk_emit(ix->pts32z, ix->ustart, ix->ukeys, nruns, dz, qmax, coff, b, k, (uint32_t)ix->n, st);
  if (e != cudaSuccess) return cuda_fail(e, "height chunks");
  *cbeg = b;
  *ckey = k;
  *nchunks = nch;
  return CG_OK;
}

// Mapped pinned words the small count writes for the host (total, longest
// row, status word, rows copied): one block per host thread, used between a
// count's launch and its stream sync in the same call.
struct SmallHostBlock {
  unsigned long long* h = nullptr;  // host address
  unsigned long long* d = nullptr;  // the same words as the device addresses them
  ~SmallHostBlock() {
    if (h) cudaFreeHost(h);
  }
};
thread_local SmallHostBlock t_small_host;

// Radius pass state kept on the index between the count and fill calls.
cg_status radius_pass(cg_index* ix, QueryCtx& C, bool all_points, const double* q, int64_t nq, double r,
                      int kernel, bool fill, int64_t* offsets, int32_t* out, int64_t* total_host,
                      cudaStream_t st) {
  if (!(r > 0) || !isfinite(r)) return fail(CG_ERR_INVALID, "radius must be positive and finite");
  if (kernel != CG_SPHERE && kernel != CG_CUBE && kernel != CG_CYLINDER) return fail(CG_ERR_INVALID, "unknown kernel");
  if (nq < 0 || nq >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "nq out of range");
  if (!all_points && ix->ntiles != 1)
    return fail(CG_ERR_UNIMPLEMENTED, "external queries on a batched index");
  RadiusState& R = C.radius;
  // small batches: one block per query, no plan (the count reads its sizes
  // back, so it is taken only when the caller asks for the total)
  if (!all_points && ix->ntiles == 1 && nq > 0 && nq <= kSmallBatch && (fill ? R.small : total_host != nullptr)) {
    if (!fill) {
      R.bufs.release(st);
      R.valid = false;
      R.small = false;
      if (!R.small_counts) {
        R.small_counts = (uint32_t*)R.small_bufs.get(4 * (size_t)kSmallBatch, st);
        R.small_stats = (uint32_t*)R.small_bufs.get(64, st);
        R.small_rows = (int32_t*)R.small_bufs.get(4 * (size_t)kSmallRowCap * (size_t)kSmallBatch, st);
        if (!R.small_counts || !R.small_stats || !R.small_rows ||
            cudaMemsetAsync(R.small_stats, 0, 64, st) != cudaSuccess) {  // [8]: the count's finish counter
          R.small_bufs.release(st);
          R.small_counts = R.small_stats = nullptr;
          R.small_rows = nullptr;
          return fail(CG_ERR_OOM, "device allocation failed (small radius pass)");
        }
      }
      if (!t_small_host.h) {
        void* hp = nullptr;
        void* dp = nullptr;
        if (cudaHostAlloc(&hp, 64, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
          cudaGetLastError();
          return fail(CG_ERR_OOM, "pinned host allocation failed (small radius pass)");
        }
        if (cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) {
          cudaGetLastError();
          cudaFreeHost(hp);
          return fail(CG_ERR_CUDA, "mapped host pointer (small radius pass)");
        }
        t_small_host.h = (unsigned long long*)hp;
        t_small_host.d = (unsigned long long*)dp;
      }
      volatile unsigned long long* hw = t_small_host.h;
      uint32_t* counts = R.small_counts;
      uint32_t* stats = R.small_stats;
      int32_t* rows = R.small_rows;
      // a search-into call: small results are copied by the count itself,
      // larger ones by a copy kernel issued before the one sync
      cudaError_t e = launch_small_count(ix->view(), ix->tiles_host[0], kernel, q, (uint32_t)nq, r, counts, rows,
                                         offsets, stats, C.status, t_small_host.d, R.direct_out, R.direct_cap, st);
      R.direct_done = false;
      bool copy_kernel = false;
      if (e == cudaSuccess && R.direct_out && (R.direct_cap > kSmallDirectMax || (uint32_t)nq > kSmallDirectQueries)) {
        e = launch_small_fill(rows, (uint32_t)nq, offsets, R.direct_out, C.status, st, R.direct_cap, stats + 9);
        copy_kernel = e == cudaSuccess;
      }
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_fail(e, "small radius count");
      *total_host = (int64_t)hw[0];
      const uint32_t maxrow = (uint32_t)hw[1];
      const uint32_t w = (uint32_t)hw[2];
      R.direct_done = copy_kernel || hw[3] != 0ull;
      cg_status s = status_verdict(w, C.status, st);
      if (s != CG_OK) return s;
      if (maxrow <= (uint32_t)kSmallRowCap) {
        R.small = true;
        R.valid = true;
        R.all_points = false;
        R.q = q;
        R.nq = nq;
        R.r = r;
        R.kernel = kernel;
        R.plan_version = C.plan.version;
        return CG_OK;
      }
      // a row too long for the warp's buffer: the regular path below
    } else {
      if (!R.valid || R.all_points || R.q != q || R.nq != nq || R.r != r || R.kernel != kernel)
        return fail(CG_ERR_INVALID, "radius fill without a matching count pass");
      cudaError_t e = launch_small_fill(R.small_rows, (uint32_t)nq, offsets, out, C.status, st);
      if (e != cudaSuccess) return cuda_fail(e, "small radius fill");
      return CG_OK;
    }
  }
  if (!fill) R.small = false;
  if (!all_points) {
    cg_status s = prepare_queries(ix, C, q, nq, fill, st);
    if (s != CG_OK) return s;
  }
  // per-call device state (counts, heavy list, thresholds, counters)
  const int64_t nqq = all_points ? ix->n : nq;
  if (!fill) {
    R.bufs.release(st);
    R.valid = false;
    R.counts = (uint32_t*)R.bufs.get(4 * std::max<int64_t>(nqq, 1), st);
    R.heavy_list = (uint32_t*)R.bufs.get(4 * std::max<int64_t>(nqq, 1), st);
    R.heavy_soff = (uint32_t*)R.bufs.get(4 * std::max<int64_t>(nqq, 1), st);
    R.ctrs = (uint32_t*)R.bufs.get(256, st);
    R.thr = (Thresholds*)R.bufs.get(sizeof(Thresholds), st);
    R.scan_scratch = R.bufs.get(scan_scratch_bytes(std::max<int64_t>(nqq, 1)), st);
    if (!R.counts || !R.heavy_list || !R.heavy_soff || !R.ctrs || !R.thr || !R.scan_scratch)
      return fail(CG_ERR_OOM, "device allocation failed (radius pass)");
    R.all_points = all_points;
    R.q = q;
    R.nq = nqq;
    R.r = r;
    R.kernel = kernel;
    R.plan_version = C.plan.version;
    cudaError_t e = cudaMemsetAsync(R.ctrs, 0, 256, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
    double emax = 0;
    for (const Tile& T : ix->tiles_host) emax = std::max(emax, (double)T.enc_err);
    if (all_points) {
      Thresholds th = make_thresholds(r, emax, emax);
      e = host_put(R.thr, &th, sizeof th, st);
      static_assert(sizeof(th) <= sizeof(R.thr_host), "threshold copy");
      memcpy(R.thr_host, &th, sizeof th);
    } else {
      thresholds_kernel<<<1, 1, 0, st>>>(R.thr, r, emax, C.plan.nblocks_dev + 4); note_launch();
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return cuda_fail(e, "thresholds");
  } else {
    if (!R.counts || R.all_points != all_points || R.q != q || R.nq != nqq || R.r != r ||
        R.kernel != kernel || R.plan_version != C.plan.version)
      return fail(CG_ERR_INVALID, "radius fill without a matching count pass");
  }
  RadiusLaunch L;
  L.iv = ix->view();
  L.thr = R.thr;
  if (all_points) {
    L.qs.all_points = 1;
    L.qs.nq = (uint32_t)ix->n;
    L.qs.nblocks = ix->nkeys;
    L.qs.blk_beg = ix->ustart;
    L.qs.blk_key = ix->ukeys;
    L.qs.qrec = ix->pts32;
    L.qs.qrec64 = ix->pts64s;
    L.qs.q64 = ix->xyz64;
  } else {
    QueryPlan& P = C.plan;
    L.qs.all_points = 0;
    L.qs.nq = (uint32_t)nq;
    L.qs.nblocks = 0xffffffffu;  // read from the device below
    L.qs.blk_beg = P.blk_beg;
    L.qs.blk_key = P.blk_key;
    L.qs.qrec = P.qrec;
    L.qs.qrec64 = P.qrec64;
    L.qs.q64 = q;
  }
  HeavyOut H;
  H.list = R.heavy_list;
  H.scratch_off = R.heavy_soff;
  H.count = R.ctrs + 0;
  H.max_len = R.ctrs + 1;
  H.scratch_total = (unsigned long long*)(R.ctrs + 2);
  H.cap = (uint32_t)std::max<int64_t>(nqq, 1);
  unsigned* work = R.ctrs + (fill ? 8 : 6);
  cudaError_t e = cudaSuccess;
  if (fill) {
    e = cudaMemsetAsync(work, 0, 4, st);
    if (e != cudaSuccess) return cuda_fail(e, "memset");
  }
  if (!all_points) {
    // the block count lives on the device: copy it into the launch struct
    // through a tiny synchronous read only once per plan
    if (C.plan.nblocks_host_version != C.plan.version) {
      HostRead rd;
      rd.get(&C.plan.nblocks, C.plan.nblocks_dev, 4);
      e = rd.sync(st);
      if (e != cudaSuccess) return cuda_fail(e, "query plan readback");
      C.plan.nblocks_host_version = C.plan.version;
    }
    L.qs.nblocks = C.plan.nblocks;
  }
  const int grid = radius_grid(ix->precision);
  // binary32 2D grids, sphere and cube: candidates (and all-points queries)
  // come from the height-sorted columns; all-points voxel groups are cut
  // into height chunks (made by the count pass, kept for its fill)
  const bool zw = zw_applies(ix, kernel);
  if (zw) {
    L.iv.pts32 = ix->pts32z;
    L.iv.sid = ix->sidz;
    if (all_points) {
      if (!fill) {
        const cg_tuning_t tun = current_tuning();
        cg_status zs = make_zchunks(ix, tun.radius_chunk_height * (float)r, tun.radius_chunk_max, R.bufs, C.status,
                                    st, &R.zbeg, &R.zkey, &R.znb);
        if (zs != CG_OK) return zs;
      }
      L.qs.nblocks = R.znb;
      L.qs.blk_beg = R.zbeg;
      L.qs.blk_key = R.zkey;
      L.qs.qrec = ix->pts32z;
    }
  }
  if (nqq > 0 && L.qs.nblocks > 0) {
    const uint32_t nb = L.qs.nblocks;
    // groups too large for the fast kernels go through the general CTA kernel
    RadiusLaunch Lbig = L;
    Lbig.qs.blk_list = R.big_list;
    Lbig.qs.blk_list_n = R.ctrs + 12;
    if (!fill) {
      R.plans = (BlockPlan*)R.bufs.get(sizeof(BlockPlan) * (size_t)nb, st);
      R.msize = (uint32_t*)R.bufs.get(4 * (size_t)(nb + 1), st);
      R.isize = (uint32_t*)R.bufs.get(4 * (size_t)(nb + 1), st);
      R.moff = (int64_t*)R.bufs.get(8 * (size_t)(nb + 1), st);
      R.idoff = (int64_t*)R.bufs.get(8 * (size_t)(nb + 1), st);
      R.big_list = (uint32_t*)R.bufs.get(4 * (size_t)nb, st);
      void* sscr = R.bufs.get(scan_scratch_bytes(nb), st);
      if (!R.plans || !R.msize || !R.isize || !R.moff || !R.idoff || !R.big_list || !sscr)
        return fail(CG_ERR_OOM, "device allocation failed (radius plan)");
      Lbig.qs.blk_list = R.big_list;
      e = launch_radius_plan(ix->precision, kernel, L.iv, L.qs, R.thr, R.plans, R.msize, R.isize, R.big_list,
                             R.ctrs + 12, C.status, st, zw, reinterpret_cast<unsigned long long*>(R.ctrs + 30));
      // 64-bit offsets: a call's mask words may exceed 2^32 (hundreds of
      // millions of queries with wide candidate sets)
      if (e == cudaSuccess) e = exclusive_scan_u32_i64(R.msize, R.moff, nb, sscr, C.status, st);
      if (e == cudaSuccess) e = exclusive_scan_u32_i64(R.isize, R.idoff, nb, sscr, C.status, st);
      int64_t tots[2] = {0, 0};
      uint32_t nbig = 0;
      HostRead rd;
      rd.get(&tots[0], R.moff + nb, 8);
      rd.get(&tots[1], R.idoff + nb, 8);
      rd.get(&nbig, R.ctrs + 12, 4);
      if (e == cudaSuccess) e = rd.sync(st);
      if (e != cudaSuccess) return cuda_fail(e, "radius plan");
      if (tots[0] < 0 || tots[1] < 0) return fail(CG_ERR_INTERNAL, "radius plan: negative buffer size");
      R.masks = (uint32_t*)R.bufs.get(4 * (size_t)std::max<int64_t>(tots[0], 1), st);
      R.ids = (uint32_t*)R.bufs.get(4 * (size_t)std::max<int64_t>(tots[1], 1), st);
      if (!R.masks || !R.ids) return fail(CG_ERR_OOM, "device allocation failed (radius masks)");
      R.big_n = nbig;
      R.mtot = tots[0];
      R.itot = tots[1];
      {
        // the size classes and the general kernel's groups are disjoint: they
        // run concurrently, so that each fills the others' tails
        ProfScope prof("radius_count_kernels", st);
        Fork f(st, 4);
        const cudaStream_t sts[3] = {f[0], f[1], f[2]};
        if (ix->precision == CG_FP32_OFFSET) {
          e = launch_radius_count32(kernel, L.iv, L.qs, R.thr, R.plans, R.moff, R.idoff, R.counts, R.masks,
                                    R.ids, R.ctrs + 20, C.status, sts, zw);
        } else {
          e = launch_radius_count2(ix->precision, kernel, L.iv, L.qs, R.thr, R.plans, R.moff, R.idoff, R.counts,
                                   R.masks, R.ids, R.ctrs + 14, C.status, f[0]);
        }
        if (e == cudaSuccess && R.big_n > 0)
          e = dispatch_radius<false>(ix->precision, kernel, Lbig, R.counts, nullptr, nullptr, H, work, C.status,
                                     grid, f[3]);
      }
    } else {
      e = cudaMemsetAsync(R.ctrs + 16, 0, 48, st);  // fill counters (binary64: 16, binary32: 24..26)
      if (e == cudaSuccess) {
        ProfScope prof("radius_fill_kernels", st);
        Fork f(st, 4);
        const cudaStream_t sts[3] = {f[0], f[1], f[2]};
        if (ix->precision == CG_FP32_OFFSET)
          e = launch_radius_fill32(L.iv, L.qs, R.plans, R.moff, R.idoff, R.masks, R.ids, offsets, out,
                                   R.ctrs + 24, C.status, sts);
        else
          e = launch_radius_fill2(ix->precision, L.iv, L.qs, R.plans, R.moff, R.idoff, R.masks, R.ids, offsets,
                                  out, R.ctrs + 16, C.status, f[0]);
        if (e == cudaSuccess && R.big_n > 0)
          e = dispatch_radius<true>(ix->precision, kernel, Lbig, nullptr, offsets, out, H, work, C.status, grid,
                                    f[3]);
      }
    }
    if (e != cudaSuccess) return cuda_fail(e, "radius kernel");
  }
  if (!fill) {
    if (nqq > 0) {
      ProfScope prof("offsets_scan", st);
      e = exclusive_scan_u32_i64(R.counts, offsets, nqq, R.scan_scratch, C.status, st);
    } else {
      e = cudaMemsetAsync(offsets, 0, 8, st);
    }
    if (e != cudaSuccess) return cuda_fail(e, "offsets scan");
    uint32_t stats[4] = {0, 0, 0, 0};
    if (total_host) {
      uint32_t w = 0;
      HostRead rd;
      rd.get(total_host, offsets + nqq, 8);
      rd.get(stats, R.ctrs, 16);
      rd.get(&w, C.status, 4);
      e = rd.sync(st);
      if (e != cudaSuccess) return cuda_fail(e, "count readback");
      R.heavy_count = stats[0];
      R.heavy_scratch = ((uint64_t)stats[3] << 32) | stats[2];
      R.stats_known = true;
      cg_status s = status_verdict(w, C.status, st);
      if (s != CG_OK) return s;
    } else {
      R.stats_known = false;
    }
    R.valid = true;
    return CG_OK;
  }
  // fill: sort the rows that were assembled from several runs
  if (!R.stats_known) {
    uint32_t stats[4] = {0, 0, 0, 0};
    HostRead rd;
    rd.get(stats, R.ctrs, 16);
    e = rd.sync(st);
    if (e != cudaSuccess) return cuda_fail(e, "heavy readback");
    R.heavy_count = stats[0];
    R.heavy_scratch = ((uint64_t)stats[3] << 32) | stats[2];
    R.stats_known = true;
  }
  if (R.heavy_count > 0) {
    int32_t* scratch = nullptr;
    if (R.heavy_scratch > 0) {
      scratch = (int32_t*)dev_alloc(4 * R.heavy_scratch, st);
      if (!scratch) return fail(CG_ERR_OOM, "device allocation failed (row sort scratch)");
    }
    const size_t smem = 4 * kSmemSortCap;
    ProfScope prof("radius_row_sort", st);
    row_sort_kernel<<<grid_for(R.heavy_count, 1, 152 * 4), 512, smem, st>>>(
        R.heavy_list, R.heavy_soff, R.ctrs + 0, (uint32_t)std::max<int64_t>(nqq, 1), offsets, out, scratch,
        C.status); note_launch();
    e = cudaGetLastError();
    if (scratch) dev_free(scratch, st);
    if (e != cudaSuccess) return cuda_fail(e, "row sort");
  }
  return CG_OK;
}


cg_status radius_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, double r, int kernel,
                      bool fill, int64_t* offsets, int32_t* out, int64_t* total_host, cudaStream_t st) {
  return radius_pass(ix, ix->ctx, all_points, q, nq, r, kernel, fill, offsets, out, total_host, st);
}

cg_status radius_search_into(cg_index* ix, QueryCtx& C, const double* q, int64_t nq, double r, int kernel,
                             int64_t* offsets, int32_t* out, int64_t cap, int64_t* total_host, cudaStream_t st) {
  RadiusState& R = C.radius;
  R.direct_out = cap > 0 ? out : nullptr;
  R.direct_cap = cap;
  R.direct_done = false;
  int64_t total = 0;
  cg_status s = radius_pass(ix, C, false, q, nq, r, kernel, false, offsets, nullptr, &total, st);
  const bool copied = R.small && R.direct_done;
  R.direct_out = nullptr;
  R.direct_done = false;
  if (s != CG_OK) return s;
  *total_host = total;
  if (total > cap) return fail(CG_ERR_OVERFLOW, "the rows exceed the output capacity (the count stands)");
  if (copied) return CG_OK;  // the small count has written the rows
  return radius_pass(ix, C, false, q, nq, r, kernel, true, offsets, out, nullptr, st);
}

// ------------------------------------------------- replayed (graph) pass

cg_status radius_work_alloc(cg_index* ix, RadiusWork& w, uint32_t cap_nb, double headroom, int64_t total,
                            cudaStream_t st) {
  const RadiusState& R = ix->ctx.radius;
  const int64_t n = std::max<int64_t>(ix->n, 1);
  auto grow = [&](double v, double slack) { return v * headroom + slack; };
  w.cap_nb = std::max<uint32_t>(cap_nb, 1);
  w.cap_m = (int64_t)grow((double)R.mtot, 65536.0);
  w.cap_i = (int64_t)grow((double)R.itot, 65536.0);
  w.cap_scr = (uint64_t)grow((double)R.heavy_scratch, 1 << 20);
  w.cap_out = (int64_t)grow((double)total, 1 << 20);
  w.counts = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.heavy_list = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.heavy_soff = (uint32_t*)w.bufs.get(4 * (size_t)n, st);
  w.ctrs = (uint32_t*)w.bufs.get(256, st);
  w.thr = (Thresholds*)w.bufs.get(sizeof(Thresholds), st);
  w.scan_scr = w.bufs.get(scan_scratch_bytes(n), st);
  w.plan_scr = w.bufs.get(scan_scratch_bytes(w.cap_nb), st);
  w.plans = (BlockPlan*)w.bufs.get(sizeof(BlockPlan) * (size_t)w.cap_nb, st);
  w.msize = (uint32_t*)w.bufs.get(4 * ((size_t)w.cap_nb + 1), st);
  w.isize = (uint32_t*)w.bufs.get(4 * ((size_t)w.cap_nb + 1), st);
  w.moff = (int64_t*)w.bufs.get(8 * ((size_t)w.cap_nb + 1), st);
  w.idoff = (int64_t*)w.bufs.get(8 * ((size_t)w.cap_nb + 1), st);
  w.big_list = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_nb, st);
  w.masks = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_m, st);
  w.ids = (uint32_t*)w.bufs.get(4 * (size_t)w.cap_i, st);
  w.row_scratch = (int32_t*)w.bufs.get(4 * (size_t)w.cap_scr, st);
  if (!w.counts || !w.heavy_list || !w.heavy_soff || !w.ctrs || !w.thr || !w.scan_scr || !w.plan_scr || !w.plans ||
      !w.msize || !w.isize || !w.moff || !w.idoff || !w.big_list || !w.masks || !w.ids || !w.row_scratch)
    return fail(CG_ERR_OOM, "device allocation failed (pipeline radius work)");
  return CG_OK;
}

// The all-points radius pass (count, scan, fill, row sort) with no host
// synchronisation or allocation: sizes come from the device (block count,
// totals), checked against the capacities of the work buffers.
cg_status radius_replay(cg_index* ix, RadiusWork& w, const uint32_t* nkeys_dev, double r, int kernel,
                        int64_t* offsets, int32_t* out, cudaStream_t st) {
  const int64_t n = ix->n;
  cudaError_t e = cudaMemsetAsync(w.ctrs, 0, 256, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay memset");
  replay_thresholds_kernel<<<1, 32, 0, st>>>(w.thr, ix->tiles, ix->ntiles, r); note_launch();
  RadiusLaunch L;
  L.iv = ix->view();
  L.thr = w.thr;
  L.qs.all_points = 1;
  L.qs.nq = (uint32_t)n;
  L.qs.nblocks = w.cap_nb;
  L.qs.nblocks_dev = nkeys_dev;
  L.qs.blk_beg = ix->ustart;
  L.qs.blk_key = ix->ukeys;
  L.qs.qrec = ix->pts32;
  L.qs.qrec64 = ix->pts64s;
  L.qs.q64 = ix->xyz64;
  RadiusLaunch Lbig = L;
  Lbig.qs.blk_list = w.big_list;
  Lbig.qs.blk_list_n = w.ctrs + 12;
  HeavyOut H;
  H.list = w.heavy_list;
  H.scratch_off = w.heavy_soff;
  H.count = w.ctrs + 0;
  H.max_len = w.ctrs + 1;
  H.scratch_total = (unsigned long long*)(w.ctrs + 2);
  H.cap = (uint32_t)std::max<int64_t>(n, 1);
  const int grid = radius_grid(ix->precision);
  const uint32_t nb = w.cap_nb;
  e = launch_radius_plan(ix->precision, kernel, L.iv, L.qs, w.thr, w.plans, w.msize, w.isize, w.big_list, w.ctrs + 12,
                         ix->status, st);
  if (e == cudaSuccess) e = exclusive_scan_u32_i64(w.msize, w.moff, nb, w.plan_scr, ix->status, st);
  if (e == cudaSuccess) e = exclusive_scan_u32_i64(w.isize, w.idoff, nb, w.plan_scr, ix->status, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay plan");
  replay_check_plan_kernel<<<1, 1, 0, st>>>(w.moff + nb, w.cap_m, w.idoff + nb, w.cap_i, ix->status); note_launch();
  {
    Fork f(st, 4);
    const cudaStream_t sts[3] = {f[0], f[1], f[2]};
    if (ix->precision == CG_FP32_OFFSET)
      e = launch_radius_count32(kernel, L.iv, L.qs, w.thr, w.plans, w.moff, w.idoff, w.counts, w.masks, w.ids,
                                w.ctrs + 20, ix->status, sts);
    else
      e = launch_radius_count2(ix->precision, kernel, L.iv, L.qs, w.thr, w.plans, w.moff, w.idoff, w.counts,
                               w.masks, w.ids, w.ctrs + 14, ix->status, f[0]);
    // groups too large for the fast kernels: the list length is read on the
    // device, an empty list costs one pass over the grid
    if (e == cudaSuccess)
      e = dispatch_radius<false>(ix->precision, kernel, Lbig, w.counts, nullptr, nullptr, H, w.ctrs + 6,
                                 ix->status, grid, f[3]);
  }
  if (e == cudaSuccess) e = exclusive_scan_u32_i64(w.counts, offsets, n, w.scan_scr, ix->status, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay count");
  replay_check_out_kernel<<<1, 1, 0, st>>>(offsets + n, w.cap_out, H.scratch_total, w.cap_scr, ix->status); note_launch();
  {
    Fork f(st, 4);
    const cudaStream_t sts[3] = {f[0], f[1], f[2]};
    if (ix->precision == CG_FP32_OFFSET)
      e = launch_radius_fill32(L.iv, L.qs, w.plans, w.moff, w.idoff, w.masks, w.ids, offsets, out, w.ctrs + 24,
                               ix->status, sts);
    else
      e = launch_radius_fill2(ix->precision, L.iv, L.qs, w.plans, w.moff, w.idoff, w.masks, w.ids, offsets, out,
                              w.ctrs + 16, ix->status, f[0]);
    if (e == cudaSuccess)
      e = dispatch_radius<true>(ix->precision, kernel, Lbig, nullptr, offsets, out, H, w.ctrs + 8, ix->status,
                                grid, f[3]);
  }
  if (e != cudaSuccess) return cuda_fail(e, "replay fill");
  row_sort_kernel<<<152 * 4, 512, 4 * kSmemSortCap, st>>>(w.heavy_list, w.heavy_soff, w.ctrs + 0, H.cap, offsets, out,
                                                         w.row_scratch, ix->status); note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "replay row sort");
  return CG_OK;
}

}  // namespace cg
