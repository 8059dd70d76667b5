// cg_knn.cu -- exact k nearest neighbours on the GPU (the result of
// Algorithm 2 of arXiv 2502.11602: the k closest points under (d2, id)).
//
// Algorithm 2 grows a search radius and keeps a taboo box of visited voxels;
// its answer is final once every voxel that can hold a closer point has been
// visited.  Here the growth is ring by ring over the voxel grid: the visited
// region is always the index box [c - R, c + R] around the query's voxel (the
// taboo box of Section 3.5), and the search stops when the k-th distance is
// strictly below the distance from the query to the outside of that box (so
// no unvisited point can be closer, nor tie with a lower id).
//
// Fast path (most queries): queries are grouped by voxel; a CTA stages the
// group's R = 1 box in shared memory once, then one warp per query
//   1. histograms the binary32 d2 of the box's points into 64 buckets below
//      the wall distance and finds the bucket holding the k-th value,
//   2. collects every candidate whose binary32 d2 is within the proven error
//      band of that bucket's upper edge (a superset of the exact top k),
//   3. recomputes those candidates' binary64 d2 exactly and sorts them by
//      (d2, id), and checks the stop condition with the exact k-th d2.
// Queries that do not finish there (they need a larger ring, a box too big
// to stage, or ties that overflow the list) go to the slow path: one warp per
// query, rings R = 1, 2, ... read from global memory, every candidate's
// binary64 d2 computed exactly and inserted into a warp-wide sorted list.
#include <float.h>
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "cg_query.cuh"
#include "cg_sort.cuh"

namespace cg {


namespace {

constexpr int KT = 256;            // threads per CTA (fast path)
constexpr int KWARPS = KT / 32;
constexpr int KQB = 128;           // queries per sub-block
constexpr int KMAX_SPANS = 64;
constexpr int LCAP = 128;          // per-warp candidate list
constexpr int NB = 64;             // histogram buckets

template <int PREC> struct KRec;
template <> struct KRec<1> { using T = float4; static constexpr int KMAX = 4096; };
template <> struct KRec<0> { using T = double4_32a; static constexpr int KMAX = 2048; };

__device__ __forceinline__ uint32_t krec_id(const float4& r) { return __float_as_uint(r.w); }
__device__ __forceinline__ uint32_t krec_id(const double4_32a& r) { return (uint32_t)__double_as_longlong(r.w); }

// binary32 squared distance (the screen; exactness comes from the binary64 re-rank)
__device__ __forceinline__ float kd2f(const float4& c, const float4& q) {
  float dx = __fsub_rn(c.x, q.x), dy = __fsub_rn(c.y, q.y), dz = __fsub_rn(c.z, q.z);
  return __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
}
__device__ __forceinline__ float kd2f(const double4_32a& c, const double4_32a& q) {
  // binary64 records: the screen is the exact value rounded up to binary32
  double dx = __dsub_rn(c.x, q.x), dy = __dsub_rn(c.y, q.y), dz = __dsub_rn(c.z, q.z);
  return __double2float_ru(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ double exact_d2(const double* __restrict__ p, const double* __restrict__ c) {
  double dx = __dsub_rn(__ldg(p), __ldg(c));
  double dy = __dsub_rn(__ldg(p + 1), __ldg(c + 1));
  double dz = __dsub_rn(__ldg(p + 2), __ldg(c + 2));
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Bound on |d2f - d2| for candidates with d2 about tau (the model of the
// radius thresholds, two-sided, doubled).  Zero for binary64 records.
struct KBound {
  float c1, c0, c2;
  __device__ __forceinline__ float at(float tau) const {
    float t = fmaxf(tau, 0.f);
    return 2.0f * (c1 * sqrtf(t) * 1.0001f + c0 + c2 * t) + 1e-30f;
  }
};

__device__ __forceinline__ float rec_u_k(const float4& q, const Tile& T, int a) {
  float x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__fadd_rn(x, T.D[a]), T.inv_sf[a]);
}
__device__ __forceinline__ float rec_u_k(const double4_32a& q, const Tile& T, int a) {
  double x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__double2float_rn(__dsub_rn(x, T.lo[a])), T.inv_sf[a]);
}
__device__ __forceinline__ float rec_abs_k(const float4& q, int a) { return fabsf(a == 0 ? q.x : (a == 1 ? q.y : q.z)); }
__device__ __forceinline__ float rec_abs_k(const double4_32a&, int) { return 0.f; }

// Certified lower bound on the squared distance from the query to any point
// outside the voxel box [lo, hi] (indexed axes only); +inf if the box covers
// the grid on every side.
template <class R>
__device__ float wall2_lower(const R& q, const Tile& T, int dim, const int* lo, const int* hi, float e_q) {
  float w = INFINITY;
  for (int a = 0; a < dim; ++a) {
    float u = rec_u_k(q, T, a);
    float eta = T.eta + (fabsf(u) + rec_abs_k(q, a) * T.inv_sf[a]) * 3.0e-7f + e_q * T.inv_sf[a];
    if (lo[a] > 0) w = fminf(w, (u - (float)lo[a] - eta) * (float)T.s[a]);
    if (hi[a] < T.n[a] - 1) w = fminf(w, ((float)(hi[a] + 1) - u - eta) * (float)T.s[a]);
  }
  if (w == INFINITY) return INFINITY;
  if (w <= 0.f) return 0.f;
  return __fmul_rd(__fmul_rd(w, w), 0.99999f);
}

// Sorts entries (d2, id) of a per-warp list in shared memory (P a power of 2).
__device__ void warp_sort_list(double* d2, uint32_t* id, int P) {
  const unsigned lane = threadIdx.x & 31u;
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < P / 2; i += 32) {
        int lo = 2 * j * (i / j) + (i % j), hi = lo + j;
        bool asc = (lo & k) == 0;
        double a = d2[lo], b = d2[hi];
        uint32_t ia = id[lo], ib = id[hi];
        bool gt = (a > b) || (a == b && ia > ib);
        if (gt == asc) { d2[lo] = b; d2[hi] = a; id[lo] = ib; id[hi] = ia; }
      }
      __syncwarp();
    }
}

template <int PREC>
__global__ void __launch_bounds__(KT) knn_fast_kernel(IndexView ix, QuerySet qs, const Thresholds* __restrict__ thr_p,
                                                     int k, int32_t* __restrict__ out_idx, double* __restrict__ out_d2,
                                                     uint32_t* __restrict__ slow_list, uint32_t* slow_cnt,
                                                     unsigned* work, uint32_t* status) {
  if (replan_pending(status)) return;  // the slow kernel then finds an empty list
  using R = typename KRec<PREC>::T;
  constexpr int KMAX = KRec<PREC>::KMAX;
  extern __shared__ __align__(32) unsigned char smem[];
  R* rec = reinterpret_cast<R*>(smem);
  R* qr = rec + KMAX;
  double* l_d2 = reinterpret_cast<double*>(qr + KQB);     // [KWARPS][LCAP]
  uint32_t* l_id = reinterpret_cast<uint32_t*>(l_d2 + KWARPS * LCAP);
  uint32_t* hist = l_id + KWARPS * LCAP;                    // [KWARPS][NB]
  uint32_t* s_start = hist + KWARPS * NB;
  uint32_t* s_off = s_start + KMAX_SPANS;                   // [KMAX_SPANS + 1]
  __shared__ uint32_t s_blk;

  const Thresholds thr = *thr_p;
  KBound kb;
  {
    const double u = 5.9604644775390625e-08, U = 1.1102230246251565e-16;
    const double alpha = PREC == 1 ? (double)thr.pad_[0] * (1.0 + u) : 0.0;
    const double beta = PREC == 1 ? (u + U) * (1.0 + 2.0 * U) : 0.0;
    kb.c1 = (float)(2.0 * alpha * (1.0 + beta) * 1.7320508075688774);
    kb.c0 = (float)(3.0 * alpha * alpha);
    kb.c2 = PREC == 1 ? (float)(2.0 * beta + beta * beta + 3.0000002 * u + 4.0 * U) : 1.2e-7f;
  }
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
  const R* __restrict__ qsrc = qs.all_points ? pts
                                             : (PREC == 1 ? reinterpret_cast<const R*>(qs.qrec)
                                                          : reinterpret_cast<const R*>(qs.qrec64));
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  double* wd2 = l_d2 + warp * LCAP;
  uint32_t* wid = l_id + warp * LCAP;
  uint32_t* wh = hist + warp * NB;

  for (;;) {
    if (threadIdx.x == 0) s_blk = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t b = s_blk;
    if (b >= qs_nblocks(qs)) break;
    const uint32_t qb0 = qs.blk_beg[b], qb1 = qs.blk_beg[b + 1];
    const uint32_t bkey = qs.blk_key[b];
    const int ti = ix.ntiles == 1 ? 0 : tile_of_key(ix.tiles, ix.ntiles, bkey);
    const Tile& T = ix.tiles[ti];
    const int dim = ix.dim;
    // the block's voxel and its R = 1 box
    uint32_t g = bkey - T.key_base;
    int c[3] = {0, 0, 0};
    if (dim == 2) { c[0] = (int)(g / (uint32_t)T.n[1]); c[1] = (int)(g % (uint32_t)T.n[1]); }
    else { c[2] = (int)(g % (uint32_t)T.n[2]); uint32_t ij = g / (uint32_t)T.n[2]; c[0] = (int)(ij / (uint32_t)T.n[1]); c[1] = (int)(ij % (uint32_t)T.n[1]); }
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      if (a < dim) { lo[a] = max(c[a] - 1, 0); hi[a] = min(c[a] + 1, T.n[a] - 1); }
      else { lo[a] = 0; hi[a] = T.n[a] - 1; }
    }
    const int ni = hi[0] - lo[0] + 1, nj = hi[1] - lo[1] + 1;
    const int nsp = dim == 2 ? ni : ni * nj;
    for (int s = threadIdx.x; s < nsp; s += KT) {
      uint32_t k0, k1;
      if (dim == 2) {
        uint32_t row = (uint32_t)(lo[0] + s) * (uint32_t)T.n[1];
        k0 = T.key_base + row + (uint32_t)lo[1];
        k1 = T.key_base + row + (uint32_t)hi[1];
      } else {
        int i = lo[0] + s / nj, j = lo[1] + s % nj;
        uint32_t col = ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
        k0 = T.key_base + col + (uint32_t)lo[2];
        k1 = T.key_base + col + (uint32_t)hi[2];
      }
      uint2 sp = row_span(ix, T, k0, k1);
      s_start[s] = sp.x;
      s_off[s] = sp.y - sp.x;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (int s = 0; s < nsp; ++s) { uint32_t t = s_off[s]; s_off[s] = acc; acc += t; }
      s_off[nsp] = acc;
    }
    __syncthreads();
    const uint32_t K = s_off[nsp];
    const bool staged = K <= (uint32_t)KMAX;
    if (staged) {
      for (uint32_t t = threadIdx.x; t < K; t += KT) {
        int a = 0, bb = nsp - 1;
        while (a < bb) { int m = (a + bb + 1) >> 1; if (s_off[m] <= t) a = m; else bb = m - 1; }
        rec[t] = pts[s_start[a] + (t - s_off[a])];
      }
    }
    __syncthreads();
    for (uint32_t q0 = qb0; q0 < qb1; q0 += KQB) {
      const int nqb = (int)min((uint32_t)KQB, qb1 - q0);
      for (int t = threadIdx.x; t < nqb; t += KT) qr[t] = qsrc[q0 + t];
      __syncthreads();
      for (int qi = warp; qi < nqb; qi += KWARPS) {
        const R q = qr[qi];
        const uint32_t qid = krec_id(q);
        if (!staged) {
          if (lane == 0) { uint32_t sl = atomicAdd(slow_cnt, 1u); slow_list[sl] = qid; }
          continue;
        }
        const float W2 = wall2_lower(q, T, dim, lo, hi, thr.e_q);
        const bool exhausted = W2 == INFINITY;
        if (!exhausted && !(W2 > 0.f)) {  // on the wall: this ring cannot decide
          if (lane == 0) { uint32_t sl = atomicAdd(slow_cnt, 1u); slow_list[sl] = qid; }
          continue;
        }
        float W = W2;
        if (exhausted) {  // every point is a candidate: bucket up to the farthest one
          float mx = 0.f;
          for (uint32_t t = lane; t < K; t += 32) mx = fmaxf(mx, kd2f(rec[t], q));
          for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
          W = fmaxf(mx, 1e-30f) * 1.0001f;
        }
        // 1. histogram below W
        for (int t = lane; t < NB; t += 32) wh[t] = 0;
        __syncwarp();
        const float inv_bw = (float)NB / W;
        for (uint32_t t = lane; t < K; t += 32) {
          float d = kd2f(rec[t], q);
          if (d <= W) atomicAdd(&wh[min(NB - 1, max(0, (int)(d * inv_bw)))], 1u);
        }
        __syncwarp();
        uint32_t h0 = wh[2 * lane], h1 = wh[2 * lane + 1];
        uint32_t inc = h0 + h1;
        for (int o = 1; o < 32; o <<= 1) {
          uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= (unsigned)o) inc += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        const uint32_t need = min((uint32_t)k, exhausted ? K : (uint32_t)k);
        if (!exhausted && total < (uint32_t)k) {  // the k-th lies beyond this ring
          if (lane == 0) { uint32_t sl = atomicAdd(slow_cnt, 1u); slow_list[sl] = qid; }
          continue;
        }
        // bucket holding the need-th value
        const uint32_t exc = inc - h0 - h1;
        int bstar = NB - 1;
        {
          bool in0 = need > 0 && exc < need && exc + h0 >= need;
          bool in1 = need > 0 && exc + h0 < need && inc >= need;
          unsigned m0 = __ballot_sync(0xffffffffu, in0), m1 = __ballot_sync(0xffffffffu, in1);
          int c0 = m0 ? 2 * (__ffs(m0) - 1) : INT_MAX, c1 = m1 ? 2 * (__ffs(m1) - 1) + 1 : INT_MAX;
          bstar = min(c0, c1);
          if (bstar == INT_MAX) bstar = NB - 1;
        }
        const float edge = (float)(bstar + 1) / inv_bw;
        const float cut = exhausted ? INFINITY : __fadd_ru(edge, 2.0f * kb.at(edge));
        // 2. collect the certified superset
        uint32_t m = 0;
        bool overflow = false;
        for (uint32_t t0 = 0; t0 < K; t0 += 32) {
          uint32_t t = t0 + lane;
          bool pick = false;
          if (t < K) pick = kd2f(rec[t], q) <= cut;
          unsigned bm = __ballot_sync(0xffffffffu, pick);
          uint32_t pos = m + __popc(bm & lanemask_lt());
          if (pick && pos < LCAP) wid[pos] = krec_id(rec[t]);
          m += __popc(bm);
        }
        if (m > LCAP) overflow = true;
        if (overflow || m < need) {
          if (lane == 0) { uint32_t sl = atomicAdd(slow_cnt, 1u); slow_list[sl] = qid; }
          __syncwarp();
          continue;
        }
        __syncwarp();
        // 3. exact binary64 values, order (d2, id)
        int P = 32;
        while (P < (int)m) P <<= 1;
        for (int t = lane; t < P; t += 32) {
          if (t < (int)m) wd2[t] = exact_d2(ix.xyz64 + 3 * (size_t)wid[t], q64 + 3 * (size_t)qid);
          else { wd2[t] = INFINITY; wid[t] = 0xffffffffu; }
        }
        __syncwarp();
        warp_sort_list(wd2, wid, P);
        const uint32_t kk = min((uint32_t)k, m);
        const double kth = wd2[kk - 1];
        if (!exhausted && !(kth < (double)W2)) {
          if (lane == 0) { uint32_t sl = atomicAdd(slow_cnt, 1u); slow_list[sl] = qid; }
          __syncwarp();
          continue;
        }
        for (int t = lane; t < k; t += 32) {
          bool ok = t < (int)kk;
          out_idx[(size_t)qid * k + t] = ok ? (int32_t)wid[t] : -1;
          if (out_d2) out_d2[(size_t)qid * k + t] = ok ? wd2[t] : INFINITY;
        }
        __syncwarp();
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------- slow path

// Warp-wide sorted list of up to 64 (d2, id) entries: lane l holds slots l
// and l + 32.
struct WarpList {
  double d[2];
  uint32_t id[2];
};

__device__ __forceinline__ bool lt(double a, uint32_t ia, double b, uint32_t ib) {
  return a < b || (a == b && ia < ib);
}

__device__ void wl_insert(WarpList& L, double d, uint32_t id, int cap) {
  const unsigned lane = threadIdx.x & 31u;
  // position = number of entries smaller than (d, id)
  unsigned b0 = __ballot_sync(0xffffffffu, lt(L.d[0], L.id[0], d, id));
  unsigned b1 = __ballot_sync(0xffffffffu, lt(L.d[1], L.id[1], d, id));
  int pos = __popc(b0) + __popc(b1);
  if (pos >= cap) return;
  double d0u = __shfl_up_sync(0xffffffffu, L.d[0], 1), d1u = __shfl_up_sync(0xffffffffu, L.d[1], 1);
  uint32_t i0u = __shfl_up_sync(0xffffffffu, L.id[0], 1), i1u = __shfl_up_sync(0xffffffffu, L.id[1], 1);
  double d031 = __shfl_sync(0xffffffffu, L.d[0], 31);
  uint32_t i031 = __shfl_sync(0xffffffffu, L.id[0], 31);
  if (lane == 0) { d1u = d031; i1u = i031; }
  int s0 = (int)lane, s1 = (int)lane + 32;
  if (s1 > pos) { L.d[1] = d1u; L.id[1] = i1u; } else if (s1 == pos) { L.d[1] = d; L.id[1] = id; }
  if (s0 > pos) { L.d[0] = d0u; L.id[0] = i0u; } else if (s0 == pos) { L.d[0] = d; L.id[0] = id; }
}

__device__ __forceinline__ double wl_get(const WarpList& L, int slot) {
  double a = __shfl_sync(0xffffffffu, L.d[0], slot & 31);
  double b = __shfl_sync(0xffffffffu, L.d[1], slot & 31);
  return slot < 32 ? a : b;
}

template <int PREC>
__global__ void __launch_bounds__(128) knn_slow_kernel(IndexView ix, QuerySet qs, int k,
                                                       const uint32_t* __restrict__ slow_list,
                                                       const uint32_t* slow_cnt,
                                                       int32_t* __restrict__ out_idx, double* __restrict__ out_d2) {
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t nslow = *slow_cnt;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  for (uint32_t e = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); e < nslow;
       e += gridDim.x * (blockDim.x / 32)) {
    const uint32_t qid = slow_list[e];
    const double* c = q64 + 3 * (size_t)qid;
    const Tile& T = ix.tiles[(qs.all_points && ix.ntiles > 1) ? tile_of_id(ix.tiles, ix.ntiles, qid) : 0];
    // the query's voxel (clamped), from binary64
    int cc[3] = {0, 0, 0};
    for (int a = 0; a < ix.dim; ++a) {
      double v = floor(__ddiv_rn(__dsub_rn(__ldg(c + a), T.lo[a]), T.s[a]));
      v = fmin(fmax(v, 0.0), (double)(T.n[a] - 1));
      cc[a] = (int)v;
    }
    WarpList L;
    L.d[0] = L.d[1] = INFINITY;
    L.id[0] = L.id[1] = 0xffffffffu;
    int plo[3] = {1, 1, 1}, phi[3] = {0, 0, 0};  // previous box (empty)
    for (int Rr = 0;; ++Rr) {
      int lo[3], hi[3];
      bool covers = true;
      for (int a = 0; a < 3; ++a) {
        if (a < ix.dim) {
          lo[a] = max(cc[a] - Rr, 0);
          hi[a] = min(cc[a] + Rr, T.n[a] - 1);
          covers &= lo[a] == 0 && hi[a] == T.n[a] - 1;
        } else {
          lo[a] = 0;
          hi[a] = T.n[a] - 1;
        }
      }
      // visit the voxels of the box outside the previous box (the taboo box)
      const int ni = hi[0] - lo[0] + 1, nj = hi[1] - lo[1] + 1;
      const int ncol = ix.dim == 2 ? ni * nj : ni * nj;
      for (int col = 0; col < ncol; ++col) {
        const int i = lo[0] + col / nj, j = lo[1] + col % nj;
        int k0 = ix.dim == 3 ? lo[2] : 0, k1 = ix.dim == 3 ? hi[2] : 0;
        for (int kz = k0; kz <= k1; ++kz) {
          bool inprev = i >= plo[0] && i <= phi[0] && j >= plo[1] && j <= phi[1] &&
                        (ix.dim == 2 || (kz >= plo[2] && kz <= phi[2]));
          if (inprev) continue;
          uint32_t key = T.key_base + (ix.dim == 2 ? (uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j
                                                   : ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2] + (uint32_t)kz);
          uint2 sp = voxel_span(ix, T, key);
          for (uint32_t t0 = sp.x; t0 < sp.y; t0 += 32) {
            uint32_t t = t0 + lane;
            double d = INFINITY;
            uint32_t id = 0xffffffffu;
            if (t < sp.y) {
              id = PREC == 1 ? __float_as_uint(ix.pts32[t].w) : (uint32_t)__double_as_longlong(ix.pts64s[t].w);
              d = exact_d2(ix.xyz64 + 3 * (size_t)id, c);
            }
            const double worst = wl_get(L, k - 1);
            const uint32_t worst_id = __shfl_sync(0xffffffffu, (k - 1) < 32 ? L.id[0] : L.id[1], (k - 1) & 31);
            unsigned cand = __ballot_sync(0xffffffffu, t < sp.y && lt(d, id, worst, worst_id));
            while (cand) {
              int src = __ffs(cand) - 1;
              cand &= cand - 1;
              double dd = __shfl_sync(0xffffffffu, d, src);
              uint32_t ii = __shfl_sync(0xffffffffu, id, src);
              wl_insert(L, dd, ii, k);
            }
          }
        }
      }
      for (int a = 0; a < 3; ++a) { plo[a] = lo[a]; phi[a] = hi[a]; }
      if (covers) break;
      // stop when the k-th is strictly inside the visited box (binary64 wall)
      const double kth = wl_get(L, k - 1);
      if (kth < INFINITY) {
        double w = INFINITY;
        for (int a = 0; a < ix.dim; ++a) {
          double x = __ldg(c + a);
          if (lo[a] > 0) w = fmin(w, x - (T.lo[a] + (double)lo[a] * T.s[a]));
          if (hi[a] < T.n[a] - 1) w = fmin(w, (T.lo[a] + (double)(hi[a] + 1) * T.s[a]) - x);
        }
        // margin for the rounding of the voxel keys and of the wall itself
        double slack = 1e-12 * (fabs(T.lo[0]) + fabs(T.lo[1]) + fabs(T.lo[2]) + 1.0);
        w -= slack;
        if (w > 0 && kth < w * w * (1.0 - 1e-12)) break;
      }
    }
    // write out: slot s lives in lane s % 32, register s / 32
    for (int s = 0; s < k; ++s) {
      double d = wl_get(L, s);
      uint32_t id = __shfl_sync(0xffffffffu, s < 32 ? L.id[0] : L.id[1], s & 31);
      if (lane == 0) {
        bool ok = d < INFINITY;
        out_idx[(size_t)qid * k + s] = ok ? (int32_t)id : -1;
        if (out_d2) out_d2[(size_t)qid * k + s] = ok ? d : INFINITY;
      }
    }
  }
}

template <int PREC>
size_t knn_smem() {
  using R = typename KRec<PREC>::T;
  return sizeof(R) * (KRec<PREC>::KMAX + KQB) + KWARPS * LCAP * (8 + 4) + KWARPS * NB * 4 +
         4 * (2 * KMAX_SPANS + 1);
}

// k-NN error terms: pad_[0] = alpha = e_p + e_q (per-axis bound on the
// binary32 difference error), e_q = the queries' own encode bound.
__device__ void knn_thresholds(Thresholds* out, double e_p, double e_q) {
  Thresholds t = make_thresholds(1.0, e_p, e_q);
  t.pad_[0] = __double2float_ru((e_p + e_q) * (1.0 + 1e-6));
  *out = t;
}

__global__ void knn_thr_kernel(Thresholds* out, double e_p, const uint32_t* maxoff_bits) {
  double m = maxoff_bits ? (double)__uint_as_float(*maxoff_bits) : 0.0;
  double e_q = maxoff_bits ? ldexp(m, -24) * (1.0 + 1e-6) + ldexp(m, -52) + 1e-30 : e_p;
  knn_thresholds(out, e_p, e_q);
}

// replayed pipelines: the encode bound of the refreshed tiles
__global__ void knn_thr_tiles_kernel(Thresholds* out, const Tile* __restrict__ tiles, int ntiles) {
  float e = 0.f;
  for (int t = threadIdx.x; t < ntiles; t += 32) e = fmaxf(e, tiles[t].enc_err);
  for (int o = 16; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(0xffffffffu, e, o));
  if (threadIdx.x == 0) knn_thresholds(out, (double)e, (double)e);
}

}  // namespace

cg_status knn_pass(cg_index* ix, QueryCtx& C, bool all_points, const double* q, int64_t nq, int k, int32_t* idx, double* d2,
                   cudaStream_t st) {
  if (k < 1 || k > 64) return fail(CG_ERR_INVALID, "k must be in [1, 64]");
  if (nq < 0 || nq >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "nq out of range");
  if (!all_points && ix->ntiles != 1)
    return fail(CG_ERR_UNIMPLEMENTED, "external k-NN queries on a batched index (every point queries its own tile)");
  if (!all_points) {
    cg_status s = prepare_queries(ix, C, q, nq, false, st);
    if (s != CG_OK) return s;
  }
  if (nq == 0) return CG_OK;
  DevBufs tmp;
  uint32_t* slow = (uint32_t*)tmp.get(4 * (size_t)nq, st);
  uint32_t* ctrs = (uint32_t*)tmp.get(256, st);
  Thresholds* thr = (Thresholds*)tmp.get(sizeof(Thresholds), st);
  if (!slow || !ctrs || !thr) { tmp.release(st); return fail(CG_ERR_OOM, "device allocation failed (k-NN)"); }
  cudaError_t e = cudaMemsetAsync(ctrs, 0, 256, st);
  double emax = 0;
  for (const Tile& T : ix->tiles_host) emax = std::max(emax, (double)T.enc_err);
  knn_thr_kernel<<<1, 1, 0, st>>>(thr, emax, all_points ? nullptr : C.plan.nblocks_dev + 4); note_launch();
  QuerySet qs;
  if (all_points) {
    qs.all_points = 1;
    qs.nq = (uint32_t)ix->n;
    qs.nblocks = ix->nkeys;
    qs.blk_beg = ix->ustart;
    qs.blk_key = ix->ukeys;
    qs.qrec = ix->pts32;
    qs.qrec64 = ix->pts64s;
    qs.q64 = ix->xyz64;
  } else {
    QueryPlan& P = C.plan;
    if (P.nblocks_host_version != P.version) {
      if (e == cudaSuccess) e = cudaMemcpyAsync(&P.nblocks, P.nblocks_dev, 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      P.nblocks_host_version = P.version;
    }
    qs.all_points = 0;
    qs.nq = (uint32_t)nq;
    qs.nblocks = P.nblocks;
    qs.blk_beg = P.blk_beg;
    qs.blk_key = P.blk_key;
    qs.qrec = P.qrec;
    qs.qrec64 = P.qrec64;
    qs.q64 = q;
  }
  if (e != cudaSuccess) { tmp.release(st); return cuda_fail(e, "k-NN setup"); }
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const IndexView iv = ix->view();
  if (ix->precision == CG_FP32_OFFSET) {
    const size_t smem = knn_smem<1>();
    cudaFuncSetAttribute(knn_fast_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    {
      ProfScope prof("knn_fast", st);
      knn_fast_kernel<1><<<sms * per, KT, smem, st>>>(iv, qs, thr, k, idx, d2, slow, ctrs, ctrs + 4, C.status);
    }
    note_launch();
    {
      ProfScope prof("knn_slow", st);
      knn_slow_kernel<1><<<sms * 8, 128, 0, st>>>(iv, qs, k, slow, ctrs, idx, d2);
    }
    note_launch();
  } else {
    const size_t smem = knn_smem<0>();
    cudaFuncSetAttribute(knn_fast_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    {
      ProfScope prof("knn_fast", st);
      knn_fast_kernel<0><<<sms * per, KT, smem, st>>>(iv, qs, thr, k, idx, d2, slow, ctrs, ctrs + 4, C.status);
    }
    note_launch();
    {
      ProfScope prof("knn_slow", st);
      knn_slow_kernel<0><<<sms * 8, 128, 0, st>>>(iv, qs, k, slow, ctrs, idx, d2);
    }
    note_launch();
  }
  e = cudaGetLastError();
  tmp.release(st);
  if (e != cudaSuccess) return cuda_fail(e, "k-NN kernels");
  return CG_OK;
}


cg_status knn_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, int k, int32_t* idx, double* d2,
                   cudaStream_t st) {
  return knn_pass(ix, ix->ctx, all_points, q, nq, k, idx, d2, st);
}

cg_status knn_work_alloc(cg_index* ix, KnnWork& w, cudaStream_t st) {
  w.slow = (uint32_t*)w.bufs.get(4 * (size_t)std::max<int64_t>(ix->n, 1), st);
  w.ctrs = (uint32_t*)w.bufs.get(256, st);
  w.thr = (Thresholds*)w.bufs.get(sizeof(Thresholds), st);
  if (!w.slow || !w.ctrs || !w.thr) return fail(CG_ERR_OOM, "device allocation failed (pipeline k-NN work)");
  return CG_OK;
}

// All-points k-NN with the block count read on the device (no host
// synchronisation or allocation).
cg_status knn_replay(cg_index* ix, KnnWork& w, const uint32_t* nkeys_dev, uint32_t cap_nb, int k, int32_t* idx,
                     double* d2, cudaStream_t st) {
  if (k < 1 || k > 64) return fail(CG_ERR_INVALID, "k must be in [1, 64]");
  cudaError_t e = cudaMemsetAsync(w.ctrs, 0, 256, st);
  if (e != cudaSuccess) return cuda_fail(e, "replay memset");
  knn_thr_tiles_kernel<<<1, 32, 0, st>>>(w.thr, ix->tiles, ix->ntiles); note_launch();
  QuerySet qs;
  qs.all_points = 1;
  qs.nq = (uint32_t)ix->n;
  qs.nblocks = cap_nb;
  qs.nblocks_dev = nkeys_dev;
  qs.blk_beg = ix->ustart;
  qs.blk_key = ix->ukeys;
  qs.qrec = ix->pts32;
  qs.qrec64 = ix->pts64s;
  qs.q64 = ix->xyz64;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const IndexView iv = ix->view();
  if (ix->precision == CG_FP32_OFFSET) {
    const size_t smem = knn_smem<1>();
    cudaFuncSetAttribute(knn_fast_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    knn_fast_kernel<1><<<sms * per, KT, smem, st>>>(iv, qs, w.thr, k, idx, d2, w.slow, w.ctrs, w.ctrs + 4,
                                                     ix->status); note_launch();
    knn_slow_kernel<1><<<sms * 8, 128, 0, st>>>(iv, qs, k, w.slow, w.ctrs, idx, d2); note_launch();
  } else {
    const size_t smem = knn_smem<0>();
    cudaFuncSetAttribute(knn_fast_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per = (int)std::max<size_t>(1, std::min<size_t>(8, (227 * 1024) / (smem + 1024)));
    knn_fast_kernel<0><<<sms * per, KT, smem, st>>>(iv, qs, w.thr, k, idx, d2, w.slow, w.ctrs, w.ctrs + 4,
                                                     ix->status); note_launch();
    knn_slow_kernel<0><<<sms * 8, 128, 0, st>>>(iv, qs, k, w.slow, w.ctrs, idx, d2); note_launch();
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "replay k-NN kernels");
  return CG_OK;
}

}  // namespace cg
