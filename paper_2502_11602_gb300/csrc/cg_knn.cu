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
template <> struct KRec<1> { using T = float4; };
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

// Squared distances are non-negative binary64 values or +inf: their bit
// patterns order as unsigned integers, so the comparisons, minima and maxima
// of the (d2, id) order run on the integer pipes (the binary64 pipe of a
// GB300 is about 1/64 of the binary32 rate and is kept for the distances).
__device__ __forceinline__ unsigned long long dbits(double d) { return (unsigned long long)__double_as_longlong(d); }
constexpr unsigned long long kInfBits = 0x7ff0000000000000ull;

// Bound on |d2f - d2| for candidates with d2 about tau (the model of the
// radius thresholds, two-sided, doubled).  Zero for binary64 records.
struct KBound {
  float c1, c0, c2;
  __device__ __forceinline__ float at(float tau) const {
    float t = fmaxf(tau, 0.f);
    return 2.0f * (c1 * sqrtf(t) * 1.0001f + c0 + c2 * t) + 1e-30f;
  }
};

// The band of a precision: alpha = per-axis bound on the binary32 difference
// error (pad_[0] of the k-NN thresholds), beta = relative rounding of the
// squares and sums; zero width for binary64 records (their screen value is
// the exact one rounded up).
template <int PREC>
__device__ __forceinline__ KBound make_kbound(const Thresholds& thr) {
  KBound kb;
  const double u = 5.9604644775390625e-08, U = 1.1102230246251565e-16;
  const double alpha = PREC == 1 ? (double)thr.pad_[0] * (1.0 + u) : 0.0;
  const double beta = PREC == 1 ? (u + U) * (1.0 + 2.0 * U) : 0.0;
  kb.c1 = (float)(2.0 * alpha * (1.0 + beta) * 1.7320508075688774);
  kb.c0 = (float)(3.0 * alpha * alpha);
  kb.c2 = PREC == 1 ? (float)(2.0 * beta + beta * beta + 3.0000002 * u + 4.0 * U) : 1.2e-7f;
  return kb;
}

__device__ __forceinline__ float rec_u_k(const double4_32a& q, const Tile& T, int a) {
  double x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__double2float_rn(__dsub_rn(x, T.lo[a])), T.inv_sf[a]);
}
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
        const unsigned long long ka = dbits(a), kb = dbits(b);
        bool gt = ka > kb || (ka == kb && ia > ib);
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
  const KBound kb = make_kbound<PREC>(thr);
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

// ------------------------------------------------ fast path, binary32 records

// One warp per voxel group, lanes = queries.  The group's box (RB voxels
// around its voxel on each indexed axis) is staged in shared memory, its
// candidates bucketed by their distance D from the group voxel's centre
// (64 buckets, bucket u holds D in [u bw, (u+1) bw)).  Each lane keeps the
// L = k + spare smallest binary32 values of its query in registers (sorted);
// candidates below a lane's current L-th value are queued (8 per lane) and
// merged into the lists whenever a queue fills, so the warp pays for the
// insertions of its busiest lane, not for every lane's.  Before each bucket,
// |p - q| >= D - |q - c| >= u bw - |q - c| bounds every later candidate:
// once that exceeds a lane's L-th value nothing later can enter its list, and
// when it holds for every lane the warp stops scanning.  Then, per lane: the
// certified band (every candidate within twice the error bound of the k-th
// value is in the list, as the list keeps every candidate below its L-th
// value, which must lie beyond that band), binary64 values of the band,
// order (d2, id), and the stop test against the box wall.
// A query the box cannot decide (its k-th may lie outside the box) goes to
// the bounded search with the box's exact k-th value as an upper bound of
// the true one; groups too large to stage go to the ring-by-ring path.
constexpr int K5_NB = 64;
constexpr int K5_Q = 12;  // queued candidates per lane

// Shared memory of a slot of gw warps: the group's staged box (records,
// buckets, spans, a few broadcast words), then one candidate queue per warp.
template <int KC>
struct K5Smem {
  static constexpr size_t tables = (16 * (size_t)KC + (size_t)KC + 4 * (2 * K5_NB + 2) + 4 * 2 * 12 + 4 * 4 + 15) / 16 * 16;
  static constexpr size_t queue = 4 * (size_t)K5_Q * 32;
  __host__ __device__ static constexpr size_t per_slot(int gw) { return tables + queue * (size_t)gw; }
};

// A candidate's binary32 value with its staged slot j (< 2048) in the low 11
// mantissa bits: the lists and queues then move one word per entry.  The
// packed value p orders as the value up to a relative 2^-12 (|p - d| <
// 2^-12 d, plus 2^-138 at d = 0); the band and the stop test below widen by
// that much.  d is clamped below +inf so that no NaN pattern arises.
__device__ __forceinline__ float k5_pack(float d, uint32_t j) {
  return __uint_as_float((__float_as_uint(fminf(d, 3.0e38f)) & ~0x7ffu) | j);
}
__device__ __forceinline__ uint32_t k5_slot(float p) { return __float_as_uint(p) & 0x7ffu; }

template <int L>
__device__ __forceinline__ void topl_insert1(float (&v)[L], float p) {
  // v ascending: p goes before the first entry it is below; every position
  // is computed from the old list (no dependent chain of selects)
  bool c[L];
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = p < v[i];
#pragma unroll
  for (int i = L - 1; i > 0; --i) v[i] = c[i - 1] ? v[i - 1] : (c[i] ? p : v[i]);
  v[0] = c[0] ? p : v[0];
}

// Barrier of the GW warps of one slot (named barrier 1 + slot).
template <int GW>
__device__ __forceinline__ void k5_slot_sync(int slot) {
  if (GW == 1) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(GW * 32) : "memory");
}

// wall2_lower for one box given by scalars (no array whose address is taken)
__device__ __forceinline__ float wall2_box(const float4& q, const Tile& T, int dim, int lo0, int lo1, int lo2, int hi0,
                                          int hi1, int hi2, float e_q) {
  float w = INFINITY;
  const float qa[3] = {q.x, q.y, q.z};
  const int lov[3] = {lo0, lo1, lo2}, hiv[3] = {hi0, hi1, hi2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      const float u = __fmul_rn(__fadd_rn(qa[a], T.D[a]), T.inv_sf[a]);
      const float eta = T.eta + (fabsf(u) + fabsf(qa[a]) * T.inv_sf[a]) * 3.0e-7f + e_q * T.inv_sf[a];
      if (lov[a] > 0) w = fminf(w, (u - (float)lov[a] - eta) * (float)T.s[a]);
      if (hiv[a] < T.n[a] - 1) w = fminf(w, ((float)(hiv[a] + 1) - u - eta) * (float)T.s[a]);
    }
  }
  if (w == INFINITY) return INFINITY;
  if (w <= 0.f) return 0.f;
  return __fmul_rd(__fmul_rd(w, w), 0.99999f);
}

__device__ __forceinline__ float centre_dist(const float4& r, float cx, float cy, float cz, float zw) {
  const float dx = r.x - cx, dy = r.y - cy, dz = (r.z - cz) * zw;
  return sqrtf(dx * dx + dy * dy + dz * dz);
}

template <int L>
__device__ __forceinline__ void topl_insert(float (&v)[L], uint32_t (&id)[L], float d, uint32_t j) {
  // v ascending: d goes before the first entry it is below (after equal
  // ones); every position is computed from the old list, so the selects do
  // not form one dependent chain
  bool c[L];
#pragma unroll
  for (int i = 0; i < L; ++i) c[i] = d < v[i];
#pragma unroll
  for (int i = L - 1; i > 0; --i) {
    v[i] = c[i - 1] ? v[i - 1] : (c[i] ? d : v[i]);
    id[i] = c[i - 1] ? id[i - 1] : (c[i] ? j : id[i]);
  }
  v[0] = c[0] ? d : v[0];
  id[0] = c[0] ? j : id[0];
}

template <int KC, int L, int NWARP, int GW>
__global__ void __launch_bounds__(NWARP * 32) knn5_kernel(IndexView ix, QuerySet qs, const Thresholds* __restrict__ thr_p,
                                                          int k, int32_t* __restrict__ out_idx,
                                                          double* __restrict__ out_d2, uint32_t* __restrict__ slow_list,
                                                          uint32_t* slow_cnt, uint32_t* __restrict__ bslot,
                                                          float* __restrict__ br2, uint32_t* bcnt, unsigned* work,
                                                          uint32_t* status, uint32_t kcls) {
  if (replan_pending(status)) return;  // the later kernels then find empty lists
  constexpr int RB = 1;
  using S = K5Smem<KC>;
  static_assert(NWARP % GW == 0 && NWARP / GW <= 15, "slot shape");
  constexpr int ST = GW * 32;  // threads per slot
  extern __shared__ __align__(32) unsigned char smem[];
  const int warp = (int)(threadIdx.x >> 5), slot = warp / GW, wis = warp % GW;
  const unsigned lane = threadIdx.x & 31u;
  const uint32_t tis = (uint32_t)wis * 32u + lane;  // thread in slot
  unsigned char* base = smem + (size_t)slot * S::per_slot(GW);
  float4* recs = reinterpret_cast<float4*>(base);                 // [KC] in bucket order
  uint8_t* bkt = reinterpret_cast<uint8_t*>(recs + KC);           // [KC] bucket of each span-order candidate
  uint32_t* bstart = reinterpret_cast<uint32_t*>(bkt + KC);       // [NB + 1]
  uint32_t* cursor = bstart + K5_NB + 1;                          // [NB + 1]
  uint32_t* sp_start = cursor + K5_NB + 1;                        // [12]
  uint32_t* sp_off = sp_start + 12;                               // [12]
  uint32_t* sbox = sp_off + 12;                                   // [4]: group, K
  float* qd = reinterpret_cast<float*>(base + S::tables + S::queue * (size_t)wis);  // [Q][32] queued packed values
  const Thresholds thr = *thr_p;
  const KBound kb = make_kbound<1>(thr);
  const float4* __restrict__ pts = ix.pts32;
  const float4* __restrict__ qsrc = qs.all_points ? pts : qs.qrec;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  const int dim = ix.dim;
  for (;;) {
    // the slot's next group; its box is staged by all GW warps, whose
    // chunks of 32 queries then share it
    if (tis == 0) sbox[0] = atomicAdd(work, 1u);
    k5_slot_sync<GW>(slot);
    const uint32_t b = sbox[0];
    k5_slot_sync<GW>(slot);
    if (b >= qs_nblocks(qs)) break;
    const uint32_t qb0 = qs.blk_beg[b], qb1 = qs.blk_beg[b + 1];
    const uint32_t bkey = qs.blk_key[b];
    const Tile& T = ix.tiles[ix.ntiles == 1 ? 0 : tile_of_key(ix.tiles, ix.ntiles, bkey)];
    const uint32_t g = bkey - T.key_base;
    int c0, c1, c2 = 0;
    if (dim == 2) { c0 = (int)(g / (uint32_t)T.n[1]); c1 = (int)(g % (uint32_t)T.n[1]); }
    else { c2 = (int)(g % (uint32_t)T.n[2]); const uint32_t ij = g / (uint32_t)T.n[2]; c0 = (int)(ij / (uint32_t)T.n[1]); c1 = (int)(ij % (uint32_t)T.n[1]); }
    const int lo0 = max(c0 - RB, 0), hi0 = min(c0 + RB, T.n[0] - 1);
    const int lo1 = max(c1 - RB, 0), hi1 = min(c1 + RB, T.n[1] - 1);
    const int lo2 = dim == 3 ? max(c2 - RB, 0) : 0, hi2 = dim == 3 ? min(c2 + RB, T.n[2] - 1) : T.n[2] - 1;
    const bool exhausted = lo0 == 0 && hi0 == T.n[0] - 1 && lo1 == 0 && hi1 == T.n[1] - 1 &&
                           (dim == 2 || (lo2 == 0 && hi2 == T.n[2] - 1));
    const int ni = hi0 - lo0 + 1, nj = hi1 - lo1 + 1;
    const int nsp = dim == 2 ? ni : ni * nj;  // <= NSP
    // spans (one contiguous run of sorted points per grid row / column),
    // computed by every warp of the slot
    uint32_t len = 0, st0 = 0;
    if ((int)lane < nsp) {
      uint32_t k0, k1;
      if (dim == 2) {
        const uint32_t row = (uint32_t)(lo0 + (int)lane) * (uint32_t)T.n[1];
        k0 = T.key_base + row + (uint32_t)lo1;
        k1 = T.key_base + row + (uint32_t)hi1;
      } else {
        const int i = lo0 + (int)lane / nj, j = lo1 + (int)lane % nj;
        const uint32_t col = ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
        k0 = T.key_base + col + (uint32_t)lo2;
        k1 = T.key_base + col + (uint32_t)hi2;
      }
      const uint2 sp = row_span(ix, T, k0, k1);
      st0 = sp.x;
      len = sp.y - sp.x;
    }
    uint32_t incl = len;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    const uint32_t K = __shfl_sync(0xffffffffu, incl, 31);
    // size classes: 0: K <= 512, 1: K <= 1024, 2: K <= 2048 (and the groups too large to stage)
    if (kcls == 0 ? K > 512u : (kcls == 1 ? (K <= 512u || K > 1024u) : K <= 1024u)) continue;
    if (K > (uint32_t)KC) {  // too large to stage: the ring-by-ring path
      for (uint32_t t = qb0 + tis; t < qb1; t += ST) slow_list[atomicAdd(slow_cnt, 1u)] = __float_as_uint(qsrc[t].w);
      continue;
    }
    if (wis == 0 && (int)lane < nsp) { sp_start[lane] = st0; sp_off[lane] = incl - len; }
    // the group voxel's centre in offset coordinates and the bucket width
    const float cx = __fsub_rn(__fmul_rn((float)c0 + 0.5f, (float)T.s[0]), T.D[0]);
    const float cy = __fsub_rn(__fmul_rn((float)c1 + 0.5f, (float)T.s[1]), T.D[1]);
    const float cz = dim == 3 ? __fsub_rn(__fmul_rn((float)c2 + 0.5f, (float)T.s[2]), T.D[2]) : 0.f;
    const float zw = dim == 3 ? 1.f : 0.f;  // z counts in the centre distance of 3D grids only
    const float smax = fmaxf(fmaxf((float)T.s[0], (float)T.s[1]), dim == 3 ? (float)T.s[2] : 0.f);
    const float bw = (dim == 2 ? 1.42f : 1.74f) * ((float)RB + 0.5f) * smax / (float)K5_NB;
    const float inv_bw = 1.0f / bw;
    for (int u = (int)tis; u <= K5_NB; u += ST) bstart[u] = 0u;
    k5_slot_sync<GW>(slot);
    // bucket counts, then starts, then the records in bucket order
    for (int r = 0; r < nsp; ++r) {
      const uint32_t o = sp_off[r], l = (r + 1 < nsp ? sp_off[r + 1] : K) - o, s0 = sp_start[r];
      for (uint32_t t = tis; t < l; t += ST) {
        const float4 r4 = __ldg(pts + s0 + t);
        const int u = min(K5_NB - 1, (int)(centre_dist(r4, cx, cy, cz, zw) * inv_bw));
        bkt[o + t] = (uint8_t)u;
        atomicAdd(&bstart[u], 1u);
      }
    }
    k5_slot_sync<GW>(slot);
    if (wis == 0) {
      const uint32_t a0 = bstart[2 * lane], a1 = bstart[2 * lane + 1];
      uint32_t inc2 = a0 + a1;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc2, o);
        if (lane >= (unsigned)o) inc2 += y;
      }
      const uint32_t ex = inc2 - a0 - a1;
      __syncwarp();
      bstart[2 * lane] = ex;
      bstart[2 * lane + 1] = ex + a0;
      cursor[2 * lane] = ex;
      cursor[2 * lane + 1] = ex + a0;
      if (lane == 31) bstart[K5_NB] = K;
    }
    k5_slot_sync<GW>(slot);
    for (int r = 0; r < nsp; ++r) {
      const uint32_t o = sp_off[r], l = (r + 1 < nsp ? sp_off[r + 1] : K) - o, s0 = sp_start[r];
      for (uint32_t t = tis; t < l; t += ST) recs[atomicAdd(&cursor[bkt[o + t]], 1u)] = __ldg(pts + s0 + t);
    }
    k5_slot_sync<GW>(slot);
    // queries, one per lane; each warp of the slot its own chunks of 32
    for (uint32_t qc = qb0 + 32u * (uint32_t)wis; qc < qb1; qc += 32u * GW) {
      __syncwarp();
      const bool live = qc + lane < qb1;
      const float4 q = live ? qsrc[qc + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
      const uint32_t qid = __float_as_uint(q.w);
      const float rq = centre_dist(q, cx, cy, cz, zw);
      float v[L];  // packed values (k5_pack), ascending
#pragma unroll
      for (int i = 0; i < L; ++i) v[i] = INFINITY;
      float gate = INFINITY;  // the L-th packed value at the last merge
      uint32_t nqd = 0;       // queued candidates of this lane
      for (int u = 0; u < K5_NB; ++u) {
        const uint32_t s0 = bstart[u], s1 = bstart[u + 1];
        if (s0 == s1) continue;
        // later candidates p have |p - q| >= t, so d2(p) >= t^2, their
        // binary32 value is at least t^2 - B(t^2) (B grows slower than d2)
        // and their packed value at least that times 1 - 2^-11
        const float t = __fsub_rd(__fsub_rd((float)u * bw, rq), 1e-3f * bw + 1e-5f);
        const float t2 = __fmul_rd(t, t);
        const bool done = !live || (t > 0.f && __fmul_rd(__fsub_rd(t2, kb.at(t2)), 0.99951171875f) > gate);
        if (__all_sync(0xffffffffu, done)) break;
        for (uint32_t j = s0; j < s1; j += 2) {  // two candidates per step
          const bool two = j + 1 < s1;
          const float4 p = recs[j];
          const float4 p1 = recs[two ? j + 1 : j];
          const float dx = __fsub_rn(p.x, q.x), dy = __fsub_rn(p.y, q.y), dz = __fsub_rn(p.z, q.z);
          const float d = k5_pack(__fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx))), j);
          const float ex1 = __fsub_rn(p1.x, q.x), ey1 = __fsub_rn(p1.y, q.y), ez1 = __fsub_rn(p1.z, q.z);
          const float d1 = k5_pack(__fmaf_rn(ez1, ez1, __fmaf_rn(ey1, ey1, __fmul_rn(ex1, ex1))), j + 1);
          if (live && d < gate) qd[(nqd++) * 32 + lane] = d;
          if (live && two && d1 < gate) qd[(nqd++) * 32 + lane] = d1;
          if (__any_sync(0xffffffffu, nqd >= (uint32_t)K5_Q - 1u)) {  // merge the queues
            for (uint32_t e = 0; e < nqd; ++e) {
              const float de = qd[e * 32 + lane];
              if (de < v[L - 1]) topl_insert1<L>(v, de);
            }
            nqd = 0;
            gate = v[L - 1];
          }
        }
      }
      for (uint32_t e = 0; e < nqd; ++e) {
        const float de = qd[e * 32 + lane];
        if (de < v[L - 1]) topl_insert1<L>(v, de);
      }
      if (!live) continue;
      // found: candidates in the list (all of the box when it holds fewer than L)
      int found = 0;
#pragma unroll
      for (int i = 0; i < L; ++i) found += v[i] < INFINITY ? 1 : 0;
      const int kk = min(k, found);
      bool undecided = false;
      float W2 = INFINITY;
      if (!exhausted) {
        W2 = wall2_box(q, T, dim, lo0, lo1, lo2, hi0, hi1, hi2, thr.e_q);
        undecided = !(W2 > 0.f) || found < k;
      }
      // the certified band: every candidate within 2 B of the k-th value
      int m = 0;
      if (!undecided && kk > 0) {
        float tau = 0.f;  // v is ascending: the k-th value is the largest of the first kk
#pragma unroll
        for (int i = 0; i < L; ++i) tau = fmaxf(tau, i < kk ? v[i] : 0.f);
        // k packed values <= tau: their binary32 values are at most
        // tau / (1 - 2^-12), the exact k-th at most that plus B; every point
        // with an exact value up to there has a packed value up to
        // (tau / (1 - 2^-12) + 2 B) (1 + 2^-12) <= cut
        const float cut = __fadd_ru(__fadd_ru(__fmul_ru(tau, 1.0009765625f), 2.0f * __fmul_ru(kb.at(tau), 1.001f)),
                                    1.0e-37f);
#pragma unroll
        for (int i = 0; i < L; ++i) m += v[i] <= cut ? 1 : 0;
        if (m == L && v[L - 1] < INFINITY) undecided = true;  // the band may continue past the list
      }
      double ex[L];
      uint32_t cid[L];
      double kth = INFINITY;
      if (!undecided) {
        kth = 0.0;
        // binary64 values of the band, order (d2, id)
#pragma unroll
        for (int i = 0; i < L; ++i) {
          if (i < m) {
            cid[i] = __float_as_uint(recs[k5_slot(v[i])].w);
            ex[i] = exact_d2(ix.xyz64 + 3 * (size_t)cid[i], q64 + 3 * (size_t)qid);
          } else {
            cid[i] = 0xffffffffu;
            ex[i] = INFINITY;
          }
        }
        for (int pass = 0; pass < L; ++pass) {  // nearly sorted already: a few passes
          bool sw = false;
#pragma unroll
          for (int i = 0; i + 1 < L; ++i) {
            const unsigned long long ka = dbits(ex[i]), kb = dbits(ex[i + 1]);
            const bool gt = ka > kb || (ka == kb && cid[i] > cid[i + 1]);
            if (gt) {
              const double te = ex[i]; ex[i] = ex[i + 1]; ex[i + 1] = te;
              const uint32_t tc = cid[i]; cid[i] = cid[i + 1]; cid[i + 1] = tc;
              sw = true;
            }
          }
          if (!sw) break;
        }
        unsigned long long kbits = 0;
#pragma unroll
        for (int i = 0; i < L; ++i) kbits = max(kbits, i < kk ? dbits(ex[i]) : 0ull);  // ex ascending
        kth = __longlong_as_double((long long)kbits);
        undecided = !exhausted && !(kth < (double)W2);
      }
      if (undecided) {
        if (found >= k && kk > 0 && dbits(kth) < kInfBits) {
          // the k-th value inside the box bounds the true k-th from above:
          // the bounded search covers that sphere
          const uint32_t e = atomicAdd(bcnt, 1u);
          bslot[e] = qc + lane;
          br2[e] = __double2float_ru(kth);
        } else {
          slow_list[atomicAdd(slow_cnt, 1u)] = qid;
        }
        continue;
      }
      int32_t* oi = out_idx + (size_t)qid * k;
      double* od = out_d2 ? out_d2 + (size_t)qid * k : nullptr;
#pragma unroll
      for (int i = 0; i < L; ++i) {
        if (i < k) {
          const bool ok = i < kk;
          oi[i] = ok ? (int32_t)cid[i] : -1;
          if (od) od[i] = ok ? ex[i] : INFINITY;
        }
      }
    }
  }
}

// ------------------------------------------------------------ bounded search

// Queries whose k-th neighbour may lie outside their group's box, with an
// exact upper bound r2u on the true k-th squared distance (the k-th inside
// the box): one warp per query visits every voxel meeting the sphere of
// radius sqrt(r2u) (the range of Algorithm 1, widened by the proven pad),
// keeps the candidates whose binary32 value is within the error band of
// r2u (a superset of every point with d2 <= r2u, hence of the k nearest),
// computes their binary64 values and sorts them by (d2, id).  More than
// KB_CAP such candidates send the query to the ring-by-ring path.
constexpr int KB_CAP = 512;  // a power of two: the sort pads the list to one
constexpr int KB_WARPS = 4;

__global__ void __launch_bounds__(KB_WARPS * 32, 7) knn_bounded_kernel(IndexView ix, QuerySet qs,
                                                                     const Thresholds* __restrict__ thr_p, int k,
                                                                     const uint32_t* __restrict__ bslot,
                                                                     const float* __restrict__ br2,
                                                                     const uint32_t* bcnt, int32_t* __restrict__ out_idx,
                                                                     double* __restrict__ out_d2,
                                                                     uint32_t* __restrict__ slow_list,
                                                                     uint32_t* slow_cnt, const uint32_t* status) {
  if (replan_pending(status)) return;
  // per warp: the candidates' ids and binary32 values, then the band's ids
  // and exact values (at most KB_CAP / 2 of them)
  __shared__ double s_d2[KB_WARPS][KB_CAP / 2];
  __shared__ float s_f[KB_WARPS][KB_CAP];
  __shared__ uint32_t s_id[KB_WARPS][KB_CAP];
  __shared__ uint32_t s_bid[KB_WARPS][KB_CAP / 2];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  __shared__ uint32_t s_zst[KB_WARPS][64], s_zoff[KB_WARPS][64];  // height-cut column spans
  double* wd2 = s_d2[warp];
  float* wf = s_f[warp];
  uint32_t* wid = s_id[warp];
  uint32_t* bid = s_bid[warp];
  uint32_t* zst = s_zst[warp];
  uint32_t* zoff = s_zoff[warp];
  const Thresholds thr = *thr_p;
  const KBound kb = make_kbound<1>(thr);
  const float4* __restrict__ pts = ix.pts32;
  const float4* __restrict__ qsrc = qs.all_points ? pts : qs.qrec;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  const int dim = ix.dim;
  const uint32_t n = *bcnt;
  for (uint32_t e = blockIdx.x * KB_WARPS + warp; e < n; e += gridDim.x * KB_WARPS) {
    const float4 q = qsrc[bslot[e]];
    const uint32_t qid = __float_as_uint(q.w);
    const float r2u = br2[e];
    const Tile& T = ix.tiles[(qs.all_points && ix.ntiles > 1) ? tile_of_id(ix.tiles, ix.ntiles, qid) : 0];
    const float r = __fsqrt_ru(r2u);
    const float qa[3] = {q.x, q.y, q.z};
    int lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        const float u = __fmul_rn(__fadd_rn(qa[a], T.D[a]), T.inv_sf[a]);
        const float rr = __fmul_ru(__fmul_ru(r, T.inv_sf[a]), 1.0000005f);
        float pad = __fadd_ru(__fadd_ru(rr, T.eta), __fmul_ru(__fadd_ru(fabsf(u), fabsf(qa[a]) * T.inv_sf[a]), 3.0e-7f));
        pad = __fadd_ru(pad, __fmul_ru(thr.e_q, T.inv_sf[a]));
        const float ul = fminf(fmaxf(__fsub_rd(u, pad), -1.0e9f), 1.0e9f);
        const float uh = fminf(fmaxf(__fadd_ru(u, pad), -1.0e9f), 1.0e9f);
        lo[a] = max((int)floorf(ul), 0);
        hi[a] = min((int)floorf(uh), T.n[a] - 1);
      } else {
        lo[a] = 0;
        hi[a] = T.n[a] - 1;
      }
    }
    const float cut = __fadd_ru(r2u, 2.0f * kb.at(r2u));
    uint32_t m = 0;
    const int ni = hi[0] - lo[0] + 1, nj = hi[1] - lo[1] + 1;
    // 2D grids with height-sorted columns: every voxel column of the box cut
    // to the candidate test's height range.  A record passes the test only
    // if RN(dz^2) <= cut (dz = RN(z~_p - z~_q)), so |z~_p - z~_q| <=
    // sqrt(cut) (1 + 2^-23); the window takes 1 + 1e-6.  The columns' spans
    // are found lane-parallel (a bisection per column), then all lanes walk
    // the concatenation.
    const bool zcut = dim == 2 && ix.pts32z != nullptr && ni > 0 && nj > 0 && ni * nj <= 64;
    if (zcut) {
      const float4* __restrict__ zs = ix.pts32z;
      const int nc = ni * nj;
      const float zh = __fmul_ru(__fsqrt_ru(cut), 1.000001f);
      const float zlo = __fsub_rd(q.z, zh), zhi = __fadd_ru(q.z, zh);
      uint32_t st2[2] = {0u, 0u}, ln2[2] = {0u, 0u};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int c = (int)lane + 32 * h;
        if (c < nc) {
          const uint32_t key = T.key_base + (uint32_t)(lo[0] + c / nj) * (uint32_t)T.n[1] + (uint32_t)(lo[1] + c % nj);
          uint2 sp = voxel_span(ix, T, key);
          if (sp.y - sp.x > 1u && sp.y - sp.x <= kZsortMax) {  // a height-sorted run
            // first height >= zlo (a), first height > zhi (d); the two
            // bisections step together, so their loads overlap
            uint32_t a = sp.x, b = sp.y, d = sp.x, f = sp.y;
            while (a < b || d < f) {
              const uint32_t m1 = (a + b) >> 1, m2 = (d + f) >> 1;
              const float z1 = a < b ? __ldg(&zs[m1].z) : 0.f;
              const float z2 = d < f ? __ldg(&zs[m2].z) : 0.f;
              if (a < b) {
                if (z1 < zlo) a = m1 + 1;
                else b = m1;
              }
              if (d < f) {
                if (z2 <= zhi) d = m2 + 1;
                else f = m2;
              }
            }
            sp = make_uint2(a, d > a ? d : a);
          }
          st2[h] = sp.x;
          ln2[h] = sp.y - sp.x;
        }
      }
      // offsets of the columns in the order c = 0 .. nc - 1
      uint32_t base = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t incl = ln2[h];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= (uint32_t)o) incl += y;
        }
        const int c = (int)lane + 32 * h;
        if (c < nc) {
          zst[c] = st2[h];
          zoff[c] = base + incl - ln2[h];
        }
        base += __shfl_sync(0xffffffffu, incl, 31);
      }
      const uint32_t total = base;
      __syncwarp();
      for (uint32_t i0 = 0; i0 < total; i0 += 128) {  // four loads in flight per lane
        float4 p[4];
        bool pick[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t i = i0 + 32u * u + lane;
          pick[u] = i < total;
          p[u] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (pick[u]) {
            int a = 0, b = nc - 1;  // the column holding candidate i
            while (a < b) {
              const int mid = (a + b + 1) >> 1;
              if (zoff[mid] <= i) a = mid;
              else b = mid - 1;
            }
            p[u] = __ldg(zs + zst[a] + (i - zoff[a]));
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float dx = __fsub_rn(p[u].x, q.x), dy = __fsub_rn(p[u].y, q.y), dz = __fsub_rn(p[u].z, q.z);
          const float dv = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
          pick[u] = pick[u] && dv <= cut;
          const unsigned bm = __ballot_sync(0xffffffffu, pick[u]);
          const uint32_t pos = m + __popc(bm & lanemask_lt());
          if (pick[u] && pos < (uint32_t)KB_CAP) {
            wid[pos] = __float_as_uint(p[u].w);
            wf[pos] = dv;
          }
          m += __popc(bm);
        }
      }
      __syncwarp();
    }
    const int ncol = (zcut || ni <= 0 || nj <= 0) ? 0 : (dim == 2 ? ni : ni * nj);
    for (int cidx = 0; cidx < ncol; ++cidx) {
      uint32_t k0, k1;
      if (dim == 2) {
        const uint32_t row = (uint32_t)(lo[0] + cidx) * (uint32_t)T.n[1];
        k0 = T.key_base + row + (uint32_t)lo[1];
        k1 = T.key_base + row + (uint32_t)hi[1];
      } else {
        const int i = lo[0] + cidx / nj, j = lo[1] + cidx % nj;
        const uint32_t col = ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2];
        k0 = T.key_base + col + (uint32_t)lo[2];
        k1 = T.key_base + col + (uint32_t)hi[2];
      }
      const uint2 sp = row_span(ix, T, k0, k1);
      for (uint32_t t0 = sp.x; t0 < sp.y; t0 += 128) {  // four loads in flight per lane
        float4 p[4];
        bool pick[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint32_t t = t0 + 32u * u + lane;
          pick[u] = t < sp.y;
          p[u] = pick[u] ? __ldg(pts + t) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float dx = __fsub_rn(p[u].x, q.x), dy = __fsub_rn(p[u].y, q.y), dz = __fsub_rn(p[u].z, q.z);
          const float dv = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
          pick[u] = pick[u] && dv <= cut;
          const unsigned bm = __ballot_sync(0xffffffffu, pick[u]);
          const uint32_t pos = m + __popc(bm & lanemask_lt());
          if (pick[u] && pos < (uint32_t)KB_CAP) {
            wid[pos] = __float_as_uint(p[u].w);
            wf[pos] = dv;
          }
          m += __popc(bm);
        }
      }
    }
    if (m > (uint32_t)KB_CAP || m < (uint32_t)k) {  // too many (or, impossibly, too few): the ring path
      if (lane == 0) slow_list[atomicAdd(slow_cnt, 1u)] = qid;
      __syncwarp();
      continue;
    }
    __syncwarp();
    // the k-th smallest binary32 value tau (bisection on the bit patterns of
    // the non-negative values), then the band d2f <= tau + 2 B(tau): it
    // holds every point of the true k nearest (there are k candidates with
    // d2f <= tau, so the exact k-th is at most tau + B(tau))
    uint32_t klo = 0u, khi = 0x7f800000u;
    while (klo < khi) {
      const uint32_t mid = klo + ((khi - klo) >> 1);
      uint32_t c = 0;
      for (uint32_t i = lane; i < m; i += 32) c += __float_as_uint(wf[i]) <= mid ? 1u : 0u;
      c = __reduce_add_sync(0xffffffffu, c);
      if (c >= (uint32_t)k) khi = mid;
      else klo = mid + 1u;
    }
    const float tau = __uint_as_float(klo);
    const float bcut = __fadd_ru(tau, 2.0f * kb.at(tau));
    // the band, compacted to the front of the exact list (slots [0, mb))
    uint32_t mb = 0;
    for (uint32_t i0 = 0; i0 < m; i0 += 32) {
      const uint32_t i = i0 + lane;
      const bool in = i < m && wf[i] <= bcut;
      const uint32_t cid = in ? wid[i] : 0u;
      const unsigned bm = __ballot_sync(0xffffffffu, in);
      const uint32_t pos = mb + __popc(bm & lanemask_lt());
      if (in && pos < (uint32_t)(KB_CAP / 2)) bid[pos] = cid;
      mb += __popc(bm);
    }
    if (mb > (uint32_t)(KB_CAP / 2)) {  // a band this wide (ties): the ring path
      if (lane == 0) slow_list[atomicAdd(slow_cnt, 1u)] = qid;
      __syncwarp();
      continue;
    }
    __syncwarp();
    int P = 32;
    while (P < (int)mb) P <<= 1;
    for (int i = (int)lane; i < P; i += 32) {
      if (i < (int)mb) wd2[i] = exact_d2(ix.xyz64 + 3 * (size_t)bid[i], q64 + 3 * (size_t)qid);
      else { wd2[i] = INFINITY; bid[i] = 0xffffffffu; }
    }
    __syncwarp();
    warp_sort_list(wd2, bid, P);
    for (int i = (int)lane; i < k; i += 32) {
      out_idx[(size_t)qid * k + i] = (int32_t)bid[i];
      if (out_d2) out_d2[(size_t)qid * k + i] = wd2[i];
    }
    __syncwarp();
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
  const unsigned long long ka = dbits(a), kb = dbits(b);
  return ka < kb || (ka == kb && ia < ib);
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

__device__ void knn_thresholds(Thresholds* out, double e_p, double e_q);

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
    // the query's voxel (clamped), from binary64 on lane 0 (the binary64
    // pipe is narrow), then broadcast
    int cc[3] = {0, 0, 0};
    if (lane == 0)
      for (int a = 0; a < ix.dim; ++a) {
        double v = floor(__ddiv_rn(__dsub_rn(__ldg(c + a), T.lo[a]), T.s[a]));
        v = fmin(fmax(v, 0.0), (double)(T.n[a] - 1));
        cc[a] = (int)v;
      }
    for (int a = 0; a < 3; ++a) cc[a] = __shfl_sync(0xffffffffu, cc[a], 0);
    // the query's record in the tile's frame and the screen's error bound
    using R = typename KRec<PREC>::T;
    const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
    R qr;
    KBound kb;
    if constexpr (PREC == 1) {
      float4 qf = make_float4(0.f, 0.f, 0.f, 0.f);
      KBound k0 = {0.f, 0.f, 0.f};
      if (lane == 0) {  // binary64 on one lane
        qf.x = __double2float_rn(__dsub_rn(__ldg(c), T.origin[0]));
        qf.y = __double2float_rn(__dsub_rn(__ldg(c + 1), T.origin[1]));
        qf.z = __double2float_rn(__dsub_rn(__ldg(c + 2), T.origin[2]));
        const double m = (double)fmaxf(fabsf(qf.x), fmaxf(fabsf(qf.y), fabsf(qf.z)));
        Thresholds th;
        knn_thresholds(&th, (double)T.enc_err, ldexp(m, -24) * (1.0 + 1e-6) + ldexp(m, -52) + 1e-30);
        k0 = make_kbound<1>(th);
      }
      qr = make_float4(__shfl_sync(0xffffffffu, qf.x, 0), __shfl_sync(0xffffffffu, qf.y, 0),
                       __shfl_sync(0xffffffffu, qf.z, 0), 0.f);
      kb.c1 = __shfl_sync(0xffffffffu, k0.c1, 0);
      kb.c0 = __shfl_sync(0xffffffffu, k0.c0, 0);
      kb.c2 = __shfl_sync(0xffffffffu, k0.c2, 0);
    } else {
      qr = make_double4_32a(__ldg(c), __ldg(c + 1), __ldg(c + 2), 0.0);
      Thresholds th;
      th.pad_[0] = 0.f;
      kb = make_kbound<0>(th);
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
            const double worst = wl_get(L, k - 1);
            const uint32_t worst_id = __shfl_sync(0xffffffffu, (k - 1) < 32 ? L.id[0] : L.id[1], (k - 1) & 31);
            const float wf = __double2float_ru(worst);
            if (t < sp.y) {
              // the binary32 screen: a candidate whose value, less its error
              // bound, exceeds the current k-th cannot enter the list
              const R rec = pts[t];
              id = krec_id(rec);
              const float df = kd2f(rec, qr);
              if (!(__fsub_rd(df, kb.at(df)) > wf)) d = exact_d2(ix.xyz64 + 3 * (size_t)id, c);
            }
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
      if (dbits(kth) < kInfBits) {
        int stop = 0;
        if (lane == 0) {  // binary64 on one lane, then broadcast
          double w = INFINITY;
          for (int a = 0; a < ix.dim; ++a) {
            double x = __ldg(c + a);
            if (lo[a] > 0) w = fmin(w, x - (T.lo[a] + (double)lo[a] * T.s[a]));
            if (hi[a] < T.n[a] - 1) w = fmin(w, (T.lo[a] + (double)(hi[a] + 1) * T.s[a]) - x);
          }
          // margin for the rounding of the voxel keys and of the wall itself
          double slack = 1e-12 * (fabs(T.lo[0]) + fabs(T.lo[1]) + fabs(T.lo[2]) + 1.0);
          w -= slack;
          stop = (w > 0 && kth < w * w * (1.0 - 1e-12)) ? 1 : 0;
        }
        if (__shfl_sync(0xffffffffu, stop, 0)) break;
      }
    }
    // write out: slot s lives in lane s % 32, register s / 32
    for (int s = 0; s < k; ++s) {
      double d = wl_get(L, s);
      uint32_t id = __shfl_sync(0xffffffffu, s < 32 ? L.id[0] : L.id[1], s & 31);
      if (lane == 0) {
        bool ok = dbits(d) < kInfBits;
        out_idx[(size_t)qid * k + s] = ok ? (int32_t)id : -1;
        if (out_d2) out_d2[(size_t)qid * k + s] = ok ? d : INFINITY;
      }
    }
  }
}

// Algorithm 2 step by step (Section 3.4.2), one warp per query: the radius r
// in binary64, each iteration visiting the voxels of the bounding box of
// B(c, r) (widened by one voxel on each side and clamped, as the kernel
// search's voxel range) outside the taboo box T of Section 3.5, the k best
// candidates under (d2, id) in the warp's list, and r grown by the policy:
//   0 (monotone)  r + s, s the smallest voxel side;
//   1 (density)   with P^ non-empty and |P^| changed since the previous
//                 iteration, r = (3 k / (4 pi rho))^(1/3) for the density
//                 rho = |P^| / ((4/3) pi r^3) of the ball; else r + s.
// |P^| (the candidates within r) is read off the list: at least k when its
// k-th entry is within r, else every candidate within r is in the list.  The
// search ends when |P^| >= k or T covers the grid; visited = |T|.
// One query (e) of Algorithm 2 step by step, by one warp.
template <int PREC>
__device__ void knn_grow_one(const IndexView& ix, const double* __restrict__ q, uint32_t e, int k, int policy,
                             int32_t* __restrict__ out_idx, double* __restrict__ out_d2,
                             long long* __restrict__ visited, uint32_t* status) {
  const unsigned lane = threadIdx.x & 31u;
  const Tile& T = ix.tiles[0];
  const int nax = ix.dim;
  double smin = fmin(T.s[0], T.s[1]);
  if (nax == 3) smin = fmin(smin, T.s[2]);
  const double kPi = 3.14159265358979323846;
  {
    const double* c = q + 3 * (size_t)e;
    const double cx[3] = {__ldg(c), __ldg(c + 1), __ldg(c + 2)};
    WarpList L;
    L.d[0] = L.d[1] = INFINITY;
    L.id[0] = L.id[1] = 0xffffffffu;
    long long vis = 0;
    if (!(isfinite(cx[0]) && isfinite(cx[1]) && isfinite(cx[2]))) {
      if (lane == 0) atomicOr(status, ST_NONFINITE);
    } else {
      // the voxel of c (clamped) and the distance to its nearest wall
      double r = INFINITY;
      for (int a = 0; a < nax; ++a) {
        double v = floor(__ddiv_rn(__dsub_rn(cx[a], T.lo[a]), T.s[a]));
        v = fmin(fmax(v, 0.0), (double)(T.n[a] - 1));
        const double wlo = __dadd_rn(T.lo[a], __dmul_rn(v, T.s[a]));
        const double whi = __dadd_rn(wlo, T.s[a]);
        r = fmin(r, fmin(fabs(__dsub_rn(cx[a], wlo)), fabs(__dsub_rn(cx[a], whi))));
      }
      bool have_t = false;
      int t0[3] = {0, 0, 0}, t1[3] = {-1, -1, -1};
      long long inside_prev = -1;
      for (;;) {
        int b0[3], b1[3];
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
          if (a < nax) {
            const double lo = floor(__ddiv_rn(__dsub_rn(__dsub_rn(cx[a], r), T.lo[a]), T.s[a])) - 1.0;
            const double hi = floor(__ddiv_rn(__dsub_rn(__dadd_rn(cx[a], r), T.lo[a]), T.s[a])) + 1.0;
            if (hi < 0.0 || lo > (double)(T.n[a] - 1)) empty = true;
            b0[a] = lo < 0.0 ? 0 : (int)lo;
            b1[a] = hi > (double)(T.n[a] - 1) ? T.n[a] - 1 : (int)hi;
          } else {
            b0[a] = 0;
            b1[a] = T.n[a] - 1;
          }
        }
        if (!empty) {
          for (int i = b0[0]; i <= b1[0]; ++i)
            for (int j = b0[1]; j <= b1[1]; ++j)
              for (int kz = b0[2]; kz <= b1[2]; ++kz) {
                if (have_t && i >= t0[0] && i <= t1[0] && j >= t0[1] && j <= t1[1] && kz >= t0[2] && kz <= t1[2])
                  continue;  // taboo: visited in an earlier iteration
                const uint32_t key = T.key_base + (nax == 2 ? (uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j
                                                            : ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) *
                                                                      (uint32_t)T.n[2] + (uint32_t)kz);
                const uint2 sp = voxel_span(ix, T, key);
                for (uint32_t s0 = sp.x; s0 < sp.y; s0 += 32) {
                  const uint32_t t = s0 + lane;
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
                    const int src = __ffs(cand) - 1;
                    cand &= cand - 1;
                    wl_insert(L, __shfl_sync(0xffffffffu, d, src), __shfl_sync(0xffffffffu, id, src), k);
                  }
                }
              }
          for (int a = 0; a < 3; ++a) {
            t0[a] = b0[a];
            t1[a] = b1[a];
          }
          have_t = true;
        }
        const double r2 = __dmul_rn(r, r);
        long long inside;
        if (wl_get(L, k - 1) <= r2) {
          inside = k;
        } else {
          const unsigned m0 = __ballot_sync(0xffffffffu, (int)lane < k && L.d[0] <= r2);
          const unsigned m1 = __ballot_sync(0xffffffffu, (int)lane + 32 < k && L.d[1] <= r2);
          inside = __popc(m0) + __popc(m1);
        }
        bool covers = have_t;
        for (int a = 0; a < nax; ++a) covers &= t0[a] == 0 && t1[a] == T.n[a] - 1;
        if (inside >= k || covers) break;
        if (policy == 1 && inside > 0 && inside != inside_prev) {
          const double vol = __dmul_rn(__dmul_rn(__dmul_rn(__dmul_rn(4.0 / 3.0, kPi), r), r), r);
          const double rho = __ddiv_rn((double)inside, vol);
          r = cbrt(__ddiv_rn(__dmul_rn(3.0, (double)k), __dmul_rn(__dmul_rn(4.0, kPi), rho)));
        } else {
          r = __dadd_rn(r, smin);
        }
        inside_prev = inside;
      }
      if (have_t) vis = (long long)(t1[0] - t0[0] + 1) * (t1[1] - t0[1] + 1) * (t1[2] - t0[2] + 1);
    }
    for (int s = 0; s < k; ++s) {
      const double d = wl_get(L, s);
      const uint32_t id = __shfl_sync(0xffffffffu, s < 32 ? L.id[0] : L.id[1], s & 31);
      if (lane == 0) {
        const bool ok = dbits(d) < kInfBits;
        out_idx[(size_t)e * k + s] = ok ? (int32_t)id : -1;
        if (out_d2) out_d2[(size_t)e * k + s] = ok ? d : INFINITY;
      }
    }
    if (lane == 0 && visited) visited[e] = vis;
  }
}

template <int PREC>
__global__ void __launch_bounds__(128) knn_grow_kernel(IndexView ix, const double* __restrict__ q, uint32_t nq,
                                                       int k, int policy, int32_t* __restrict__ out_idx,
                                                       double* __restrict__ out_d2,
                                                       long long* __restrict__ visited, uint32_t* status) {
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < nq; w += gridDim.x * (blockDim.x / 32))
    knn_grow_one<PREC>(ix, q, w, k, policy, out_idx, out_d2, visited, status);
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

// ---------------------------------------------------------------- small batches

// Small batches of external queries (at most kSmallBatch): one block of
// KS_T threads per query, no query plan.  Boxes of R = 1, 2, ... voxel rings
// around the query's voxel are gathered until they hold k points (every
// candidate: one record load, its binary32 screen value); the k-th smallest
// screen value tau (bisection on the bit patterns) gives the band
// d2f <= tau + 2 B(tau), which holds the box's k nearest; their binary64
// values sorted by (d2, id) give the box's k-th value kth.  If kth is below
// the squared distance to the box's walls the answer is final; else the
// true k nearest all lie within sqrt(kth) (the box already holds k points
// that close), and the voxel range of Algorithm 1 for that radius is
// gathered and searched once more (final).  A box of more than KS_CAP
// points or a band wider than KS_BAND: the block's first warp runs
// Algorithm 2 step by step for the query instead.
constexpr int KS_T = kBoxThreads;
constexpr int KS_CAP = 4096;
constexpr int KS_BAND = 256;
constexpr int KS_MAX_RING = 64;

template <int PREC>
__global__ void __launch_bounds__(KS_T) knn_small_kernel(IndexView ix, const double* __restrict__ q, uint32_t nq,
                                                         int k, int32_t* __restrict__ out_idx,
                                                         double* __restrict__ out_d2, uint32_t* status, float m_host,
                                                         float alpha_host, float eq_host) {
  using R = typename KRec<PREC>::T;
  __shared__ float s_f[KS_CAP];
  __shared__ uint32_t s_id[KS_CAP];
  __shared__ double s_d[KS_BAND];
  __shared__ uint32_t s_bid[KS_BAND];
  __shared__ uint32_t s_red[KS_T / 32];
  __shared__ uint32_t s_start[kBoxThreads + 1], s_off[kBoxThreads + 1];
  __shared__ uint32_t s_n, s_mb, s_pick, s_pick_below;
  __shared__ float s_fcut;
  __shared__ uint32_t s_hist[KS_T];  // 256 bins
  static_assert(KS_T == 256, "one histogram bin per thread");
  __shared__ int s_box[8];  // lo[3], hi[3], covers, final
  __shared__ R s_q;
  __shared__ KBound s_kb;
  const uint32_t e = blockIdx.x;
  if (e >= nq) return;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const Tile& T = ix.tiles[0];
  const int nax = ix.dim;
  const double* c = q + 3 * (size_t)e;
  const double cx[3] = {__ldg(c), __ldg(c + 1), __ldg(c + 2)};
  int32_t* oi = out_idx + (size_t)e * k;
  double* od = out_d2 ? out_d2 + (size_t)e * k : nullptr;
  if (!(isfinite(cx[0]) && isfinite(cx[1]) && isfinite(cx[2]))) {
    if (threadIdx.x == 0) atomicOr(status, ST_NONFINITE);
    for (int i = (int)threadIdx.x; i < k; i += KS_T) {
      oi[i] = -1;
      if (od) od[i] = INFINITY;
    }
    return;
  }
  // set-up on thread 0 (the binary64 pipe is narrow: a division by all 256
  // threads costs more than the whole gather): the query's record in the
  // tile's frame, the screen's error bound (from the host's bound for query
  // offsets up to m_host, else its own), the query's voxel (clamped; any
  // voxel would do, the walls are measured exactly)
  int cc[3] = {0, 0, 0};
  float eq = 0.f;
  if (threadIdx.x == 0) {
    if constexpr (PREC == 1) {
      const float x = __double2float_rn(__dsub_rn(cx[0], T.origin[0]));
      const float y = __double2float_rn(__dsub_rn(cx[1], T.origin[1]));
      const float z = __double2float_rn(__dsub_rn(cx[2], T.origin[2]));
      s_q = make_float4(x, y, z, 0.f);
      const float mf = fmaxf(fabsf(x), fmaxf(fabsf(y), fabsf(z)));
      Thresholds th;
      if (mf <= m_host) {
        th.pad_[0] = alpha_host;
        eq = eq_host;
      } else {
        const double m = (double)mf;
        const double e_q = ldexp(m, -24) * (1.0 + 1e-6) + ldexp(m, -52) + 1e-30;
        th.pad_[0] = __double2float_ru(((double)T.enc_err + e_q) * (1.0 + 1e-6));
        eq = __double2float_ru(e_q);
      }
      s_kb = make_kbound<1>(th);
      const float qa[3] = {x, y, z};
      for (int a = 0; a < nax; ++a) {
        const float u = floorf(__fmul_rn(__fadd_rn(qa[a], T.D[a]), T.inv_sf[a]));
        cc[a] = u < 0.f ? 0 : (u > (float)(T.n[a] - 1) ? T.n[a] - 1 : (int)u);
      }
    } else {
      s_q = make_double4_32a(cx[0], cx[1], cx[2], 0.0);
      Thresholds th;
      th.pad_[0] = 0.f;
      s_kb = make_kbound<0>(th);
      for (int a = 0; a < nax; ++a) {
        double v = floor(__ddiv_rn(__dsub_rn(cx[a], T.lo[a]), T.s[a]));
        v = fmin(fmax(v, 0.0), (double)(T.n[a] - 1));
        cc[a] = (int)v;
      }
    }
  }
  __syncthreads();
  const R qr = s_q;
  const KBound kb = s_kb;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
  int Rr = 1;
  bool final_box = false;
  uint32_t mb = 0;
  for (;;) {
    // the box (thread 0): rings around the query's voxel, or the final
    // ball's range
    if (threadIdx.x == 0) {
      const double rb = (final_box && PREC == 0) ? sqrt(s_d[k - 1]) : 0.0;
      // binary32 records: the final ball's range in binary32 with the proven
      // pad of the voxel coordinates (the k-NN bounded search's formula)
      const float rbf = (final_box && PREC == 1) ? __fmul_ru(__fsqrt_ru(__double2float_ru(s_d[k - 1])), 1.000001f) : 0.f;
      int cov = 1;
      for (int a = 0; a < 3; ++a) {
        int l0, h0;
        if (a >= nax) {
          l0 = 0;
          h0 = T.n[a] - 1;
        } else if (!final_box) {
          l0 = max(cc[a] - Rr, 0);
          h0 = min(cc[a] + Rr, T.n[a] - 1);
        } else if constexpr (PREC == 1) {
          const float qv = a == 0 ? s_q.x : (a == 1 ? s_q.y : s_q.z);
          const float u = __fmul_rn(__fadd_rn(qv, T.D[a]), T.inv_sf[a]);
          const float rr = __fmul_ru(__fmul_ru(rbf, T.inv_sf[a]), 1.0000005f);
          float pad = __fadd_ru(__fadd_ru(rr, T.eta), __fmul_ru(__fadd_ru(fabsf(u), fabsf(qv) * T.inv_sf[a]), 3.0e-7f));
          pad = __fadd_ru(pad, __fmul_ru(eq, T.inv_sf[a]));
          const float ul = fminf(fmaxf(__fsub_rd(u, pad), -1.0e9f), 1.0e9f);
          const float uh = fminf(fmaxf(__fadd_ru(u, pad), -1.0e9f), 1.0e9f);
          l0 = min(max((int)floorf(ul), 0), T.n[a] - 1);
          h0 = max(min((int)floorf(uh), T.n[a] - 1), 0);
        } else {
          const double l = floor(__ddiv_rn(__dsub_rn(__dsub_rn(cx[a], rb), T.lo[a]), T.s[a])) - 1.0;
          const double h = floor(__ddiv_rn(__dsub_rn(__dadd_rn(cx[a], rb), T.lo[a]), T.s[a])) + 1.0;
          l0 = l < 0.0 ? 0 : (l > (double)(T.n[a] - 1) ? T.n[a] - 1 : (int)l);
          h0 = h < 0.0 ? 0 : (h > (double)(T.n[a] - 1) ? T.n[a] - 1 : (int)h);
        }
        if (a < nax) cov &= (l0 == 0 && h0 == T.n[a] - 1) ? 1 : 0;
        s_box[a] = l0;
        s_box[3 + a] = h0;
      }
      s_box[6] = cov;
      s_n = 0;
      if (final_box) {
        const float kf = __double2float_ru(s_d[k - 1]);
        s_fcut = __fadd_ru(kf, 2.0f * kb.at(kf));
      } else {
        s_fcut = INFINITY;
      }
    }
    __syncthreads();  // also: every thread has read s_d before the band is rebuilt
    const int lo[3] = {s_box[0], s_box[1], s_box[2]}, hi[3] = {s_box[3], s_box[4], s_box[5]};
    const bool covers = s_box[6] != 0;
    // gather: every point of the box, its screen value and id (the final
    // box keeps only the points whose screen value may lie within the
    // k-th value found so far, kth: the true k nearest are among them)
    const float fcut = s_fcut;
    for_each_in_box(ix, T, lo, hi, s_start, s_off, [&](uint32_t t, bool valid) {
      float df = 0.f;
      uint32_t id = 0;
      if (valid) {
        const R rec = pts[t];
        df = kd2f(rec, qr);
        id = krec_id(rec);
        valid = df <= fcut;
      }
      const unsigned bm = __ballot_sync(0xffffffffu, valid);
      uint32_t base = 0;
      if (lane == 0 && bm) base = atomicAdd(&s_n, (uint32_t)__popc(bm));
      const uint32_t pos = __shfl_sync(0xffffffffu, base, 0) + __popc(bm & lanemask_lt());
      if (valid && pos < (uint32_t)KS_CAP) {
        s_f[pos] = df;
        s_id[pos] = id;
      }
    });
    __syncthreads();
    const uint32_t n = s_n;
    if (n > (uint32_t)KS_CAP) break;  // too many points: the step-by-step kernel
    if (n < (uint32_t)k && !covers && !final_box) {
      if (++Rr > KS_MAX_RING) break;
      continue;
    }
    // an upper bound tau of the k-th smallest screen value, within 2^-8 of
    // it: two 256-bin histograms of the values' bit patterns (non-negative
    // binary32 values order as their bits), bits 30..23, then 22..15 of the
    // bin that holds the k-th; tau = the top of that second bin
    const uint32_t kk = min((uint32_t)k, n);
    float tau = 0.f;
    if (kk > 0 && kk == (uint32_t)k) {
      uint32_t below = 0, prefix = 0;
      for (int level = 0; level < 2; ++level) {
        const int shift = level == 0 ? 23 : 15;
        s_hist[threadIdx.x] = 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < n; i += KS_T) {
          const uint32_t b = __float_as_uint(s_f[i]);
          if (level == 0 || (b >> 23) == prefix) atomicAdd(&s_hist[(b >> shift) & 255u], 1u);
        }
        __syncthreads();
        // inclusive scan of the 256 bins (one per thread)
        const uint32_t h = s_hist[threadIdx.x];
        uint32_t inc = h;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
          if (lane >= (uint32_t)o) inc += y;
        }
        if (lane == 31) s_red[warp] = inc;
        __syncthreads();
        uint32_t wb = 0;
        for (uint32_t w2 = 0; w2 < warp; ++w2) wb += s_red[w2];
        inc += wb + below;
        if (inc >= kk && inc - h < kk) s_pick = threadIdx.x;  // the bin holding the k-th
        __syncthreads();
        const uint32_t pick = s_pick;
        // the count below the picked bin, from its own thread
        if (threadIdx.x == pick) s_pick_below = inc - h;
        __syncthreads();
        below = s_pick_below;
        prefix = level == 0 ? pick : (prefix << 8) | pick;
        __syncthreads();  // s_hist, s_red and s_pick are reused
      }
      tau = (prefix >> 8) == 255u ? INFINITY : __uint_as_float((prefix << 15) | 0x7fffu);
    }
    const float bcut = kk < (uint32_t)k ? INFINITY : __fadd_ru(tau, 2.0f * kb.at(tau));
    if (threadIdx.x == 0) s_mb = 0;
    __syncthreads();
    for (uint32_t i0 = 0; i0 < n; i0 += KS_T) {
      const uint32_t i = i0 + threadIdx.x;
      const bool in = i < n && s_f[i] <= bcut;
      const unsigned bm = __ballot_sync(0xffffffffu, in);
      uint32_t base = 0;
      if (lane == 0 && bm) base = atomicAdd(&s_mb, (uint32_t)__popc(bm));
      base = __shfl_sync(0xffffffffu, base, 0);
      const uint32_t pos = base + __popc(bm & lanemask_lt());
      if (in && pos < (uint32_t)KS_BAND) s_bid[pos] = s_id[i];
    }
    __syncthreads();
    mb = s_mb;
    if (mb > (uint32_t)KS_BAND) break;  // a band this wide (ties): the step-by-step kernel
    uint32_t P = 1;
    while (P < mb) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += KS_T) {
      if (i < mb) s_d[i] = exact_d2(ix.xyz64 + 3 * (size_t)s_bid[i], c);
      else { s_d[i] = INFINITY; s_bid[i] = 0xffffffffu; }
    }
    __syncthreads();
    for (uint32_t kq = 2; kq <= P; kq <<= 1)  // bitonic sort by (d2, id)
      for (uint32_t j = kq >> 1; j > 0; j >>= 1) {
        for (uint32_t i = threadIdx.x; i < P; i += KS_T) {
          const uint32_t l = i ^ j;
          if (l > i) {
            const unsigned long long ka = dbits(s_d[i]), kv = dbits(s_d[l]);
            const uint32_t ia = s_bid[i], il = s_bid[l];
            const bool gt = ka > kv || (ka == kv && ia > il);
            if (gt == ((i & kq) == 0)) {
              const double td = s_d[i];
              s_d[i] = s_d[l];
              s_d[l] = td;
              s_bid[i] = il;
              s_bid[l] = ia;
            }
          }
        }
        __syncthreads();
      }
    if (final_box || covers || kk < (uint32_t)k) {
      mb = min(mb, (uint32_t)k);
      goto out;
    }
    {
      // final when the k-th value lies strictly inside the box's walls
      if (threadIdx.x == 0) {
        const double kth = s_d[k - 1];
        double w = INFINITY;
        for (int a = 0; a < nax; ++a) {
          if (lo[a] > 0) w = fmin(w, cx[a] - (T.lo[a] + (double)lo[a] * T.s[a]));
          if (hi[a] < T.n[a] - 1) w = fmin(w, (T.lo[a] + (double)(hi[a] + 1) * T.s[a]) - cx[a]);
        }
        w -= 1e-12 * (fabs(T.lo[0]) + fabs(T.lo[1]) + fabs(T.lo[2]) + 1.0);
        s_box[7] = (w > 0 && kth < w * w * (1.0 - 1e-12)) ? 1 : 0;
      }
      __syncthreads();
      if (s_box[7]) {
        mb = (uint32_t)k;
        goto out;
      }
    }
    final_box = true;
  }
  // not decided here (a box or band too large for shared memory): the
  // block's first warp runs Algorithm 2 step by step for the query
  if (warp == 0) knn_grow_one<PREC>(ix, q, e, k, 1, out_idx, out_d2, nullptr, status);
  return;
out:
  for (int i = (int)threadIdx.x; i < k; i += KS_T) {
    const bool ok = (uint32_t)i < mb;
    oi[i] = ok ? (int32_t)s_bid[i] : -1;
    if (od) od[i] = ok ? s_d[i] : INFINITY;
  }
}

}  // namespace

// Binary32 fast path (k <= 64): group boxes of radius 1 in three size
// classes (staged boxes of <= 512, 1024 and 2048 candidates; list length
// the class's largest k + 2: 4, 6, 10, 18, 34 or 66), then the bounded search of the queries
// left undecided.  bslot / br2 have room for every query; ctrs[4..6] are
// the box launches' group counters, ctrs[9] the bounded list's length,
// ctrs[0] the ring-by-ring list's.
cudaError_t launch_knn5(const IndexView& iv, const QuerySet& qs, const Thresholds* thr, int k, int32_t* idx,
                        double* d2, uint32_t* slow, uint32_t* bslot, float* br2, uint32_t* ctrs, uint32_t* status,
                        cudaStream_t st) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // the classes' groups are disjoint: their launches run concurrently
  ProfScope prof_all("knn_fast_kernels", st);  // box classes + bounded search
  Fork f(st, 3);
#define CG_K5(KC, L, NW, GW, CLS)                                                                            \
  do {                                                                                                       \
    auto kfn = knn5_kernel<KC, L, NW, GW>;                                                                   \
    const size_t smem = K5Smem<KC>::per_slot(GW) * (NW / GW);                                                \
    cudaError_t le = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
    if (le != cudaSuccess) return le;                                                                        \
    int per = 0;                                                                                             \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kfn, NW * 32, smem);                                 \
    cudaStream_t cs = f[CLS];                                                                                \
    ProfScope prof(CLS == 2 ? "knn5_2k" : (CLS ? "knn5_1k" : "knn5_512"), cs);                               \
    kfn<<<sms * (per > 0 ? per : 1), NW * 32, smem, cs>>>(iv, qs, thr, k, idx, d2, slow, ctrs, bslot, br2,    \
                                                          ctrs + 9, ctrs + 4 + CLS, status, CLS);              \
    note_launch();                                                                                           \
    if ((le = cudaGetLastError()) != cudaSuccess) return le;                                                 \
  } while (0)
  // warps per group: 1, 2, 4 for the three classes (their groups hold about
  // 1, 2.5 and 4 chunks of 32 queries), sharing the staged box
  if (k <= 2) {
    CG_K5(512, 4, 4, 1, 0u);
    CG_K5(1024, 4, 4, 2, 1u);
    CG_K5(2048, 4, 4, 4, 2u);
  } else if (k <= 4) {
    CG_K5(512, 6, 4, 1, 0u);
    CG_K5(1024, 6, 4, 2, 1u);
    CG_K5(2048, 6, 4, 4, 2u);
  } else if (k <= 8) {
    CG_K5(512, 10, 4, 1, 0u);
    CG_K5(1024, 10, 4, 2, 1u);
    CG_K5(2048, 10, 4, 4, 2u);
  } else if (k <= 16) {
    CG_K5(512, 18, 4, 1, 0u);
    CG_K5(1024, 18, 4, 2, 1u);
    CG_K5(2048, 18, 4, 4, 2u);
  } else if (k <= 32) {
    CG_K5(512, 34, 4, 1, 0u);
    CG_K5(1024, 34, 4, 2, 1u);
    CG_K5(2048, 34, 4, 4, 2u);
  } else {
    CG_K5(512, 66, 4, 1, 0u);
    CG_K5(1024, 66, 4, 2, 1u);
    CG_K5(2048, 66, 4, 4, 2u);
  }
#undef CG_K5
  f.join();
  {
    ProfScope prof("knn_bounded", st);
    knn_bounded_kernel<<<sms * 7, KB_WARPS * 32, 0, st>>>(iv, qs, thr, k, bslot, br2, ctrs + 9, idx, d2, slow, ctrs,
                                                          status);
    note_launch();
  }
  return cudaGetLastError();
}

cg_status knn_pass(cg_index* ix, QueryCtx& C, bool all_points, const double* q, int64_t nq, int k, int32_t* idx, double* d2,
                   cudaStream_t st) {
  if (k < 1 || k > 64) return fail(CG_ERR_INVALID, "k must be in [1, 64]");
  if (nq < 0 || nq >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "nq out of range");
  if (!all_points && ix->ntiles != 1)
    return fail(CG_ERR_UNIMPLEMENTED, "external k-NN queries on a batched index (every point queries its own tile)");
  // small batches: one block per query, no query plan; the queries it
  // cannot decide (boxes or bands too large for its shared memory) run
  // Algorithm 2 step by step with the density rule (the same result)
  if (!all_points && nq > 0 && nq <= kSmallBatch && ix->ntiles == 1) {
    // the screen's bound for query offsets up to the tile's extent plus
    // 64 cells (farther queries make their own)
    const Tile& T0 = ix->tiles_host[0];
    double mh = 0.0;
    for (int a = 0; a < 3; ++a)
      mh = std::max(mh, std::max(std::fabs(T0.lo[a] - T0.origin[a]), std::fabs(T0.hi[a] - T0.origin[a])) + 64.0 * T0.s[a]);
    const float m_host = (float)mh;
    const double mq = (double)m_host;
    const double eqh = std::ldexp(mq, -24) * (1.0 + 1e-6) + std::ldexp(mq, -52) + 1e-30;
    const float alpha_host = f_up(((double)T0.enc_err + eqh) * (1.0 + 1e-6));
    const float eq_host = f_up(eqh);
    {
      ProfScope prof("knn_small", st);
      if (ix->precision == CG_FP32_OFFSET)
        knn_small_kernel<1><<<(int)nq, KS_T, 0, st>>>(ix->view(), q, (uint32_t)nq, k, idx, d2, C.status, m_host,
                                                      alpha_host, eq_host);
      else
        knn_small_kernel<0><<<(int)nq, KS_T, 0, st>>>(ix->view(), q, (uint32_t)nq, k, idx, d2, C.status, m_host,
                                                      alpha_host, eq_host);
      note_launch();
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "small k-NN kernel");
    return CG_OK;
  }
  if (!all_points) {
    cg_status s = prepare_queries(ix, C, q, nq, false, st);
    if (s != CG_OK) return s;
  }
  if (nq == 0) return CG_OK;
  DevBufs tmp;
  uint32_t* slow = (uint32_t*)tmp.get(4 * (size_t)nq, st);
  // queries for the bounded search (room for every query)
  uint32_t* bslot = (uint32_t*)tmp.get(4 * (size_t)nq, st);
  float* br2 = (float*)tmp.get(4 * (size_t)nq, st);
  uint32_t* ctrs = (uint32_t*)tmp.get(256, st);
  Thresholds* thr = (Thresholds*)tmp.get(sizeof(Thresholds), st);
  if (!slow || !ctrs || !thr || !bslot || !br2) { tmp.release(st); return fail(CG_ERR_OOM, "device allocation failed (k-NN)"); }
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
      HostRead rd;
      rd.get(&P.nblocks, P.nblocks_dev, 4);
      if (e == cudaSuccess) e = rd.sync(st);
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
  if (ix->precision == CG_FP32_OFFSET && k <= 64) {
    e = launch_knn5(iv, qs, thr, k, idx, d2, slow, bslot, br2, ctrs, C.status, st);
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


cg_status knn_grow_pass(cg_index* ix, const double* q, int64_t nq, int k, int policy, int32_t* idx, double* d2,
                        int64_t* visited, cudaStream_t st, uint32_t* status) {
  if (!status) status = ix->status;
  if (k < 1 || k > 64) return fail(CG_ERR_INVALID, "k must be in [1, 64]");
  if (policy != 0 && policy != 1) return fail(CG_ERR_INVALID, "policy must be 0 (monotone) or 1 (density)");
  if (nq < 0 || nq >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "nq out of range");
  if (ix->ntiles != 1) return fail(CG_ERR_UNIMPLEMENTED, "external queries on a batched index");
  if (nq == 0) return CG_OK;
  const int sms = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 152;
  }();
  const int grid = (int)std::min<int64_t>((nq + 3) / 4, (int64_t)sms * 16);
  ProfScope prof("knn_grow", st);
  if (ix->precision == CG_FP32_OFFSET)
    knn_grow_kernel<1><<<grid, 128, 0, st>>>(ix->view(), q, (uint32_t)nq, k, policy, idx, d2,
                                             reinterpret_cast<long long*>(visited), status);
  else
    knn_grow_kernel<0><<<grid, 128, 0, st>>>(ix->view(), q, (uint32_t)nq, k, policy, idx, d2,
                                             reinterpret_cast<long long*>(visited), status);
  note_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "k-NN growth kernel");
  return CG_OK;
}

cg_status knn_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, int k, int32_t* idx, double* d2,
                   cudaStream_t st) {
  return knn_pass(ix, ix->ctx, all_points, q, nq, k, idx, d2, st);
}

cg_status knn_work_alloc(cg_index* ix, KnnWork& w, cudaStream_t st) {
  w.slow = (uint32_t*)w.bufs.get(4 * (size_t)std::max<int64_t>(ix->n, 1), st);
  w.bslot = (uint32_t*)w.bufs.get(4 * (size_t)std::max<int64_t>(ix->n, 1), st);
  w.br2 = (float*)w.bufs.get(4 * (size_t)std::max<int64_t>(ix->n, 1), st);
  w.ctrs = (uint32_t*)w.bufs.get(256, st);
  w.thr = (Thresholds*)w.bufs.get(sizeof(Thresholds), st);
  if (!w.slow || !w.ctrs || !w.thr || !w.bslot || !w.br2)
    return fail(CG_ERR_OOM, "device allocation failed (pipeline k-NN work)");
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
  if (ix->precision == CG_FP32_OFFSET && k <= 64) {
    e = launch_knn5(iv, qs, w.thr, k, idx, d2, w.slow, w.bslot, w.br2, w.ctrs, ix->status, st);
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
