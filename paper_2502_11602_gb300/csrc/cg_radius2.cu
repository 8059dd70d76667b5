// cg_radius2.cu -- fast kernels of the two-pass radius search.
//
// The count pass and the fill pass of Algorithm 1 share one expensive step:
// testing every staged candidate against every query of a voxel group.  Here
// the count pass does that test once and keeps its outcome, and the fill
// pass only expands it:
//
//   plan  (one warp per voxel group): union of the group's voxel ranges (the
//         kernel bounding boxes through Eq. chs-point-to-idcs, widened by the
//         proven rounding pad), its row spans (one contiguous span of sorted
//         points per grid row / column), the candidate count K and the sizes
//         of the group's outputs.  Groups that are too large for the fast
//         kernels are listed for the general CTA kernel.
//   count (one 128-thread CTA per group): TMA bulk copies (cp.async.bulk +
//         mbarrier, bounded wait) stage the spans and the queries in shared
//         memory; a CTA radix sort orders the candidates by original id; one
//         thread per (query, 32-candidate word) tests the candidates against
//         broadcast shared-memory records and writes one 32-bit hit mask per
//         word; the group's sorted ids and the per-query counts go to global
//         memory.
//   fill  (one CTA per group): expands each query's masks into its CSR row:
//         bits are visited in candidate (= id) order, so rows are ascending
//         without any per-row sort.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "cg_query.cuh"
#include "cg_sort.cuh"

namespace cg {
namespace {

constexpr int PT = 128;   // plan kernel threads (one warp per group)
constexpr int CT = 256;   // count / fill CTA threads
constexpr int CW = CT / 32;
constexpr int QB2 = 512;  // queries per group handled by the fast kernels

template <int PREC> struct R2;
template <> struct R2<1> { using T = float4; static constexpr int KW = 2048; };
template <> struct R2<0> { using T = double4_32a; static constexpr int KW = 1024; };

__device__ __forceinline__ uint32_t rid(const float4& r) { return __float_as_uint(r.w); }
__device__ __forceinline__ uint32_t rid(const double4_32a& r) { return (uint32_t)__double_as_longlong(r.w); }
__device__ __forceinline__ float4 sentinel(float4*) {
  return make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                     __uint_as_float(0xffffffffu));
}
__device__ __forceinline__ double4_32a sentinel(double4_32a*) {
  double nan = __longlong_as_double(0x7ff8000000000000ll);
  return make_double4_32a(nan, nan, nan, __longlong_as_double(0xffffffffll));
}

__device__ __forceinline__ float ru(const float4& q, const Tile& T, int a) {
  float x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__fadd_rn(x, T.D[a]), T.inv_sf[a]);
}
__device__ __forceinline__ float ru(const double4_32a& q, const Tile& T, int a) {
  double x = a == 0 ? q.x : (a == 1 ? q.y : q.z);
  return __fmul_rn(__double2float_rn(__dsub_rn(x, T.lo[a])), T.inv_sf[a]);
}
__device__ __forceinline__ float rabs(const float4& q, int a) { return fabsf(a == 0 ? q.x : (a == 1 ? q.y : q.z)); }
__device__ __forceinline__ float rabs(const double4_32a&, int) { return 0.f; }

template <int KERN>
__device__ __forceinline__ bool exact_in(const double* __restrict__ p, const double* __restrict__ c, double r2) {
  double dx = __dsub_rn(__ldg(p), __ldg(c));
  double dy = __dsub_rn(__ldg(p + 1), __ldg(c + 1));
  double dz = __dsub_rn(__ldg(p + 2), __ldg(c + 2));
  if (KERN == CG_SPHERE)
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
  return fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
}
template <int KERN>
__device__ __forceinline__ bool exact_in4(const double4_32a& p, const double4_32a& c, double r2) {
  double dx = __dsub_rn(p.x, c.x), dy = __dsub_rn(p.y, c.y), dz = __dsub_rn(p.z, c.z);
  if (KERN == CG_SPHERE)
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
  return fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ plan

template <int PREC>
__global__ void __launch_bounds__(PT) radius_plan_kernel(IndexView ix, QuerySet qs,
                                                         const Thresholds* __restrict__ thr_p,
                                                         BlockPlan* __restrict__ plans,
                                                         uint32_t* __restrict__ msize,
                                                         uint32_t* __restrict__ isize,
                                                         uint32_t* __restrict__ big_list, uint32_t* big_n,
                                                         const uint32_t* status) {
  using R = typename R2<PREC>::T;
  constexpr int KW = R2<PREC>::KW;
  if (replan_pending(status)) return;
  const Thresholds thr = *thr_p;
  const unsigned lane = threadIdx.x & 31u;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
  const R* __restrict__ qsrc = qs.all_points ? pts
                                             : (PREC == 1 ? reinterpret_cast<const R*>(qs.qrec)
                                                          : reinterpret_cast<const R*>(qs.qrec64));
  const uint32_t nwarps = gridDim.x * (PT / 32);
  for (uint32_t b = blockIdx.x * (PT / 32) + (threadIdx.x >> 5); b < qs_nblocks(qs); b += nwarps) {
    const uint32_t qb0 = qs.blk_beg[b], qb1 = qs.blk_beg[b + 1], nq = qb1 - qb0;
    const uint32_t bkey = qs.blk_key[b];
    const Tile& T = ix.tiles[ix.ntiles == 1 ? 0 : tile_of_key(ix.tiles, ix.ntiles, bkey)];
    const int dim = ix.dim;
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    for (uint32_t t = lane; t < nq; t += 32) {
      const R q = qsrc[qb0 + t];
      for (int a = 0; a < dim; ++a) {
        float u = ru(q, T, a);
        float rr = __fmul_ru(__fmul_ru(thr.r_f, T.inv_sf[a]), 1.0000005f);
        float pad = __fadd_ru(__fadd_ru(rr, T.eta), __fmul_ru(__fadd_ru(fabsf(u), rabs(q, a) * T.inv_sf[a]), 3.0e-7f));
        pad = __fadd_ru(pad, __fmul_ru(thr.e_q, T.inv_sf[a]));
        float ul = fminf(fmaxf(__fsub_rd(u, pad), -1.0e9f), 1.0e9f);
        float uh = fminf(fmaxf(__fadd_ru(u, pad), -1.0e9f), 1.0e9f);
        lo[a] = min(lo[a], (int)floorf(ul));
        hi[a] = max(hi[a], (int)floorf(uh));
      }
    }
    bool empty = false;
    for (int a = 0; a < 3; ++a) {
      if (a < dim) {
        for (int o = 16; o > 0; o >>= 1) {
          lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
          hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        lo[a] = max(lo[a], 0);
        hi[a] = min(hi[a], T.n[a] - 1);
        empty |= lo[a] > hi[a];
      } else {
        lo[a] = 0;
        hi[a] = T.n[a] - 1;
      }
    }
    // one run per non-empty voxel of the range (each run is sorted by id)
    const int ni = empty ? 0 : hi[0] - lo[0] + 1, nj = empty ? 0 : hi[1] - lo[1] + 1;
    const int nk = empty ? 0 : (dim == 3 ? hi[2] - lo[2] + 1 : 1);
    const int nvox = ni * nj * nk;
    bool big = nq > (uint32_t)QB2 || nvox > 32;
    uint32_t start = 0, len = 0;
    if (!big && (int)lane < nvox) {
      const int i = lo[0] + (int)lane / (nj * nk), j = lo[1] + ((int)lane / nk) % nj;
      uint32_t key;
      if (dim == 2) key = T.key_base + (uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j;
      else key = T.key_base + ((uint32_t)i * (uint32_t)T.n[1] + (uint32_t)j) * (uint32_t)T.n[2] + (uint32_t)(lo[2] + (int)lane % nk);
      const uint2 sp = voxel_span(ix, T, key);
      start = sp.x;
      len = sp.y - sp.x;
    }
    const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
    const int nsp = __popc(nonempty);
    const int slot = __popc(nonempty & lanemask_lt());
    uint32_t K = len;
    for (int o = 16; o > 0; o >>= 1) K += __shfl_xor_sync(0xffffffffu, K, o);
    big |= K > (uint32_t)KW;
    const uint32_t W = big ? 0u : (K + 31u) / 32u;
    BlockPlan* P = plans + b;
    if (len > 0) {
      P->start[slot] = start;
      P->len[slot] = len;
    }
    if (lane == 0) {
      P->q0 = qb0;
      P->nq = nq;
      P->K = big ? 0u : K;
      P->nsp = (uint16_t)(big ? 0 : nsp);
      P->W = (uint16_t)W;
      P->heavy = big ? 1u : 0u;
      P->pad_[0] = (PREC == 1 && K > 1024u) ? 1u : 0u;  // size class for the binary32 kernels
      // binary32 path: query masks, window masks of up to min(32, nq) z-groups,
      // one group id per query; binary64 path: query masks only
      msize[b] = big ? 0u : (PREC == 1 ? nq * W + min(32u, nq) * W + nq : nq * W);
      isize[b] = big ? 0u : K;
      if (big) big_list[atomicAdd(big_n, 1u)] = b;
    }
  }
  // replayed pipelines scan the whole capacity: groups past the true count
  // contribute nothing
  if (qs.nblocks_dev != nullptr)
    for (uint32_t b = qs_nblocks(qs) + blockIdx.x * PT + threadIdx.x; b < qs.nblocks; b += gridDim.x * PT) {
      msize[b] = 0u;
      isize[b] = 0u;
    }
}

// ------------------------------------------------------------------ count

// Layout of the id-sorted candidates used by the binary32 test: candidate
// pairs (2p, 2p+1) as {x0, x1, y0, y1} and {z0, z1}, so that packed
// f32x2 arithmetic evaluates two candidates per instruction; one padding pair
// after every 16 pairs (one 32-candidate word) keeps the words on different
// shared-memory banks.  ids are kept in a plain array.
struct PairLayout {
  ulonglong2* xy;       // [pair_cap]
  unsigned long long* z;  // [pair_cap]
  uint32_t* id;         // [KW]
};
__device__ __forceinline__ int pair_slot(int j) { int p = j >> 1; return p + (p >> 4); }

__device__ __forceinline__ void put_pair(const PairLayout& L, int j, const float4& r) {
  const int ps = pair_slot(j);
  float* xy = reinterpret_cast<float*>(L.xy + ps);
  float* z = reinterpret_cast<float*>(L.z + ps);
  const int h = j & 1;
  xy[h] = r.x;
  xy[2 + h] = r.y;
  z[h] = r.z;
  L.id[j] = __float_as_uint(r.w);
}

// CTA-wide stable LSD radix sort of K records by id (8-bit digits, per-warp
// ranking with match_any).  Pass p reads A (even p) or B and writes the
// other; the last pass (passes is odd, so it reads A) hands each record and
// its sorted position to `final_store`.
template <class R, int EPL, class Final>
__device__ void cta_sort_by_id(const R* A, R* B, int K, int passes, uint16_t* hist, uint32_t* dbase,
                               Final final_store) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const int C = ((K + CW * 32 - 1) / (CW * 32)) * 32;  // elements per warp
  for (int p = 0; p < passes; ++p) {
    const R* src = (p & 1) ? B : A;
    R* dst = (p & 1) ? const_cast<R*>(A) : B;
    const bool last = p == passes - 1;
    const int shift = 8 * p;
    for (int i = threadIdx.x; i < CW * 256; i += CT) hist[i] = 0;
    __syncthreads();
    R v[EPL];
    uint32_t rank[EPL], dig[EPL];
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = (int)warp * C + j * 32 + (int)lane;
      const bool ok = j * 32 < C && e < K;
      if (ok) v[j] = src[e];
      const uint32_t id = ok ? rid(v[j]) : 0u;
      const uint32_t d = shift < 32 ? (id >> shift) & 255u : 0u;
      dig[j] = d;
      const unsigned peers = __match_any_sync(0xffffffffu, ok ? d : 256u + lane);
      const uint32_t before = ok ? hist[warp * 256 + d] : 0u;
      __syncwarp();
      const unsigned lower = peers & lanemask_lt();
      rank[j] = before + __popc(lower);
      if (ok && lower == 0) hist[warp * 256 + d] = (uint16_t)(before + __popc(peers));
      __syncwarp();
    }
    __syncthreads();
    {  // digit totals -> exclusive scan over 256 digits (one per thread)
      const int d = threadIdx.x;
      uint32_t tot = 0;
#pragma unroll
      for (int w = 0; w < CW; ++w) tot += hist[w * 256 + d];
      uint32_t incl = tot;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += y;
      }
      if (lane == 31) dbase[256 + warp] = incl;
      __syncthreads();
      uint32_t run = incl - tot;
      for (unsigned w = 0; w < warp; ++w) run += dbase[256 + w];
#pragma unroll
      for (int w = 0; w < CW; ++w) {
        uint32_t a = hist[w * 256 + d];
        hist[w * 256 + d] = (uint16_t)run;
        run += a;
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = (int)warp * C + j * 32 + (int)lane;
      if (j * 32 < C && e < K) {
        const int pos = (int)(hist[warp * 256 + dig[j]] + rank[j]);
        if (last) final_store(pos, v[j]);
        else dst[pos] = v[j];
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned long long pk(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

template <int PREC>
struct CountSmem;
template <>
struct CountSmem<1> {
  static constexpr int KW = R2<1>::KW;
  static constexpr int PAIRS = KW / 2 + KW / 32 + 8;
  static constexpr size_t A = sizeof(float4) * KW;
  static constexpr size_t Bpairs = (16 + 8) * (size_t)PAIRS + 4 * (size_t)KW;
  static constexpr size_t Brec = sizeof(float4) * KW;
  static constexpr size_t B = Bpairs > Brec ? Bpairs : Brec;
};
template <>
struct CountSmem<0> {
  static constexpr int KW = R2<0>::KW;
  static constexpr size_t A = sizeof(double4_32a) * KW;
  static constexpr size_t B = sizeof(double4_32a) * (KW + KW / 32 + 64);
};
constexpr size_t kCountTail = 2 * CW * 256 + 4 * (256 + CW) + 4 * QB2;

template <int PREC, int KERN>
__global__ void __launch_bounds__(CT) radius_count2_kernel(IndexView ix, QuerySet qs,
                                                           const Thresholds* __restrict__ thr_p,
                                                           const BlockPlan* __restrict__ plans,
                                                           const uint32_t* __restrict__ moff,
                                                           const uint32_t* __restrict__ idoff,
                                                           uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ masks,
                                                           uint32_t* __restrict__ ids, unsigned* work,
                                                           uint32_t* status, int passes) {
  if (replan_pending(status)) return;
  using R = typename R2<PREC>::T;
  using SM = CountSmem<PREC>;
  constexpr int EPL = SM::KW / CT;
  extern __shared__ __align__(128) unsigned char smem[];
  R* recA = reinterpret_cast<R*>(smem);
  unsigned char* Bmem = smem + SM::A;
  uint16_t* hist = reinterpret_cast<uint16_t*>(Bmem + SM::B);    // [CW][256]
  uint32_t* dbase = reinterpret_cast<uint32_t*>(hist + CW * 256);  // [256 + CW]
  uint32_t* cnt_s = dbase + 256 + CW;                              // [QB2]
  __shared__ uint32_t s_b, s_hdr[6];
  __shared__ uint32_t s_start[kPlanSpans], s_len[kPlanSpans], s_dst[kPlanSpans];
  __shared__ __align__(8) unsigned long long s_mbar;

  const Thresholds thr = *thr_p;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
  const R* __restrict__ qsrc = qs.all_points ? pts
                                             : (PREC == 1 ? reinterpret_cast<const R*>(qs.qrec)
                                                          : reinterpret_cast<const R*>(qs.qrec64));
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  const uint32_t mbar = smem_addr(&s_mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_b = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t b = s_b;
    if (b >= qs_nblocks(qs)) break;
    if (threadIdx.x < 6) s_hdr[threadIdx.x] = reinterpret_cast<const uint32_t*>(plans + b)[threadIdx.x];
    if (threadIdx.x < kPlanSpans) {
      s_start[threadIdx.x] = plans[b].start[threadIdx.x];
      s_len[threadIdx.x] = plans[b].len[threadIdx.x];
    }
    __syncthreads();
    const uint32_t q0 = s_hdr[0], nq = s_hdr[1], K = s_hdr[2];
    const uint32_t nsp = s_hdr[3] & 0xffffu, W = s_hdr[3] >> 16, heavy = s_hdr[4];
    if (heavy || nq == 0) continue;
    if (K > 0) {
      // ---- stage the spans with TMA bulk copies (one per span)
      if (threadIdx.x == 0) {
        uint32_t acc = 0;
        for (uint32_t s = 0; s < nsp; ++s) { s_dst[s] = acc; acc += s_len[s]; }
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar),
                     "r"(K * (uint32_t)sizeof(R))
                     : "memory");
      }
      __syncthreads();
      if (threadIdx.x < nsp && s_len[threadIdx.x] > 0) {
        const uint32_t s = threadIdx.x;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                         "r"(smem_addr(recA + s_dst[s])), "l"(pts + s_start[s]), "r"(s_len[s] * (uint32_t)sizeof(R)),
                     "r"(mbar)
                     : "memory");
      }
      uint32_t done = 0;
      for (uint32_t it = 0; it < kSpinLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
      if (!done) {
        atomicOr(status, ST_TIMEOUT);
        for (uint32_t it = 0; it < kSpinLimit && !done; ++it)  // still bounded
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(done)
              : "r"(mbar), "r"(phase)
              : "memory");
      }
      phase ^= 1u;
    }
    for (uint32_t t = threadIdx.x; t < nq; t += CT) cnt_s[t] = 0;
    uint32_t* mb = masks + moff[b];
    const uint32_t io = idoff[b];
    if constexpr (PREC == 1) {
      PairLayout PL;
      PL.xy = reinterpret_cast<ulonglong2*>(Bmem);
      PL.z = reinterpret_cast<unsigned long long*>(Bmem + 16 * (size_t)SM::PAIRS);
      PL.id = reinterpret_cast<uint32_t*>(Bmem + 24 * (size_t)SM::PAIRS);
      if (K > 0)
        cta_sort_by_id<float4, EPL>(recA, reinterpret_cast<float4*>(Bmem), (int)K, passes, hist, dbase,
                                    [&](int pos, const float4& r) { put_pair(PL, pos, r); });
      const float4 sent = make_float4(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000),
                                      __int_as_float(0x7fc00000), __uint_as_float(0xffffffffu));
      for (uint32_t j = K + threadIdx.x; j < W * 32u; j += CT) put_pair(PL, (int)j, sent);
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < K; j += CT) ids[io + j] = PL.id[j];
      const float slo = KERN == CG_SPHERE ? thr.s_lo : thr.c_lo;
      const float shi = KERN == CG_SPHERE ? thr.s_hi : thr.c_hi;
      for (uint32_t qg = 0; qg < nq; qg += CT) {
        const uint32_t nqg = min((uint32_t)CT, nq - qg);
        const uint32_t S = max(1u, min(W, (uint32_t)CT / nqg));
        if (threadIdx.x < nqg * S) {
          const uint32_t q = qg + threadIdx.x % nqg, s = threadIdx.x / nqg;
          const float4 qq = qsrc[q0 + q];
          const uint32_t qid = __float_as_uint(qq.w);
          const unsigned long long QX = pk(qq.x, qq.x), QY = pk(qq.y, qq.y), QZ = pk(qq.z, qq.z);
          uint32_t cnt = 0;
          for (uint32_t w = s; w < W; w += S) {
            const ulonglong2* xyw = PL.xy + w * 17u;
            const unsigned long long* zw = PL.z + w * 17u;
            uint32_t m_in = 0, m_hi = 0;
#pragma unroll
            for (int pr = 0; pr < 16; ++pr) {
              const ulonglong2 xy = xyw[pr];
              const unsigned long long zz = zw[pr];
              const unsigned long long DX = sub2(xy.x, QX), DY = sub2(xy.y, QY), DZ = sub2(zz, QZ);
              float v0, v1;
              if (KERN == CG_SPHERE) {
                upk(fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX))), v0, v1);
              } else {
                float a0, a1, b0, b1, c0, c1;
                upk(mul2(DX, DX), a0, a1);
                upk(mul2(DY, DY), b0, b1);
                upk(mul2(DZ, DZ), c0, c1);
                v0 = fmaxf(fmaxf(a0, b0), c0);
                v1 = fmaxf(fmaxf(a1, b1), c1);
              }
              m_in |= (v0 <= slo ? 1u : 0u) << (2 * pr);
              m_in |= (v1 <= slo ? 1u : 0u) << (2 * pr + 1);
              m_hi |= (v0 <= shi ? 1u : 0u) << (2 * pr);
              m_hi |= (v1 <= shi ? 1u : 0u) << (2 * pr + 1);
            }
            uint32_t band = m_hi & ~m_in;
            while (band) {  // rare: decide in binary64 on the original coordinates
              const int bb = __ffs(band) - 1;
              band &= band - 1;
              const uint32_t cid = PL.id[w * 32u + bb];
              if (exact_in<KERN>(ix.xyz64 + 3 * (size_t)cid, q64 + 3 * (size_t)qid, thr.r2)) m_in |= 1u << bb;
            }
            mb[q * W + w] = m_in;
            cnt += __popc(m_in);
          }
          atomicAdd(&cnt_s[q], cnt);
        }
      }
    } else {
      R* recB = reinterpret_cast<R*>(Bmem);
      if (K > 0)
        cta_sort_by_id<R, EPL>(recA, recB, (int)K, passes, hist, dbase,
                               [&](int pos, const R& r) { recB[pos + (pos >> 5)] = r; });
      for (uint32_t j = K + threadIdx.x; j < W * 32u; j += CT) recB[j + (j >> 5)] = sentinel((R*)nullptr);
      __syncthreads();
      for (uint32_t j = threadIdx.x; j < K; j += CT) ids[io + j] = rid(recB[j + (j >> 5)]);
      for (uint32_t qg = 0; qg < nq; qg += CT) {
        const uint32_t nqg = min((uint32_t)CT, nq - qg);
        const uint32_t S = max(1u, min(W, (uint32_t)CT / nqg));
        if (threadIdx.x < nqg * S) {
          const uint32_t q = qg + threadIdx.x % nqg, s = threadIdx.x / nqg;
          const R qq = qsrc[q0 + q];
          uint32_t cnt = 0;
          for (uint32_t w = s; w < W; w += S) {
            const R* base = recB + w * 33u;
            uint32_t m_in = 0;
#pragma unroll 8
            for (int bb = 0; bb < 32; ++bb) m_in |= (exact_in4<KERN>(base[bb], qq, thr.r2) ? 1u : 0u) << bb;
            mb[q * W + w] = m_in;
            cnt += __popc(m_in);
          }
          atomicAdd(&cnt_s[q], cnt);
        }
      }
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += CT) counts[rid(qsrc[q0 + t])] = cnt_s[t];
  }
}

// ------------------------------------------------------------------ count (z-grouped)

// The binary32 count kernel used for every group that fits the fast path.
// On a 2D grid a voxel column holds points at every height, but a point can
// only be a neighbour if |z_p - z_q| <= r.  The group's queries are binned by
// z into at most 32 z-groups (bins at least r wide); a candidate is kept only
// if it lies inside the z-window of some group (window = bin extended by r
// plus the binary32 error pad, so no true neighbour is ever dropped).  The
// kept candidates are ordered by id by merging the voxel runs (each run is
// already ascending in id): the rank of a candidate is its position in its
// run plus, for every other run, the number of ids below it.  Each z-group
// then tests only its own window's candidates (compacted, in id order) and
// stores masks over that compacted list, plus the window membership over the
// group's sorted list for the fill pass.
template <int KWc>
struct Count3Smem {
  static constexpr int KW = KWc;
  static constexpr int PAIRS = KW / 2 + KW / 32 + 8;
  static constexpr size_t A = sizeof(float4) * KW;                          // staging, then sorted
  static constexpr size_t Bpair = 24 * (size_t)PAIRS + 4 * (size_t)KW;     // pairs + candidate index
  static constexpr size_t B = Bpair > A ? Bpair : A;                        // filtered runs, then pairs
  static constexpr size_t Q = (size_t)QB2 * (4 + 2 + 2 + 4);               // qz, qgrp, qlist, cnt
  static constexpr size_t total = A + B + Q + 4 * (32 + 80 + 64 + 64 + 64 + 72);
};

template <int NW>
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  uint32_t pre = 0, tot = 0;
  for (int w = 0; w < NW; ++w) {
    const uint32_t t = s_warp[w];
    if (w < (int)warp) pre += t;
    tot += t;
  }
  __syncthreads();
  total = tot;
  return pre + incl - v;
}

template <int KERN, int TPB, int KWc>
__global__ void __launch_bounds__(TPB) radius_count3_kernel(IndexView ix, QuerySet qs,
                                                           const Thresholds* __restrict__ thr_p,
                                                           const BlockPlan* __restrict__ plans,
                                                           const uint32_t* __restrict__ moff,
                                                           const uint32_t* __restrict__ idoff,
                                                           uint32_t* __restrict__ counts,
                                                           uint32_t* __restrict__ masks,
                                                           uint32_t* __restrict__ ids,
                                                           uint32_t* __restrict__ meta, unsigned* work,
                                                           uint32_t* status, uint32_t cls) {
  if (replan_pending(status)) return;
  using SM = Count3Smem<KWc>;
  constexpr int NW = TPB / 32;
  extern __shared__ __align__(128) unsigned char smem[];
  float4* A = reinterpret_cast<float4*>(smem);
  unsigned char* Bm = smem + SM::A;
  float4* Bf = reinterpret_cast<float4*>(Bm);
  float* qz = reinterpret_cast<float*>(Bm + SM::B);      // [QB2]
  uint32_t* cnt_s = reinterpret_cast<uint32_t*>(qz + QB2);  // [QB2]
  uint16_t* qgrp = reinterpret_cast<uint16_t*>(cnt_s + QB2);  // [QB2]
  uint16_t* qlist = qgrp + QB2;                               // [QB2]
  uint32_t* s_warp = reinterpret_cast<uint32_t*>(qlist + QB2);  // [32]
  uint32_t* s_gcnt = s_warp + 32;                          // [64] bin / group counts, cursors at +40
  uint32_t* s_rs = s_gcnt + 80;                            // [33] run starts (filtered)
  uint32_t* s_misc = s_rs + 64;                            // [64]
  uint32_t* s_wm = s_misc + 64;                            // [64] window-mask words
  uint32_t* s_wp = s_wm + 64;                              // [65] their exclusive prefix
  __shared__ uint32_t s_b, s_hdr[6];
  __shared__ uint32_t s_start[kPlanSpans], s_len[kPlanSpans], s_dst[kPlanSpans + 1];
  __shared__ __align__(8) unsigned long long s_mbar;
  __shared__ float s_zr[2];
  __shared__ unsigned s_nonempty;

  const Thresholds thr = *thr_p;
  const float4* __restrict__ pts = ix.pts32;
  const float4* __restrict__ qsrc = qs.all_points ? pts : qs.qrec;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t mbar = smem_addr(&s_mbar);
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  uint32_t phase = 0;
  // z pad: r plus the binary32 error of both offsets (alpha = e_p + e_q), doubled
  const float R = __fadd_ru(thr.r_f, __fmul_ru(4.0f, __fadd_ru(thr.e_q, thr.e_q)) + 1e-6f * thr.r_f);
  const float slo = KERN == CG_SPHERE ? thr.s_lo : thr.c_lo;
  const float shi = KERN == CG_SPHERE ? thr.s_hi : thr.c_hi;
  PairLayout PL;
  PL.xy = reinterpret_cast<ulonglong2*>(Bm);
  PL.z = reinterpret_cast<unsigned long long*>(Bm + 16 * (size_t)SM::PAIRS);
  PL.id = reinterpret_cast<uint32_t*>(Bm + 24 * (size_t)SM::PAIRS);

  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_b = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t b = s_b;
    if (b >= qs_nblocks(qs)) break;
    if (threadIdx.x < 6) s_hdr[threadIdx.x] = reinterpret_cast<const uint32_t*>(plans + b)[threadIdx.x];
    if (threadIdx.x < kPlanSpans) {
      s_start[threadIdx.x] = plans[b].start[threadIdx.x];
      s_len[threadIdx.x] = plans[b].len[threadIdx.x];
    }
    __syncthreads();
    const uint32_t q0 = s_hdr[0], nq = s_hdr[1], K = s_hdr[2];
    const uint32_t nsp = s_hdr[3] & 0xffffu, heavy = s_hdr[4];
    if (heavy || nq == 0 || s_hdr[5] != cls) continue;
    uint32_t* mb = masks + moff[b];
    const uint32_t Wp = (K + 31u) / 32u;  // plan word count (upper bound of every group's)
    if (K == 0) {
      for (uint32_t t = threadIdx.x; t < nq; t += TPB) counts[__float_as_uint(qsrc[q0 + t].w)] = 0;
      if (threadIdx.x == 0) { meta[4 * b] = 0; meta[4 * b + 1] = 0; meta[4 * b + 2] = 0; }
      continue;
    }
    // ---- stage the voxel runs (TMA bulk copies, one per run)
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (uint32_t s = 0; s < nsp; ++s) { s_dst[s] = acc; acc += s_len[s]; }
      s_dst[nsp] = acc;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(K * 16u) : "memory");
    }
    __syncthreads();
    if (threadIdx.x < nsp) {
      const uint32_t s = threadIdx.x;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
                       "r"(smem_addr(A + s_dst[s])), "l"(pts + s_start[s]), "r"(s_len[s] * 16u), "r"(mbar)
                   : "memory");
    }
    // queries' z while the copies fly; z range of the group
    float zmn = INFINITY, zmx = -INFINITY;
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) {
      const float z = qsrc[q0 + t].z;
      qz[t] = z;
      zmn = fminf(zmn, z);
      zmx = fmaxf(zmx, z);
      cnt_s[t] = 0;
    }
    for (int o = 16; o > 0; o >>= 1) {
      zmn = fminf(zmn, __shfl_xor_sync(0xffffffffu, zmn, o));
      zmx = fmaxf(zmx, __shfl_xor_sync(0xffffffffu, zmx, o));
    }
    if (threadIdx.x == 0) {  // ordered-int encodings: min slot high, max slot low
      reinterpret_cast<int*>(s_zr)[0] = INT_MAX;
      reinterpret_cast<int*>(s_zr)[1] = INT_MIN;
      s_nonempty = 0;
    }
    {
      uint32_t done = 0;
      for (uint32_t it = 0; it < kSpinLimit && !done; ++it)
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
      if (!done) {
        atomicOr(status, ST_TIMEOUT);
        for (uint32_t it = 0; it < kSpinLimit && !done; ++it)
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(done)
              : "r"(mbar), "r"(phase)
              : "memory");
      }
      phase ^= 1u;
    }
    __syncthreads();
    // float min / max through ordered int encodings
    {
      int* zi = reinterpret_cast<int*>(s_zr);
      if (lane == 0) {
        auto ord = [](float f) { int i = __float_as_int(f); return i >= 0 ? i : i ^ 0x7fffffff; };
        atomicMin(&zi[0], ord(zmn));
        atomicMax(&zi[1], ord(zmx));
      }
    }
    __syncthreads();
    auto unord = [](int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); };
    const float zlo = unord(reinterpret_cast<int*>(s_zr)[0]), zhi = unord(reinterpret_cast<int*>(s_zr)[1]);
    // ---- z-groups: bins at least r wide (at most 32); adjacent non-empty bins
    // merge into one group unless separated by an empty bin, or unless the
    // group already holds 32 queries over 4 bins (keeps groups busy enough)
    const float binw = fmaxf(thr.r_f, (zhi - zlo) * (1.0f / 31.5f)) * 1.0001f;
    const bool one_group = (zhi - zlo) <= thr.r_f;
    if (threadIdx.x < 32) s_gcnt[threadIdx.x] = 0;  // per-bin query counts
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) {
      const int bin = one_group ? 0 : min(31, max(0, (int)floorf((qz[t] - zlo) / binw)));
      qgrp[t] = (uint16_t)bin;
      atomicOr(&s_nonempty, 1u << bin);
      atomicAdd(&s_gcnt[bin], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      // s_misc[b] = group of bin b; s_misc[32 + g] = (first bin, last bin) of group g
      uint32_t g = 0, cnt = 0;
      int first = -1, last = -1;
      for (int bn = 0; bn < 32; ++bn) {
        const uint32_t c = s_gcnt[bn];
        if (c == 0) continue;
        const bool close = first >= 0 && (bn - last > 1 || (cnt >= 32 && last - first >= 3));
        if (close) {
          s_misc[32 + g] = (uint32_t)first | ((uint32_t)last << 16);
          ++g;
          first = -1;
          cnt = 0;
        }
        if (first < 0) first = bn;
        last = bn;
        cnt += c;
        s_misc[bn] = g;
      }
      s_misc[32 + g] = (uint32_t)first | ((uint32_t)last << 16);
      s_hdr[5] = g + 1;  // number of groups
    }
    __syncthreads();
    const unsigned nonempty = s_nonempty;
    const uint32_t G = s_hdr[5];
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) qgrp[t] = (uint16_t)s_misc[qgrp[t]];
    // ---- filter the runs by the union of the group windows (stable, per run)
    const uint32_t per = (K + TPB - 1) / TPB;
    const uint32_t e0 = min(threadIdx.x * per, K), e1 = min(e0 + per, K);
    auto keep = [&](float cz) -> bool {
      if (one_group) return cz >= zlo - R && cz <= zhi + R;
      const int blo = max(0, (int)floorf((cz - zlo - R) / binw) - 1);
      const int bhi = min(31, (int)floorf((cz - zlo + R) / binw) + 1);
      if (bhi < blo) return false;
      const unsigned span = (bhi - blo >= 31) ? 0xffffffffu : (((2u << (bhi - blo)) - 1u) << blo);
      return (span & nonempty) != 0u;
    };
    uint32_t kept = 0;
    for (uint32_t e = e0; e < e1; ++e) kept += keep(A[e].z) ? 1u : 0u;
    uint32_t Kp;
    uint32_t pos = cta_excl_scan<NW>(kept, s_warp, Kp);
    {
      // first run starting at or after e0
      uint32_t rs = 0;
      while (rs < nsp && s_dst[rs] < e0) ++rs;
      for (uint32_t e = e0; e < e1; ++e) {
        while (rs < nsp && s_dst[rs] == e) { s_rs[rs] = pos; ++rs; }
        if (keep(A[e].z)) Bf[pos++] = A[e];
      }
    }
    if (threadIdx.x == 0) s_rs[nsp] = Kp;
    __syncthreads();
    const uint32_t W = (Kp + 31u) / 32u;
    // ---- order the kept candidates by id.  Ids are unique, so a one-pass
    // bucket sort is exact once every bucket is ordered: 512 buckets over
    // the block's id range, an atomic slot per element, then a short
    // insertion sort per bucket.  If some bucket is crowded (ids clustered in
    // a narrow range), merge the id-sorted voxel runs by rank instead.
    uint32_t* bk = reinterpret_cast<uint32_t*>(qz);  // 512 counters (qz is dead)
    {
      uint32_t mn = 0xffffffffu, mx = 0u;
      for (uint32_t e = threadIdx.x; e < Kp; e += TPB) {
        const uint32_t id = __float_as_uint(Bf[e].w);
        mn = min(mn, id);
        mx = max(mx, id);
      }
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      }
      if (threadIdx.x == 0) { s_misc[0] = 0xffffffffu; s_misc[1] = 0u; s_misc[2] = 0u; }
      for (uint32_t bb = threadIdx.x; bb < 512u; bb += TPB) bk[bb] = 0u;
      __syncthreads();
      if (lane == 0) { atomicMin(&s_misc[0], mn); atomicMax(&s_misc[1], mx); }
      __syncthreads();
    }
    const uint32_t idmin = s_misc[0];
    const uint32_t span = Kp ? s_misc[1] - idmin : 0u;
    int shift = 0;
    while (shift < 32 && (span >> shift) >= 512u) ++shift;
    for (uint32_t e = threadIdx.x; e < Kp; e += TPB)
      atomicAdd(&bk[(__float_as_uint(Bf[e].w) - idmin) >> shift], 1u);
    __syncthreads();
    {
      constexpr int BPT = 512 / TPB;  // buckets per thread
      uint32_t c[BPT], sum = 0;
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        c[u] = bk[BPT * threadIdx.x + u];
        sum += c[u];
        if (c[u] > 16u) s_misc[2] = 1u;  // crowded bucket: use the run merge
      }
      uint32_t tot;
      uint32_t pre = cta_excl_scan<NW>(sum, s_warp, tot);
#pragma unroll
      for (int u = 0; u < BPT; ++u) {
        bk[BPT * threadIdx.x + u] = pre;
        pre += c[u];
      }
    }
    __syncthreads();
    if (s_misc[2] == 0u) {
      for (uint32_t e = threadIdx.x; e < Kp; e += TPB) {
        const float4 v = Bf[e];
        A[atomicAdd(&bk[(__float_as_uint(v.w) - idmin) >> shift], 1u)] = v;
      }
      __syncthreads();
      // bk[b] is now the end of bucket b; order each bucket
      for (uint32_t bb = threadIdx.x; bb < 512u; bb += TPB) {
        const uint32_t e1 = bk[bb], e0 = bb ? bk[bb - 1] : 0u;
        for (uint32_t x = e0 + 1; x < e1; ++x) {
          const float4 v = A[x];
          const uint32_t id = __float_as_uint(v.w);
          uint32_t y = x;
          while (y > e0 && __float_as_uint(A[y - 1].w) > id) { A[y] = A[y - 1]; --y; }
          A[y] = v;
        }
      }
    } else {
      for (uint32_t e = threadIdx.x; e < Kp; e += TPB) {
        int r = 0, rh = (int)nsp - 1;  // last run whose start <= e
        while (r < rh) {
          const int m = (r + rh + 1) >> 1;
          if (s_rs[m] <= e) r = m; else rh = m - 1;
        }
        const float4 v = Bf[e];
        const uint32_t id = __float_as_uint(v.w);
        uint32_t rank = e - s_rs[r];
        for (int o = 0; o < (int)nsp; ++o) {
          if (o == r) continue;
          uint32_t a = s_rs[o], c = s_rs[o + 1];
          while (a < c) {
            const uint32_t m = (a + c) >> 1;
            if (__float_as_uint(Bf[m].w) < id) a = m + 1; else c = m;
          }
          rank += a - s_rs[o];
        }
        A[rank] = v;
      }
    }
    __syncthreads();
    const uint32_t io = idoff[b];
    for (uint32_t j = threadIdx.x; j < Kp; j += TPB) ids[io + j] = __float_as_uint(A[j].w);
    if (threadIdx.x == 0) { meta[4 * b] = Kp; meta[4 * b + 1] = W; meta[4 * b + 2] = G; }
    // ---- queries by group (group-major list)
    if (threadIdx.x < 33) s_gcnt[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) atomicAdd(&s_gcnt[qgrp[t]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (uint32_t g = 0; g < G; ++g) { uint32_t c = s_gcnt[g]; s_gcnt[g] = acc; s_gcnt[40 + g] = acc; acc += c; }
      s_gcnt[G] = acc;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) qlist[atomicAdd(&s_gcnt[40 + qgrp[t]], 1u)] = (uint16_t)t;
    uint32_t* mgid = mb + nq * Wp + min(32u, nq) * Wp;
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) mgid[t] = qgrp[t];
    __syncthreads();
    // ---- groups in batches that fit the pair pool: one warp compacts one
    // group's window (in id order), then all queries of the batch test
    // group regions are whole 32-candidate words of the padded pair layout
    // (KW / 32 words available): region of group g = words [(g - g0) W, (g - g0 + 1) W)
    const uint32_t per_batch = max(1u, (uint32_t)(KWc / 32) / max(W, 1u));
    for (uint32_t g0 = 0; g0 < G; g0 += per_batch) {
      const uint32_t g1 = min(G, g0 + per_batch);
      for (uint32_t g = g0 + warp; g < g1; g += NW) {
        const uint32_t fb = s_misc[32 + g] & 0xffffu, lb = s_misc[32 + g] >> 16;
        const float wlo = one_group ? zlo - R : zlo + (float)fb * binw - R;
        const float whi = one_group ? zhi + R : zlo + (float)(lb + 1) * binw + R;
        uint32_t* wmask = mb + nq * Wp + g * Wp;
        const uint32_t rb = (g - g0) * W * 32u;  // candidate index base of the region
        uint32_t run = 0;
        for (uint32_t w = 0; w < W; ++w) {
          const uint32_t j = w * 32u + lane;
          const bool in = j < Kp && A[j].z >= wlo && A[j].z <= whi;
          const unsigned bm = __ballot_sync(0xffffffffu, in);
          if (lane == 0) wmask[w] = bm;
          if (in) put_pair(PL, (int)(rb + run + __popc(bm & lanemask_lt())), A[j]);
          run += __popc(bm);
        }
        const uint32_t Wg = (run + 31u) / 32u;
        const float4 sent = make_float4(1.0e30f, 1.0e30f, 1.0e30f, __uint_as_float(0xffffffffu));
        for (uint32_t t = run + lane; t < Wg * 32u; t += 32) put_pair(PL, (int)(rb + t), sent);
        if (lane == 0) s_wp[g] = Wg;
      }
      __syncthreads();
      // tests: one thread per (query of the batch, slice of words)
      const uint32_t qa = s_gcnt[g0], nqb = s_gcnt[g1] - s_gcnt[g0];
      for (uint32_t qg0 = 0; qg0 < nqb; qg0 += TPB) {
        const uint32_t nqg = min((uint32_t)TPB, nqb - qg0);
        const uint32_t S = max(1u, min(W, (uint32_t)TPB / nqg));
        if (threadIdx.x < nqg * S) {
          const uint32_t qs_ = qlist[qa + qg0 + threadIdx.x % nqg];
          const uint32_t s = threadIdx.x / nqg;
          const uint32_t g = qgrp[qs_];
          const uint32_t Wg = s_wp[g];
          const uint32_t pb = (g - g0) * W * 17u;  // pair base of the group's region
          const uint32_t cb = (g - g0) * W * 32u;  // candidate index base
          const float4 qq = qsrc[q0 + qs_];
          const uint32_t qid = __float_as_uint(qq.w);
          const unsigned long long QX = pk(qq.x, qq.x), QY = pk(qq.y, qq.y), QZ = pk(qq.z, qq.z);
          uint32_t cnt = 0;
          for (uint32_t w = s; w < Wg; w += S) {
            const ulonglong2* xyw = PL.xy + pb + w * 17u;
            const unsigned long long* zw = PL.z + pb + w * 17u;
            uint32_t mi[4] = {0u, 0u, 0u, 0u}, mh[4] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int pr = 0; pr < 16; ++pr) {
              const ulonglong2 xy = xyw[pr];
              const unsigned long long zz = zw[pr];
              const unsigned long long DX = sub2(xy.x, QX), DY = sub2(xy.y, QY), DZ = sub2(zz, QZ);
              float v0, v1;
              if (KERN == CG_SPHERE) {
                upk(fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX))), v0, v1);
              } else {
                float a0, a1, b0, b1, c0, c1;
                upk(mul2(DX, DX), a0, a1);
                upk(mul2(DY, DY), b0, b1);
                upk(mul2(DZ, DZ), c0, c1);
                v0 = fmaxf(fmaxf(a0, b0), c0);
                v1 = fmaxf(fmaxf(a1, b1), c1);
              }
              const int part = pr >> 2, sh = 2 * (pr & 3);
              mi[part] |= ((v0 <= slo ? 1u : 0u) | (v1 <= slo ? 2u : 0u)) << sh;
              mh[part] |= ((v0 <= shi ? 1u : 0u) | (v1 <= shi ? 2u : 0u)) << sh;
            }
            uint32_t m_in = mi[0] | (mi[1] << 8) | (mi[2] << 16) | (mi[3] << 24);
            const uint32_t m_hi = mh[0] | (mh[1] << 8) | (mh[2] << 16) | (mh[3] << 24);
            uint32_t band = m_hi & ~m_in;
            while (band) {  // rare: decide in binary64 on the original coordinates
              const int bb = __ffs(band) - 1;
              band &= band - 1;
              const uint32_t cid = PL.id[cb + w * 32u + bb];
              if (exact_in<KERN>(ix.xyz64 + 3 * (size_t)cid, q64 + 3 * (size_t)qid, thr.r2)) m_in |= 1u << bb;
            }
            mb[qs_ * Wp + w] = m_in;
            cnt += __popc(m_in);
          }
          atomicAdd(&cnt_s[qs_], cnt);
        }
      }
      __syncthreads();
    }
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) counts[__float_as_uint(qsrc[q0 + t].w)] = cnt_s[t];
  }
}

// ------------------------------------------------------------ count (warp per group)

// Groups of up to 1024 candidates (almost all of them on ALS tiles): one
// warp owns a group from start to end, so no CTA barrier ever waits on
// another group's phases and many groups are in flight per SM.  The warp
// bucket-sorts the candidates' ids into a shared-memory index (sorted
// position -> index of the candidate in the point array), then its lanes,
// one per (query, slice of 32-candidate words), read the candidates in id
// order through the L1 / L2 and test them.  Output layout is the one the
// fill kernel reads: a single z-group whose window holds every candidate.
constexpr int W4 = 4;       // warps per CTA
constexpr int KW4 = 1024;   // candidates per group
struct Count4Warp {
  uint32_t gidx[KW4];       // id-sorted candidates (their sorted-array index)
  uint32_t bk[512];         // bucket counters, then cursors
  uint32_t rstart[33], roff[33];
};

template <int KERN>
__global__ void __launch_bounds__(W4 * 32) radius_count4_kernel(IndexView ix, QuerySet qs,
                                                                const Thresholds* __restrict__ thr_p,
                                                                const BlockPlan* __restrict__ plans,
                                                                const uint32_t* __restrict__ moff,
                                                                const uint32_t* __restrict__ idoff,
                                                                uint32_t* __restrict__ counts,
                                                                uint32_t* __restrict__ masks,
                                                                uint32_t* __restrict__ ids,
                                                                uint32_t* __restrict__ meta, unsigned* work,
                                                                const uint32_t* status) {
  if (replan_pending(status)) return;
  extern __shared__ __align__(16) unsigned char smem[];
  Count4Warp& S = reinterpret_cast<Count4Warp*>(smem)[threadIdx.x >> 5];
  const unsigned lane = threadIdx.x & 31u;
  const Thresholds thr = *thr_p;
  const float4* __restrict__ pts = ix.pts32;
  const uint32_t* __restrict__ sid = ix.sid;
  const float4* __restrict__ qsrc = qs.all_points ? pts : qs.qrec;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  const float slo = KERN == CG_SPHERE ? thr.s_lo : thr.c_lo;
  const float shi = KERN == CG_SPHERE ? thr.s_hi : thr.c_hi;
  for (;;) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(work, 1u);
    b = __shfl_sync(0xffffffffu, b, 0);
    if (b >= qs_nblocks(qs)) break;
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(plans + b);
    const uint32_t q0 = __ldg(hp), nq = __ldg(hp + 1), K = __ldg(hp + 2);
    const uint32_t nsp = __ldg(hp + 3) & 0xffffu, heavy = __ldg(hp + 4), cls = __ldg(hp + 5);
    if (heavy || cls != 0u || nq == 0) continue;
    uint32_t* mb = masks + moff[b];
    const uint32_t Wp = (K + 31u) / 32u;
    if (K == 0) {
      for (uint32_t t = lane; t < nq; t += 32) counts[__float_as_uint(qsrc[q0 + t].w)] = 0;
      if (lane < 3) meta[4 * b + lane] = 0;
      continue;
    }
    // runs (one per non-empty voxel) and their offsets in the concatenation
    uint32_t rl = lane < nsp ? __ldg(plans[b].len + lane) : 0u;
    uint32_t incl = rl;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    if (lane < nsp) { S.rstart[lane] = __ldg(plans[b].start + lane); S.roff[lane] = incl - rl; }
    if (lane == 0) S.roff[nsp] = K;
    __syncwarp();
    auto gindex = [&](uint32_t p) -> uint32_t {  // concatenated position -> sorted-array index
      int r = 0, rh = (int)nsp - 1;
      while (r < rh) {
        const int m = (r + rh + 1) >> 1;
        if (S.roff[m] <= p) r = m; else rh = m - 1;
      }
      return S.rstart[r] + (p - S.roff[r]);
    };
    // id range -> 512 buckets
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (uint32_t p = lane; p < K; p += 32) {
      const uint32_t id = __ldg(sid + gindex(p));
      mn = min(mn, id);
      mx = max(mx, id);
    }
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    int shift = 0;
    while (shift < 32 && ((mx - mn) >> shift) >= 512u) ++shift;
    for (uint32_t u = lane; u < 512u; u += 32) S.bk[u] = 0u;
    __syncwarp();
    for (uint32_t p = lane; p < K; p += 32) atomicAdd(&S.bk[(__ldg(sid + gindex(p)) - mn) >> shift], 1u);
    __syncwarp();
    // exclusive scan of the 512 counters (16 per lane)
    bool crowded = false;
    {
      uint32_t c[16], sum = 0;
#pragma unroll
      for (int u = 0; u < 16; ++u) { c[u] = S.bk[16 * lane + u]; sum += c[u]; crowded |= c[u] > 16u; }
      uint32_t in2 = sum;
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, in2, o);
        if (lane >= (unsigned)o) in2 += y;
      }
      uint32_t pre = in2 - sum;
#pragma unroll
      for (int u = 0; u < 16; ++u) { S.bk[16 * lane + u] = pre; pre += c[u]; }
    }
    crowded = __any_sync(0xffffffffu, crowded);
    __syncwarp();
    if (!crowded) {
      for (uint32_t p = lane; p < K; p += 32) {
        const uint32_t gi = gindex(p);
        S.gidx[atomicAdd(&S.bk[(__ldg(sid + gi) - mn) >> shift], 1u)] = gi;
      }
      __syncwarp();
      for (uint32_t u = lane; u < 512u; u += 32) {  // bucket u now ends at bk[u]
        const uint32_t e1 = S.bk[u], e0 = u ? S.bk[u - 1] : 0u;
        for (uint32_t x = e0 + 1; x < e1; ++x) {
          const uint32_t g = S.gidx[x], id = __ldg(sid + g);
          uint32_t y = x;
          while (y > e0 && __ldg(sid + S.gidx[y - 1]) > id) { S.gidx[y] = S.gidx[y - 1]; --y; }
          S.gidx[y] = g;
        }
      }
    } else {
      // ids clustered in a narrow range: merge the id-sorted voxel runs by rank
      for (uint32_t p = lane; p < K; p += 32) {
        int r = 0, rh = (int)nsp - 1;
        while (r < rh) {
          const int m = (r + rh + 1) >> 1;
          if (S.roff[m] <= p) r = m; else rh = m - 1;
        }
        const uint32_t gi = S.rstart[r] + (p - S.roff[r]), id = __ldg(sid + gi);
        uint32_t rank = p - S.roff[r];
        for (int o = 0; o < (int)nsp; ++o) {
          if (o == r) continue;
          uint32_t a = 0, c = S.roff[o + 1] - S.roff[o];
          const uint32_t* run = sid + S.rstart[o];
          while (a < c) {
            const uint32_t m = (a + c) >> 1;
            if (__ldg(run + m) < id) a = m + 1; else c = m;
          }
          rank += a;
        }
        S.gidx[rank] = gi;
      }
    }
    __syncwarp();
    // outputs read by the fill: sorted ids, one z-group whose window is everything
    const uint32_t io = idoff[b];
    for (uint32_t j = lane; j < K; j += 32) ids[io + j] = __ldg(sid + S.gidx[j]);
    uint32_t* wmask = mb + nq * Wp;
    for (uint32_t w = lane; w < Wp; w += 32)
      wmask[w] = (w + 1 < Wp || (K & 31u) == 0) ? 0xffffffffu : ((1u << (K & 31u)) - 1u);
    uint32_t* mgid = mb + nq * Wp + min(32u, nq) * Wp;
    for (uint32_t t = lane; t < nq; t += 32) mgid[t] = 0u;
    if (lane == 0) { meta[4 * b] = K; meta[4 * b + 1] = Wp; meta[4 * b + 2] = 1u; }
    // tests: lanes = (query, slice), slices a power of two <= words
    for (uint32_t qg0 = 0; qg0 < nq; qg0 += 32) {
      const uint32_t nqg = min(32u, nq - qg0);
      uint32_t Sl = 1;
      while (Sl * 2 <= 32u / nqg && Sl * 2 <= Wp) Sl *= 2;
      const uint32_t qi = lane / Sl, s = lane % Sl;
      const bool active = qi < nqg;
      uint32_t cnt = 0, qid = 0;
      if (active) {
        const uint32_t q = qg0 + qi;
        const float4 qq = qsrc[q0 + q];
        qid = __float_as_uint(qq.w);
        for (uint32_t w = s; w < Wp; w += Sl) {
          uint32_t m_in = 0, m_hi = 0;
          const uint32_t jb = w * 32u;
#pragma unroll 8
          for (int bb = 0; bb < 32; ++bb) {
            const uint32_t j = jb + bb;
            if (j < K) {
              const float4 c = __ldg(pts + S.gidx[j]);
              const float dx = __fsub_rn(c.x, qq.x), dy = __fsub_rn(c.y, qq.y), dz = __fsub_rn(c.z, qq.z);
              float v;
              if (KERN == CG_SPHERE) v = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
              else v = fmaxf(fmaxf(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
              m_in |= (v <= slo ? 1u : 0u) << bb;
              m_hi |= (v <= shi ? 1u : 0u) << bb;
            }
          }
          uint32_t band = m_hi & ~m_in;
          while (band) {  // rare: decide in binary64 on the original coordinates
            const int bb = __ffs(band) - 1;
            band &= band - 1;
            const uint32_t cid = __ldg(sid + S.gidx[jb + bb]);
            if (exact_in<KERN>(ix.xyz64 + 3 * (size_t)cid, q64 + 3 * (size_t)qid, thr.r2)) m_in |= 1u << bb;
          }
          mb[q * Wp + w] = m_in;
          cnt += __popc(m_in);
        }
      }
      for (uint32_t o = 1; o < Sl; o <<= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
      if (active && s == 0) counts[qid] = cnt;
    }
    __syncwarp();
  }
}

// Fill of the z-grouped layout: per group, the window mask gives the list of
// sorted candidates the group tested (idx), and each query's masks index
// into that list.
template <int TPB>
__global__ void __launch_bounds__(TPB) radius_fill3_kernel(IndexView ix, QuerySet qs,
                                                          const BlockPlan* __restrict__ plans,
                                                          const uint32_t* __restrict__ moff,
                                                          const uint32_t* __restrict__ idoff,
                                                          const uint32_t* __restrict__ masks,
                                                          const uint32_t* __restrict__ ids,
                                                          const uint32_t* __restrict__ meta,
                                                          const int64_t* __restrict__ offsets,
                                                          int32_t* __restrict__ out, unsigned* work,
                                                          const uint32_t* status) {
  if (replan_pending(status)) return;
  constexpr int KW = R2<1>::KW;
  __shared__ uint32_t sids[KW];
  __shared__ uint16_t idxg[KW];
  __shared__ long long soff[QB2];
  __shared__ uint32_t qst[QB2];
  __shared__ uint16_t qlist[QB2];
  __shared__ uint32_t s_gc[40], s_go[40];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_b, s_hdr[6], s_meta[3];
  constexpr int NW = TPB / 32;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const float4* __restrict__ qsrc = qs.all_points ? ix.pts32 : qs.qrec;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_b = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t b = s_b;
    if (b >= qs_nblocks(qs)) break;
    if (threadIdx.x < 6) s_hdr[threadIdx.x] = reinterpret_cast<const uint32_t*>(plans + b)[threadIdx.x];
    if (threadIdx.x < 3) s_meta[threadIdx.x] = meta[4 * b + threadIdx.x];
    __syncthreads();
    const uint32_t q0 = s_hdr[0], nq = s_hdr[1], K = s_hdr[2], heavy = s_hdr[4];
    const uint32_t Kp = s_meta[0], W = s_meta[1], G = s_meta[2];
    if (heavy || nq == 0 || Kp == 0) continue;
    const uint32_t Wp = (K + 31u) / 32u;
    const uint32_t io = idoff[b];
    const uint32_t* __restrict__ mb = masks + moff[b];
    const uint32_t* __restrict__ mgid = mb + nq * Wp + min(32u, nq) * Wp;
    for (uint32_t j = threadIdx.x; j < Kp; j += TPB) sids[j] = ids[io + j];
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) soff[t] = offsets[__float_as_uint(qsrc[q0 + t].w)];
    if (threadIdx.x < 40) s_gc[threadIdx.x] = 0;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) atomicAdd(&s_gc[mgid[t]], 1u);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (uint32_t g = 0; g < G; ++g) { uint32_t c = s_gc[g]; s_gc[g] = acc; s_go[g] = acc; acc += c; }
      s_gc[G] = acc;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += TPB) qlist[atomicAdd(&s_go[mgid[t]], 1u)] = (uint16_t)t;
    __syncthreads();
    for (uint32_t g = 0; g < G; ++g) {
      // candidates of the group: positions of the window mask's bits
      const uint32_t* wmask = mb + nq * Wp + g * Wp;
      if (warp == 0) {
        uint32_t base = 0;
        for (uint32_t w0 = 0; w0 < W; w0 += 32) {
          const uint32_t w = w0 + lane;
          uint32_t m = w < W ? wmask[w] : 0u;
          uint32_t c = __popc(m), incl = c;
          for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (unsigned)o) incl += y;
          }
          uint32_t p = base + incl - c;
          while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            idxg[p++] = (uint16_t)(w * 32u + bit);
          }
          base += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) s_warp[16] = base;
      }
      __syncthreads();
      const uint32_t Kg = s_warp[16];
      const uint32_t Wg = (Kg + 31u) / 32u;
      const uint32_t gq0 = s_gc[g], ngq = s_gc[g + 1] - s_gc[g];
      const uint32_t Pw = ngq * Wg;
      const uint32_t C = (Pw + TPB - 1) / TPB;
      const uint32_t e0 = min(threadIdx.x * C, Pw), e1 = min(e0 + C, Pw);
      uint32_t local = 0;
      {
        uint32_t qq = Wg ? e0 / Wg : 0, w = e0 - qq * Wg;
        for (uint32_t e = e0; e < e1; ++e) {
          local += __popc(mb[qlist[gq0 + qq] * Wp + w]);
          if (++w == Wg) { w = 0; ++qq; }
        }
      }
      uint32_t tot;
      const uint32_t tpre = cta_excl_scan<NW>(local, s_warp, tot);
      {
        uint32_t qq = Wg ? e0 / Wg : 0, w = e0 - qq * Wg;
        uint32_t run = tpre;
        for (uint32_t e = e0; e < e1; ++e) {
          if (w == 0) qst[qq] = run;
          run += __popc(mb[qlist[gq0 + qq] * Wp + w]);
          if (++w == Wg) { w = 0; ++qq; }
        }
      }
      __syncthreads();
      {
        uint32_t qq = Wg ? e0 / Wg : 0, w = e0 - qq * Wg;
        uint32_t run = tpre;
        for (uint32_t e = e0; e < e1; ++e) {
          const uint32_t t = qlist[gq0 + qq];
          uint32_t word = mb[t * Wp + w];
          long long p = soff[t] + (long long)(run - qst[qq]);
          run += __popc(word);
          const uint16_t* iw = idxg + w * 32u;
          while (word) {
            const int bit = __ffs(word) - 1;
            word &= word - 1;
            out[p++] = (int32_t)sids[iw[bit]];
          }
          if (++w == Wg) { w = 0; ++qq; }
        }
      }
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------ fill

// Expands the masks of a group into its rows.  The group's (query, word)
// pairs, query-major, are split into equal contiguous chunks over the CTA's
// threads; one CTA-wide scan of the words' popcounts gives every word its
// position inside its query's row.
template <int PREC>
__global__ void __launch_bounds__(CT) radius_fill2_kernel(IndexView ix, QuerySet qs,
                                                          const BlockPlan* __restrict__ plans,
                                                          const uint32_t* __restrict__ moff,
                                                          const uint32_t* __restrict__ idoff,
                                                          const uint32_t* __restrict__ masks,
                                                          const uint32_t* __restrict__ ids,
                                                          const int64_t* __restrict__ offsets,
                                                          int32_t* __restrict__ out, unsigned* work,
                                                          const uint32_t* status) {
  if (replan_pending(status)) return;
  using R = typename R2<PREC>::T;
  constexpr int KW = R2<PREC>::KW;
  __shared__ uint32_t sids[KW];
  __shared__ long long soff[QB2];
  __shared__ uint32_t qst[QB2];
  __shared__ uint32_t s_warp[CW];
  __shared__ uint32_t s_b, s_hdr[6];
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const R* __restrict__ pts = PREC == 1 ? reinterpret_cast<const R*>(ix.pts32) : reinterpret_cast<const R*>(ix.pts64s);
  const R* __restrict__ qsrc = qs.all_points ? pts
                                             : (PREC == 1 ? reinterpret_cast<const R*>(qs.qrec)
                                                          : reinterpret_cast<const R*>(qs.qrec64));
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_b = atomicAdd(work, 1u);
    __syncthreads();
    const uint32_t b = s_b;
    if (b >= qs_nblocks(qs)) break;
    if (threadIdx.x < 6) s_hdr[threadIdx.x] = reinterpret_cast<const uint32_t*>(plans + b)[threadIdx.x];
    __syncthreads();
    const uint32_t q0 = s_hdr[0], nq = s_hdr[1], K = s_hdr[2];
    const uint32_t W = s_hdr[3] >> 16, heavy = s_hdr[4];
    if (heavy || nq == 0 || K == 0) continue;
    const uint32_t io = idoff[b];
    const uint32_t* __restrict__ mb = masks + moff[b];
    for (uint32_t j = threadIdx.x; j < K; j += CT) sids[j] = ids[io + j];
    for (uint32_t t = threadIdx.x; t < nq; t += CT) soff[t] = offsets[rid(qsrc[q0 + t])];
    const uint32_t Pw = nq * W;
    const uint32_t C = (Pw + CT - 1) / CT;
    const uint32_t e0 = min(threadIdx.x * C, Pw), e1 = min(e0 + C, Pw);
    uint32_t local = 0;
    for (uint32_t e = e0; e < e1; ++e) local += __popc(mb[e]);
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    uint32_t tpre = incl - local;
    for (unsigned w = 0; w < warp; ++w) tpre += s_warp[w];
    // start of every query inside the scan (owned by the thread holding word 0)
    uint32_t q = e0 / max(W, 1u), w = e0 - q * W;
    uint32_t run = tpre;
    for (uint32_t e = e0; e < e1; ++e) {
      if (w == 0) qst[q] = run;
      run += __popc(mb[e]);
      if (++w == W) { w = 0; ++q; }
    }
    __syncthreads();
    q = e0 / max(W, 1u);
    w = e0 - q * W;
    run = tpre;
    for (uint32_t e = e0; e < e1; ++e) {
      uint32_t word = mb[e];
      long long p = soff[q] + (long long)(run - qst[q]);
      run += __popc(word);
      const uint32_t* idw = sids + w * 32u;
      while (word) {
        const int bit = __ffs(word) - 1;
        word &= word - 1;
        out[p++] = (int32_t)idw[bit];
      }
      if (++w == W) { w = 0; ++q; }
    }
  }
}

template <int PREC>
size_t count2_smem() { return CountSmem<PREC>::A + CountSmem<PREC>::B + kCountTail; }

int sm_count() {
  static const int sms = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 152;
  }();
  return sms;
}

template <class F>
int resident_grid(F kern, int threads, size_t smem) {
  int per = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
  if (per < 1) per = 1;
  return sm_count() * per;
}

}  // namespace

// ------------------------------------------------------------------ host

cudaError_t launch_radius_plan(int prec, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                               BlockPlan* plans, uint32_t* msize, uint32_t* isize, uint32_t* big_list,
                               uint32_t* big_n, const uint32_t* status, cudaStream_t st) {
  const int grid = (int)std::min<int64_t>((qs.nblocks + 3) / 4 + 1, (int64_t)sm_count() * 16);
  ProfScope prof("radius_plan", st);
  if (prec == CG_FP32_OFFSET)
    radius_plan_kernel<1><<<grid, PT, 0, st>>>(iv, qs, thr, plans, msize, isize, big_list, big_n, status);
  else
    radius_plan_kernel<0><<<grid, PT, 0, st>>>(iv, qs, thr, plans, msize, isize, big_list, big_n, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_count2(int prec, int kern, const IndexView& iv, const QuerySet& qs,
                                 const Thresholds* thr, const BlockPlan* plans, const uint32_t* moff,
                                 const uint32_t* idoff, uint32_t* counts, uint32_t* masks, uint32_t* ids,
                                 unsigned* work, uint32_t* status, cudaStream_t st) {
  int bits = 1;
  while (bits < 32 && ((uint64_t)1 << bits) < (uint64_t)iv.n) ++bits;
  int passes = (bits + 7) / 8;
  if ((passes & 1) == 0) ++passes;
  ProfScope prof("radius_count2", st);
#define CG_LAUNCH_C2(P, KN)                                                                      \
  do {                                                                                           \
    auto kfn = radius_count2_kernel<P, KN>;                                                      \
    const size_t smem = count2_smem<P>();                                                        \
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    kfn<<<resident_grid(kfn, CT, smem), CT, smem, st>>>(iv, qs, thr, plans, moff, idoff, counts, \
                                                        masks, ids, work, status, passes);       \
  } while (0)
  if (prec == CG_FP32_OFFSET) {
    if (kern == CG_SPHERE) CG_LAUNCH_C2(1, CG_SPHERE); else CG_LAUNCH_C2(1, CG_CUBE);
  } else {
    if (kern == CG_SPHERE) CG_LAUNCH_C2(0, CG_SPHERE); else CG_LAUNCH_C2(0, CG_CUBE);
  }
#undef CG_LAUNCH_C2
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_fill2(int prec, const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                const uint32_t* moff, const uint32_t* idoff, const uint32_t* masks,
                                const uint32_t* ids, const int64_t* offsets, int32_t* out, unsigned* work,
                                const uint32_t* status, cudaStream_t st) {
  ProfScope prof("radius_fill2", st);
  if (prec == CG_FP32_OFFSET) {
    auto kfn = radius_fill2_kernel<1>;
    kfn<<<resident_grid(kfn, CT, 0), CT, 0, st>>>(iv, qs, plans, moff, idoff, masks, ids, offsets, out, work, status);
  } else {
    auto kfn = radius_fill2_kernel<0>;
    kfn<<<resident_grid(kfn, CT, 0), CT, 0, st>>>(iv, qs, plans, moff, idoff, masks, ids, offsets, out, work, status);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_count3(int kern, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                                 const BlockPlan* plans, const uint32_t* moff, const uint32_t* idoff,
                                 uint32_t* counts, uint32_t* masks, uint32_t* ids, uint32_t* meta,
                                 unsigned* work, uint32_t* status, cudaStream_t st) {
  // size class 0: K <= 1024 (128 threads, half the shared memory, more groups
  // in flight); class 1: 1024 < K <= 2048 (256 threads)
#define CG_C3(KN, TPB, KWc, CLS, WORK)                                                                   \
  do {                                                                                                    \
    auto kfn = radius_count3_kernel<KN, TPB, KWc>;                                                        \
    const size_t smem = Count3Smem<KWc>::total;                                                            \
    cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                   \
    const int g3 = resident_grid(kfn, TPB, smem);                                                        \
    ProfScope prof("radius_count3", st);                                                                 \
    kfn<<<g3, TPB, smem, st>>>(iv, qs, thr, plans, moff, idoff, counts, masks,                           \
                               ids, meta, WORK, status, CLS);                                            \
    note_launch();                                                                                        \
  } while (0)
  const size_t smem4 = sizeof(Count4Warp) * W4;
  if (kern == CG_SPHERE) {
    auto k4 = radius_count4_kernel<CG_SPHERE>;
    cudaFuncSetAttribute(k4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4);
    {
      const int g4 = resident_grid(k4, W4 * 32, smem4);
      ProfScope prof("radius_count4", st);
      k4<<<g4, W4 * 32, smem4, st>>>(iv, qs, thr, plans, moff, idoff, counts, masks, ids, meta, work, status);
    }
    note_launch();
    CG_C3(CG_SPHERE, 256, 2048, 1u, work + 1);
  } else {
    auto k4 = radius_count4_kernel<CG_CUBE>;
    cudaFuncSetAttribute(k4, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem4);
    {
      const int g4 = resident_grid(k4, W4 * 32, smem4);
      ProfScope prof("radius_count4", st);
      k4<<<g4, W4 * 32, smem4, st>>>(iv, qs, thr, plans, moff, idoff, counts, masks, ids, meta, work, status);
    }
    note_launch();
    CG_C3(CG_CUBE, 256, 2048, 1u, work + 1);
  }
#undef CG_C3
  return cudaGetLastError();
}

cudaError_t launch_radius_fill3(const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                const uint32_t* moff, const uint32_t* idoff, const uint32_t* masks,
                                const uint32_t* ids, const uint32_t* meta, const int64_t* offsets, int32_t* out,
                                unsigned* work, const uint32_t* status, cudaStream_t st) {
  auto kfn = radius_fill3_kernel<256>;
  const int g = resident_grid(kfn, 256, 0);
  ProfScope prof("radius_fill3", st);
  kfn<<<g, 256, 0, st>>>(iv, qs, plans, moff, idoff, masks, ids, meta, offsets, out, work,
                                                   status);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cg
