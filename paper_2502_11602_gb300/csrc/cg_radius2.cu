// cg_radius2.cu -- fast kernels of the two-pass radius search.
//
// The count pass and the fill pass of Algorithm 1 share one expensive step:
// testing every staged candidate against every query of a voxel group.  Here
// the count pass does that test once and keeps its outcome, and the fill
// pass only expands it:
//
//   plan  (one warp per voxel group): union of the group's voxel ranges (the
//         kernel bounding boxes through Eq. chs-point-to-idcs, widened by the
//         proven rounding pad), its runs (one per non-empty voxel), the
//         candidate count K, the size class and the sizes of the group's
//         outputs.  Groups too large for the fast kernels are listed for the
//         general CTA kernel.
//   count, binary32 records (one warp per group, radius_count5_kernel): ids
//         and records staged in shared memory, a shared-memory bucket sort by
//         original id, packed f32x2 tests from broadcast reads, one 32-bit
//         hit mask per (word, query).
//   count, binary64 records (one CTA per group, radius_count2_kernel): TMA
//         bulk copies (cp.async.bulk + mbarrier, bounded wait) stage the runs
//         and the queries, a CTA radix sort orders the candidates by id.
//   fill  (radius_fill5_kernel / radius_fill2_kernel): expands each query's
//         masks into its CSR row; bits are visited in candidate (= id)
//         order, so rows are ascending without any per-row sort.
#include <limits.h>
#include <math.h>

#include <algorithm>

#include "cg_f32x2.cuh"
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
                                                         const uint32_t* status, int zfull, int zw,
                                                         unsigned long long* pairs) {
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
    const int dimr = (zfull && dim == 3) ? 2 : dim;  // the cylinder spans every z slice
    int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {INT_MIN, INT_MIN, INT_MIN};
    // zw: the group's height range widened by the kernel's half height.  A
    // kernel point has |dz| <= r for dz = fl64(p_z - c_z) (the sphere's and
    // the cube's values are at least fl64(dz^2), squaring is monotone), so
    // |z~_p - z~_c| <= r (1 + 2^-52) + e_p + e_q, e the bound on
    // |z~ - (z - O)|; rounded up with margin, then applied rounding outward.
    const float zh = __fadd_ru(__fmul_ru(thr.r_f, 1.000001f), __fmul_ru(fmaxf(T.enc_err, thr.e_q), 2.000001f));
    float zlo = INFINITY, zhi = -INFINITY;
    for (uint32_t t = lane; t < nq; t += 32) {
      const R q = qsrc[qb0 + t];
      if (PREC == 1 && zw) {
        zlo = fminf(zlo, __fsub_rd((float)q.z, zh));
        zhi = fmaxf(zhi, __fadd_ru((float)q.z, zh));
      }
      for (int a = 0; a < dimr; ++a) {
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
      if (a < dimr) {
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
    if (PREC == 1 && zw)
      for (int o = 16; o > 0; o >>= 1) {
        zlo = fminf(zlo, __shfl_xor_sync(0xffffffffu, zlo, o));
        zhi = fmaxf(zhi, __shfl_xor_sync(0xffffffffu, zhi, o));
      }
    // one run per non-empty voxel of the range (sorted by id; zw: by height,
    // and only the part within [zlo, zhi])
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
      if (PREC == 1 && zw && len > 0 && len <= kZsortMax) {
        // the first height >= zlo (a) and the first height > zhi (d): the two
        // bisections step together, so their loads overlap
        uint32_t a = 0, c = len, d = 0, f = len;
        while (a < c || d < f) {
          const uint32_t m1 = (a + c) >> 1, m2 = (d + f) >> 1;
          const float z1 = a < c ? (float)pts[start + m1].z : 0.f;
          const float z2 = d < f ? (float)pts[start + m2].z : 0.f;
          if (a < c) {
            if (z1 < zlo) a = m1 + 1;
            else c = m1;
          }
          if (d < f) {
            if (z2 <= zhi) d = m2 + 1;
            else f = m2;
          }
        }
        start += a;
        len = d > a ? d - a : 0u;
      }
    }
    const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
    const int nsp = __popc(nonempty);
    const int slot = __popc(nonempty & lanemask_lt());
    uint32_t K = len;
    for (int o = 16; o > 0; o >>= 1) K += __shfl_xor_sync(0xffffffffu, K, o);
    big |= K > (uint32_t)KW;
    // the binary32 warp kernels compare against finite thresholds only
    if (PREC == 1) big |= !(fmaxf(thr.s_hi, thr.c_hi) < 3.0e38f);
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
      // size class of the binary32 kernels: K <= 512, <= 1024, <= 2048
      P->pad_[0] = PREC == 1 ? (K > 1024u ? 2u : (K > 512u ? 1u : 0u)) : 0u;
      // one hit mask per (32-candidate word, query)
      msize[b] = big ? 0u : nq * W;
      isize[b] = big ? 0u : K;
      if (big) big_list[atomicAdd(big_n, 1u)] = b;
      else if (pairs) atomicAdd(pairs, (unsigned long long)K * nq);  // the tests the count kernels run
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
// shared-memory banks.
struct PairLayout {
  ulonglong2* xy;         // [pair_cap]
  unsigned long long* z;  // [pair_cap]
};
__device__ __forceinline__ int pair_slot(int j) { int p = j >> 1; return p + (p >> 4); }

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

template <int PREC>
struct CountSmem;
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
                                                           const int64_t* __restrict__ moff,
                                                           const int64_t* __restrict__ idoff,
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
      if (__syncthreads_or(!done)) {
        // The pass is void (the host rejects every kernel of it, the other
        // size classes included, on ST_TIMEOUT): wait once more, still
        // bounded, for the copies in flight, then stop without computing or
        // writing anything.
        if (threadIdx.x == 0) atomicOr(status, ST_TIMEOUT);
        for (uint32_t it = 0; it < kSpinLimit && !done; ++it)
          asm volatile(
              "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
              : "=r"(done)
              : "r"(mbar), "r"(phase)
              : "memory");
        break;
      }
      phase ^= 1u;
    }
    for (uint32_t t = threadIdx.x; t < nq; t += CT) cnt_s[t] = 0;
    uint32_t* mb = masks + moff[b];
    const size_t io = (size_t)idoff[b];
    // binary64 records: the exact predicate directly
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
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nq; t += CT) counts[rid(qsrc[q0 + t])] = cnt_s[t];
  }
}

// ------------------------------------------------------------ binary32 count / fill (warp per group)

// Binary32 records, groups of up to KC candidates (KC = 1024 or 2048, the
// plan's size class): one warp owns a group from start to end, so no CTA
// barrier ever waits on another group's phases.
//   1. the candidates' ids, run by run (a run is one non-empty voxel, its ids
//      ascending), go to shared memory;
//   2. a bucket sort by id in shared memory (NBK buckets over the group's id
//      range, insertion sort inside a bucket) gives every candidate its slot
//      in id order; when ids crowd a few buckets the sorted runs are merged
//      by rank instead;
//   3. the records are gathered run by run into their slots, in the pair
//      layout (pair_slot), so that packed f32x2 arithmetic tests two
//      candidates per instruction from broadcast shared-memory reads;
//   4. the (word, query) items of the group, word-major, spread evenly over
//      the slot's lanes: one 32-bit hit mask per item, stored word-major
//      ([word][query], coalesced); candidates inside the proven error band
//      of r2 are decided in binary64 on the exact coordinates.
// The fill pass reads the sorted ids and the masks back.
template <int KC>
struct C5 {
  static constexpr int NBK = KC / 2;                                                // id buckets
  static constexpr int PAIRS = KC / 2 + KC / 32 + 2;                                // pair slots
  static constexpr size_t PH2 = 24 * (size_t)PAIRS;                                 // xy + z pairs
  static constexpr size_t PH1 = 4 * (size_t)KC + 4 * (size_t)NBK + 2 * (size_t)KC;  // ids, buckets, order
  static constexpr size_t R1 = ((PH2 > PH1 ? PH2 : PH1) + 15) / 16 * 16;
  static constexpr size_t SLOT = 2 * (size_t)KC;                                    // id-order slot of each candidate
  static constexpr size_t RUNS = 4 * (2 * 36 + 4 + 2 * 8);                          // runs, sbox, wred (GW <= 8)
  // 16-bit hit counter per query, two per word: in the slot table, which
  // the tests no longer need
  static_assert(2 * (size_t)QB2 <= SLOT, "query counters overlay the slot table");
  // the crowded-id radix sort's histogram sits after the phase-1 tables
  static_assert(PH1 == 8 * (size_t)KC && PH1 + 4 * 256 <= R1, "radix histogram overlay");
  // a slot of gw warps: the group's tables
  __host__ __device__ static constexpr size_t per_slot(int) { return (R1 + SLOT + RUNS + 15) / 16 * 16; }
};

// Hit masks of one 32-candidate word against one query: bit j of *in is set
// when the binary32 value of candidate j is <= lo, bit j of *hi when it is
// <= hi.  TL = pk(T_lo, T_lo) with T_lo the next binary32 above lo (0 when
// lo < 0), TH likewise for hi (hi finite): v <= lo exactly when
// fl(v - T_lo) < 0, since a rounded difference keeps the sign of the exact
// one and is +0 when v == T_lo; values are >= +0 or +inf (padding, never
// below a finite T).
template <int KERN>
__device__ __forceinline__ void word_masks(const ulonglong2* __restrict__ xyw, const unsigned long long* __restrict__ zw,
                                           unsigned long long QX, unsigned long long QY, unsigned long long QZ,
                                           unsigned long long TL, unsigned long long TH, uint32_t& in,
                                           uint32_t& hi) {
  // four independent chains of 8 candidates (bytes 3..0), candidate 8c+7
  // first in chain c, so that it ends in bit 8c+7
  uint32_t mi[4] = {0, 0, 0, 0}, mh[4] = {0, 0, 0, 0};
#pragma unroll
  for (int k = 3; k >= 0; --k) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int pr = 4 * c + k;
      const unsigned long long V = pair_vals<KERN>(xyw[pr], zw[pr], QX, QY, QZ);
      float l0, l1, h0, h1;
      upk(sub2(V, TL), l0, l1);
      upk(sub2(V, TH), h0, h1);
      mi[c] = push_sign(push_sign(mi[c], l1), l0);
      mh[c] = push_sign(push_sign(mh[c], h1), h0);
    }
  }
  in = (mi[3] << 24) | (mi[2] << 16) | (mi[1] << 8) | mi[0];
  hi = (mh[3] << 24) | (mh[2] << 16) | (mh[1] << 8) | mh[0];
}

// GW warps share a group (a slot of the CTA): they stage and sort its
// candidates together (per-slot named barriers), then each takes its own
// chunks of 32 queries.  GW = 1 for the smallest size class.
template <int GW>
__device__ __forceinline__ void slot_sync(int slot) {
  if (GW == 1) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(1 + slot), "r"(GW * 32) : "memory");
}

// Positions [0, K) ordered by ids[position] (one warp; the ids are unique):
// stable LSD radix sort of id - min(id), 8-bit digits, as many passes as the
// id range needs, between A (initially the identity) and B; returns the
// buffer holding the result.  hist: 256 words.
__device__ uint16_t* warp_order_by_id(uint32_t K, const uint32_t* __restrict__ ids, uint16_t* A, uint16_t* B,
                                      uint32_t* hist, uint32_t lane) {
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (uint32_t e = lane; e < K; e += 32) {
    A[e] = (uint16_t)e;
    mn = min(mn, ids[e]);
    mx = max(mx, ids[e]);
  }
  mn = __reduce_min_sync(0xffffffffu, mn);
  mx = __reduce_max_sync(0xffffffffu, mx);
  __syncwarp();
  const uint32_t range = mx - mn;
  const int passes = range == 0u ? 0 : (32 - __clz((int)range) + 7) / 8;
  for (int p = 0; p < passes; ++p) {
    const uint32_t sh = 8u * (uint32_t)p;
    for (uint32_t i = lane; i < 256u; i += 32) hist[i] = 0u;
    __syncwarp();
    for (uint32_t e = lane; e < K; e += 32) atomicAdd(&hist[((ids[A[e]] - mn) >> sh) & 255u], 1u);
    __syncwarp();
    {  // exclusive scan of the 256 digit counts, eight per lane
      uint32_t c[8], s = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        c[u] = hist[8 * lane + u];
        s += c[u];
      }
      uint32_t incl = s;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      uint32_t pre = incl - s;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        hist[8 * lane + u] = pre;
        pre += c[u];
      }
    }
    __syncwarp();
    for (uint32_t e0 = 0; e0 < K; e0 += 32) {
      const uint32_t e = e0 + lane;
      const bool valid = e < K;
      const uint32_t s = valid ? A[e] : 0u;
      const uint32_t d = valid ? ((ids[s] - mn) >> sh) & 255u : 256u + lane;
      const unsigned peers = __match_any_sync(0xffffffffu, d);
      const uint32_t lt = (uint32_t)__popc(peers & lanemask_lt());
      const uint32_t at = valid ? hist[d] : 0u;
      __syncwarp();
      if (valid) {
        B[at + lt] = (uint16_t)s;
        if (lt == 0u) hist[d] = at + (uint32_t)__popc(peers);
      }
      __syncwarp();
    }
    uint16_t* t = A;
    A = B;
    B = t;
  }
  return A;
}

template <int KERN, int KC, int NWARP, int GW>
__global__ void __launch_bounds__(NWARP * 32) radius_count5_kernel(IndexView ix, QuerySet qs,
                                                                   const Thresholds* __restrict__ thr_p,
                                                                   const BlockPlan* __restrict__ plans,
                                                                   const int64_t* __restrict__ moff,
                                                                   const int64_t* __restrict__ idoff,
                                                                   uint32_t* __restrict__ counts,
                                                                   uint32_t* __restrict__ masks,
                                                                   uint32_t* __restrict__ ids, unsigned* work,
                                                                   const uint32_t* status, uint32_t cls,
                                                                   int zspan) {
  if (replan_pending(status)) return;
  using L = C5<KC>;
  constexpr int ST = GW * 32;  // threads per slot
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = threadIdx.x & 31u;
  const int warp = (int)(threadIdx.x >> 5), slot = warp / GW, wis = warp % GW;
  const uint32_t tis = (uint32_t)wis * 32u + lane;  // thread in slot
  unsigned char* base = smem + (size_t)slot * L::per_slot(GW);
  uint32_t* ids_r = reinterpret_cast<uint32_t*>(base);           // phase 1: ids in run order
  uint32_t* bk = ids_r + KC;                                      // phase 1: bucket counters
  uint16_t* order = reinterpret_cast<uint16_t*>(bk + L::NBK);     // phase 1: id order -> run position
  PairLayout PL;                                                  // phase 2: records in id order
  PL.xy = reinterpret_cast<ulonglong2*>(base);
  PL.z = reinterpret_cast<unsigned long long*>(base + 16 * (size_t)L::PAIRS);
  uint16_t* slot_of = reinterpret_cast<uint16_t*>(base + L::R1);  // run position -> id order
  uint32_t* rstart = reinterpret_cast<uint32_t*>(base + L::R1 + L::SLOT);
  uint32_t* roff = rstart + 36;
  uint32_t* sbox = roff + 36;                  // [4]: group, crowded flag, id range
  uint32_t* wred = sbox + 4;                   // [2 GW]: per-warp id minima / maxima
  static_assert(GW <= 8 && NWARP % GW == 0, "slot shape");
  uint32_t* qcnt = reinterpret_cast<uint32_t*>(slot_of);  // phase 4: [QB2 / 2] hits per query, 16 bits each
  const Thresholds thr = *thr_p;
  const float4* __restrict__ pts = ix.pts32;
  const uint32_t* __restrict__ sid = ix.sid;
  const float4* __restrict__ qsrc = qs.all_points ? pts : qs.qrec;
  const double* __restrict__ q64 = qs.all_points ? ix.xyz64 : qs.q64;
  // the cylinder's two-term value has a smaller error than the sphere's
  // three-term one: the sphere's band bounds it
  // (the plan sends every group to the general kernel when hi is not finite)
  const unsigned long long TL = above(KERN == CG_CUBE ? thr.c_lo : thr.s_lo);
  const unsigned long long TH = above(KERN == CG_CUBE ? thr.c_hi : thr.s_hi);
  const float far = __int_as_float(0x7f000000);  // padding candidate: its square overflows to +inf
  for (;;) {
    if (tis == 0) sbox[0] = atomicAdd(work, 1u);
    slot_sync<GW>(slot);
    const uint32_t b = sbox[0];
    slot_sync<GW>(slot);
    if (b >= qs_nblocks(qs)) break;
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(plans + b);
    const uint32_t q0 = __ldg(hp), nq = __ldg(hp + 1), K = __ldg(hp + 2);
    const uint32_t nsp = __ldg(hp + 3) & 0xffffu, heavy = __ldg(hp + 4), gcls = __ldg(hp + 5);
    if (heavy || gcls != cls || nq == 0) continue;
    if (K == 0) {
      for (uint32_t t = tis; t < nq; t += ST) counts[__float_as_uint(qsrc[q0 + t].w)] = 0;
      continue;
    }
    uint32_t* mb = masks + moff[b];
    const size_t io = (size_t)idoff[b];
    const uint32_t Wp = (K + 31u) / 32u;
    // runs and their offsets in the run-order concatenation
    if (wis == 0) {
      const uint32_t rl = lane < nsp ? __ldg(plans[b].len + lane) : 0u;
      uint32_t incl = rl;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += y;
      }
      if (lane < nsp) {
        rstart[lane] = __ldg(plans[b].start + lane);
        roff[lane] = incl - rl;
      }
      if (lane == 0) roff[nsp] = K;
    }
    slot_sync<GW>(slot);
    // 1. ids, run by run
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (uint32_t r = 0; r < nsp; ++r) {
      const uint32_t o = roff[r], len = roff[r + 1] - o, s0 = rstart[r];
      for (uint32_t t = tis; t < len; t += ST) {
        const uint32_t id = __ldg(sid + s0 + t);
        ids_r[o + t] = id;
        mn = min(mn, id);
        mx = max(mx, id);
      }
    }
    mn = __reduce_min_sync(0xffffffffu, mn);
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (GW > 1) {
      if (lane == 0) { wred[wis] = mn; wred[GW + wis] = mx; }
      slot_sync<GW>(slot);
#pragma unroll
      for (int w = 0; w < GW; ++w) { mn = min(mn, wred[w]); mx = max(mx, wred[GW + w]); }
    }
    int shift = 0;
    while (shift < 31 && ((mx - mn) >> shift) >= (uint32_t)L::NBK) ++shift;
    for (uint32_t u = tis; u < (uint32_t)L::NBK; u += ST) bk[u] = 0u;
    slot_sync<GW>(slot);
    for (uint32_t p = tis; p < K; p += ST) atomicAdd(&bk[(ids_r[p] - mn) >> shift], 1u);
    slot_sync<GW>(slot);
    // 2. exclusive scan of the buckets (warp 0 of the slot, a contiguous chunk per lane)
    constexpr int PER = L::NBK / 32;
    if (wis == 0) {
      bool crowded = false;
      uint32_t c[PER], sum = 0;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        c[u] = bk[PER * lane + u];
        sum += c[u];
        crowded |= c[u] > 16u;
      }
      uint32_t in2 = sum;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, in2, o);
        if (lane >= (unsigned)o) in2 += y;
      }
      uint32_t pre = in2 - sum;
#pragma unroll
      for (int u = 0; u < PER; ++u) {
        bk[PER * lane + u] = pre;
        pre += c[u];
      }
      crowded = __any_sync(0xffffffffu, crowded);
      if (lane == 0) sbox[1] = crowded ? 1u : 0u;
    }
    slot_sync<GW>(slot);
    if (!sbox[1]) {
      for (uint32_t p = tis; p < K; p += ST) order[atomicAdd(&bk[(ids_r[p] - mn) >> shift], 1u)] = (uint16_t)p;
      slot_sync<GW>(slot);
      for (uint32_t u = tis; u < (uint32_t)L::NBK; u += ST) {  // bucket u now spans [bk[u-1], bk[u])
        const uint32_t e1 = bk[u], e0 = u ? bk[u - 1] : 0u;
        for (uint32_t x = e0 + 1; x < e1; ++x) {
          const uint16_t g = order[x];
          const uint32_t id = ids_r[g];
          uint32_t y = x;
          while (y > e0 && ids_r[order[y - 1]] > id) {
            order[y] = order[y - 1];
            --y;
          }
          order[y] = g;
        }
      }
    } else if (zspan) {
      // ids packed into a narrow range, spans in height order: radix sort
      // (the first warp of the slot; its histogram in the phase-1 area's
      // unused tail)
      if (wis == 0) {
        uint16_t* res = warp_order_by_id(K, ids_r, order, reinterpret_cast<uint16_t*>(bk),
                                         reinterpret_cast<uint32_t*>(base + 8 * (size_t)KC), lane);
        if (res != order)
          for (uint32_t j = lane; j < K; j += 32) order[j] = res[j];
      }
    } else {
      // ids packed into a narrow range: merge the sorted runs by rank
      for (uint32_t r = 0; r < nsp; ++r) {
        const uint32_t o = roff[r], len = roff[r + 1] - o;
        for (uint32_t t = tis; t < len; t += ST) {
          const uint32_t id = ids_r[o + t];
          uint32_t rank = t;
          for (uint32_t r2 = 0; r2 < nsp; ++r2) {
            if (r2 == r) continue;
            uint32_t a = roff[r2], c = roff[r2 + 1];
            const uint32_t a0 = a;
            while (a < c) {
              const uint32_t m = (a + c) >> 1;
              if (ids_r[m] < id) a = m + 1;
              else c = m;
            }
            rank += a - a0;
          }
          order[rank] = (uint16_t)(o + t);
        }
      }
    }
    slot_sync<GW>(slot);
    for (uint32_t j = tis; j < K; j += ST) {
      const uint32_t p = order[j];
      slot_of[p] = (uint16_t)j;
      ids[io + j] = ids_r[p];
    }
    slot_sync<GW>(slot);
    // 3. records into their id-order slots (overwrites the phase-1 tables)
    for (uint32_t r = 0; r < nsp; ++r) {
      const uint32_t o = roff[r], len = roff[r + 1] - o, s0 = rstart[r];
      for (uint32_t t = tis; t < len; t += ST) {
        const float4 rec = __ldg(pts + s0 + t);
        const int ps = pair_slot(slot_of[o + t]), h = slot_of[o + t] & 1;
        float* xy = reinterpret_cast<float*>(PL.xy + ps);
        float* z = reinterpret_cast<float*>(PL.z + ps);
        xy[h] = rec.x;
        xy[2 + h] = rec.y;
        z[h] = rec.z;
      }
    }
    for (uint32_t j = K + tis; j < Wp * 32u; j += ST) {
      const int ps = pair_slot((int)j), h = (int)(j & 1u);
      float* xy = reinterpret_cast<float*>(PL.xy + ps);
      float* z = reinterpret_cast<float*>(PL.z + ps);
      xy[h] = far;
      xy[2 + h] = far;
      z[h] = far;
    }
    slot_sync<GW>(slot);
    // 4. tests: items (word w, query q) in word-major order, spread evenly
    // over the slot's lanes; consecutive lanes take consecutive queries of
    // one word, so that candidate reads are broadcasts and the mask stores
    // coalesce
    for (uint32_t t = tis; t < (nq + 1u) / 2u; t += ST) qcnt[t] = 0u;
    slot_sync<GW>(slot);
    const uint32_t items = Wp * nq;
    const float inv_nq = 1.0f / (float)nq;
    for (uint32_t it = tis; it < items; it += ST) {
      uint32_t w = (uint32_t)((float)it * inv_nq);  // exact after one correction (items < 2^16)
      if (w * nq > it) --w;
      else if ((w + 1u) * nq <= it) ++w;
      const uint32_t q = it - w * nq;
      const float4 qq = qsrc[q0 + q];
      const unsigned long long QX = pk(qq.x, qq.x), QY = pk(qq.y, qq.y), QZ = pk(qq.z, qq.z);
      uint32_t m_in, m_hi;
      word_masks<KERN>(PL.xy + w * 17u, PL.z + w * 17u, QX, QY, QZ, TL, TH, m_in, m_hi);
      for (uint32_t band = m_hi & ~m_in; band != 0u; band &= band - 1u) {  // rare: decide in binary64
        const uint32_t j = w * 32u + (uint32_t)(__ffs(band) - 1);
        const uint32_t cid = __ldcg(ids + io + j);
        if (exact_in<KERN>(ix.xyz64 + 3 * (size_t)cid, q64 + 3 * (size_t)__float_as_uint(qq.w), thr.r2))
          m_in |= band & (0u - band);
      }
      mb[w * nq + q] = m_in;
      atomicAdd(&qcnt[q >> 1], (uint32_t)__popc(m_in) << (16u * (q & 1u)));
    }
    slot_sync<GW>(slot);
    for (uint32_t t = tis; t < nq; t += ST)
      counts[__float_as_uint(qsrc[q0 + t].w)] = (qcnt[t >> 1] >> (16u * (t & 1u))) & 0xffffu;
    slot_sync<GW>(slot);  // the next group overwrites the slot's tables
  }
}

// Fill of the binary32 groups: the group's sorted ids to shared memory
// (once per slot of GW warps), then each warp takes its own chunks of 32
// queries: their masks (word-major, one coalesced row per word) to shared
// memory; rows are expanded in lane segments of seg = 2^ceil(log2 Wp) lanes,
// 32 / seg rows at a time (one word per lane): a segmented scan of the
// words' popcounts places each word's hits (ids ascending) in the row.  The
// row is assembled in the segment's share of a per-warp staging buffer and
// then written out by consecutive lanes (coalesced); a row longer than its
// share is written hit by hit instead.  Groups of more than 32 words use
// the whole warp per row, words 32..63 placed after all of words 0..31.
template <int KC>
struct F5 {
  static constexpr int WMAX = KC / 32;
  static constexpr int RB = 512;  // staging entries per warp
  __host__ __device__ static constexpr size_t per_warp() { return 4 * (size_t)WMAX * 33 + 8 * 32 + 4 * (size_t)RB; }
  __host__ __device__ static constexpr size_t per_slot(int gw) {
    return (4 * (size_t)KC + per_warp() * (size_t)gw + 15) / 16 * 16;
  }
};

template <int KC, int NWARP, int GW>
__global__ void __launch_bounds__(NWARP * 32) radius_fill5_kernel(IndexView ix, QuerySet qs,
                                                                  const BlockPlan* __restrict__ plans,
                                                                  const int64_t* __restrict__ moff,
                                                                  const int64_t* __restrict__ idoff,
                                                                  const uint32_t* __restrict__ masks,
                                                                  const uint32_t* __restrict__ ids,
                                                                  const int64_t* __restrict__ offsets,
                                                                  int32_t* __restrict__ out, unsigned* work,
                                                                  const uint32_t* status, uint32_t cls) {
  if (replan_pending(status)) return;
  using L = F5<KC>;
  constexpr int ST = GW * 32;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ uint32_t s_grp[NWARP / GW];
  const unsigned lane = threadIdx.x & 31u;
  const int warp = (int)(threadIdx.x >> 5), slot = warp / GW, wis = warp % GW;
  const uint32_t tis = (uint32_t)wis * 32u + lane;
  unsigned char* base = smem + (size_t)slot * L::per_slot(GW);
  uint32_t* sids = reinterpret_cast<uint32_t*>(base);                                  // [KC]
  unsigned char* wbase = base + 4 * (size_t)KC + (size_t)wis * L::per_warp();
  uint32_t* ms = reinterpret_cast<uint32_t*>(wbase);                                   // [WMAX][33]
  long long* soff = reinterpret_cast<long long*>(ms + L::WMAX * 33);                  // [32]
  int32_t* rbuf = reinterpret_cast<int32_t*>(soff + 32);                               // [RB]
  const float4* __restrict__ qsrc = qs.all_points ? ix.pts32 : qs.qrec;
  for (;;) {
    if (tis == 0) s_grp[slot] = atomicAdd(work, 1u);
    slot_sync<GW>(slot);
    const uint32_t b = s_grp[slot];
    slot_sync<GW>(slot);
    if (b >= qs_nblocks(qs)) break;
    const uint32_t* hp = reinterpret_cast<const uint32_t*>(plans + b);
    const uint32_t q0 = __ldg(hp), nq = __ldg(hp + 1), K = __ldg(hp + 2);
    const uint32_t heavy = __ldg(hp + 4), gcls = __ldg(hp + 5);
    if (heavy || gcls != cls || nq == 0 || K == 0) continue;
    const uint32_t Wp = (K + 31u) / 32u;
    const size_t io = (size_t)idoff[b];
    const uint32_t* __restrict__ mb = masks + moff[b];
    for (uint32_t j = tis; j < K; j += ST) sids[j] = __ldg(ids + io + j);
    slot_sync<GW>(slot);
    uint32_t seg = 1;
    while (seg < Wp && seg < 32) seg <<= 1;
    for (uint32_t c0 = 32u * wis; c0 < nq; c0 += 32u * GW) {
      const uint32_t nc = min(32u, nq - c0);
      __syncwarp();
      if (lane < nc) {
        soff[lane] = offsets[__float_as_uint(qsrc[q0 + c0 + lane].w)];
        for (uint32_t w = 0; w < Wp; ++w) ms[w * 33 + lane] = __ldg(mb + w * nq + c0 + lane);
      }
      __syncwarp();
      if (L::WMAX <= 32 || Wp <= 32) {
        // each word's hits go straight to their place in the row
        const uint32_t rows = 32u / seg, j = lane / seg, wl = lane % seg;
        const uint32_t share = (uint32_t)L::RB / rows;  // staging entries of this segment
        int32_t* rb = rbuf + j * share;
        for (uint32_t t0 = 0; t0 < nc; t0 += rows) {
          const uint32_t t = t0 + j;
          const bool live = t < nc;
          uint32_t m = (live && wl < Wp) ? ms[wl * 33 + t] : 0u;
          const uint32_t c = __popc(m);
          uint32_t incl = c;
          for (uint32_t o = 1; o < seg; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o, seg);
            if (wl >= o) incl += y;
          }
          const uint32_t H = __shfl_sync(0xffffffffu, incl, seg - 1, seg);  // hits of the row
          const bool staged = H <= share;
          int32_t* dst = (staged ? rb : out + (live ? soff[t] : 0)) + (incl - c);
          while (m) {
            const int bit = __ffs(m) - 1;
            m &= m - 1;
            *dst++ = (int32_t)sids[wl * 32 + bit];
          }
          __syncwarp();
          if (staged && live) {
            int32_t* row = out + soff[t];
            for (uint32_t u = wl; u < H; u += seg) row[u] = rb[u];
          }
          __syncwarp();  // the next rows reuse the staging buffer
        }
      } else {
        for (uint32_t t = 0; t < nc; ++t) {
          // words 0..31 (lane = word), then words 32..63 after all of them
          uint32_t m[2], c[2], incl[2];
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const uint32_t w = lane + 32u * half;
            m[half] = w < Wp ? ms[w * 33 + t] : 0u;
            c[half] = __popc(m[half]);
            incl[half] = c[half];
            for (int o = 1; o < 32; o <<= 1) {
              const uint32_t y = __shfl_up_sync(0xffffffffu, incl[half], o);
              if (lane >= (unsigned)o) incl[half] += y;
            }
          }
          const uint32_t T0 = __shfl_sync(0xffffffffu, incl[0], 31);
          const uint32_t H = T0 + __shfl_sync(0xffffffffu, incl[1], 31);
          const bool staged = H <= (uint32_t)L::RB;
          int32_t* row = out + soff[t];
          int32_t* base = staged ? rbuf : row;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            int32_t* dst = base + (half ? T0 : 0u) + (incl[half] - c[half]);
            uint32_t mm = m[half];
            while (mm) {
              const int bit = __ffs(mm) - 1;
              mm &= mm - 1;
              *dst++ = (int32_t)sids[(lane + 32u * half) * 32 + bit];
            }
          }
          __syncwarp();
          if (staged)
            for (uint32_t u = lane; u < H; u += 32) row[u] = rbuf[u];
          __syncwarp();  // the next row reuses the staging buffer
        }
      }
    }
    slot_sync<GW>(slot);  // the next group overwrites the slot's ids
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
                                                          const int64_t* __restrict__ moff,
                                                          const int64_t* __restrict__ idoff,
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
    const size_t io = (size_t)idoff[b];
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

cudaError_t launch_radius_plan(int prec, int kern, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                               BlockPlan* plans, uint32_t* msize, uint32_t* isize, uint32_t* big_list,
                               uint32_t* big_n, const uint32_t* status, cudaStream_t st, bool zw,
                               unsigned long long* pairs) {
  const int zfull = kern == CG_CYLINDER ? 1 : 0;
  const int grid = (int)std::min<int64_t>((qs.nblocks + 3) / 4 + 1, (int64_t)sm_count() * 16);
  ProfScope prof("radius_plan", st);
  if (prec == CG_FP32_OFFSET)
    radius_plan_kernel<1><<<grid, PT, 0, st>>>(iv, qs, thr, plans, msize, isize, big_list, big_n, status, zfull,
                                               zw ? 1 : 0, pairs);
  else
    radius_plan_kernel<0><<<grid, PT, 0, st>>>(iv, qs, thr, plans, msize, isize, big_list, big_n, status, zfull, 0,
                                               pairs);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_count2(int prec, int kern, const IndexView& iv, const QuerySet& qs,
                                 const Thresholds* thr, const BlockPlan* plans, const int64_t* moff,
                                 const int64_t* idoff, uint32_t* counts, uint32_t* masks, uint32_t* ids,
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
  (void)prec;  // binary64 records only (binary32 records use the warp-per-group kernels)
  if (kern == CG_SPHERE) CG_LAUNCH_C2(0, CG_SPHERE);
  else if (kern == CG_CYLINDER) CG_LAUNCH_C2(0, CG_CYLINDER);
  else CG_LAUNCH_C2(0, CG_CUBE);
#undef CG_LAUNCH_C2
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_fill2(int prec, const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                const int64_t* moff, const int64_t* idoff, const uint32_t* masks,
                                const uint32_t* ids, const int64_t* offsets, int32_t* out, unsigned* work,
                                const uint32_t* status, cudaStream_t st) {
  ProfScope prof("radius_fill2", st);
  (void)prec;  // binary64 records only
  auto kfn = radius_fill2_kernel<0>;
  kfn<<<resident_grid(kfn, CT, 0), CT, 0, st>>>(iv, qs, plans, moff, idoff, masks, ids, offsets, out, work, status);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_radius_count32(int kern, const IndexView& iv, const QuerySet& qs, const Thresholds* thr,
                                  const BlockPlan* plans, const int64_t* moff, const int64_t* idoff,
                                  uint32_t* counts, uint32_t* masks, uint32_t* ids, unsigned* work,
                                  uint32_t* status, const cudaStream_t* sts, bool zspan) {
  // size classes: K <= 512 (a warp per group, 7 warps per CTA), <= 1024
  // (two warps per group, 16 per CTA), <= 2048 (four, 4 per CTA): shapes
  // measured fastest on the 12M ALS tile; work[0..2] are their group
  // counters, sts[0..2] their streams
#define CG_C5(KN, KC, NW, GW, CLS, WORK)                                                         \
  do {                                                                                            \
    auto kfn = radius_count5_kernel<KN, KC, NW, GW>;                                             \
    const size_t smem = C5<KC>::per_slot(GW) * (NW / GW);                                        \
    cudaError_t le = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (le != cudaSuccess) return le;                                                             \
    const int g = resident_grid(kfn, NW * 32, smem);                                             \
    cudaStream_t st = sts[CLS];                                                                  \
    ProfScope prof(CLS == 2 ? "radius_count5_2k" : (CLS ? "radius_count5_1k" : "radius_count5_512"), st); \
    kfn<<<g, NW * 32, smem, st>>>(iv, qs, thr, plans, moff, idoff, counts, masks, ids, WORK, status, \
                                  CLS, zspan ? 1 : 0);                                            \
    note_launch();                                                                                \
    if ((le = cudaGetLastError()) != cudaSuccess) return le;                                      \
  } while (0)
  // launch shapes (warps per CTA, warps per group) of the three classes:
  // 0 = (7, 1), (16, 2), (4, 4); 1 = (14, 2), (8, 1), (8, 4); 2 = (8, 1),
  // (16, 4), (4, 2)
#define CG_C5_ALL(KN)                                      \
  do {                                                     \
    if (shape == 1) {                                      \
      CG_C5(KN, 512, 14, 2, 0u, work);                     \
      CG_C5(KN, 1024, 8, 1, 1u, work + 1);                 \
      CG_C5(KN, 2048, 8, 4, 2u, work + 2);                 \
    } else if (shape == 2) {                               \
      CG_C5(KN, 512, 8, 1, 0u, work);                      \
      CG_C5(KN, 1024, 16, 4, 1u, work + 1);                \
      CG_C5(KN, 2048, 4, 2, 2u, work + 2);                 \
    } else {                                               \
      CG_C5(KN, 512, 7, 1, 0u, work);                      \
      CG_C5(KN, 1024, 16, 2, 1u, work + 1);                \
      CG_C5(KN, 2048, 4, 4, 2u, work + 2);                 \
    }                                                      \
  } while (0)
  const int shape = current_tuning().count_shape;
  if (kern == CG_SPHERE) CG_C5_ALL(CG_SPHERE);
  else if (kern == CG_CYLINDER) CG_C5_ALL(CG_CYLINDER);
  else CG_C5_ALL(CG_CUBE);
#undef CG_C5_ALL
#undef CG_C5
  return cudaGetLastError();
}

cudaError_t launch_radius_fill32(const IndexView& iv, const QuerySet& qs, const BlockPlan* plans,
                                 const int64_t* moff, const int64_t* idoff, const uint32_t* masks,
                                 const uint32_t* ids, const int64_t* offsets, int32_t* out, unsigned* work,
                                 const uint32_t* status, const cudaStream_t* sts) {
#define CG_F5(KC, NW, GW, CLS, WORK)                                                              \
  do {                                                                                            \
    auto kfn = radius_fill5_kernel<KC, NW, GW>;                                                  \
    const size_t smem = F5<KC>::per_slot(GW) * (NW / GW);                                        \
    cudaError_t le = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (le != cudaSuccess) return le;                                                             \
    const int g = resident_grid(kfn, NW * 32, smem);                                             \
    cudaStream_t st = sts[CLS];                                                                  \
    ProfScope prof(CLS == 2 ? "radius_fill5_2k" : (CLS ? "radius_fill5_1k" : "radius_fill5_512"), st); \
    kfn<<<g, NW * 32, smem, st>>>(iv, qs, plans, moff, idoff, masks, ids, offsets, out, WORK, status, CLS); \
    note_launch();                                                                                \
    if ((le = cudaGetLastError()) != cudaSuccess) return le;                                      \
  } while (0)
  // launch shapes (warps per CTA, warps per group) of the three classes:
  // 0 = (16, 1), (8, 1), (4, 2) (measured fastest on the 12M ALS tile);
  // 1 = (8, 1), (8, 2), (8, 4); 2 = (16, 2), (16, 2), (4, 1)
  const int shape = current_tuning().fill_shape;
  if (shape == 1) {
    CG_F5(512, 8, 1, 0u, work);
    CG_F5(1024, 8, 2, 1u, work + 1);
    CG_F5(2048, 8, 4, 2u, work + 2);
  } else if (shape == 2) {
    CG_F5(512, 16, 2, 0u, work);
    CG_F5(1024, 16, 2, 1u, work + 1);
    CG_F5(2048, 4, 1, 2u, work + 2);
  } else {
    CG_F5(512, 16, 1, 0u, work);
    CG_F5(1024, 8, 1, 1u, work + 1);
    CG_F5(2048, 4, 2, 2u, work + 2);
  }
#undef CG_F5
  return cudaGetLastError();
}

}  // namespace cg
