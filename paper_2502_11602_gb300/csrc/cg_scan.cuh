// cg_scan.cuh -- single-pass exclusive scan with decoupled look-back
// (Merrill & Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", 2016), shared by the library's scans (cg_sort.cu) and the
// allocation-free offsets scan (cg_noalloc.cu) (internal).
//
// Every look-back spin is bounded (kSpinLimit); on the bound the kernel
// records ST_TIMEOUT in `err` and carries on with a zero partial, so a wait
// can never hang the GPU.
#pragma once
#include <stdint.h>
#include <string.h>

#include "cg_internal.cuh"

namespace cg {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr unsigned long long kFlagAgg = 1ull << 62;
constexpr unsigned long long kFlagPre = 2ull << 62;
constexpr unsigned long long kValMask = (1ull << 62) - 1;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Exclusive prefix of the tiles before `tile` for one running total.
__device__ unsigned long long look_back(unsigned long long* status, long long tile,
                                        uint32_t* err) {
  unsigned long long prefix = 0;
  long long t = tile - 1;
  uint32_t spins = 0;
  while (t >= 0) {
    unsigned long long s = ld_volatile(status + t);
    if ((s & ~kValMask) == 0) {
      if (++spins > kSpinLimit) {
        atomicOr(err, ST_TIMEOUT);
        break;
      }
      continue;
    }
    prefix += s & kValMask;
    if ((s & ~kValMask) == kFlagPre) break;
    --t;
  }
  return prefix;
}

// done == nullptr: the thread holding element n - 1 writes out[n] (the
// total).  done != nullptr (a finish counter, zero before the launch): the
// last tile to finish writes out[n], or -1 if any look-back of the launch
// gave up (err != 0), so that a caller without a status word can tell.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const Tin* __restrict__ in,
                                                            Tout* __restrict__ out, int64_t n,
                                                            unsigned long long* status,
                                                            unsigned* tile_ctr, uint32_t* err,
                                                            unsigned* done = nullptr) {
  __shared__ long long s_tile;
  __shared__ unsigned long long s_warp[kScanThreads / 32];
  __shared__ unsigned long long s_prefix;
  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const int64_t base = tile * (int64_t)kScanTile + (int64_t)threadIdx.x * kScanItems;

  unsigned long long v[kScanItems];
  unsigned long long run = 0;
  // the thread's 8 inputs as two 16-byte loads where they are whole and
  // aligned (4-byte inputs), else one by one
  Tin xin[kScanItems];
  if (sizeof(Tin) == 4 && base + kScanItems <= n && ((reinterpret_cast<uintptr_t>(in + base) & 15u) == 0)) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(in + base));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(in + base) + 1);
    const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) xin[i] = (Tin)w[i];
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) xin[i] = (base + i < n) ? in[base + i] : (Tin)0;
  }
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = run;  // exclusive within the thread
    run += (unsigned long long)xin[i];
  }
  // block-wide exclusive scan of the thread totals
  unsigned long long incl = run;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
      unsigned long long t = s_warp[w];
      s_warp[w] = acc;
      acc += t;
    }
    // acc = tile aggregate
    if (tile == 0) {
      st_release(status, kFlagPre | (acc & kValMask));
      s_prefix = 0;
    } else {
      st_release(status + tile, kFlagAgg | (acc & kValMask));
      unsigned long long p = look_back(status, tile, err);
      st_release(status + tile, kFlagPre | ((p + acc) & kValMask));
      s_prefix = p;
    }
  }
  __syncthreads();
  const unsigned long long off = s_prefix + s_warp[warp] + (incl - run);
  Tout o[kScanItems];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) o[i] = (Tout)(off + v[i]);
  if (base + kScanItems <= n && ((reinterpret_cast<uintptr_t>(out + base) & 15u) == 0)) {
    // whole and aligned: 16-byte stores
    uint4* d = reinterpret_cast<uint4*>(out + base);
#pragma unroll
    for (int i = 0; i < (int)(kScanItems * sizeof(Tout) / 16); ++i) {
      uint4 q;
      memcpy(&q, reinterpret_cast<const char*>(o) + 16 * i, 16);
      d[i] = q;
    }
  } else {
#pragma unroll
    for (int i = 0; i < kScanItems; ++i)
      if (base + i < n) out[base + i] = o[i];
  }
  if (done == nullptr) {
    if (base <= n - 1 && n - 1 < base + kScanItems) out[n] = (Tout)(off + run);
    if (n == 0 && tile == 0 && threadIdx.x == 0) out[0] = (Tout)0;
  } else if (threadIdx.x == 0) {
    __threadfence();
    const unsigned ntiles = gridDim.x;
    if (atomicAdd(done, 1u) == ntiles - 1) {
      __threadfence();
      const bool bad = *((volatile uint32_t*)err) != 0u;
      const unsigned long long last = ld_volatile(status + (ntiles - 1));
      out[n] = bad ? (Tout)-1 : (Tout)(last & kValMask);
    }
  }
}

}  // namespace
}  // namespace cg
