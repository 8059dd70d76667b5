// cg_zwin.cu -- height order of the voxel columns of a 2D grid (binary32
// records), and the height chunks of the radius search's voxel groups.
//
// On a 2D grid a voxel is a vertical column, and Algorithm 1 tests every
// point of every column that meets the kernel's bounding box, whatever its
// height.  In an airborne tile with walls and trees most of those points are
// far above or below the query.  Every column therefore also exists as a
// copy sorted by height (`pts32z`, with the original ids in the same order in
// `sidz`), built once with the index:
//
//   zsort   each voxel run sorted by binary32 height, ties in id order; runs
//           longer than kZsortMax keep id order (searched whole).
//   chunks  for an all-points radius pass, each column's height-sorted
//           queries are cut into chunks whose heights span at most the
//           radius (and at most kChunkMax queries); each chunk is a voxel
//           group of its own.  The plan then takes, from every column that
//           meets a chunk's kernel boxes, only the contiguous height range
//           [lowest - h, highest + h] (h the kernel's half height plus the
//           rounding pad), so the candidate set stays a superset of the
//           chunk's kernels while shrinking with the chunk's height span.
//
// Everything after the plan (the count and fill kernels, the exact decision
// of the binary32 path) is unchanged: a group's candidates are still staged,
// sorted by id and tested against all of its queries.
#include <math.h>

#include <algorithm>

#include "cg_f32x2.cuh"
#include "cg_query.cuh"

namespace cg {
namespace {

constexpr int ZS_WARPS = 8;      // build sort: warps per CTA
constexpr int ZS_SHORT = 256;    // runs up to this length: one warp each

__device__ __forceinline__ uint32_t z_order_key(float z) {
  const uint32_t u = __float_as_uint(z);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// Bitonic sort of n2 (a power of two) 64-bit keys in shared memory by the
// threads [0, nth) of `tid`, with `sync` between the steps.
template <class Sync>
__device__ __forceinline__ void bitonic_u64(unsigned long long* K, uint32_t n2, uint32_t tid, uint32_t nth,
                                            Sync sync) {
  for (uint32_t k = 2; k <= n2; k <<= 1)
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = tid; i < n2; i += nth) {
        const uint32_t l = i ^ j;
        if (l > i) {
          const unsigned long long a = K[i], b = K[l];
          const bool up = (i & k) == 0;
          if (up ? a > b : a < b) {
            K[i] = b;
            K[l] = a;
          }
        }
      }
      sync();
    }
}

// One compare-exchange step of a bitonic network held in registers: element
// e of the network, partner e ^ j (a lane of the same register), block size k.
__device__ __forceinline__ unsigned long long bitonic_step(unsigned long long key, uint32_t e, uint32_t j,
                                                           uint32_t k) {
  const unsigned long long o = __shfl_xor_sync(0xffffffffu, key, (int)j);
  const bool keep_min = ((e & j) == 0) == ((e & k) == 0);
  return keep_min ? (o < key ? o : key) : (o > key ? o : key);
}

// Runs of up to ZS_SHORT points: one warp each, sorted by (height, position
// in the id-ordered run): up to 64 points in registers (two per lane),
// longer in shared memory; runs longer than ZS_SHORT are listed for
// zsort_long_kernel.
__global__ void __launch_bounds__(ZS_WARPS * 32) zsort_short_kernel(const float4* __restrict__ in,
                                                                    float4* __restrict__ out,
                                                                    uint32_t* __restrict__ sid_out,
                                                                    const uint32_t* __restrict__ ustart,
                                                                    uint32_t cap, const uint32_t* ndev, uint32_t n,
                                                                    uint32_t* __restrict__ long_list,
                                                                    uint32_t* long_n, const uint32_t* status) {
  if (replan_pending(status)) return;
  __shared__ unsigned long long keys[ZS_WARPS][ZS_SHORT];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t nruns = ndev ? min(*ndev, cap) : cap;
  unsigned long long* K = keys[warp];
  for (uint32_t run = blockIdx.x * ZS_WARPS + warp; run < nruns; run += gridDim.x * ZS_WARPS) {
    const uint32_t s = ustart[run], e = ustart[run + 1];
    if (e < s || e > n) continue;  // tables of a replay that outgrew them (flagged; never written past n)
    const uint32_t len = e - s;
    if (len > (uint32_t)ZS_SHORT) {
      if (lane == 0) long_list[atomicAdd(long_n, 1u)] = run;
      continue;
    }
    if (len <= 1) {
      if (lane == 0 && len == 1) {
        out[s] = in[s];
        sid_out[s] = __float_as_uint(in[s].w);
      }
      continue;
    }
    if (len <= 64) {
      // elements lane and lane + 32; padding keys sort last
      unsigned long long k0 = lane < len ? ((unsigned long long)z_order_key(in[s + lane].z) << 32) | lane : ~0ull;
      unsigned long long k1 =
          lane + 32 < len ? ((unsigned long long)z_order_key(in[s + lane + 32].z) << 32) | (lane + 32) : ~0ull;
      const uint32_t n2 = len <= 32 ? 32u : 64u;
      for (uint32_t k = 2; k <= n2; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
          if (j == 32) {  // elements lane and lane + 32: in one lane
            const bool up = (lane & k) == 0;
            const unsigned long long lo = k0 < k1 ? k0 : k1, hi = k0 < k1 ? k1 : k0;
            k0 = up ? lo : hi;
            k1 = up ? hi : lo;
          } else {
            k0 = bitonic_step(k0, lane, j, k);
            if (n2 == 64) k1 = bitonic_step(k1, lane + 32, j, k);
          }
        }
      if (lane < len) {
        const float4 rec = in[s + (uint32_t)k0];
        out[s + lane] = rec;
        sid_out[s + lane] = __float_as_uint(rec.w);
      }
      if (lane + 32 < len) {
        const float4 rec = in[s + (uint32_t)k1];
        out[s + lane + 32] = rec;
        sid_out[s + lane + 32] = __float_as_uint(rec.w);
      }
      continue;
    }
    uint32_t n2 = 2;
    while (n2 < len) n2 <<= 1;
    for (uint32_t i = lane; i < n2; i += 32)
      K[i] = i < len ? ((unsigned long long)z_order_key(in[s + i].z) << 32) | i : ~0ull;
    __syncwarp();
    bitonic_u64(K, n2, lane, 32u, [] { __syncwarp(); });
    for (uint32_t i = lane; i < len; i += 32) {
      const float4 rec = in[s + (uint32_t)K[i]];
      out[s + i] = rec;
      sid_out[s + i] = __float_as_uint(rec.w);
    }
    __syncwarp();
  }
}

// Runs longer than ZS_SHORT: one CTA each; runs over kZsortMax are copied
// in id order (the query kernels search them whole).
__global__ void __launch_bounds__(256) zsort_long_kernel(const float4* __restrict__ in, float4* __restrict__ out,
                                                         uint32_t* __restrict__ sid_out,
                                                         const uint32_t* __restrict__ ustart,
                                                         const uint32_t* __restrict__ long_list,
                                                         const uint32_t* long_n, const uint32_t* status) {
  if (replan_pending(status)) return;
  __shared__ unsigned long long K[kZsortMax];
  const uint32_t nl = *long_n;
  for (uint32_t li = blockIdx.x; li < nl; li += gridDim.x) {
    const uint32_t run = long_list[li];
    const uint32_t s = ustart[run], len = ustart[run + 1] - s;  // checked by zsort_short_kernel
    if (len > kZsortMax) {
      for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
        out[s + i] = in[s + i];
        sid_out[s + i] = __float_as_uint(in[s + i].w);
      }
      continue;
    }
    uint32_t n2 = 2;
    while (n2 < len) n2 <<= 1;
    for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x)
      K[i] = i < len ? ((unsigned long long)z_order_key(in[s + i].z) << 32) | i : ~0ull;
    __syncthreads();
    bitonic_u64(K, n2, threadIdx.x, blockDim.x, [] { __syncthreads(); });
    for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) {
      const float4 rec = in[s + (uint32_t)K[i]];
      out[s + i] = rec;
      sid_out[s + i] = __float_as_uint(rec.w);
    }
    __syncthreads();
  }
}

// Walks run [s, e) of the height-sorted records and calls emit(c, i) for
// the start i of its c-th chunk: a chunk ends before the first point more
// than dz above the chunk's lowest point, or after qmax points (runs that
// are not sorted by height, longer than kZsortMax: every qmax points).
template <class Emit>
__device__ __forceinline__ uint32_t z_chunks_of_run(const float4* __restrict__ pz, uint32_t s, uint32_t e,
                                                    float dz, uint32_t qmax, Emit emit) {
  // one warp per run: the next chunk starts at the first point, at or after
  // the current chunk's next candidate, that is qmax points past the chunk's
  // first or more than dz above it; 32 points tested per step (a ballot).
  // The same chunks as a point-by-point scan (the tests are identical and
  // taken in the same order).  Chunk c starting at point i: emit(c, i),
  // called by lane 0.
  const uint32_t lane = threadIdx.x & 31u;
  if (e <= s) return 0u;
  const bool sorted = e - s <= kZsortMax;
  uint32_t c = 0, start = s;
  float z0 = pz[s].z;
  if (lane == 0) emit(0u, s);
  for (uint32_t i0 = s + 1; i0 < e;) {
    const uint32_t i = i0 + lane;
    bool brk = false;
    float z = z0;
    if (i < e) {
      z = sorted ? pz[i].z : z0;
      brk = i - start >= qmax || z - z0 > dz;
    }
    const unsigned bm = __ballot_sync(0xffffffffu, brk);
    if (bm == 0u) {
      i0 += 32u;
      continue;
    }
    const int src = __ffs(bm) - 1;
    start = i0 + (uint32_t)src;
    z0 = __shfl_sync(0xffffffffu, z, src);
    ++c;
    if (lane == 0) emit(c, start);
    i0 = start + 1u;
  }
  return c + 1u;
}

__global__ void zchunk_count_kernel(const float4* __restrict__ pz, const uint32_t* __restrict__ ustart,
                                    uint32_t nruns, float dz, uint32_t qmax, uint32_t* __restrict__ cnt) {
  const uint32_t lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nruns; r += nw) {
    const uint32_t c = z_chunks_of_run(pz, ustart[r], ustart[r + 1], dz, qmax, [](uint32_t, uint32_t) {});
    if (lane == 0) cnt[r] = c;
  }
}

__global__ void zchunk_emit_kernel(const float4* __restrict__ pz, const uint32_t* __restrict__ ustart,
                                   const uint32_t* __restrict__ ukeys, uint32_t nruns, float dz, uint32_t qmax,
                                   const uint32_t* __restrict__ coff, uint32_t* __restrict__ cbeg,
                                   uint32_t* __restrict__ ckey, uint32_t n) {
  const uint32_t lane = threadIdx.x & 31u, nw = gridDim.x * (blockDim.x >> 5);
  for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < nruns; r += nw) {
    const uint32_t o = coff[r], key = ukeys[r];
    z_chunks_of_run(pz, ustart[r], ustart[r + 1], dz, qmax, [&](uint32_t c, uint32_t i) {
      cbeg[o + c] = i;
      ckey[o + c] = key;
    });
    if (r == nruns - 1 && lane == 0) cbeg[coff[nruns]] = n;
  }
}

int zw_sm_count() {
  static const int sms = [] {
    int dev = 0, m = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m, cudaDevAttrMultiProcessorCount, dev);
    return m > 0 ? m : 152;
  }();
  return sms;
}

}  // namespace

// ------------------------------------------------------------------ host

cudaError_t launch_zsort(const float4* in, float4* out, uint32_t* sid_out, const uint32_t* ustart, uint32_t cap,
                         const uint32_t* ndev, uint32_t n, uint32_t* long_list, uint32_t* long_n,
                         const uint32_t* status, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(long_n, 0, 4, st);
  if (e != cudaSuccess) return e;
  const int sms = zw_sm_count();
  const int g1 = (int)std::min<int64_t>(((int64_t)cap + ZS_WARPS - 1) / ZS_WARPS, (int64_t)sms * 8);
  {
    ProfScope prof("build_zsort_short", st);
    zsort_short_kernel<<<g1 > 0 ? g1 : 1, ZS_WARPS * 32, 0, st>>>(in, out, sid_out, ustart, cap, ndev, n,
                                                                  long_list, long_n, status);
  }
  note_launch();
  {
    ProfScope prof("build_zsort_long", st);
    zsort_long_kernel<<<sms * 4, 256, 0, st>>>(in, out, sid_out, ustart, long_list, long_n, status);
  }
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zchunk_count(const float4* pz, const uint32_t* ustart, uint32_t nruns, float dz, uint32_t qmax,
                                uint32_t* cnt, cudaStream_t st) {
  if (nruns == 0) return cudaSuccess;
  const int g = (int)std::min<int64_t>(((int64_t)nruns + 7) / 8, (int64_t)zw_sm_count() * 8);
  zchunk_count_kernel<<<g, 256, 0, st>>>(pz, ustart, nruns, dz, qmax, cnt);
  note_launch();
  return cudaGetLastError();
}

cudaError_t launch_zchunk_emit(const float4* pz, const uint32_t* ustart, const uint32_t* ukeys, uint32_t nruns,
                               float dz, uint32_t qmax, const uint32_t* coff, uint32_t* cbeg, uint32_t* ckey,
                               uint32_t n, cudaStream_t st) {
  if (nruns == 0) return cudaSuccess;
  const int g = (int)std::min<int64_t>(((int64_t)nruns + 7) / 8, (int64_t)zw_sm_count() * 8);
  zchunk_emit_kernel<<<g, 256, 0, st>>>(pz, ustart, ukeys, nruns, dz, qmax, coff, cbeg, ckey, n);
  note_launch();
  return cudaGetLastError();
}

}  // namespace cg
