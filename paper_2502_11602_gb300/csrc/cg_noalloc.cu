// cg_noalloc.cu -- cg_offsets_scan_noalloc: the exclusive scan that turns
// per-query neighbour counts into CSR offsets, for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc (or a framework allocator
// call) is not an option -- a serving loop whose device memory was reserved
// up front by another allocator and must not grow, a real-time path where an
// allocation may block or fail at the worst moment, or a host that hands the
// library only the input and output buffers it owns.  The regular count pass
// allocates its scan scratch per call; this variant never does.
//
// How: the single-pass scan with decoupled look-back keeps its per-tile
// status words and its tile ticket in `g_scan_scratch`, a file-scope device
// array of fixed size that every GPU loading this library holds until the
// process exits.  The host never uses the array's name as an address (in
// host code it only names a host-side stand-in); it asks the runtime for the
// device address once per device and passes that pointer to the kernel.
#include <mutex>

#include "cg_index.h"

namespace cg {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaItems = 8;
constexpr int kNaTile = kNaThreads * kNaItems;          // 2048 counts per tile
constexpr int64_t kNaMaxTiles = 65536;
constexpr int64_t kNaMaxN = kNaMaxTiles * kNaTile;      // 134,217,728 counts
constexpr int kNaHeaderWords = 32;                      // 256 bytes: ticket, done, error
constexpr unsigned long long kNaFlagAgg = 1ull << 62;
constexpr unsigned long long kNaFlagPre = 2ull << 62;
constexpr unsigned long long kNaValMask = (1ull << 62) - 1;

// [0] tile ticket, [1] finished tiles, [2] error flag, [32 ...] tile status.
// 256 B + 512 KiB of device memory per GPU, for the lifetime of the process.
static __device__ __align__(256) unsigned long long g_scan_scratch[kNaHeaderWords + kNaMaxTiles];

__device__ __forceinline__ unsigned long long na_ld(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void na_st(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__global__ void __launch_bounds__(kNaThreads) noalloc_scan_kernel(const uint32_t* __restrict__ in,
                                                                  int64_t* __restrict__ out, int64_t n,
                                                                  unsigned long long* scratch,
                                                                  unsigned ntiles) {
  __shared__ long long s_tile;
  __shared__ unsigned long long s_warp[kNaThreads / 32];
  __shared__ unsigned long long s_prefix;
  unsigned* ticket = reinterpret_cast<unsigned*>(scratch);
  unsigned long long* status = scratch + kNaHeaderWords;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  __syncthreads();
  const long long tile = s_tile;
  const int64_t base = tile * (int64_t)kNaTile + (int64_t)threadIdx.x * kNaItems;
  unsigned long long v[kNaItems];
  unsigned long long run = 0;
#pragma unroll
  for (int i = 0; i < kNaItems; ++i) {
    const int64_t e = base + i;
    v[i] = run;
    run += (e < n) ? (unsigned long long)in[e] : 0ull;
  }
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  unsigned long long incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long acc = 0;
    for (int w = 0; w < kNaThreads / 32; ++w) {
      unsigned long long t = s_warp[w];
      s_warp[w] = acc;
      acc += t;
    }
    unsigned long long prefix = 0;
    if (tile == 0) {
      na_st(status, kNaFlagPre | (acc & kNaValMask));
    } else {
      na_st(status + tile, kNaFlagAgg | (acc & kNaValMask));
      long long t = tile - 1;
      uint32_t spins = 0;
      while (t >= 0) {  // bounded look-back: gives up with an error flag
        unsigned long long s = na_ld(status + t);
        if ((s & ~kNaValMask) == 0) {
          if (++spins > kSpinLimit) {
            atomicExch(scratch + 2, 1ull);
            break;
          }
          continue;
        }
        prefix += s & kNaValMask;
        if ((s & ~kNaValMask) == kNaFlagPre) break;
        --t;
      }
      na_st(status + tile, kNaFlagPre | ((prefix + acc) & kNaValMask));
    }
    s_prefix = prefix;
  }
  __syncthreads();
  const unsigned long long off = s_prefix + s_warp[warp] + (incl - run);
#pragma unroll
  for (int i = 0; i < kNaItems; ++i) {
    const int64_t e = base + i;
    if (e < n) out[e] = (int64_t)(off + v[i]);
  }
  // the last tile to finish writes the total (or -1 if any wait gave up)
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned done = atomicAdd(reinterpret_cast<unsigned*>(scratch + 1), 1u);
    if (done == ntiles - 1) {
      __threadfence();
      const bool err = na_ld(scratch + 2) != 0;
      const unsigned long long last = na_ld(status + (ntiles - 1));
      out[n] = err ? (int64_t)-1 : (int64_t)(last & kNaValMask);
    }
  }
}

std::mutex g_na_mutex;
void* g_na_ptr[256] = {};  // device address of g_scan_scratch, per device ordinal

}  // namespace
}  // namespace cg

using namespace cg;

extern "C" cg_status cg_offsets_scan_noalloc(const uint32_t* counts_dev, int64_t n,
                                             int64_t* offsets_dev, void* stream) {
  if (!offsets_dev) return fail(CG_ERR_INVALID, "offsets_dev is NULL");
  if (n < 0) return fail(CG_ERR_INVALID, "n must be >= 0");
  if (n > kNaMaxN)
    return fail(CG_ERR_INVALID, "n exceeds the fixed scratch of cg_offsets_scan_noalloc (max 134217728 counts)");
  if (n > 0 && !counts_dev) return fail(CG_ERR_INVALID, "counts_dev is NULL");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 256) return fail(CG_ERR_INVALID, "device ordinal out of range");
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
      // set-up, once per device, with that device current
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scan_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scan_scratch)");
      g_na_ptr[dev] = p;
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t tiles = n > 0 ? (n + kNaTile - 1) / kNaTile : 1;
  // the ticket, the finish counter, the error flag and the used status words
  // must start at zero; the previous call's contents are still there
  e = cudaMemsetAsync(scratch, 0, (size_t)(kNaHeaderWords + tiles) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
  noalloc_scan_kernel<<<(unsigned)tiles, kNaThreads, 0, st>>>(counts_dev, offsets_dev, n,
                                                             (unsigned long long*)scratch,
                                                             (unsigned)tiles);
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc scan launch");
  return CG_OK;
}
