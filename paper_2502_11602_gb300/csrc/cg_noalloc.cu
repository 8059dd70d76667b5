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
// How: the single-pass scan with decoupled look-back of the library's other
// scans (cg_scan.cuh, the kernel with its "last tile writes the total" mode)
// keeps its per-tile status words, its tile ticket, its finish counter and
// its error word in `g_scan_scratch`, a file-scope device array of fixed size
// that every GPU loading this library holds until the process exits.  The
// host never uses the array's name as an address (in host code it only names
// a host-side stand-in); it asks the runtime for the device address and
// passes that pointer to the kernel.  The address belongs to the CUDA context
// that loaded the module, so it is asked for again on every call made while
// the stream is not capturing (a reset device reloads the module elsewhere);
// a call on a capturing stream uses the address the last such call found.
#include <mutex>

#include "cg_index.h"
#include "cg_scan.cuh"

namespace cg {
namespace {

constexpr int64_t kNaMaxTiles = 65536;
constexpr int64_t kNaMaxN = kNaMaxTiles * kScanTile;   // 134,217,728 counts
constexpr int kNaHeaderWords = 32;                      // 256 bytes: ticket, done, error

// [0] tile ticket, [1] finished tiles, [2] error word, [32 ...] tile status.
// 256 B + 512 KiB of device memory per GPU, for the lifetime of the process.
static __device__ __align__(256) unsigned long long g_scan_scratch[kNaHeaderWords + kNaMaxTiles];

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
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (cap == cudaStreamCaptureStatusNone) {
      // the current context's address of the array (the module may have been
      // reloaded since the last call, e.g. after a device reset)
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scan_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_scan_scratch)");
      g_na_ptr[dev] = p;
    } else if (!g_na_ptr[dev]) {
      return fail(CG_ERR_INVALID,
                  "cg_offsets_scan_noalloc: first call on this device made on a capturing stream");
    }
    scratch = g_na_ptr[dev];
  }
  const int64_t tiles = n > 0 ? (n + kScanTile - 1) / kScanTile : 1;
  // the ticket, the finish counter, the error flag and the used status words
  // must start at zero; the previous call's contents are still there
  e = cudaMemsetAsync(scratch, 0, (size_t)(kNaHeaderWords + tiles) * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(scratch)");
  unsigned long long* w = (unsigned long long*)scratch;
  scan_kernel<uint32_t, int64_t><<<(unsigned)tiles, kScanThreads, 0, st>>>(
      counts_dev, offsets_dev, n, w + kNaHeaderWords, reinterpret_cast<unsigned*>(w),
      reinterpret_cast<uint32_t*>(w + 2), reinterpret_cast<unsigned*>(w + 1));
  note_launch();
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "noalloc scan launch");
  return CG_OK;
}
