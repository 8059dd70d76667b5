// cg_sort.cu -- device-wide primitives of the index build and the query
// offsets: a single-pass exclusive scan with decoupled look-back (Merrill &
// Garland, "Single-pass Parallel Prefix Scan with Decoupled Look-back",
// 2016) and a stable LSD radix sort of (key, index) pairs with one kernel
// per 8-bit digit that also uses decoupled look-back for the digit offsets
// (the Onesweep scheme of Adinets & Merrill, 2022).  Ties keep input order,
// so equal voxel keys stay in ascending original point id (the reordering
// remark of Section 3.5 with a deterministic order inside a voxel).
//
// Every look-back spin is bounded (kSpinLimit); on the bound the kernel
// records ST_TIMEOUT in the status word and carries on with a zero partial,
// so a wait can never hang the GPU.
#include "cg_scan.cuh"
#include "cg_sort.cuh"

namespace cg {

namespace {

// ---------------------------------------------------------------- radix sort

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;  // per thread
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint32_t* __restrict__ keys,
                                                                  int64_t n, int passes,
                                                                  uint32_t* __restrict__ hist) {
  __shared__ uint32_t sh[4][kRadix];
  for (int i = threadIdx.x; i < 4 * kRadix; i += blockDim.x) (&sh[0][0])[i] = 0;
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t k = keys[e];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(k >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += blockDim.x) {
    uint32_t c = (&sh[0][0])[i];
    if (c) atomicAdd(hist + i, c);
  }
}

// exclusive scan of each pass's 256-bin histogram, in place
__global__ void radix_hist_scan_kernel(uint32_t* hist, int passes) {
  __shared__ uint32_t s[kRadix];
  for (int p = 0; p < passes; ++p) {
    uint32_t v = hist[p * kRadix + threadIdx.x];
    s[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t acc = 0;
      for (int d = 0; d < kRadix; ++d) {
        uint32_t t = s[d];
        s[d] = acc;
        acc += t;
      }
    }
    __syncthreads();
    hist[p * kRadix + threadIdx.x] = s[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSortThreads) onesweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int64_t n, int shift,
    const uint32_t* __restrict__ digit_base, unsigned long long* status, unsigned* tile_ctr,
    uint32_t* err) {
  __shared__ uint32_t s_keys[kSortTile];
  __shared__ uint32_t s_vals[kSortTile];
  __shared__ uint32_t s_whist[kSortWarps][kRadix];
  __shared__ uint32_t s_dstart[kRadix];   // tile-local start of each digit
  __shared__ uint32_t s_gbase[kRadix];    // global start of each digit's slice of this tile
  __shared__ uint32_t s_wsum[kSortWarps]; // per-warp sums of the digit totals
  __shared__ long long s_tile;

  if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&s_whist[0][0])[i] = 0;
  __syncthreads();
  const long long tile = s_tile;
  const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const int64_t wbase = tile * (int64_t)kSortTile + (int64_t)warp * (32 * kSortItems);

  uint32_t key[kSortItems], val[kSortItems], rank[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    int64_t e = wbase + j * 32 + lane;
    bool ok = e < n;
    key[j] = ok ? keys_in[e] : 0xffffffffu;
    val[j] = ok ? (vals_in ? vals_in[e] : (uint32_t)e) : 0u;
  }
  // stable rank inside the warp's sub-tile (order: j-major, then lane)
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    int64_t e = wbase + j * 32 + lane;
    bool ok = e < n;
    uint32_t d = (key[j] >> shift) & 255u;
    unsigned peers = __match_any_sync(0xffffffffu, ok ? d : (256u + lane));
    uint32_t before = ok ? s_whist[warp][d] : 0u;
    __syncwarp();
    unsigned lower = peers & lanemask_lt();
    rank[j] = before + __popc(lower);
    if (ok && lower == 0) s_whist[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: warp-exclusive offsets and the tile total
  uint32_t total;
  {
    const int d = threadIdx.x;  // kSortThreads == kRadix
    uint32_t acc = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t t = s_whist[w][d];
      s_whist[w][d] = acc;
      acc += t;
    }
    total = acc;
  }
  // tile-local start of each digit: block-wide exclusive scan of the digit
  // totals (thread d holds digit d)
  {
    uint32_t incl = total;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= (unsigned)o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t add = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) add += w < (int)warp ? s_wsum[w] : 0u;
    s_dstart[threadIdx.x] = add + incl - total;
  }
  // decoupled look-back per digit (thread d owns digit d)
  {
    const int d = threadIdx.x;
    unsigned long long* st = status + d;  // status[tile * 256 + d]
    const long long stride = kRadix;
    unsigned long long prefix = 0;
    if (tile == 0) {
      st_release(st, kFlagPre | total);
    } else {
      st_release(st + tile * stride, kFlagAgg | total);
      long long t = tile - 1;
      uint32_t spins = 0;
      while (t >= 0) {
        unsigned long long s = ld_volatile(st + t * stride);
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
      st_release(st + tile * stride, kFlagPre | ((prefix + total) & kValMask));
    }
    s_gbase[d] = digit_base[d] + (uint32_t)prefix;
  }
  __syncthreads();
  // scatter into shared memory in digit order
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    int64_t e = wbase + j * 32 + lane;
    if (e < n) {
      uint32_t d = (key[j] >> shift) & 255u;
      uint32_t slot = s_dstart[d] + s_whist[warp][d] + rank[j];
      s_keys[slot] = key[j];
      s_vals[slot] = val[j];
    }
  }
  __syncthreads();
  int64_t valid = n - tile * (int64_t)kSortTile;
  if (valid > kSortTile) valid = kSortTile;
  for (int i = threadIdx.x; i < valid; i += kSortThreads) {
    uint32_t k = s_keys[i];
    uint32_t d = (k >> shift) & 255u;
    uint32_t pos = s_gbase[d] + (uint32_t)i - s_dstart[d];
    keys_out[pos] = k;
    vals_out[pos] = s_vals[i];
  }
}

__global__ void iota_kernel(uint32_t* v, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    v[e] = (uint32_t)e;
}

int grid_for(int64_t n, int threads, int max_blocks = 152 * 16) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > max_blocks) b = max_blocks;
  return (int)b;
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  return 256 + (size_t)tiles * 8;
}

template <class Tin, class Tout>
static cudaError_t scan_impl(const Tin* in, Tout* out, int64_t n, void* scratch, uint32_t* err,
                             cudaStream_t st) {
  int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles < 1) tiles = 1;
  unsigned* ctr = (unsigned*)scratch;
  unsigned long long* status = (unsigned long long*)((char*)scratch + 256);
  cudaError_t e = cudaMemsetAsync(scratch, 0, scan_scratch_bytes(n), st);
  if (e != cudaSuccess) return e;
  scan_kernel<Tin, Tout><<<(unsigned)tiles, kScanThreads, 0, st>>>(in, out, n, status, ctr, err); note_launch();
  return cudaGetLastError();
}

cudaError_t exclusive_scan_u32_i64(const uint32_t* in, int64_t* out, int64_t n, void* scratch,
                                   uint32_t* err, cudaStream_t st) {
  return scan_impl<uint32_t, int64_t>(in, out, n, scratch, err, st);
}
cudaError_t exclusive_scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t n, void* scratch,
                                   uint32_t* err, cudaStream_t st) {
  return scan_impl<uint32_t, uint32_t>(in, out, n, scratch, err, st);
}

size_t radix_sort_scratch_bytes(int64_t n) {
  int64_t tiles = (n + kSortTile - 1) / kSortTile;
  if (tiles < 1) tiles = 1;
  // keys/vals ping-pong + histograms + per-pass counters + status
  return (size_t)n * 16 + 4 * kRadix * 4 + 256 + (size_t)tiles * kRadix * 8 + 1024;
}

cudaError_t radix_sort_pairs(const uint32_t* keys, int64_t n, int key_bits, uint32_t* keys_sorted,
                             uint32_t* vals_sorted, void* scratch, uint32_t* err,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int passes = (key_bits + 7) / 8;
  if (passes > 4) passes = 4;
  if (passes == 0) {
    cudaError_t e = dev_copy(keys_sorted, keys, (size_t)n * 4, st);
    if (e != cudaSuccess) return e;
    iota_kernel<<<grid_for(n, 256), 256, 0, st>>>(vals_sorted, n); note_launch();
    return cudaGetLastError();
  }
  int64_t tiles = (n + kSortTile - 1) / kSortTile;
  char* p = (char*)scratch;
  uint32_t* kb = (uint32_t*)p; p += (size_t)n * 4;
  uint32_t* vb = (uint32_t*)p; p += (size_t)n * 4;
  uint32_t* kc = (uint32_t*)p; p += (size_t)n * 4;
  uint32_t* vc = (uint32_t*)p; p += (size_t)n * 4;
  uint32_t* hist = (uint32_t*)p; p += 4 * kRadix * 4;
  unsigned* ctrs = (unsigned*)p; p += 256;
  unsigned long long* status = (unsigned long long*)p;
  size_t status_bytes = (size_t)tiles * kRadix * 8;

  cudaError_t e = cudaMemsetAsync(hist, 0, 4 * kRadix * 4 + 256, st);
  if (e != cudaSuccess) return e;
  radix_hist_kernel<<<grid_for(n, kSortThreads, 152 * 4), kSortThreads, 0, st>>>(keys, n, passes, hist); note_launch();
  radix_hist_scan_kernel<<<1, kRadix, 0, st>>>(hist, passes); note_launch();
  const uint32_t* kin = keys;
  const uint32_t* vin = nullptr;
  for (int pass = 0; pass < passes; ++pass) {
    bool last = pass == passes - 1;
    uint32_t* kout = last ? keys_sorted : ((pass & 1) ? kc : kb);
    uint32_t* vout = last ? vals_sorted : ((pass & 1) ? vc : vb);
    e = cudaMemsetAsync(status, 0, status_bytes, st);
    if (e != cudaSuccess) return e;
    onesweep_kernel<<<(unsigned)tiles, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, 8 * pass,
                                                             hist + pass * kRadix, status,
                                                             ctrs + pass, err); note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    kin = kout;
    vin = vout;
  }
  return cudaSuccess;
}

}  // namespace cg
