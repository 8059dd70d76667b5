// cg_capi.cu -- the C ABI declared in include/cheesegpu.h: argument checks,
// error reporting, allocation hooks and the calls into the build / query
// implementations.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cg_index.h"
#include "cg_query.cuh"

namespace cg {

cg_status build_index(const double* xyz, int64_t n, const int64_t* toff_host, int ntiles,
                      const double* cell_xy, const double* cell_z, int dim, int flavor,
                      int precision, cudaStream_t st, cg_index** out);
cg_status radius_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, double r,
                      int kernel, bool fill, int64_t* offsets, int32_t* out, int64_t* total_host,
                      cudaStream_t st);
cg_status knn_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, int k, int32_t* idx,
                   double* d2, cudaStream_t st);

namespace {
std::atomic<unsigned long long> g_launches{0};
thread_local std::string g_last_error;
cg_alloc_fn g_alloc = nullptr;
cg_free_fn g_free = nullptr;
void* g_user = nullptr;
}  // namespace

void set_error(const std::string& msg) { g_last_error = msg; }

namespace {
struct ProfPending {
  std::string name;
  cudaEvent_t a, b;
};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
std::vector<ProfPending> g_prof_pending;
std::map<std::string, std::pair<int64_t, double>> g_prof_acc;  // launches, total ms

// Folds finished event pairs into the totals (waits for them).
void prof_resolve() {
  std::vector<ProfPending> p;
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    p.swap(g_prof_pending);
  }
  for (auto& r : p) {
    float ms = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
      std::lock_guard<std::mutex> g(g_prof_mu);
      auto& e = g_prof_acc[r.name];
      e.first += 1;
      e.second += ms;
    }
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  cudaGetLastError();
}
}  // namespace

namespace {
struct AuxStreams {
  int dev = -1;
  bool ok = false;
  cudaStream_t s[Fork::kMax - 1] = {};
  cudaEvent_t fork = nullptr, join[Fork::kMax - 1] = {};
  ~AuxStreams() { release(); }
  void release() {
    if (!ok) return;
    for (int i = 0; i < Fork::kMax - 1; ++i) {
      cudaStreamDestroy(s[i]);
      cudaEventDestroy(join[i]);
    }
    cudaEventDestroy(fork);
    ok = false;
  }
  bool ensure() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return false;
    if (ok && d == dev) return true;
    release();
    bool good = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    // the last branch carries the longest single blocks of a pass (the
    // general kernel's largest groups): it gets the highest priority so that
    // they start first instead of ending the pass
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    for (int i = 0; good && i < Fork::kMax - 1; ++i)
      good = cudaStreamCreateWithPriority(&s[i], cudaStreamNonBlocking, i == Fork::kMax - 2 ? greatest : least) ==
                 cudaSuccess &&
             cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) == cudaSuccess;
    cudaGetLastError();
    ok = good;
    dev = d;
    return ok;
  }
};
thread_local AuxStreams t_aux;
}  // namespace

// Without extra streams (creation failed) every branch is the origin itself.
Fork::Fork(cudaStream_t origin, int branches) : origin_(origin) {
  for (int i = 0; i < kMax - 1; ++i) aux_[i] = origin;
  n_ = branches < 1 ? 1 : (branches > kMax ? kMax : branches);
  if (n_ == 1 || !t_aux.ensure()) {
    n_ = 1;
    return;
  }
  cudaEventRecord(t_aux.fork, origin);
  for (int i = 0; i < n_ - 1; ++i) {
    aux_[i] = t_aux.s[i];
    join_[i] = t_aux.join[i];
    cudaStreamWaitEvent(aux_[i], t_aux.fork, 0);
  }
}

void Fork::join() {
  if (joined_) return;
  joined_ = true;
  for (int i = 0; i < n_ - 1; ++i) {
    cudaEventRecord(join_[i], aux_[i]);
    cudaStreamWaitEvent(origin_, join_[i], 0);
  }
}

ProfScope::ProfScope(const char* nm, cudaStream_t s) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  if (cudaEventCreate(&a) != cudaSuccess) {
    a = nullptr;
    cudaGetLastError();
    return;
  }
  cudaEventRecord(a, s);
  name = nm;
  st = s;
}

ProfScope::~ProfScope() {
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    cudaGetLastError();
    return;
  }
  cudaEventRecord(b, st);
  std::lock_guard<std::mutex> g(g_prof_mu);
  g_prof_pending.push_back({name, a, b});
}

void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

// ---------------------------------------------------------------------------
// Copy-engine-free small transfers (HostRead, host_put, dev_copy)
// ---------------------------------------------------------------------------
namespace {
struct XferItem {
  const void* src;
  void* dst;
  unsigned long long bytes;
};
constexpr int kXferItems = 8;
struct XferBatch {
  XferItem it[kXferItems];
  int n;
};

// Every item is copied by the whole grid, in 16-, 8-, 4- or 1-byte units as
// the alignment of both ends and of the length allows.
__global__ void __launch_bounds__(256) xfer_kernel(XferBatch b) {
  const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int i = 0; i < b.n; ++i) {
    const XferItem x = b.it[i];
    const uintptr_t a = (uintptr_t)x.src | (uintptr_t)x.dst | (uintptr_t)x.bytes;
    if ((a & 15) == 0) {
      const uint4* s = (const uint4*)x.src;
      uint4* d = (uint4*)x.dst;
      for (size_t w = t; w < x.bytes / 16; w += stride) d[w] = s[w];
    } else if ((a & 7) == 0) {
      const uint2* s = (const uint2*)x.src;
      uint2* d = (uint2*)x.dst;
      for (size_t w = t; w < x.bytes / 8; w += stride) d[w] = s[w];
    } else if ((a & 3) == 0) {
      const uint32_t* s = (const uint32_t*)x.src;
      uint32_t* d = (uint32_t*)x.dst;
      for (size_t w = t; w < x.bytes / 4; w += stride) d[w] = s[w];
    } else {
      const unsigned char* s = (const unsigned char*)x.src;
      unsigned char* d = (unsigned char*)x.dst;
      for (size_t w = t; w < x.bytes; w += stride) d[w] = s[w];
    }
  }
}

cudaError_t launch_xfer(const XferBatch& b, size_t max_bytes, int max_blocks, cudaStream_t st) {
  if (b.n == 0) return cudaSuccess;
  size_t units = (max_bytes + 15) / 16;
  int blocks = (int)std::min<size_t>((units + 255) / 256, (size_t)max_blocks);
  xfer_kernel<<<std::max(blocks, 1), 256, 0, st>>>(b);
  note_launch();
  return cudaGetLastError();
}

bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return cs != cudaStreamCaptureStatusNone;
}

// Mapped pinned host buffer of one host thread; `done` marks the last
// kernel that used it.
struct Mapped {
  char* p = nullptr;   // host address
  char* dp = nullptr;  // the same bytes as the device addresses them
  size_t cap = 0;
  cudaEvent_t done = nullptr;
  bool pending = false;
  ~Mapped() {
    if (pending) cudaEventSynchronize(done);
    if (p) cudaFreeHost(p);
    if (done) cudaEventDestroy(done);
    cudaGetLastError();
  }
  // waits for the buffer's last user, then grows it to `bytes` if needed
  cudaError_t take(size_t bytes) {
    cudaError_t e = cudaSuccess;
    if (!done && (e = cudaEventCreateWithFlags(&done, cudaEventDisableTiming)) != cudaSuccess) return e;
    if (pending && (e = cudaEventSynchronize(done)) != cudaSuccess) return e;
    pending = false;
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFreeHost(p);
    p = dp = nullptr;
    cap = 0;
    size_t want = std::max<size_t>(bytes, 64 << 10);
    if ((e = cudaHostAlloc((void**)&p, want, cudaHostAllocMapped | cudaHostAllocPortable)) != cudaSuccess) {
      p = nullptr;
      return e;
    }
    if ((e = cudaHostGetDevicePointer((void**)&dp, p, 0)) != cudaSuccess) {
      cudaFreeHost(p);
      p = dp = nullptr;
      return e;
    }
    cap = want;
    return cudaSuccess;
  }
  cudaError_t used_on(cudaStream_t st) {
    cudaError_t e = cudaEventRecord(done, st);
    pending = e == cudaSuccess;
    return e;
  }
};
// Reads and puts use separate buffers; puts rotate over a few so that a
// put seldom waits for the previous one's kernel.
thread_local Mapped t_read;
thread_local Mapped t_put[4];
thread_local unsigned t_put_next = 0;

size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }
}  // namespace

void HostRead::get(void* host, const void* dev, size_t bytes) {
  if (n_ < kMax) {
    host_[n_] = host;
    dev_[n_] = dev;
    bytes_[n_] = bytes;
  }
  ++n_;
}

cudaError_t HostRead::sync(cudaStream_t st) {
  int n = n_;
  n_ = 0;
  if (n > kMax) return cudaErrorInvalidValue;
  if (capturing(st)) return cudaErrorStreamCaptureUnsupported;
  size_t total = 0, most = 0;
  for (int i = 0; i < n; ++i) {
    total += align16(bytes_[i]);
    most = std::max(most, bytes_[i]);
  }
  cudaError_t e = t_read.take(total);
  if (e != cudaSuccess) return e;
  XferBatch b{};
  b.n = n;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    b.it[i] = {dev_[i], t_read.dp + off, bytes_[i]};
    off += align16(bytes_[i]);
  }
  if ((e = launch_xfer(b, most, 64, st)) != cudaSuccess) return e;
  if ((e = t_read.used_on(st)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  t_read.pending = false;
  off = 0;
  for (int i = 0; i < n; ++i) {
    memcpy(host_[i], t_read.p + off, bytes_[i]);
    off += align16(bytes_[i]);
  }
  return cudaSuccess;
}

cudaError_t host_put(void* dev, const void* host, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  if (capturing(st)) return cudaErrorStreamCaptureUnsupported;
  Mapped& m = t_put[t_put_next++ % 4];
  cudaError_t e = m.take(bytes);
  if (e != cudaSuccess) return e;
  memcpy(m.p, host, bytes);
  XferBatch b{};
  b.n = 1;
  b.it[0] = {m.dp, dev, bytes};
  if ((e = launch_xfer(b, bytes, 64, st)) != cudaSuccess) return e;
  return m.used_on(st);
}

cudaError_t dev_copy(void* dst, const void* src, size_t bytes, cudaStream_t st) {
  if (bytes == 0) return cudaSuccess;
  XferBatch b{};
  b.n = 1;
  b.it[0] = {src, dst, bytes};
  int sms = 152;
  int d = 0;
  if (cudaGetDevice(&d) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
  cudaGetLastError();
  return launch_xfer(b, bytes, 8 * sms, st);
}

cg_status fail(cg_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

cg_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? CG_ERR_OOM : CG_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

// Keeps freed memory in the device's default stream-ordered pool across
// synchronisations (the default threshold of 0 hands it back to the driver
// at every sync, and re-mapping gigabytes costs milliseconds per call).
static void keep_pool_warm() {
  static std::atomic<uint64_t> done_mask{0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  const uint64_t bit = 1ull << dev;
  if (done_mask.load() & bit) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t threshold = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold);
  }
  cudaGetLastError();
  done_mask.fetch_or(bit);
}

void* dev_alloc(size_t bytes, cudaStream_t st) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) return g_alloc(bytes, (void*)st, g_user);
  keep_pool_warm();
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}

void dev_free(void* p, cudaStream_t st) {
  if (!p) return;
  if (g_free) {
    g_free(p, (void*)st, g_user);
    return;
  }
  cudaFreeAsync(p, st);
}

cg_status check_status(cg_index* ix, cudaStream_t st) { return check_status_word(ix->status, st); }

cg_status check_status_word(uint32_t* status, cudaStream_t st) {
  uint32_t w = 0;
  HostRead rd;
  rd.get(&w, status, 4);
  cudaError_t e = rd.sync(st);
  if (e != cudaSuccess) return cuda_fail(e, "status readback");
  return status_verdict(w, status, st);
}

cg_status status_verdict(uint32_t w, uint32_t* status, cudaStream_t st) {
  if (w & (ST_NONFINITE | ST_TIMEOUT | ST_OVERFLOW | ST_INTERNAL)) {
    cudaMemsetAsync(status, 0, 4, st);
    if (w & ST_NONFINITE) return fail(CG_ERR_INVALID, "non-finite query coordinate");
    if (w & ST_TIMEOUT) return fail(CG_ERR_TIMEOUT, "a bounded device wait gave up");
    if (w & ST_OVERFLOW) return fail(CG_ERR_OVERFLOW, "an internal capacity was exceeded");
    return fail(CG_ERR_INTERNAL, "device consistency check failed");
  }
  return CG_OK;
}

}  // namespace cg

using namespace cg;

static bool finite_pos(double v) { return isfinite(v) && v > 0; }

extern "C" {

cg_status cg_set_allocator(cg_alloc_fn alloc_fn, cg_free_fn free_fn, void* user) {
  if ((alloc_fn == nullptr) != (free_fn == nullptr))
    return fail(CG_ERR_INVALID, "allocator hook needs both functions or neither");
  g_alloc = alloc_fn;
  g_free = free_fn;
  g_user = user;
  return CG_OK;
}

const char* cg_last_error(void) { return g_last_error.c_str(); }

const char* cg_version(void) { return "cheesegpu 0.1 (sm_103a)"; }

uint64_t cg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

cg_status cg_set_tuning(const cg_tuning_t* t) {
  cg_tuning_t v = default_tuning();
  if (t) {
    if (!(t->radius_chunk_height > 0.f) || !isfinite(t->radius_chunk_height))
      return fail(CG_ERR_INVALID, "radius_chunk_height must be positive and finite");
    if (t->radius_chunk_max < 1 || t->radius_chunk_max > 512)
      return fail(CG_ERR_INVALID, "radius_chunk_max must be in [1, 512]");
    if (t->count_shape < 0 || t->count_shape > 2 || t->fill_shape < 0 || t->fill_shape > 2)
      return fail(CG_ERR_INVALID, "count_shape and fill_shape must be 0, 1 or 2");
    v = *t;
  }
  set_tuning(v);
  return CG_OK;
}

cg_status cg_get_tuning(cg_tuning_t* t) {
  if (!t) return fail(CG_ERR_INVALID, "NULL argument");
  *t = current_tuning();
  return CG_OK;
}

cg_status cg_profile_enable(int on) {
  if (!on) prof_resolve();
  g_prof_on.store(on != 0);
  return CG_OK;
}

cg_status cg_profile_read(char* buf, size_t cap, size_t* len, int reset) {
  prof_resolve();
  std::string out = "{";
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    bool first = true;
    char tmp[256];
    for (auto& kv : g_prof_acc) {
      snprintf(tmp, sizeof tmp, "%s\"%s\": [%lld, %.6f]", first ? "" : ", ", kv.first.c_str(),
               (long long)kv.second.first, kv.second.second);
      out += tmp;
      first = false;
    }
    if (reset) g_prof_acc.clear();
  }
  out += "}";
  if (len) *len = out.size() + 1;
  if (!buf || cap < out.size() + 1) return buf ? fail(CG_ERR_INVALID, "profile buffer too small") : CG_OK;
  memcpy(buf, out.c_str(), out.size() + 1);
  return CG_OK;
}

cg_status cg_build(const double* xyz_dev, int64_t n, double cell_xy, double cell_z, int dim,
                   cg_flavor flavor, cg_precision precision, void* stream, cg_index_t* out) {
  if (!out) return fail(CG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!xyz_dev) return fail(CG_ERR_INVALID, "xyz_dev is NULL");
  if (n < 1 || n >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "n must be in [1, 2^31)");
  if (!finite_pos(cell_xy) || !finite_pos(cell_z)) return fail(CG_ERR_INVALID, "cell sizes must be positive and finite");
  if (dim != 2 && dim != 3) return fail(CG_ERR_INVALID, "dim must be 2 or 3");
  if (flavor < CG_DENSE || flavor > CG_MIXED) return fail(CG_ERR_INVALID, "unknown flavor");
  if (precision != CG_FP64 && precision != CG_FP32_OFFSET) return fail(CG_ERR_INVALID, "unknown precision");
  int64_t toff[2] = {0, n};
  return build_index(xyz_dev, n, toff, 1, &cell_xy, &cell_z, dim, flavor, precision,
                     (cudaStream_t)stream, out);
}

cg_status cg_build_batched(const double* xyz_dev, const int64_t* tile_offsets, int32_t T,
                           const double* cell_xy_host, int dim, cg_flavor flavor,
                           cg_precision precision, void* stream, cg_index_t* out) {
  if (!out) return fail(CG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!xyz_dev || !tile_offsets || !cell_xy_host) return fail(CG_ERR_INVALID, "NULL argument");
  if (T < 1) return fail(CG_ERR_INVALID, "T must be >= 1");
  if (dim != 2 && dim != 3) return fail(CG_ERR_INVALID, "dim must be 2 or 3");
  if (flavor < CG_DENSE || flavor > CG_MIXED) return fail(CG_ERR_INVALID, "unknown flavor");
  if (precision != CG_FP64 && precision != CG_FP32_OFFSET) return fail(CG_ERR_INVALID, "unknown precision");
  if (tile_offsets[0] != 0) return fail(CG_ERR_INVALID, "tile_offsets[0] must be 0");
  for (int t = 0; t < T; ++t) {
    if (tile_offsets[t + 1] <= tile_offsets[t]) return fail(CG_ERR_INVALID, "every tile must be non-empty");
    if (!finite_pos(cell_xy_host[t])) return fail(CG_ERR_INVALID, "cell sizes must be positive and finite");
  }
  const int64_t n = tile_offsets[T];
  if (n >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "too many points");
  return build_index(xyz_dev, n, tile_offsets, T, cell_xy_host, cell_xy_host, dim, flavor,
                     precision, (cudaStream_t)stream, out);
}

cg_status cg_index_info(cg_index_t ix, cg_index_info_t* info) {
  if (!ix || !info) return fail(CG_ERR_INVALID, "NULL argument");
  memset(info, 0, sizeof *info);
  info->n = ix->n;
  info->dim = ix->dim;
  info->flavor = ix->flavor;
  info->precision = ix->precision;
  info->ntiles = ix->ntiles;
  info->ncell = ix->ncell;
  info->nonempty = ix->nkeys;
  info->nslices = ix->nslices;
  info->dense_slices = ix->dense_slices;
  info->device_bytes = (int64_t)ix->bufs.bytes;
  const Tile& T = ix->tiles_host[0];
  for (int a = 0; a < 3; ++a) {
    info->lo[a] = T.lo[a];
    info->hi[a] = T.hi[a];
    info->nc[a] = T.n[a];
    info->cell[a] = T.s[a];
    info->origin[a] = T.origin[a];
  }
  info->enc_err = T.enc_err;
  return CG_OK;
}

cg_status cg_index_free(cg_index_t ix) {
  if (!ix) return fail(CG_ERR_INVALID, "NULL index");
  ix->ctx.release(ix->stream);
  ix->bufs.release(ix->stream);
  delete ix;
  return CG_OK;
}

cg_status cg_radius_count(cg_index_t ix, const double* q_dev, int64_t nq, double r,
                          cg_kernel kernel, int64_t* offsets_dev, int64_t* total_host,
                          void* stream) {
  if (!ix || !offsets_dev || (nq > 0 && !q_dev)) return fail(CG_ERR_INVALID, "NULL argument");
  return radius_pass(ix, false, q_dev, nq, r, kernel, false, offsets_dev, nullptr, total_host,
                     (cudaStream_t)stream);
}

cg_status cg_radius_fill(cg_index_t ix, const double* q_dev, int64_t nq, double r,
                         cg_kernel kernel, const int64_t* offsets_dev, int32_t* indices_dev,
                         void* stream) {
  if (!ix || !offsets_dev || (nq > 0 && !q_dev)) return fail(CG_ERR_INVALID, "NULL argument");
  return radius_pass(ix, false, q_dev, nq, r, kernel, true, (int64_t*)offsets_dev, indices_dev,
                     nullptr, (cudaStream_t)stream);
}

cg_status cg_radius_search_into(cg_index_t ix, const double* q_dev, int64_t nq, double r, cg_kernel kernel,
                                int64_t* offsets_dev, int32_t* indices_dev, int64_t capacity, int64_t* total_host,
                                void* stream) {
  if (!ix || !offsets_dev || !total_host || (nq > 0 && !q_dev) || (capacity > 0 && !indices_dev))
    return fail(CG_ERR_INVALID, "NULL argument");
  if (capacity < 0) return fail(CG_ERR_INVALID, "capacity must be >= 0");
  return radius_search_into(ix, ix->ctx, q_dev, nq, r, kernel, offsets_dev, indices_dev, capacity, total_host,
                            (cudaStream_t)stream);
}

cg_status cg_all_points_count(cg_index_t ix, double r, cg_kernel kernel, int64_t* offsets_dev,
                              int64_t* total_host, void* stream) {
  if (!ix || !offsets_dev) return fail(CG_ERR_INVALID, "NULL argument");
  return radius_pass(ix, true, nullptr, ix->n, r, kernel, false, offsets_dev, nullptr, total_host,
                     (cudaStream_t)stream);
}

cg_status cg_all_points_fill(cg_index_t ix, double r, cg_kernel kernel, const int64_t* offsets_dev,
                             int32_t* indices_dev, void* stream) {
  if (!ix || !offsets_dev) return fail(CG_ERR_INVALID, "NULL argument");
  return radius_pass(ix, true, nullptr, ix->n, r, kernel, true, (int64_t*)offsets_dev, indices_dev,
                     nullptr, (cudaStream_t)stream);
}

cg_status cg_radius_search(cg_index_t ix, const double* q_dev, int64_t nq, double r,
                           cg_kernel kernel, int64_t** offsets_dev, int32_t** indices_dev,
                           int64_t* total, void* stream) {
  if (!ix || !offsets_dev || !indices_dev || !total || (nq > 0 && !q_dev))
    return fail(CG_ERR_INVALID, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  *offsets_dev = nullptr;
  *indices_dev = nullptr;
  int64_t* off = (int64_t*)dev_alloc(8 * (size_t)(nq + 1), st);
  if (!off) return fail(CG_ERR_OOM, "device allocation failed (offsets)");
  int64_t tot = 0;
  cg_status s = radius_pass(ix, false, q_dev, nq, r, kernel, false, off, nullptr, &tot, st);
  if (s != CG_OK) { dev_free(off, st); return s; }
  int32_t* ind = (int32_t*)dev_alloc(4 * (size_t)std::max<int64_t>(tot, 1), st);
  if (!ind) { dev_free(off, st); return fail(CG_ERR_OOM, "device allocation failed (indices)"); }
  s = radius_pass(ix, false, q_dev, nq, r, kernel, true, off, ind, nullptr, st);
  if (s != CG_OK) { dev_free(off, st); dev_free(ind, st); return s; }
  *offsets_dev = off;
  *indices_dev = ind;
  *total = tot;
  return CG_OK;
}

cg_status cg_index_status(cg_index_t ix, void* stream) {
  if (!ix) return fail(CG_ERR_INVALID, "NULL index");
  return check_status(ix, (cudaStream_t)stream);
}

cg_status cg_free_device(void* ptr, void* stream) {
  dev_free(ptr, (cudaStream_t)stream);
  return CG_OK;
}

cg_status cg_knn(cg_index_t ix, const double* q_dev, int64_t nq, int32_t k, int32_t* idx_dev,
                 double* d2_dev, void* stream) {
  if (!ix || !idx_dev || (nq > 0 && !q_dev)) return fail(CG_ERR_INVALID, "NULL argument");
  return knn_pass(ix, false, q_dev, nq, k, idx_dev, d2_dev, (cudaStream_t)stream);
}

cg_status cg_all_points_knn(cg_index_t ix, int32_t k, int32_t* idx_dev, double* d2_dev,
                            void* stream) {
  if (!ix || !idx_dev) return fail(CG_ERR_INVALID, "NULL argument");
  return knn_pass(ix, true, nullptr, ix->n, k, idx_dev, d2_dev, (cudaStream_t)stream);
}

cg_status cg_radius_stats(cg_index_t ix, cg_radius_stats_t* out) {
  if (!ix || !out) return fail(CG_ERR_INVALID, "NULL argument");
  memset(out, 0, sizeof *out);
  const RadiusState& R = ix->ctx.radius;
  if (!R.valid || R.small || !R.ctrs) return CG_OK;  // no planned count pass on record
  unsigned long long pairs = 0;
  uint32_t big = 0;
  HostRead rd;
  rd.get(&pairs, R.ctrs + 30, 8);
  rd.get(&big, R.ctrs + 12, 4);
  cudaError_t e = rd.sync(ix->stream);
  if (e != cudaSuccess) return cuda_fail(e, "radius stats");
  out->tested_pairs = (int64_t)pairs;
  out->general_groups = big;
  out->groups = R.all_points && R.zbeg ? (int64_t)R.znb : -1;
  return CG_OK;
}

cg_status cg_knn_grow(cg_index_t ix, const double* q_dev, int64_t nq, int32_t k, int32_t policy,
                      int32_t* idx_dev, double* d2_dev, int64_t* visited_dev, void* stream) {
  if (!ix || !idx_dev || (nq > 0 && !q_dev)) return fail(CG_ERR_INVALID, "NULL argument");
  return knn_grow_pass(ix, q_dev, nq, k, policy, idx_dev, d2_dev, visited_dev, (cudaStream_t)stream);
}

}  // extern "C"
