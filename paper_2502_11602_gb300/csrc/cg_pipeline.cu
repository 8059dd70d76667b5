// cg_pipeline.cu -- the captured batched pipeline: build (bbox, keys, radix
// sort, gather, runs, cell table) + all-points radius search (plan, count,
// scan, fill, row order) + all-points k-NN over every tile of a batch,
// recorded once as a CUDA graph and replayed on new coordinates of the same
// tile layout.  Data-dependent sizes are checked on the device; data that
// outgrows the plan sets ST_REPLAN, the rest of the replay is skipped and
// the next synchronising run re-plans.
#include <math.h>
#include <string.h>

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
}  // namespace cg

using namespace cg;

struct cg_pipeline {
  // what the plan is made for
  const double* xyz = nullptr;
  std::vector<int64_t> toff;
  std::vector<double> cell;
  int dim = 2, precision = CG_FP32_OFFSET;
  double r = 1.0, headroom = 1.25;
  int kernel = CG_SPHERE, k = 0;
  cudaStream_t create_st = nullptr, last_st = nullptr;
  // the plan
  cg_index* ix = nullptr;
  BuildWork bw;
  RadiusWork rw;
  KnnWork kw;
  DevBufs outs;
  int64_t* offsets = nullptr;
  int32_t* indices = nullptr;
  int32_t* knn_idx = nullptr;
  double* knn_d2 = nullptr;
  cudaStream_t cap_st = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_kernels = 0, graph_nodes = 0;
  int64_t replans = 0;
};

namespace {

void teardown(cg_pipeline* p, cudaStream_t st) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  p->exec = nullptr;
  p->graph = nullptr;
  p->bw.bufs.release(st);
  p->rw.bufs.release(st);
  p->kw.bufs.release(st);
  p->outs.release(st);
  p->bw = BuildWork();
  p->rw = RadiusWork();
  p->kw = KnnWork();
  p->offsets = nullptr;
  p->indices = nullptr;
  p->knn_idx = nullptr;
  p->knn_d2 = nullptr;
  if (p->ix) {
    p->ix->ctx.release(st);
    p->ix->bufs.release(st);
    delete p->ix;
    p->ix = nullptr;
  }
}

// Everything the replay needs, sized from one eager build and count on the
// current coordinates, then the graph capture.
cg_status setup(cg_pipeline* p, cudaStream_t st) {
  const int T = (int)p->toff.size() - 1;
  const int64_t n = p->toff[T];
  cg_status s = build_index(p->xyz, n, p->toff.data(), T, p->cell.data(), p->cell.data(), p->dim, CG_DENSE,
                            p->precision, st, &p->ix);
  if (s != CG_OK) return s;
  cg_index* ix = p->ix;
  p->offsets = (int64_t*)p->outs.get(8 * (size_t)(n + 1), st);
  if (!p->offsets) return fail(CG_ERR_OOM, "device allocation failed (pipeline offsets)");
  int64_t total = 0;
  s = radius_pass(ix, true, nullptr, 0, p->r, p->kernel, false, p->offsets, nullptr, &total, st);
  if (s != CG_OK) return s;
  s = build_work_alloc(ix, p->bw, st);
  if (s == CG_OK) s = radius_work_alloc(ix, p->rw, p->bw.cap_keys, p->headroom, total, st);
  if (s == CG_OK && p->k > 0) s = knn_work_alloc(ix, p->kw, st);
  if (s != CG_OK) return s;
  ix->ctx.release(st);
  // the caller's buffer stays valid for the pipeline's lifetime: the exact
  // binary64 rechecks read it in place instead of a copy
  ix->xyz64 = const_cast<double*>(p->xyz);
  p->indices = (int32_t*)p->outs.get(4 * (size_t)p->rw.cap_out, st);
  if (p->k > 0) {
    p->knn_idx = (int32_t*)p->outs.get(4 * (size_t)n * p->k, st);
    p->knn_d2 = (double*)p->outs.get(8 * (size_t)n * p->k, st);
  }
  if (!p->indices || (p->k > 0 && (!p->knn_idx || !p->knn_d2)))
    return fail(CG_ERR_OOM, "device allocation failed (pipeline outputs)");
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline setup");

  // capture: the counter of host launches must not count the recording
  const uint64_t before = cg_launch_count();
  e = cudaStreamBeginCapture(p->cap_st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin capture");
  s = build_replay(ix, p->bw, p->xyz, p->cap_st);
  if (s == CG_OK) s = radius_replay(ix, p->rw, p->bw.nkeys_dev, p->r, p->kernel, p->offsets, p->indices, p->cap_st);
  if (s == CG_OK && p->k > 0)
    s = knn_replay(ix, p->kw, p->bw.nkeys_dev, p->bw.cap_keys, p->k, p->knn_idx, p->knn_d2, p->cap_st);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(p->cap_st, &g);
  note_launch(-(int)(cg_launch_count() - before));
  if (s != CG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  p->graph = g;
  e = cudaGraphInstantiate(&p->exec, g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
  int kern = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kern;
  }
  p->graph_nodes = (int)nn;
  p->graph_kernels = kern;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pipeline capture");
  return CG_OK;
}

cg_status launch(cg_pipeline* p, cudaStream_t st) {
  cudaError_t e = cudaGraphLaunch(p->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "graph launch");
  note_launch(p->graph_kernels);
  p->last_st = st;
  return CG_OK;
}

// Synchronises, reads and clears the status word; with `total`, also reads
// the CSR total of the run in the same transfer.
cg_status read_status(cg_pipeline* p, cudaStream_t st, uint32_t* word, int64_t* total = nullptr) {
  HostRead rd;
  rd.get(word, p->ix->status, 4);
  if (total) rd.get(total, p->offsets + p->toff.back(), 8);
  cudaError_t e = rd.sync(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->ix->status, 0, 4, st);
  if (e != cudaSuccess) return cuda_fail(e, "pipeline status");
  return CG_OK;
}

cg_status status_error(uint32_t w) {
  if (w & ST_NONFINITE) return fail(CG_ERR_INVALID, "non-finite point coordinate");
  if (w & ST_TIMEOUT) return fail(CG_ERR_TIMEOUT, "a bounded device wait gave up");
  if (w & ST_OVERFLOW) return fail(CG_ERR_OVERFLOW, "an internal capacity was exceeded");
  if (w & ST_INTERNAL) return fail(CG_ERR_INTERNAL, "device consistency check failed");
  return CG_OK;
}

}  // namespace

extern "C" {

cg_status cg_pipeline_create(const double* xyz_dev, const int64_t* tile_offsets, int32_t T, const double* cell_host,
                             int dim, cg_precision precision, const cg_pipeline_opts_t* opts, void* stream,
                             cg_pipeline_t* out) {
  if (!out) return fail(CG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!xyz_dev || !tile_offsets || !cell_host || !opts) return fail(CG_ERR_INVALID, "NULL argument");
  if (T < 1) return fail(CG_ERR_INVALID, "T must be >= 1");
  if (dim != 2 && dim != 3) return fail(CG_ERR_INVALID, "dim must be 2 or 3");
  if (precision != CG_FP64 && precision != CG_FP32_OFFSET) return fail(CG_ERR_INVALID, "unknown precision");
  if (!(opts->radius > 0) || !isfinite(opts->radius)) return fail(CG_ERR_INVALID, "radius must be positive and finite");
  if (opts->kernel != CG_SPHERE && opts->kernel != CG_CUBE && opts->kernel != CG_CYLINDER) return fail(CG_ERR_INVALID, "unknown kernel");
  if (opts->k < 0 || opts->k > 64) return fail(CG_ERR_INVALID, "k must be in [0, 64]");
  if (!(opts->headroom == 0 || (opts->headroom >= 1 && opts->headroom <= 16)))
    return fail(CG_ERR_INVALID, "headroom must be 0 or in [1, 16]");
  if (tile_offsets[0] != 0) return fail(CG_ERR_INVALID, "tile_offsets[0] must be 0");
  for (int t = 0; t < T; ++t) {
    if (tile_offsets[t + 1] <= tile_offsets[t]) return fail(CG_ERR_INVALID, "every tile must be non-empty");
    if (!(cell_host[t] > 0) || !isfinite(cell_host[t])) return fail(CG_ERR_INVALID, "cell sizes must be positive and finite");
  }
  if (tile_offsets[T] >= (int64_t)0x7fffffff) return fail(CG_ERR_INVALID, "too many points");
  cg_pipeline* p = new cg_pipeline();
  p->xyz = xyz_dev;
  p->toff.assign(tile_offsets, tile_offsets + T + 1);
  p->cell.assign(cell_host, cell_host + T);
  p->dim = dim;
  p->precision = precision;
  p->r = opts->radius;
  p->kernel = opts->kernel;
  p->k = opts->k;
  p->headroom = opts->headroom == 0 ? 1.25 : opts->headroom;
  p->create_st = (cudaStream_t)stream;
  p->last_st = p->create_st;
  cudaError_t e = cudaStreamCreateWithFlags(&p->cap_st, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete p;
    return cuda_fail(e, "capture stream");
  }
  cg_status s = setup(p, p->create_st);
  if (s != CG_OK) {
    std::string msg = cg_last_error();
    cudaStreamSynchronize(p->create_st);
    teardown(p, p->create_st);
    cudaStreamDestroy(p->cap_st);
    delete p;
    return fail(s, msg);
  }
  *out = p;
  return CG_OK;
}

cg_status cg_pipeline_run(cg_pipeline_t p, void* stream, int64_t* total_host) {
  if (!p) return fail(CG_ERR_INVALID, "NULL pipeline");
  cudaStream_t st = (cudaStream_t)stream;
  cg_status s = launch(p, st);
  if (s != CG_OK || !total_host) return s;
  uint32_t w = 0;
  s = read_status(p, st, &w, total_host);
  if (s != CG_OK) return s;
  if (w & ST_REPLAN) {
    // new data outgrew the plan: plan again from the current coordinates
    teardown(p, st);
    p->replans++;
    s = setup(p, st);
    if (s != CG_OK) return s;
    s = launch(p, st);
    if (s == CG_OK) s = read_status(p, st, &w, total_host);
    if (s != CG_OK) return s;
    if (w & ST_REPLAN) return fail(CG_ERR_INTERNAL, "pipeline re-plan did not fit its own data");
  }
  return status_error(w);
}

cg_status cg_pipeline_outputs(cg_pipeline_t p, int64_t** offsets, int32_t** indices, int32_t** knn_idx,
                              double** knn_d2) {
  if (!p) return fail(CG_ERR_INVALID, "NULL pipeline");
  if (offsets) *offsets = p->offsets;
  if (indices) *indices = p->indices;
  if (knn_idx) *knn_idx = p->knn_idx;
  if (knn_d2) *knn_d2 = p->knn_d2;
  return CG_OK;
}

cg_status cg_pipeline_info(cg_pipeline_t p, cg_pipeline_info_t* info) {
  if (!p || !info) return fail(CG_ERR_INVALID, "NULL argument");
  memset(info, 0, sizeof *info);
  info->n = p->toff.back();
  info->ntiles = (int32_t)p->toff.size() - 1;
  info->k = p->k;
  info->graph_kernels = p->graph_kernels;
  info->graph_nodes = p->graph_nodes;
  info->replans = p->replans;
  info->capacity_indices = p->rw.cap_out;
  info->capacity_voxels = p->bw.cap_keys;
  info->ncell = p->ix ? p->ix->ncell : 0;
  info->device_bytes = (int64_t)(p->bw.bufs.bytes + p->rw.bufs.bytes + p->kw.bufs.bytes + p->outs.bytes +
                                 (p->ix ? p->ix->bufs.bytes : 0));
  return CG_OK;
}

cg_status cg_pipeline_free(cg_pipeline_t p) {
  if (!p) return fail(CG_ERR_INVALID, "NULL pipeline");
  cudaStreamSynchronize(p->last_st);
  teardown(p, p->create_st);
  cudaStreamSynchronize(p->create_st);
  cudaStreamDestroy(p->cap_st);
  delete p;
  return CG_OK;
}

}  // extern "C"
