// cg_server.cu -- the serving loop: continuous batching of query requests
// (radius search or k-NN, query sets of any size) against device-resident
// indexes.  Each of `slots` worker threads owns a CUDA stream and a query
// context; a request is admitted as soon as a slot is free and its memory
// fits the budget, so requests that arrive while others run start at once
// and their kernels overlap on the GPU.  Radius requests reserve their
// CSR output only after the count pass has measured it (total x 4 B); a
// request that cannot fit even alone fails with CG_ERR_OOM.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cg_index.h"

using namespace cg;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id = 0;
  cg_request_t req{};
  cg_index* ix = nullptr;
  Clock::time_point t_submit, t_admit, t_done;
  bool done = false;
  cg_status status = CG_OK;
  std::string error;
  int64_t total = 0;
  int64_t* offsets = nullptr;
  int32_t* indices = nullptr;
  int32_t* knn_idx = nullptr;
  double* knn_d2 = nullptr;
  int64_t held = 0;        // bytes of the budget held by the outputs
  int64_t known_need = 0;  // measured size after a preemption (re-admitted only when it fits)
  int64_t seq = 0;         // admission order
  int preemptions = 0;
  cudaStream_t st = nullptr;
};

// Conservative device bytes of a pass's internal work for nq queries
// (plan, sort scratch, counters, masks); corrected by the actual figure
// once the count pass has run.
int64_t work_estimate(int64_t nq) { return 160 * nq + (4 << 20); }

int64_t first_reservation(const Request* R) {
  const cg_request_t& q = R->req;
  const int64_t f = work_estimate(q.nq) + (q.op == CG_REQ_RADIUS ? 8 * (q.nq + 1) : 12 * q.nq * (int64_t)q.k);
  return std::max(f, R->known_need);
}

enum class Acq { OK, NEVER, PREEMPT };

}  // namespace

struct cg_server {
  std::vector<cg_index*> indexes;
  int dev = 0;
  int64_t budget = 0;
  int64_t in_use = 0, peak_in_use = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_mem, cv_done;
  std::deque<Request*> queue;
  std::deque<int64_t> completed;  // finished requests not yet handed out by cg_server_wait_any
  std::unordered_map<int64_t, Request*> reqs;
  std::vector<std::thread> workers;
  bool stopping = false;
  int64_t next_id = 1;
  int in_flight = 0, max_in_flight = 0;
  int64_t next_seq = 1, preemptions = 0;
  std::vector<int64_t> mem_waiters;  // admission seqs of requests waiting for output memory
  // statistics of completed requests
  std::vector<double> latencies_ms;
  int64_t queries_done = 0, requests_done = 0, requests_failed = 0;
  Clock::time_point t_first_submit, t_last_done;
  bool any_submit = false;

  // Blocks until `bytes` more fit the budget.  NEVER: the request could not
  // fit even alone.  PREEMPT: every request on the GPU is waiting for memory
  // (none can finish and free any), so the last admitted one steps back.
  Acq acquire(std::unique_lock<std::mutex>& lk, int64_t bytes, int64_t already_held, int64_t seq) {
    if (bytes + already_held > budget) return Acq::NEVER;
    mem_waiters.push_back(seq);
    cv_mem.notify_all();  // the other waiters re-check the deadlock condition
    Acq res = Acq::OK;
    cv_mem.wait(lk, [&] {
      if (stopping) { res = Acq::NEVER; return true; }
      if (in_use + bytes <= budget) { res = Acq::OK; return true; }
      if ((int)mem_waiters.size() == in_flight &&
          seq == *std::max_element(mem_waiters.begin(), mem_waiters.end())) {
        res = Acq::PREEMPT;
        return true;
      }
      return false;
    });
    mem_waiters.erase(std::find(mem_waiters.begin(), mem_waiters.end(), seq));
    if (res == Acq::OK) {
      in_use += bytes;
      peak_in_use = std::max(peak_in_use, in_use);
    }
    return res;
  }
  void give_back(int64_t bytes) {
    in_use -= bytes;
    cv_mem.notify_all();
    cv_work.notify_all();
  }

  // true when the request finished (successfully or not); false when it was
  // preempted and put back at the head of the queue
  bool run_request(Request* R, QueryCtx& C, cudaStream_t st, std::unique_lock<std::mutex>& lk, int64_t reserved);
  void worker(int slot);
};

bool cg_server::run_request(Request* R, QueryCtx& C, cudaStream_t st, std::unique_lock<std::mutex>& lk,
                            int64_t reserved) {
  const cg_request_t& q = R->req;
  cg_index* ix = R->ix;
  const int64_t nq = q.nq;
  lk.unlock();
  DevBufs out;
  cg_status s = CG_OK;
  if (q.op == CG_REQ_RADIUS) {
    R->offsets = (int64_t*)out.get(8 * (size_t)(nq + 1), st);
    if (!R->offsets) s = fail(CG_ERR_OOM, "device allocation failed (request offsets)");
    int64_t total = 0;
    if (s == CG_OK)
      s = radius_pass(ix, C, false, q.q_dev, nq, q.radius, q.kernel, false, R->offsets, nullptr, &total, st);
    if (s == CG_OK) {
      // the measured output, and the measured work in place of the estimate
      const int64_t work = (int64_t)(C.plan.bufs.bytes + C.radius.bufs.bytes);
      const int64_t need = 4 * std::max<int64_t>(total, 1) + 8 * (nq + 1) + work;
      lk.lock();
      if (need > reserved) {
        const Acq a = acquire(lk, need - reserved, reserved, R->seq);
        if (a == Acq::NEVER) {
          s = fail(CG_ERR_OOM, "request needs more device memory than the budget");
        } else if (a == Acq::PREEMPT) {
          // step back: free everything, wait at the head of the queue until
          // the measured size fits
          lk.unlock();
          C.release(st);
          out.release(st);
          cudaStreamSynchronize(st);
          R->offsets = nullptr;
          lk.lock();
          give_back(reserved);
          R->known_need = need;
          R->preemptions++;
          preemptions++;
          queue.push_front(R);
          cv_work.notify_all();
          return false;
        } else {
          reserved = need;
        }
      }
      lk.unlock();
      if (s == CG_OK) {
        R->total = total;
        R->indices = (int32_t*)out.get(4 * (size_t)std::max<int64_t>(total, 1), st);
        if (!R->indices) s = fail(CG_ERR_OOM, "device allocation failed (request indices)");
      }
      if (s == CG_OK)
        s = radius_pass(ix, C, false, q.q_dev, nq, q.radius, q.kernel, true, R->offsets, R->indices, nullptr, st);
      if (s == CG_OK) s = check_status_word(C.status, st);
    }
  } else {
    R->knn_idx = (int32_t*)out.get(4 * (size_t)std::max<int64_t>(nq * q.k, 1), st);
    R->knn_d2 = (double*)out.get(8 * (size_t)std::max<int64_t>(nq * q.k, 1), st);
    if (!R->knn_idx || !R->knn_d2) s = fail(CG_ERR_OOM, "device allocation failed (request k-NN output)");
    if (s == CG_OK) s = knn_pass(ix, C, false, q.q_dev, nq, q.k, R->knn_idx, R->knn_d2, st);
    if (s == CG_OK) s = check_status_word(C.status, st);
  }
  if (s == CG_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "request");
  }
  std::string msg = s == CG_OK ? std::string() : std::string(cg_last_error());
  C.release(st);  // the pass's work buffers; outputs stay with the request
  if (s != CG_OK) {
    out.release(st);
    cudaStreamSynchronize(st);
    R->offsets = nullptr;
    R->indices = nullptr;
    R->knn_idx = nullptr;
    R->knn_d2 = nullptr;
  }
  lk.lock();
  const int64_t keep = s == CG_OK ? (int64_t)out.bytes : 0;
  R->held = keep;
  if (reserved > keep) give_back(reserved - keep);
  else if (keep > reserved) in_use += keep - reserved;  // rounding of small buffers
  out.ptrs.clear();  // ownership moves to the request (freed by cg_server_release)
  R->status = s;
  R->error = msg;
  return true;
}

void cg_server::worker(int slot) {
  cudaSetDevice(dev);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  QueryCtx C;
  DevBufs statbuf;
  C.status = (uint32_t*)statbuf.get(64 * 4, st);
  if (C.status) cudaMemsetAsync(C.status, 0, 64 * 4, st);
  cudaStreamSynchronize(st);
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    // admission: the oldest request whose first reservation fits
    Request* R = nullptr;
    cv_work.wait(lk, [&] {
      if (stopping) return true;
      if (queue.empty()) return false;
      const int64_t first = first_reservation(queue.front());
      return first > budget || in_use + first <= budget;
    });
    if (stopping) break;
    R = queue.front();
    queue.pop_front();
    const int64_t first = first_reservation(R);
    R->t_admit = Clock::now();
    R->st = st;
    R->seq = next_seq++;
    if (!C.status) {
      R->status = CG_ERR_OOM;
      R->error = "device allocation failed (slot status)";
    } else if (first > budget) {
      R->status = CG_ERR_OOM;
      R->error = "request needs more device memory than the budget";
    } else {
      in_use += first;
      peak_in_use = std::max(peak_in_use, in_use);
      in_flight++;
      max_in_flight = std::max(max_in_flight, in_flight);
      cv_work.notify_all();  // the next request may fit beside this one
      const bool finished = run_request(R, C, st, lk, first);
      in_flight--;
      cv_mem.notify_all();  // fewer requests on the GPU: re-check waiters
      if (!finished) continue;
    }
    R->t_done = Clock::now();
    R->done = true;
    t_last_done = R->t_done;
    if (R->status == CG_OK) {
      requests_done++;
      queries_done += R->req.nq;
      latencies_ms.push_back(std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count());
    } else {
      requests_failed++;
    }
    completed.push_back(R->id);
    cv_done.notify_all();
    cv_work.notify_all();
  }
  lk.unlock();
  C.release(st);
  statbuf.release(st);
  cudaStreamSynchronize(st);
  cudaStreamDestroy(st);
}

extern "C" {

cg_status cg_server_create(const cg_index_t* indexes, int32_t n_indexes, const cg_server_opts_t* opts,
                           cg_server_t* out) {
  if (!out) return fail(CG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!indexes || n_indexes < 1 || !opts) return fail(CG_ERR_INVALID, "need at least one index and options");
  if (opts->slots < 1 || opts->slots > 64) return fail(CG_ERR_INVALID, "slots must be in [1, 64]");
  if (opts->memory_budget < 0) return fail(CG_ERR_INVALID, "memory_budget must be >= 0");
  for (int i = 0; i < n_indexes; ++i)
    if (!indexes[i]) return fail(CG_ERR_INVALID, "NULL index");
  cg_server* s = new cg_server();
  s->indexes.assign(indexes, indexes + n_indexes);
  cudaGetDevice(&s->dev);
  s->budget = opts->memory_budget;
  if (s->budget == 0) {
    size_t fr = 0, tot = 0;
    cudaError_t e = cudaMemGetInfo(&fr, &tot);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "memory info");
    }
    s->budget = (int64_t)(fr / 2);
  }
  for (int i = 0; i < opts->slots; ++i) s->workers.emplace_back([s, i] { s->worker(i); });
  *out = s;
  return CG_OK;
}

cg_status cg_server_submit(cg_server_t s, const cg_request_t* req, int64_t* id_out) {
  if (!s || !req || !id_out) return fail(CG_ERR_INVALID, "NULL argument");
  if (req->index < 0 || req->index >= (int32_t)s->indexes.size()) return fail(CG_ERR_INVALID, "no such index");
  if (req->nq < 0 || req->nq >= (int64_t)0x7fffffff || (req->nq > 0 && !req->q_dev))
    return fail(CG_ERR_INVALID, "bad query set");
  cg_index* ix = s->indexes[req->index];
  if (ix->ntiles != 1) return fail(CG_ERR_UNIMPLEMENTED, "external queries on a batched index");
  if (req->op == CG_REQ_RADIUS) {
    if (!(req->radius > 0) || !isfinite(req->radius)) return fail(CG_ERR_INVALID, "radius must be positive and finite");
    if (req->kernel != CG_SPHERE && req->kernel != CG_CUBE && req->kernel != CG_CYLINDER) return fail(CG_ERR_INVALID, "unknown kernel");
  } else if (req->op == CG_REQ_KNN) {
    if (req->k < 1 || req->k > 64) return fail(CG_ERR_INVALID, "k must be in [1, 64]");
  } else {
    return fail(CG_ERR_INVALID, "unknown request op");
  }
  Request* R = new Request();
  R->req = *req;
  R->ix = ix;
  R->t_submit = Clock::now();
  std::lock_guard<std::mutex> g(s->mu);
  if (s->stopping) {
    delete R;
    return fail(CG_ERR_INVALID, "server is shutting down");
  }
  R->id = s->next_id++;
  if (!s->any_submit) {
    s->t_first_submit = R->t_submit;
    s->any_submit = true;
  }
  s->reqs[R->id] = R;
  s->queue.push_back(R);
  s->cv_work.notify_one();
  *id_out = R->id;
  return CG_OK;
}

cg_status cg_server_wait(cg_server_t s, int64_t id, double timeout_s, cg_result_t* res) {
  if (!s || !res) return fail(CG_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return fail(CG_ERR_INVALID, "unknown request id");
  Request* R = it->second;
  auto ready = [&] { return R->done; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return fail(CG_ERR_TIMEOUT, "request not finished yet");
  }
  memset(res, 0, sizeof *res);
  res->status = R->status;
  res->nq = R->req.nq;
  res->total = R->total;
  res->offsets = R->offsets;
  res->indices = R->indices;
  res->knn_idx = R->knn_idx;
  res->knn_d2 = R->knn_d2;
  res->queue_ms = std::chrono::duration<double, std::milli>(R->t_admit - R->t_submit).count();
  res->latency_ms = std::chrono::duration<double, std::milli>(R->t_done - R->t_submit).count();
  if (R->status != CG_OK) return fail(R->status, R->error);
  return CG_OK;
}

cg_status cg_server_wait_any(cg_server_t s, double timeout_s, int64_t* id) {
  if (!s || !id) return fail(CG_ERR_INVALID, "NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] {
    // skip requests that were released meanwhile
    while (!s->completed.empty() && !s->reqs.count(s->completed.front())) s->completed.pop_front();
    return !s->completed.empty();
  };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, ready);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) {
    return fail(CG_ERR_TIMEOUT, "no request finished in time");
  }
  *id = s->completed.front();
  s->completed.pop_front();
  return CG_OK;
}

cg_status cg_server_release(cg_server_t s, int64_t id) {
  if (!s) return fail(CG_ERR_INVALID, "NULL server");
  Request* R = nullptr;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return fail(CG_ERR_INVALID, "unknown request id");
    if (!it->second->done) return fail(CG_ERR_INVALID, "request still running");
    R = it->second;
    s->reqs.erase(it);
  }
  // outputs were allocated on the slot's stream, which has finished with them
  for (void* p : {(void*)R->offsets, (void*)R->indices, (void*)R->knn_idx, (void*)R->knn_d2})
    if (p) dev_free(p, R->st);
  if (R->st) cudaStreamSynchronize(R->st);
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->give_back(R->held);
  }
  delete R;
  return CG_OK;
}

cg_status cg_server_stats(cg_server_t s, cg_server_stats_t* out) {
  if (!s || !out) return fail(CG_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> g(s->mu);
  memset(out, 0, sizeof *out);
  out->requests_done = s->requests_done;
  out->requests_failed = s->requests_failed;
  out->queries_done = s->queries_done;
  out->queued = (int64_t)s->queue.size();
  out->in_flight = s->in_flight;
  out->max_in_flight = s->max_in_flight;
  out->memory_budget = s->budget;
  out->memory_in_use = s->in_use;
  out->memory_peak = s->peak_in_use;
  out->preemptions = s->preemptions;
  std::vector<double> l = s->latencies_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    // nearest-rank percentiles
    auto pct = [&](double p) { size_t r = (size_t)ceil(p * l.size()); return l[std::max<size_t>(r, 1) - 1]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = l.back();
  }
  if (s->any_submit && s->requests_done > 0) {
    const double span = std::chrono::duration<double>(s->t_last_done - s->t_first_submit).count();
    out->queries_per_s = span > 0 ? (double)s->queries_done / span : 0.0;
  }
  return CG_OK;
}

cg_status cg_server_free(cg_server_t s) {
  if (!s) return fail(CG_ERR_INVALID, "NULL server");
  {
    // requests still queued are dropped; those on the GPU finish (one that
    // waits for memory fails), then the workers stop
    std::lock_guard<std::mutex> g(s->mu);
    s->stopping = true;
    s->cv_work.notify_all();
    s->cv_mem.notify_all();
  }
  for (auto& t : s->workers) t.join();
  for (auto& kv : s->reqs) {
    Request* R = kv.second;
    for (void* p : {(void*)R->offsets, (void*)R->indices, (void*)R->knn_idx, (void*)R->knn_d2})
      if (p) dev_free(p, nullptr);
    delete R;
  }
  cudaDeviceSynchronize();
  delete s;
  return CG_OK;
}

}  // extern "C"
