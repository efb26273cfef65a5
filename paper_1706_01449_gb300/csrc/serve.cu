// Serving runtime: a request queue over one index with continuous batching
// (mips_server_* in include/mips.h).  Host code only.  Sec. II-B notes that
// the index also serves a subset of users at a time, as in a model-serving
// system that collects requests; each batch here is such a subset and gets
// the same exact top-K as the batch problem.
//
// Threads: the caller's (submit / wait), a scheduler that forms batches and
// launches them on free stream slots, and a completion thread that polls the
// slots' events and hands results back.  One mutex guards the queue, the
// slots' busy flags and the requests' states.
#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

using namespace mips;

namespace {

struct Request {
  int64_t id = 0;
  const float* users = nullptr;
  int64_t n = 0;
  int K = 0;
  int32_t* out_idx = nullptr;
  double* out_score = nullptr;
  double t_submit = 0, t_start = 0, t_done = 0;
  int64_t batch = -1, batch_users = 0;
  int batch_K = 0, slot = -1;
  size_t batch_bytes = 0, batch_ws = 0, inflight = 0;
  bool done = false;
  mips_status status = MIPS_OK;
  std::string error;
};
using RequestP = std::shared_ptr<Request>;

struct Slot {
  mips_index_t worker = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  // pinned staging and device buffers, grown on demand
  float* h_users = nullptr;
  int32_t* h_idx = nullptr;
  double* h_score = nullptr;
  float* d_users = nullptr;
  int32_t* d_idx = nullptr;
  double* d_score = nullptr;
  int64_t cap_users = 0, cap_out = 0;    // pinned host capacity: rows x f floats, rows x K outputs
  int64_t dcap_users = 0, dcap_out = 0;  // device capacity (freed under a memory budget)
  // the batch in flight
  bool busy = false, launched = false;
  std::vector<RequestP> reqs;
  int64_t batch = -1, n = 0;
  int K = 0;
  size_t bytes = 0;     // admitted: the call's workspace plus this batch's user and result buffers
  size_t ws_used = 0;   // workspace the call took
  size_t inflight = 0;  // admitted bytes of all batches in flight when this one started
  mips_status status = MIPS_OK;
  std::string error;
};

int k_class(int K) { return K == 1 ? 0 : (K <= 10 ? 1 : (K <= 32 ? 2 : 3)); }

// status + message for mips_last_error() of the calling thread
mips_status fail(mips_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error_message(buf);
  return st;
}

mips_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  return fail(e == cudaErrorMemoryAllocation ? MIPS_ERR_NOMEM : MIPS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

}  // namespace

struct mips_server_s {
  mips_index_t idx = nullptr;
  mips_server_options opt{};
  int device = 0;
  int f = 0;
  int64_t n_items = 0;
  std::mutex mu;
  std::condition_variable cv_sched, cv_compl, cv_done;
  std::deque<RequestP> pending;
  std::unordered_map<int64_t, RequestP> requests;
  std::vector<Slot> slots;
  int64_t next_id = 0, next_batch = 0;
  size_t inflight_bytes = 0;
  bool stop = false, sched_exited = false;
  std::thread sched, compl_;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
  // Device bytes a batch of n users at this K holds while in flight: the
  // workspace its call lays out (computed by the call's own layout code on
  // the idle worker that will run it) plus its user rows and results.
  size_t batch_bytes(mips_index_t worker, int64_t n, int K) const {
    return call_workspace_bytes(worker, n, K, opt.method) + (size_t)n * (size_t)f * 4 + (size_t)n * K * 12;
  }
  // Device bytes the slots hold now (workspaces and batch buffers).
  size_t held_bytes() const {
    size_t b = 0;
    for (const Slot& sl : slots)
      b += index_workspace_held(sl.worker) + (size_t)sl.dcap_users * f * 4 + (size_t)sl.dcap_out * 12;
    return b;
  }
  bool free_slot(int* which) const {
    for (size_t i = 0; i < slots.size(); ++i)
      if (!slots[i].busy) {
        *which = (int)i;
        return true;
      }
    return false;
  }
  void scheduler();
  void completer();
  mips_status launch(Slot& sl);
};

namespace {

// grow a pinned host / device buffer (the slot is idle while this runs)
template <typename T>
cudaError_t grow_host(T*& p, size_t count) {
  if (p) cudaFreeHost(p);
  p = nullptr;
  return cudaMallocHost((void**)&p, sizeof(T) * (count > 0 ? count : 1));
}
template <typename T>
cudaError_t grow_dev(T*& p, size_t count, cudaStream_t s) {  // stream-ordered: no device-wide sync
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
  return cudaMallocAsync((void**)&p, sizeof(T) * (count > 0 ? count : 1), s);
}

}  // namespace

mips_status mips_server_s::launch(Slot& sl) {
  cudaError_t e = cudaSuccess;
  if (sl.n > sl.cap_users) {
    if ((e = grow_host(sl.h_users, (size_t)sl.n * f)) != cudaSuccess) return cuda_fail(e, "server staging allocation");
    sl.cap_users = sl.n;
  }
  if (sl.n > sl.dcap_users) {
    if ((e = grow_dev(sl.d_users, (size_t)sl.n * f, sl.stream)) != cudaSuccess)
      return cuda_fail(e, "server staging allocation");
    sl.dcap_users = sl.n;
  }
  const int64_t outs = sl.n * sl.K;
  if (outs > sl.cap_out) {
    if ((e = grow_host(sl.h_idx, outs)) != cudaSuccess || (e = grow_host(sl.h_score, outs)) != cudaSuccess)
      return cuda_fail(e, "server output allocation");
    sl.cap_out = outs;
  }
  if (outs > sl.dcap_out) {
    if ((e = grow_dev(sl.d_idx, outs, sl.stream)) != cudaSuccess ||
        (e = grow_dev(sl.d_score, outs, sl.stream)) != cudaSuccess)
      return cuda_fail(e, "server output allocation");
    sl.dcap_out = outs;
  }
  int64_t row = 0;
  for (const RequestP& r : sl.reqs) {
    memcpy(sl.h_users + row * f, r->users, sizeof(float) * r->n * f);
    row += r->n;
  }
  if ((e = cudaMemcpyAsync(sl.d_users, sl.h_users, sizeof(float) * sl.n * f, cudaMemcpyHostToDevice, sl.stream)) !=
      cudaSuccess)
    return cuda_fail(e, "server users copy");
  mips_status st = opt.method == 0
                       ? mips_topk(sl.worker, sl.d_users, sl.n, sl.K, sl.d_idx, sl.d_score, sl.stream)
                       : mips_topk_maximus(sl.worker, sl.d_users, sl.n, sl.K, sl.d_idx, sl.d_score, sl.stream);
  if (st != MIPS_OK) return st;
  sl.ws_used = index_workspace_used(sl.worker);
  if ((e = cudaMemcpyAsync(sl.h_idx, sl.d_idx, sizeof(int32_t) * outs, cudaMemcpyDeviceToHost, sl.stream)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(sl.h_score, sl.d_score, sizeof(double) * outs, cudaMemcpyDeviceToHost, sl.stream)) !=
          cudaSuccess ||
      (e = cudaEventRecord(sl.done, sl.stream)) != cudaSuccess)
    return cuda_fail(e, "server results copy");
  return MIPS_OK;
}

void mips_server_s::scheduler() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    int which = -1;
    cv_sched.wait(lk, [&] { return (stop && pending.empty()) || (!pending.empty() && free_slot(&which)); });
    if (pending.empty()) break;  // stopping, nothing left
    // the batch: the oldest request, then later ones of the same K class
    // while the users fit
    const RequestP head = pending.front();
    const int cls = k_class(head->K);
    std::vector<RequestP> take{head};
    int64_t n = head->n;
    int K = head->K;
    for (size_t i = 1; i < pending.size(); ++i) {
      const RequestP& r = pending[i];
      if (k_class(r->K) != cls || n + r->n > opt.max_batch_users) continue;
      take.push_back(r);
      n += r->n;
      K = std::max(K, r->K);
    }
    const size_t bytes = batch_bytes(slots[which].worker, n, K);
    if (opt.mem_budget > 0 && inflight_bytes > 0 && inflight_bytes + bytes > (size_t)opt.mem_budget) {
      // admission by memory: wait for a batch in flight to finish
      cv_sched.wait(lk, [&] { return stop || inflight_bytes + bytes <= (size_t)opt.mem_budget || inflight_bytes == 0; });
      continue;  // re-form the batch (the queue may have changed)
    }
    for (const RequestP& r : take) pending.erase(std::find(pending.begin(), pending.end(), r));
    Slot& sl = slots[which];
    sl.busy = true;
    sl.launched = false;
    sl.reqs = take;
    sl.n = n;
    sl.K = K;
    sl.bytes = bytes;
    sl.batch = next_batch++;
    inflight_bytes += bytes;
    sl.inflight = inflight_bytes;
    const double t = now();
    for (const RequestP& r : take) r->t_start = t;
    lk.unlock();
    const mips_status st = launch(sl);
    lk.lock();
    sl.status = st;
    sl.error = st == MIPS_OK ? std::string() : std::string(mips_last_error());
    sl.launched = true;
    cv_compl.notify_all();
  }
  sched_exited = true;
  cv_compl.notify_all();
}

void mips_server_s::completer() {
  cudaSetDevice(device);
  std::unique_lock<std::mutex> lk(mu);
  while (true) {
    bool any_busy = false;
    for (const Slot& sl : slots) any_busy |= sl.busy;
    if (!any_busy && sched_exited) break;
    if (!any_busy) {
      cv_compl.wait(lk);
      continue;
    }
    bool progressed = false;
    for (size_t i = 0; i < slots.size(); ++i) {
      Slot& sl = slots[i];
      if (!sl.busy || !sl.launched) continue;
      mips_status st = sl.status;
      if (st == MIPS_OK) {
        const cudaError_t q = cudaEventQuery(sl.done);
        if (q == cudaErrorNotReady) continue;
        lk.unlock();
        st = mips_sync(sl.worker, sl.stream);  // the batch is done: reads its error flag
        std::string err = st == MIPS_OK ? std::string() : std::string(mips_last_error());
        if (st == MIPS_OK) {
          // each request keeps the first K of its rows (batch rows hold sl.K)
          int64_t row = 0;
          for (const RequestP& r : sl.reqs) {
            for (int64_t u = 0; u < r->n; ++u) {
              memcpy(r->out_idx + u * r->K, sl.h_idx + (row + u) * sl.K, sizeof(int32_t) * r->K);
              memcpy(r->out_score + u * r->K, sl.h_score + (row + u) * sl.K, sizeof(double) * r->K);
            }
            row += r->n;
          }
        }
        lk.lock();
        sl.error = err;
      }
      const double t = now();
      for (const RequestP& r : sl.reqs) {
        r->t_done = t;
        r->batch = sl.batch;
        r->batch_users = sl.n;
        r->batch_K = sl.K;
        r->slot = (int)i;
        r->batch_bytes = sl.bytes;
        r->batch_ws = sl.ws_used;
        r->inflight = sl.inflight;
        r->status = st;
        r->error = sl.error;
        r->done = true;
      }
      sl.reqs.clear();
      sl.busy = false;
      sl.launched = false;
      inflight_bytes -= sl.bytes;
      // with a budget, an idle slot gives its workspace and buffers back
      // while the slots hold more than the budget (its next batch
      // allocates what that batch needs)
      if (opt.mem_budget > 0 && held_bytes() > (size_t)opt.mem_budget) {
        index_release_workspace(sl.worker, sl.stream);
        if (sl.d_users) cudaFreeAsync(sl.d_users, sl.stream);
        if (sl.d_idx) cudaFreeAsync(sl.d_idx, sl.stream);
        if (sl.d_score) cudaFreeAsync(sl.d_score, sl.stream);
        sl.d_users = nullptr;
        sl.d_idx = nullptr;
        sl.d_score = nullptr;
        sl.dcap_users = 0;
        sl.dcap_out = 0;
      }
      progressed = true;
    }
    if (progressed) {
      cv_done.notify_all();
      cv_sched.notify_all();
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

extern "C" {

mips_status mips_server_create(mips_index_t idx, const mips_server_options* opt, mips_server_t* out) {
  if (!out) return fail(MIPS_ERR_ARG, "null output handle");
  *out = nullptr;
  if (!idx) return fail(MIPS_ERR_ARG, "null index");
  mips_server_options o{0, 2, 8192, 0};
  if (opt) o = *opt;
  if (o.method != 0 && o.method != 1) return fail(MIPS_ERR_ARG, "method must be 0 or 1");
  if (o.slots < 1 || o.slots > 8) return fail(MIPS_ERR_ARG, "slots out of range [1,8]: %d", o.slots);
  if (o.max_batch_users < 1) return fail(MIPS_ERR_ARG, "max_batch_users must be positive");
  if (o.mem_budget < 0) return fail(MIPS_ERR_ARG, "mem_budget must be >= 0");
  auto* srv = new (std::nothrow) mips_server_s();
  if (!srv) return fail(MIPS_ERR_NOMEM, "host allocation failed");
  srv->idx = idx;
  srv->opt = o;
  srv->f = index_f(idx);
  srv->n_items = index_n_items(idx);
  cudaGetDevice(&srv->device);
  srv->slots.resize(o.slots);
  for (Slot& sl : srv->slots) {
    sl.worker = index_worker_clone(idx);
    cudaError_t e = sl.worker ? cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      srv->sched_exited = true;
      mips_server_destroy(srv);
      return cuda_fail(e, "server slot creation");
    }
  }
  srv->sched = std::thread([srv] { srv->scheduler(); });
  srv->compl_ = std::thread([srv] { srv->completer(); });
  *out = srv;
  return MIPS_OK;
}

mips_status mips_server_submit(mips_server_t srv, const float* users_host, int64_t n_users, int K,
                               int32_t* out_idx_host, double* out_score_host, int64_t* request_id) {
  if (!srv || !users_host || !out_idx_host || !out_score_host || !request_id)
    return fail(MIPS_ERR_ARG, "null argument");
  if (n_users < 1 || n_users >= (1ll << 31)) return fail(MIPS_ERR_ARG, "n_users out of range");
  auto r = std::make_shared<Request>();
  r->users = users_host;
  r->n = n_users;
  r->K = K;
  r->out_idx = out_idx_host;
  r->out_score = out_score_host;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return fail(MIPS_ERR_ARG, "server is stopping");
  // (checked here: a bad request must not fail the batch it would join)
  if (K < 1 || K > 128 || K > srv->n_items) return fail(MIPS_ERR_ARG, "K out of range: %d", K);
  r->id = srv->next_id++;
  r->t_submit = srv->now();
  srv->requests[r->id] = r;
  srv->pending.push_back(r);
  *request_id = r->id;
  srv->cv_sched.notify_all();
  return MIPS_OK;
}

mips_status mips_server_wait(mips_server_t srv, int64_t request_id, double timeout_s, mips_request_info* info) {
  if (!srv) return fail(MIPS_ERR_ARG, "null server");
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->requests.find(request_id);
  if (it == srv->requests.end()) return fail(MIPS_ERR_ARG, "unknown request id %lld", (long long)request_id);
  RequestP r = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0);
  if (!srv->cv_done.wait_until(lk, until, [&] { return r->done; }))
    return fail(MIPS_ERR_TIMEOUT, "request %lld not done within %.3f s", (long long)request_id, timeout_s);
  srv->requests.erase(it);
  if (info) {
    info->t_submit = r->t_submit;
    info->t_start = r->t_start;
    info->t_done = r->t_done;
    info->batch = r->batch;
    info->batch_users = r->batch_users;
    info->batch_K = r->batch_K;
    info->slot = r->slot;
    info->batch_bytes = (int64_t)r->batch_bytes;
    info->batch_ws_bytes = (int64_t)r->batch_ws;
    info->inflight_bytes = (int64_t)r->inflight;
  }
  if (r->status != MIPS_OK) return fail(r->status, "%s", r->error.c_str());
  return MIPS_OK;
}

mips_status mips_server_destroy(mips_server_t srv) {
  if (!srv) return MIPS_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_sched.notify_all();
  srv->cv_compl.notify_all();
  if (srv->sched.joinable()) srv->sched.join();
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->sched_exited = true;
  }
  srv->cv_compl.notify_all();
  if (srv->compl_.joinable()) srv->compl_.join();
  for (Slot& sl : srv->slots) {
    if (sl.stream) {  // device buffers first, on the stream they were allocated on
      if (sl.d_users) cudaFreeAsync(sl.d_users, sl.stream);
      if (sl.d_idx) cudaFreeAsync(sl.d_idx, sl.stream);
      if (sl.d_score) cudaFreeAsync(sl.d_score, sl.stream);
      cudaStreamSynchronize(sl.stream);
    }
    if (sl.worker) mips_free_index(sl.worker);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.h_users) cudaFreeHost(sl.h_users);
    if (sl.h_idx) cudaFreeHost(sl.h_idx);
    if (sl.h_score) cudaFreeHost(sl.h_score);
    if (sl.stream) cudaStreamDestroy(sl.stream);  // last: nothing uses it after this
  }
  delete srv;
  return MIPS_OK;
}

}  // extern "C"
