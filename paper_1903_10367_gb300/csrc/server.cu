// Request server: continuous batching of independent adAFAC solves on one GPU.
//
// Requests (a tree, eps, f, options, tolerance) are submitted from any host
// thread and queued with copies of their inputs.  A worker thread owns the
// device:
//   * admission -- a queued request is admitted when its workspace
//     (adafac_workspace_size) fits into the free part of one device pool
//     allocated when the server is created (first fit, 256-byte aligned,
//     neighbouring free ranges merged).  A request that can never fit fails
//     at once with ADAFAC_ERR_OOM;
//   * setup -- an admitted request gets a handle on one of the server's
//     streams (round robin) with its workspace carved from the pool;
//   * cycles -- every running request without work in flight gets a batch of
//     cycles (inner_cycles for MIXED, kBatchFP64 for FP64) and an asynchronous
//     copy of its control block, both on its stream.  Requests on different
//     streams overlap on the device; a request that arrives while others run
//     joins at the next pass of the loop;
//   * completion -- when a request's control block shows convergence,
//     divergence or the cycle limit, its solution is copied to host memory,
//     its handle destroyed and its workspace returned to the pool.
// Latency is measured on the host from submission to the moment the solution
// is in host memory.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "adafac.h"
#include "engine.h"

using namespace adafac;

namespace {

constexpr int kBatchFP64 = 8;       // FP64 cycles enqueued per pass
constexpr size_t kAlign = 256;

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) of the device pool.
class Pool {
 public:
  explicit Pool(size_t size) { free_[0] = size; }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + kAlign - 1) / kAlign * kAlign;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;  // offset -> length
  size_t used_ = 0;
};

struct Request {
  int64_t ticket = 0;
  adafac_tree tree{};
  adafac_options opt{};
  int eps_scalar = 0;
  std::vector<double> eps, f;
  double tol = 1e-8;
  int max_cycles = 0;
  int state = ADAFAC_REQUEST_PENDING;
  adafac_status status = ADAFAC_OK;
  std::string error;
  // running
  adafac_handle h = nullptr;
  size_t off = 0, bytes = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  Control* host_ctl = nullptr;  // pinned slot of the server
  int slot = -1;
  bool inflight = false;
  int enqueued = 0;
  // result
  int cycles = 0;
  double rel = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::vector<double> u;
};

}  // namespace

struct adafac_server_s {
  char* pool_base = nullptr;
  size_t pool_bytes = 0;
  Pool* pool = nullptr;
  std::vector<cudaStream_t> streams;
  int next_stream = 0;
  int max_running = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> pending;
  std::vector<int64_t> running;
  std::map<int64_t, Request*> all;
  int64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::thread worker;
  int device = 0;
  Control* ctl_slots = nullptr;  // pinned, one per running request
  std::vector<int> free_slots;
};

namespace {

long long vertices(const adafac_tree& t) {
  long long n = 1, v = 1;
  for (int i = 0; i < t.depth; ++i) n *= 3;
  for (int j = 0; j < t.dim; ++j) v *= n + 1;
  return v;
}

void finish(adafac_server_s* S, Request* r, int state, adafac_status st, const std::string& why) {
  r->state = state;
  r->status = st;
  r->error = why;
  r->t_done = now_ms();
}

// releases the device resources of a running request (worker thread)
void retire(adafac_server_s* S, Request* r) {
  if (r->h) adafac_destroy(r->h);
  r->h = nullptr;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  std::lock_guard<std::mutex> g(S->mu);
  if (r->slot >= 0) S->free_slots.push_back(r->slot);
  r->slot = -1;
  r->host_ctl = nullptr;
  if (r->bytes) S->pool->release(r->off, r->bytes);
  r->bytes = 0;
}

bool admit_one(adafac_server_s* S, Request* r) {
  size_t need = 0;
  if (adafac_workspace_size(&r->tree, &r->opt, &need) != ADAFAC_OK) {
    std::lock_guard<std::mutex> g(S->mu);
    finish(S, r, ADAFAC_REQUEST_FAILED, ADAFAC_ERR_INVALID_ARG, "invalid tree or options");
    return true;
  }
  {
    std::lock_guard<std::mutex> g(S->mu);
    if (S->free_slots.empty() || !S->pool->alloc(need, &r->off)) return false;
    r->bytes = need;
    r->slot = S->free_slots.back();
    S->free_slots.pop_back();
    r->host_ctl = S->ctl_slots + r->slot;
  }
  r->t_admit = now_ms();
  r->stream = S->streams[S->next_stream];
  S->next_stream = (S->next_stream + 1) % (int)S->streams.size();
  adafac_status st = adafac_setup(&r->tree, r->eps.data(), r->eps_scalar,
                                  r->f.empty() ? nullptr : r->f.data(), 0, &r->opt,
                                  S->pool_base + r->off, r->bytes, r->stream, &r->h);
  if (st == ADAFAC_OK) st = handle_arm(r->h, r->tol);
  if (st == ADAFAC_OK && cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming) != cudaSuccess)
    st = ADAFAC_ERR_CUDA;
  if (st != ADAFAC_OK) {
    const std::string why = adafac_last_error(r->h);
    retire(S, r);
    std::lock_guard<std::mutex> g(S->mu);
    finish(S, r, ADAFAC_REQUEST_FAILED, st, why);
    return true;
  }
  r->inflight = false;
  r->enqueued = 0;
  std::lock_guard<std::mutex> g(S->mu);
  r->state = ADAFAC_REQUEST_RUNNING;
  S->running.push_back(r->ticket);
  return true;
}

// enqueue the next batch of a running request
void launch_batch(Request* r) {
  const bool mixed = r->opt.precision == ADAFAC_PRECISION_MIXED;
  int k = mixed ? r->opt.inner_cycles : kBatchFP64;
  k = std::min(k, r->max_cycles - r->enqueued);
  if (k > 0) adafac_cycle(r->h, k);
  r->enqueued += k;
  cudaMemcpyAsync(r->host_ctl, handle_control(r->h), sizeof(Control), cudaMemcpyDeviceToHost,
                  r->stream);
  cudaEventRecord(r->ev, r->stream);
  r->inflight = true;
}

// checks a request whose batch completed; true when it left the running set
bool check_done(adafac_server_s* S, Request* r) {
  const Control& c = *r->host_ctl;
  const bool limit = r->enqueued >= r->max_cycles;
  if (!(c.done || c.diverged || c.fault || limit)) return false;
  std::vector<double> u;
  adafac_status st = ADAFAC_OK;
  std::string why;
  if (c.fault) {
    st = ADAFAC_ERR_TIMEOUT;
    why = "a bounded device-side wait gave up";
  } else if (c.diverged) {
    st = ADAFAC_ERR_DIVERGED;
    why = "residual diverged";
  } else if (!c.done) {
    st = ADAFAC_ERR_NOT_CONVERGED;
    why = "max_cycles reached before rel_tol";
  }
  if (st == ADAFAC_OK || st == ADAFAC_ERR_NOT_CONVERGED) {
    u.resize((size_t)vertices(r->tree));
    if (adafac_solution(r->h, u.data(), 0) != ADAFAC_OK) {
      st = ADAFAC_ERR_CUDA;
      why = adafac_last_error(r->h);
    }
  }
  const int cycles = c.applied;
  const double rel = c.rel;
  retire(S, r);
  std::lock_guard<std::mutex> g(S->mu);
  r->u.swap(u);
  r->cycles = cycles;
  r->rel = rel;
  finish(S, r, st == ADAFAC_OK ? ADAFAC_REQUEST_DONE : ADAFAC_REQUEST_FAILED, st, why);
  return true;
}

void worker_loop(adafac_server_s* S) {
  cudaSetDevice(S->device);
  while (!S->stop.load()) {
    bool busy = false;
    // admission, in submission order, of whatever fits
    std::vector<Request*> cand;
    {
      std::lock_guard<std::mutex> g(S->mu);
      const int room = S->max_running - (int)S->running.size();
      for (size_t i = 0; i < S->pending.size() && (int)cand.size() < room && i < 64; ++i)
        cand.push_back(S->all[S->pending[i]]);
    }
    for (Request* r : cand) {
      if (admit_one(S, r)) {
        busy = true;
        std::lock_guard<std::mutex> g(S->mu);
        S->pending.erase(std::find(S->pending.begin(), S->pending.end(), r->ticket));
      }
    }
    // batches and completions
    std::vector<Request*> run;
    {
      std::lock_guard<std::mutex> g(S->mu);
      for (int64_t t : S->running) run.push_back(S->all[t]);
    }
    for (Request* r : run) {
      if (!r->inflight) {
        launch_batch(r);
        busy = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) continue;
      busy = true;
      r->inflight = false;
      bool left;
      if (q != cudaSuccess) {
        cudaGetLastError();
        retire(S, r);
        std::lock_guard<std::mutex> g(S->mu);
        finish(S, r, ADAFAC_REQUEST_FAILED, ADAFAC_ERR_CUDA, cudaGetErrorString(q));
        left = true;
      } else {
        left = check_done(S, r);
        if (!left) launch_batch(r);
      }
      if (left) {
        std::lock_guard<std::mutex> g(S->mu);
        S->running.erase(std::find(S->running.begin(), S->running.end(), r->ticket));
        S->cv.notify_all();
      }
    }
    if (!busy) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
  }
  // shutdown: let running work finish, then release it
  std::vector<Request*> run;
  {
    std::lock_guard<std::mutex> g(S->mu);
    for (int64_t t : S->running) run.push_back(S->all[t]);
    S->running.clear();
  }
  for (Request* r : run) {
    if (r->inflight) cudaEventSynchronize(r->ev);
    retire(S, r);
    std::lock_guard<std::mutex> g(S->mu);
    finish(S, r, ADAFAC_REQUEST_FAILED, ADAFAC_ERR_INVALID_ARG, "server destroyed");
  }
}

}  // namespace

extern "C" {

adafac_status adafac_server_create(size_t device_bytes, int n_streams, int max_running,
                                   adafac_server* out) {
  if (!out) return ADAFAC_ERR_INVALID_ARG;
  *out = nullptr;
  if (device_bytes < kAlign || n_streams < 1 || n_streams > 256 || max_running < 1)
    return ADAFAC_ERR_INVALID_ARG;
  adafac_server_s* S = new (std::nothrow) adafac_server_s();
  if (!S) return ADAFAC_ERR_OOM;
  if (cudaGetDevice(&S->device) != cudaSuccess) {
    delete S;
    return ADAFAC_ERR_CUDA;
  }
  void* p = nullptr;
  if (cudaMalloc(&p, device_bytes) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return ADAFAC_ERR_OOM;
  }
  S->pool_base = static_cast<char*>(p);
  S->pool_bytes = device_bytes / kAlign * kAlign;
  S->pool = new Pool(S->pool_bytes);
  S->max_running = max_running;
  if (cudaMallocHost(&S->ctl_slots, sizeof(Control) * (size_t)max_running) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(p);
    delete S->pool;
    delete S;
    return ADAFAC_ERR_OOM;
  }
  for (int i = max_running - 1; i >= 0; --i) S->free_slots.push_back(i);
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      break;
    }
    S->streams.push_back(s);
  }
  if (S->streams.empty()) {
    cudaFree(p);
    delete S->pool;
    delete S;
    return ADAFAC_ERR_CUDA;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return ADAFAC_OK;
}

adafac_status adafac_submit(adafac_server S, const adafac_tree* tree, const double* eps,
                            int eps_is_scalar, const double* f, const adafac_options* opt,
                            double rel_tol, int max_cycles, int64_t* ticket) {
  if (!S || !tree || !eps || !opt || !ticket || !(rel_tol >= 0.0) || max_cycles < 1)
    return ADAFAC_ERR_INVALID_ARG;
  *ticket = 0;
  if ((tree->dim != 2 && tree->dim != 3) || tree->depth < 1 || tree->depth > 12)
    return ADAFAC_ERR_INVALID_ARG;
  size_t need = 0;
  if (adafac_workspace_size(tree, opt, &need) != ADAFAC_OK) return ADAFAC_ERR_INVALID_ARG;
  if ((need + kAlign - 1) / kAlign * kAlign > S->pool_bytes) return ADAFAC_ERR_OOM;
  Request* r = new (std::nothrow) Request();
  if (!r) return ADAFAC_ERR_OOM;
  r->tree = *tree;
  r->opt = *opt;
  r->eps_scalar = eps_is_scalar ? 1 : 0;
  long long ncell = 1, n = 1;
  for (int i = 0; i < tree->depth; ++i) n *= 3;
  for (int j = 0; j < tree->dim; ++j) ncell *= n;
  r->eps.assign(eps, eps + (eps_is_scalar ? 1 : ncell));
  if (f) r->f.assign(f, f + vertices(*tree));
  r->tol = rel_tol;
  r->max_cycles = max_cycles;
  r->t_submit = now_ms();
  std::lock_guard<std::mutex> g(S->mu);
  r->ticket = S->next_ticket++;
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  S->pending.push_back(r->ticket);
  S->cv.notify_all();
  return ADAFAC_OK;
}

adafac_status adafac_poll(adafac_server S, int64_t ticket, adafac_request_info* info) {
  if (!S || !info) return ADAFAC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return ADAFAC_ERR_INVALID_ARG;
  const Request* r = it->second;
  info->state = r->state;
  info->status = r->status;
  info->cycles = r->cycles;
  info->rel = r->rel;
  const bool ended = r->state == ADAFAC_REQUEST_DONE || r->state == ADAFAC_REQUEST_FAILED;
  const bool admitted = r->t_admit > 0.0;
  info->queue_ms = admitted ? r->t_admit - r->t_submit : -1.0;
  info->latency_ms = ended ? r->t_done - r->t_submit : -1.0;
  return ADAFAC_OK;
}

adafac_status adafac_fetch(adafac_server S, int64_t ticket, double* dst) {
  if (!S) return ADAFAC_ERR_INVALID_ARG;
  Request* r = nullptr;
  {
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return ADAFAC_ERR_INVALID_ARG;
    r = it->second;
    if (r->state != ADAFAC_REQUEST_DONE && r->state != ADAFAC_REQUEST_FAILED)
      return ADAFAC_ERR_INVALID_ARG;  // still queued or running
    S->all.erase(it);
  }
  adafac_status st = r->status;
  if (dst && !r->u.empty()) std::memcpy(dst, r->u.data(), r->u.size() * sizeof(double));
  delete r;
  return st;
}

adafac_status adafac_server_stats(adafac_server S, int* pending, int* running,
                                  size_t* bytes_in_use) {
  if (!S) return ADAFAC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(S->mu);
  if (pending) *pending = (int)S->pending.size();
  if (running) *running = (int)S->running.size();
  if (bytes_in_use) *bytes_in_use = S->pool->used();
  return ADAFAC_OK;
}

adafac_status adafac_server_destroy(adafac_server S) {
  if (!S) return ADAFAC_ERR_INVALID_ARG;
  S->stop.store(true);
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto& kv : S->all) delete kv.second;
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  cudaFreeHost(S->ctl_slots);
  cudaFree(S->pool_base);
  delete S->pool;
  delete S;
  return ADAFAC_OK;
}

}  // extern "C"
