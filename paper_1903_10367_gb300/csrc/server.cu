// Request server: continuous batching of independent adAFAC solves on one GPU.
//
// Requests (a tree, eps, f, options, tolerance) are submitted from any host
// thread and queued with copies of their inputs.  Two host threads own the
// device work:
//   * service threads (kServiceThreads) admit a queued request when a running slot is free
//     and its workspace (adafac_workspace_size) fits into the free part of one
//     device pool allocated when the server is created (first fit, 256-byte
//     aligned, neighbouring free ranges merged; the first 64 queued requests
//     are scanned in submission order), and sets it up on the slot's stream
//     with its workspace carved from the pool.  It also completes ended
//     requests: their solution is copied to host memory, the handle destroyed
//     and the workspace returned to the pool.  These calls wait on the device,
//     so each service thread takes one such job at a time;
//   * the launcher thread keeps one batch of cycles (inner_cycles for MIXED,
//     kBatchFP64 for FP64) plus an asynchronous copy of the control block in
//     flight for every running request, and never waits on the device.  When
//     a copy shows convergence, divergence, a fault or the cycle limit, the
//     request goes to the service threads.
// Requests on different streams overlap on the device; small requests (up to
// kSmallBytes of workspace) run on high-priority streams so that their short
// kernels are scheduled ahead of the blocks of large ones.  A request submitted
// while others run is admitted as soon as a slot and memory are free.
// Requests set up with path BATCHED do not get launches of their own: the
// launcher groups them by dimension and cluster size, and one launch of the
// batched kernel advances every request of a group by one refinement step (a
// cluster of CTAs per request), followed by one copy of all their control
// blocks.  A group has one launch in flight at a time; requests that became
// ready meanwhile join its next launch.
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
constexpr size_t kSmallBytes = 64u << 20;  // workspaces up to this run at high priority
constexpr int kServiceThreads = 4;         // setups and completions in parallel
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
  size_t need = 0;              // workspace bytes
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
  // batched path: the instance on the device and its launch group
  const BatchItem* bitem = nullptr;
  int group = -1;
  int onchip = 0;               // shared-memory bytes of its vectors at one CTA
  int step_k = 0;               // cycles of the launch in flight
  // result
  int cycles = 0;
  double rel = 0.0;
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  std::vector<double> u;
};

// One launch group of batched requests (same dimension and cluster size).
struct BatchGroup {
  int D = 0, C = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  Control* d_mirror = nullptr;   // device: control blocks written by the launch
  Control* h_mirror = nullptr;   // pinned copy of them
  std::vector<Request*> members; // requests of the launch in flight
  bool inflight = false;
};

}  // namespace

struct adafac_server_s {
  char* pool_base = nullptr;
  size_t pool_bytes = 0;
  Pool* pool = nullptr;
  std::vector<cudaStream_t> streams;       // lowest priority: large requests
  std::vector<cudaStream_t> fast_streams;  // highest priority: small requests
  int max_running = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<int64_t> pending;
  std::vector<int64_t> running;
  std::map<int64_t, Request*> all;
  int64_t next_ticket = 1;
  std::atomic<bool> stop{false};
  std::vector<Request*> completing;  // ended, waiting for a service thread
  int in_setup = 0;                  // admitted, being set up
  int in_completion = 0;             // ended, solution being copied
  std::thread launcher;
  std::vector<std::thread> service;
  int device = 0;
  Control* ctl_slots = nullptr;  // pinned, one per running request
  std::vector<int> free_slots;
  std::map<int, BatchGroup> groups;  // batched launch groups by D * 64 + C (launcher)
  int batch_priority = 0;
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

// releases the device resources of a request
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

// claims a slot and pool memory for a queued request (caller holds S->mu)
bool claim(adafac_server_s* S, Request* r) {
  if (S->free_slots.empty() || !S->pool->alloc(r->need, &r->off)) return false;
  r->bytes = r->need;
  r->slot = S->free_slots.back();
  S->free_slots.pop_back();
  r->host_ctl = S->ctl_slots + r->slot;
  r->state = ADAFAC_REQUEST_RUNNING;  // admitted: memory and slot reserved
  r->t_admit = now_ms();
  S->in_setup += 1;
  return true;
}

// sets up a claimed request and hands it to the launcher (service thread)
void admit(adafac_server_s* S, Request* r) {
  // small solves go to high-priority streams, so that their short kernels
  // are scheduled ahead of the blocks of large solves sharing the device
  const bool small = r->bytes <= kSmallBytes;
  const std::vector<cudaStream_t>& pool = small ? S->fast_streams : S->streams;
  r->stream = pool[r->slot % (int)pool.size()];
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
    S->in_setup -= 1;
    return;
  }
  r->inflight = false;
  r->enqueued = 0;
  int D = 0, C = 0;
  r->bitem = handle_batch_item(r->h, &D, &C, &r->onchip);
  r->group = r->bitem ? D * 64 + C : -1;
  std::lock_guard<std::mutex> g(S->mu);
  S->running.push_back(r->ticket);
  S->in_setup -= 1;
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

// true when the control block copied after the last batch ends the request
bool ended(const Request* r) {
  const Control& c = *r->host_ctl;
  return c.done || c.diverged || c.fault || r->enqueued >= r->max_cycles;
}

// copies the solution of an ended request to host memory and releases its
// device resources (service thread)
void complete(adafac_server_s* S, Request* r) {
  const Control c = *r->host_ctl;
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
  retire(S, r);
  std::lock_guard<std::mutex> g(S->mu);
  r->u.swap(u);
  r->cycles = c.applied;
  r->rel = c.rel;
  finish(S, r, st == ADAFAC_OK ? ADAFAC_REQUEST_DONE : ADAFAC_REQUEST_FAILED, st, why);
}

// The launch group of a batched request (created on first use; launcher
// thread only).  Null when its stream or buffers cannot be made.
BatchGroup* group_of(adafac_server_s* S, const Request* r) {
  auto it = S->groups.find(r->group);
  if (it != S->groups.end()) return it->second.stream ? &it->second : nullptr;
  BatchGroup& G = S->groups[r->group];
  G.D = r->group / 64;
  G.C = r->group % 64;
  if (cudaStreamCreateWithPriority(&G.stream, cudaStreamNonBlocking, S->batch_priority) !=
          cudaSuccess ||
      cudaEventCreateWithFlags(&G.ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMalloc(&G.d_mirror, sizeof(Control) * kBatchMax) != cudaSuccess ||
      cudaMallocHost(&G.h_mirror, sizeof(Control) * kBatchMax) != cudaSuccess) {
    cudaGetLastError();
    if (G.stream) cudaStreamDestroy(G.stream);
    G.stream = nullptr;
    return nullptr;
  }
  return &G;
}

// hands an ended request to the service threads (launcher thread)
void hand_over(adafac_server_s* S, Request* r) {
  std::lock_guard<std::mutex> g(S->mu);
  S->running.erase(std::find(S->running.begin(), S->running.end(), r->ticket));
  S->completing.push_back(r);
  S->cv.notify_all();
}

// One launch of the batched kernel for the ready requests of a group, then
// one copy of their control blocks.  Returns false if nothing was launched.
bool launch_group(adafac_server_s* S, BatchGroup& G, std::vector<Request*>& ready) {
  BatchLaunch bl;
  G.members.clear();
  for (Request* r : ready) {
    if ((int)G.members.size() == kBatchMax) break;
    int k = std::min(r->opt.inner_cycles, r->max_cycles - r->enqueued);
    if (k < 1) continue;
    bl.item[bl.count] = r->bitem;
    bl.k[bl.count] = k;
    bl.count += 1;
    if (G.C == 1) bl.dyn_bytes = std::max(bl.dyn_bytes, r->onchip);
    r->step_k = k;
    G.members.push_back(r);
  }
  if (!bl.count) return false;
  bl.mirror = G.d_mirror;
  cudaError_t e = launch_batch_step(G.D, G.C, bl, G.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(G.h_mirror, G.d_mirror, sizeof(Control) * bl.count,
                        cudaMemcpyDeviceToHost, G.stream);
  if (e == cudaSuccess) e = cudaEventRecord(G.ev, G.stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    for (Request* r : G.members) {
      r->host_ctl->fault = 1;  // reported as a failed request
      hand_over(S, r);
    }
    G.members.clear();
    return true;
  }
  for (Request* r : G.members) {
    r->inflight = true;
    r->enqueued += r->step_k;
  }
  G.inflight = true;
  return true;
}

// Launcher: keeps a batch in flight for every running request and hands
// ended requests to the service thread.  It never waits on the device.
void launcher_loop(adafac_server_s* S) {
  cudaSetDevice(S->device);
  std::vector<Request*> run;
  std::map<int, std::vector<Request*>> ready;
  while (!S->stop.load()) {
    bool busy = false;
    run.clear();
    {
      std::lock_guard<std::mutex> g(S->mu);
      for (int64_t t : S->running) run.push_back(S->all[t]);
    }
    // batched groups whose launch ended: their control blocks are in host memory
    for (auto& kv : S->groups) {
      BatchGroup& G = kv.second;
      if (!G.inflight) continue;
      const cudaError_t q = cudaEventQuery(G.ev);
      if (q == cudaErrorNotReady) continue;
      busy = true;
      G.inflight = false;
      if (q != cudaSuccess) cudaGetLastError();
      for (size_t i = 0; i < G.members.size(); ++i) {
        Request* r = G.members[i];
        r->inflight = false;
        if (q != cudaSuccess) r->host_ctl->fault = 1;
        else *r->host_ctl = G.h_mirror[i];
      }
    }
    ready.clear();
    for (Request* r : run) {
      if (r->bitem) {
        if (r->inflight) continue;
        if (r->enqueued > 0 && ended(r)) {
          busy = true;
          hand_over(S, r);
        } else {
          ready[r->group].push_back(r);
        }
        continue;
      }
      if (!r->inflight) {
        launch_batch(r);
        busy = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q == cudaErrorNotReady) continue;
      busy = true;
      r->inflight = false;
      if (q != cudaSuccess) {
        cudaGetLastError();
        r->host_ctl->fault = 1;  // reported as a failed request
      } else if (!ended(r)) {
        launch_batch(r);
        continue;
      }
      hand_over(S, r);
    }
    for (auto& kv : ready) {
      BatchGroup* G = group_of(S, kv.second.front());
      if (!G) {
        for (Request* r : kv.second) {
          r->host_ctl->fault = 1;
          hand_over(S, r);
        }
        busy = true;
        continue;
      }
      if (G->inflight) continue;
      if (launch_group(S, *G, kv.second)) busy = true;
    }
    if (!busy) {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv.wait_for(lk, std::chrono::microseconds(20));
    }
  }
}

// Service threads: completions (solution copies, releases) first, then
// admissions (setups) -- the calls that wait on the device.  Each thread takes
// one job at a time, so a long setup does not hold up other completions.
void service_loop(adafac_server_s* S) {
  cudaSetDevice(S->device);
  while (!S->stop.load()) {
    Request* job = nullptr;
    bool completion = false;
    {
      std::lock_guard<std::mutex> g(S->mu);
      if (!S->completing.empty()) {
        job = S->completing.front();
        S->completing.erase(S->completing.begin());
        S->in_completion += 1;
        completion = true;
      } else {
        // admission, in submission order, of the first request that fits
        for (size_t i = 0; i < S->pending.size() && i < 64; ++i) {
          Request* r = S->all[S->pending[i]];
          if (claim(S, r)) {
            S->pending.erase(S->pending.begin() + i);
            job = r;
            break;
          }
        }
      }
    }
    if (job) {
      if (completion) {
        complete(S, job);
        std::lock_guard<std::mutex> g(S->mu);
        S->in_completion -= 1;
      } else {
        admit(S, job);
      }
      continue;
    }
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait_for(lk, std::chrono::microseconds(50));
  }
}

// after both threads stopped: release whatever is still on the device
void drain_all(adafac_server_s* S) {
  for (auto& kv : S->groups)
    if (kv.second.stream) cudaStreamSynchronize(kv.second.stream);
  std::vector<Request*> left;
  {
    std::lock_guard<std::mutex> g(S->mu);
    for (int64_t t : S->running) left.push_back(S->all[t]);
    S->running.clear();
    for (Request* r : S->completing) left.push_back(r);
    S->completing.clear();
  }
  for (Request* r : left) {
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
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
    cudaGetLastError();
    least = greatest = 0;
  }
  S->batch_priority = greatest;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithPriority(&a, cudaStreamNonBlocking, least) != cudaSuccess ||
        cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, greatest) != cudaSuccess) {
      cudaGetLastError();
      if (a) cudaStreamDestroy(a);
      break;
    }
    S->streams.push_back(a);
    S->fast_streams.push_back(b);
  }
  if (S->streams.empty()) {
    cudaFree(p);
    delete S->pool;
    delete S;
    return ADAFAC_ERR_CUDA;
  }
  S->launcher = std::thread(launcher_loop, S);
  for (int i = 0; i < kServiceThreads; ++i) S->service.emplace_back(service_loop, S);
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
  r->need = need;
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
  if (running)
    *running = (int)S->running.size() + S->in_setup + (int)S->completing.size() +
               S->in_completion;
  if (bytes_in_use) *bytes_in_use = S->pool->used();
  return ADAFAC_OK;
}

adafac_status adafac_server_destroy(adafac_server S) {
  if (!S) return ADAFAC_ERR_INVALID_ARG;
  S->stop.store(true);
  S->cv.notify_all();
  if (S->launcher.joinable()) S->launcher.join();
  for (std::thread& t : S->service)
    if (t.joinable()) t.join();
  drain_all(S);
  for (auto& kv : S->all) delete kv.second;
  for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
  for (cudaStream_t s : S->fast_streams) cudaStreamDestroy(s);
  for (auto& kv : S->groups) {
    BatchGroup& G = kv.second;
    if (G.stream) cudaStreamDestroy(G.stream);
    if (G.ev) cudaEventDestroy(G.ev);
    if (G.d_mirror) cudaFree(G.d_mirror);
    if (G.h_mirror) cudaFreeHost(G.h_mirror);
  }
  cudaFreeHost(S->ctl_slots);
  cudaFree(S->pool_base);
  delete S->pool;
  delete S;
  return ADAFAC_OK;
}

}  // extern "C"
