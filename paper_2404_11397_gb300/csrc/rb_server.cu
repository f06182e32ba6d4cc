// rb_server.cu -- continuous-batching request loop over resident events.
//
// Clients call rb_submit from any thread; a scheduler thread admits pending
// requests whenever a slot (a CUDA stream with pinned and device staging
// buffers) is free and the launch's device footprint fits in the remaining
// budget.  It takes the oldest pending request and packs into the same launch
// the later pending requests for the same event and gradient flag (up to the
// slot capacity and the budget), so that requests that arrive while others
// are on the GPU share launches as well as overlapping them on other slots.
// A launch runs the packed walkers rounded up to a multiple of 256 (copies of
// its first walker fill the rest); every walker is computed independently by
// one warp, so each result is bit-identical to the same request evaluated
// alone.  With graphs, each launch is captured (copy-in, set-up, likelihood
// kernel, copy-out, completion node) and applied to the slot's instantiated
// graph for its detector count and gradient flag with cudaGraphExecUpdate;
// the graph is instantiated again only when the update is refused.  The
// scheduler thread only forms the launches; each slot's own worker thread
// stages the walkers and issues its launch, so the host work of several
// launches proceeds in parallel.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <utility>
#include <vector>

#include "rb.h"
#include "rb_api_internal.h"

namespace rb {

constexpr int64_t kPackQuantum = 256;  // launches run a multiple of this many walkers
constexpr size_t kMaxLatencies = (size_t)1 << 22;  // latencies kept between rb_server_latency resets

struct Request {
  uint64_t ticket = 0;
  std::chrono::steady_clock::time_point t_submit, t_assigned, t_issued;
  const EventEntry* ev = nullptr;
  int64_t W = 0;
  bool want_grad = false;
  std::vector<double> theta, logl, grad;
  int status = RB_OK;
  bool done = false;
  char msg[256] = "";  // error detail (set on the scheduler thread)
};

struct Server;

struct Slot {
  int idx = 0;
  Server* srv = nullptr;
  cudaStream_t stream = nullptr;
  double *h_theta = nullptr, *h_logl = nullptr, *h_grad = nullptr;  // pinned
  double *d_theta = nullptr, *d_logl = nullptr, *d_grad = nullptr;
  void* d_ws = nullptr;
  // the launch on the slot: its requests (walkers in this order from row 0)
  std::vector<Request*> reqs;
  int64_t run_w = 0;        // walkers the launch runs (requested + padding)
  size_t footprint = 0;
  bool stuck = false;       // abandoned at shutdown with work possibly in flight: never freed
  bool has_work = false;    // a launch assigned by the scheduler, not yet issued (guarded by Server::mu)
  bool gpu_done = false;    // the launch's completion node has run; results await the worker (Server::mu)
  std::condition_variable cv_work;
  std::thread worker;
  std::map<std::pair<int, bool>, cudaGraphExec_t> graphs;  // (n_det, grad) -> instantiated graph (worker only)
};

// What one launch did, for the statistics.
struct LaunchOutcome {
  bool graph = false, updated = false, instantiated = false;
};

struct Server {
  rb_server_opts opts{};
  size_t bytes_per_walker = 0;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<Request*> pending;
  std::unordered_map<uint64_t, std::unique_ptr<Request>> requests;
  std::vector<std::unique_ptr<Slot>> slots;
  std::vector<Slot*> free_slots;
  uint64_t next_ticket = 1;
  size_t hbm_in_use = 0;
  int in_flight = 0;
  bool stopping = false;
  rb_server_stats stats{};
  // per completed request: submit -> results in host memory, and its parts:
  // waiting for a slot, the host issuing the launch, the device and completion
  std::vector<float> latency_us[4];
  std::thread thread;

  void run();
  void work(Slot* s);
  int launch(Slot* s, LaunchOutcome* out);
  void gpu_finished(Slot* s);
  void complete(Slot* s);
  void fail_slot(Slot* s, int status, const char* why);  // with mu held
};

static int64_t pack_round(int64_t W) { return (W + kPackQuantum - 1) / kPackQuantum * kPackQuantum; }

// The completion node (CUDA's host-callback thread, shared by all streams):
// only flag the slot; its worker copies the results out.
static void CUDART_CB slot_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->srv->gpu_finished(s);
}

void Server::gpu_finished(Slot* s) {
  std::lock_guard<std::mutex> lk(mu);
  s->gpu_done = true;
  s->cv_work.notify_one();
}

// On the slot's worker, after gpu_finished: results to the requests, slot freed.
void Server::complete(Slot* s) {
  const auto now = std::chrono::steady_clock::now();
  {
    // the requests stay owned by the slot until marked done below
    int64_t row = 0;
    for (Request* r : s->reqs) {
      std::memcpy(r->logl.data(), s->h_logl + row, sizeof(double) * r->W);
      if (r->want_grad) std::memcpy(r->grad.data(), s->h_grad + kNPar * row, sizeof(double) * kNPar * r->W);
      row += r->W;
    }
  }
  std::lock_guard<std::mutex> lk(mu);
  if (s->reqs.empty()) return;  // failed at shutdown already
  for (Request* r : s->reqs) {
    r->status = RB_OK;
    r->done = true;
    ++stats.completed;
    if (latency_us[0].size() < kMaxLatencies) {
      using us = std::chrono::duration<float, std::micro>;
      latency_us[0].push_back(us(now - r->t_submit).count());
      latency_us[1].push_back(us(r->t_assigned - r->t_submit).count());
      latency_us[2].push_back(us(r->t_issued - r->t_assigned).count());
      latency_us[3].push_back(us(now - r->t_issued).count());
    }
    stats.walkers_requested += (uint64_t)r->W;
  }
  stats.walkers_run += (uint64_t)s->run_w;
  hbm_in_use -= s->footprint;
  --in_flight;
  s->reqs.clear();
  free_slots.push_back(s);
  cv.notify_all();
}

void Server::fail_slot(Slot* s, int status, const char* why) {
  for (Request* r : s->reqs) {
    std::snprintf(r->msg, sizeof(r->msg), "%s", why);
    r->status = status;
    r->done = true;
  }
  s->reqs.clear();
  hbm_in_use -= s->footprint;
  --in_flight;
  cv.notify_all();
}

// Issue copy-in, set-up + likelihood kernels, copy-out and the completion
// host node on the slot's stream (captured into a graph when enabled).
static int enqueue_work(Slot* s, const EventEntry* ev, int64_t W, bool grad, int mode) {
  cudaError_t err = cudaMemcpyAsync(s->d_theta, s->h_theta, sizeof(double) * kNPar * W, cudaMemcpyHostToDevice,
                                    s->stream);
  if (err != cudaSuccess) return cuda_fail(err, "server copy-in");
  int rc = run_batch(ev, s->d_theta, W, s->d_logl, grad ? s->d_grad : nullptr, mode, s->stream, s->d_ws);
  if (rc != RB_OK) return rc;
  if ((err = cudaMemcpyAsync(s->h_logl, s->d_logl, sizeof(double) * W, cudaMemcpyDeviceToHost, s->stream)) !=
      cudaSuccess)
    return cuda_fail(err, "server copy-out");
  if (grad && (err = cudaMemcpyAsync(s->h_grad, s->d_grad, sizeof(double) * kNPar * W, cudaMemcpyDeviceToHost,
                                     s->stream)) != cudaSuccess)
    return cuda_fail(err, "server copy-out grad");
  if ((err = cudaLaunchHostFunc(s->stream, slot_done, s)) != cudaSuccess) return cuda_fail(err, "server host node");
  return RB_OK;
}

int Server::launch(Slot* s, LaunchOutcome* out) {
  const Request* head = s->reqs.front();
  const EventEntry* ev = head->ev;
  const bool grad = head->want_grad;
  int64_t row = 0;
  for (const Request* r : s->reqs) {
    std::memcpy(s->h_theta + kNPar * row, r->theta.data(), sizeof(double) * kNPar * r->W);
    row += r->W;
  }
  for (int64_t w = row; w < s->run_w; ++w)  // pad with the first walker
    std::memcpy(s->h_theta + kNPar * w, head->theta.data(), sizeof(double) * kNPar);
  if (!opts.use_graphs) {
    for (Request* r : s->reqs) r->t_issued = std::chrono::steady_clock::now();
    return enqueue_work(s, ev, s->run_w, grad, opts.mode);
  }
  out->graph = true;
  cudaGraph_t graph = nullptr;
  cudaError_t err = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
  if (err != cudaSuccess) return cuda_fail(err, "begin capture");
  int rc = enqueue_work(s, ev, s->run_w, grad, opts.mode);
  err = cudaStreamEndCapture(s->stream, &graph);
  if (rc != RB_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (err != cudaSuccess) return cuda_fail(err, "end capture");
  const auto key = std::make_pair(ev->n_det, grad);
  cudaGraphExec_t exec = nullptr;
  auto it = s->graphs.find(key);
  if (it != s->graphs.end()) {
    cudaGraphExecUpdateResultInfo info{};
    if (cudaGraphExecUpdate(it->second, graph, &info) == cudaSuccess) {
      exec = it->second;
      out->updated = true;
    } else {
      cudaGetLastError();  // a refused update is not an error of the stream
      cudaGraphExecDestroy(it->second);
      s->graphs.erase(it);
    }
  }
  if (!exec) {
    err = cudaGraphInstantiate(&exec, graph, 0);
    if (err != cudaSuccess) {
      cudaGraphDestroy(graph);
      return cuda_fail(err, "graph instantiate");
    }
    s->graphs[key] = exec;
    out->instantiated = true;
  }
  cudaGraphDestroy(graph);
  for (Request* r : s->reqs) r->t_issued = std::chrono::steady_clock::now();
  err = cudaGraphLaunch(exec, s->stream);
  if (err != cudaSuccess) return cuda_fail(err, "graph launch");
  count_launches(2);
  return RB_OK;
}

// A slot's worker: issue each launch the scheduler assigns to the slot, and
// collect its results once the completion node has flagged it.  At shutdown
// the worker stays until its slot holds no launch.
void Server::work(Slot* s) {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    s->cv_work.wait(lk, [&] { return s->has_work || s->gpu_done || (stopping && s->reqs.empty()); });
    if (s->gpu_done) {
      s->gpu_done = false;
      lk.unlock();
      complete(s);
      lk.lock();
      continue;
    }
    if (!s->has_work) return;  // stopping, and nothing on the slot
    s->has_work = false;
    lk.unlock();
    LaunchOutcome o;
    const int rc = launch(s, &o);
    lk.lock();
    if (rc == RB_OK) {
      if (o.graph) ++stats.graph_launches; else ++stats.plain_launches;
      if (o.updated) ++stats.graph_updates;
      if (o.instantiated) ++stats.graphs_captured;
    } else {  // the completion node never runs: release here
      fail_slot(s, rc, rb_last_error());
      free_slots.push_back(s);
    }
  }
}

void Server::run() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv.wait(lk, [&] {
      if (stopping) return true;
      if (pending.empty() || free_slots.empty()) return false;
      const Request* r = pending.front();
      return hbm_in_use + bytes_per_walker * (size_t)pack_round(r->W) <= opts.hbm_budget_bytes || in_flight == 0;
    });
    if (stopping) break;
    // the oldest request, then the later ones for the same event and gradient flag
    Slot* s = free_slots.back();
    free_slots.pop_back();
    Request* head = pending.front();
    pending.pop_front();
    s->reqs.assign(1, head);
    int64_t W = head->W;
    for (auto it = pending.begin(); it != pending.end();) {
      Request* r = *it;
      const int64_t Wn = W + r->W;
      if (r->ev == head->ev && r->want_grad == head->want_grad && Wn <= opts.max_walkers &&
          hbm_in_use + bytes_per_walker * (size_t)pack_round(Wn) <= opts.hbm_budget_bytes) {
        s->reqs.push_back(r);
        W = Wn;
        it = pending.erase(it);
      } else {
        ++it;
      }
    }
    s->run_w = pack_round(W) < opts.max_walkers ? pack_round(W) : opts.max_walkers;
    s->footprint = bytes_per_walker * (size_t)s->run_w;
    const auto t_assigned = std::chrono::steady_clock::now();
    for (Request* r : s->reqs) r->t_assigned = t_assigned;
    hbm_in_use += s->footprint;
    ++in_flight;
    if (in_flight > stats.max_in_flight) stats.max_in_flight = in_flight;
    s->has_work = true;
    s->cv_work.notify_one();
  }
  for (auto& sp : slots) sp->cv_work.notify_one();  // workers with nothing assigned exit
  // Shutdown: wait for the launches on the GPU.  A slot whose stream reports an
  // error fails its requests now (its completion node will not run); after the
  // deadline the rest fail and their slots are left untouched.
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(30);
  while (in_flight > 0) {
    cv.wait_for(lk, std::chrono::milliseconds(20), [&] { return in_flight == 0; });
    if (in_flight == 0) break;
    for (auto& sp : slots) {
      Slot* s = sp.get();
      if (s->reqs.empty()) continue;
      const cudaError_t q = cudaStreamQuery(s->stream);
      if (q != cudaSuccess && q != cudaErrorNotReady) {
        fail_slot(s, RB_ECUDA, "the slot's stream reported a CUDA error");
        s->stuck = true;  // the failed context may still hold the buffers
        s->cv_work.notify_one();
      }
    }
    if (std::chrono::steady_clock::now() > deadline) {
      for (auto& sp : slots)
        if (!sp->reqs.empty()) {
          fail_slot(sp.get(), RB_ETIMEDOUT, "the launch did not complete before shutdown");
          sp->stuck = true;
          sp->cv_work.notify_one();
        }
    }
  }
  for (Request* r : pending) {
    r->status = RB_ECLOSED;
    std::snprintf(r->msg, sizeof(r->msg), "server shut down before the request ran");
    r->done = true;
  }
  pending.clear();
  cv.notify_all();
}

}  // namespace rb

using namespace rb;

struct rb_server_s {
  rb::Server s;
};

extern "C" {

int rb_server_create(const rb_server_opts* opts, rb_server_t* out) {
  RB_NVTX("rb_server_create");
  if (!out) return set_error(RB_EINVAL, "rb_server_create: NULL output");
  *out = nullptr;
  rb_server_opts o{};
  if (opts) o = *opts;
  if (o.hbm_budget_bytes == 0) o.hbm_budget_bytes = (size_t)1 << 30;
  if (o.max_slots == 0) o.max_slots = 8;
  if (o.max_queue == 0) o.max_queue = 4096;
  if (o.max_walkers == 0) o.max_walkers = 65536;
  if (!opts) o.use_graphs = 1;
  if (o.max_slots < 1 || o.max_slots > 64 || o.max_queue < 1 || o.max_walkers < 1 ||
      (o.mode != RB_MIXED && o.mode != RB_FP64 && o.mode != RB_MIXED_F64PHASE))
    return set_error(RB_EINVAL, "rb_server_create: invalid options");
  // slot buffers hold the largest launch: max_walkers rounded up to the packing quantum
  const int64_t cap = pack_round(o.max_walkers);
  auto* srv = new (std::nothrow) rb_server_s();
  if (!srv) return set_error(RB_ENOMEM, "rb_server_create: host allocation");
  Server& S = srv->s;
  S.opts = o;
  S.bytes_per_walker = sizeof(double) * (2 * kNPar + 1) + walker_ws_bytes(o.mode, true);
  int rc = RB_OK;
  for (int i = 0; i < o.max_slots && rc == RB_OK; ++i) {
    auto sl = std::make_unique<Slot>();
    sl->idx = i;
    sl->srv = &S;
    cudaError_t err = cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaMallocHost(&sl->h_theta, sizeof(double) * kNPar * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&sl->h_logl, sizeof(double) * cap);
    if (err == cudaSuccess) err = cudaMallocHost(&sl->h_grad, sizeof(double) * kNPar * cap);
    if (err == cudaSuccess) err = cudaMalloc(&sl->d_theta, sizeof(double) * kNPar * cap);
    if (err == cudaSuccess) err = cudaMalloc(&sl->d_logl, sizeof(double) * cap);
    if (err == cudaSuccess) err = cudaMalloc(&sl->d_grad, sizeof(double) * kNPar * cap);
    if (err == cudaSuccess) err = cudaMalloc(&sl->d_ws, walker_ws_bytes(o.mode, true) * cap);
    if (err != cudaSuccess) rc = cuda_fail(err, "rb_server_create: slot buffers");
    S.free_slots.push_back(sl.get());
    S.slots.push_back(std::move(sl));
  }
  if (rc != RB_OK) {
    rb_server_destroy(srv);
    return rc;
  }
  for (auto& sl : S.slots) {
    Slot* p = sl.get();
    sl->worker = std::thread([&S, p] { S.work(p); });
  }
  S.thread = std::thread([&S] { S.run(); });
  *out = srv;
  return RB_OK;
}

int rb_server_destroy(rb_server_t srv) {
  RB_NVTX("rb_server_destroy");
  if (!srv) return RB_OK;
  Server& S = srv->s;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stopping = true;
  }
  S.cv.notify_all();
  if (S.thread.joinable()) S.thread.join();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    for (auto& sl : S.slots) sl->cv_work.notify_one();
  }
  for (auto& sl : S.slots)
    if (sl->worker.joinable()) sl->worker.join();
  for (auto& sl : S.slots) {
    if (sl->stuck) continue;  // abandoned with work possibly in flight: leave its memory alone
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    for (auto& kv : sl->graphs) cudaGraphExecDestroy(kv.second);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    cudaFreeHost(sl->h_theta);
    cudaFreeHost(sl->h_logl);
    cudaFreeHost(sl->h_grad);
    cudaFree(sl->d_theta);
    cudaFree(sl->d_logl);
    cudaFree(sl->d_grad);
    cudaFree(sl->d_ws);
  }
  delete srv;
  return RB_OK;
}

int rb_submit(rb_server_t srv, rb_event_t ev, const double* theta_host, int64_t W, int want_grad, uint64_t* ticket) {
  RB_NVTX("rb_submit");
  if (!srv || !ev || !theta_host || !ticket) return set_error(RB_EINVAL, "rb_submit: NULL argument");
  Server& S = srv->s;
  if (W < 1 || W > S.opts.max_walkers) return set_error(RB_EINVAL, "rb_submit: W=%lld out of range", (long long)W);
  auto r = std::make_unique<Request>();
  r->ev = event_entry(ev);
  r->W = W;
  r->want_grad = want_grad != 0;
  r->theta.assign(theta_host, theta_host + kNPar * W);
  r->t_submit = std::chrono::steady_clock::now();
  r->logl.resize(W);
  if (r->want_grad) r->grad.resize(kNPar * W);
  {
    std::lock_guard<std::mutex> lk(S.mu);
    if (S.stopping) return set_error(RB_ECLOSED, "rb_submit: server shut down");
    if ((int)S.pending.size() >= S.opts.max_queue) {
      ++S.stats.rejected;
      return set_error(RB_EBUSY, "rb_submit: %d requests pending", (int)S.pending.size());
    }
    r->ticket = S.next_ticket++;
    *ticket = r->ticket;
    S.pending.push_back(r.get());
    S.requests.emplace(r->ticket, std::move(r));
    ++S.stats.submitted;
  }
  S.cv.notify_all();
  return RB_OK;
}

int rb_poll(rb_server_t srv, uint64_t ticket, int64_t timeout_us, double* logl_out, double* grad_out) {
  RB_NVTX("rb_poll");
  if (!srv) return set_error(RB_EINVAL, "rb_poll: NULL server");
  Server& S = srv->s;
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.requests.find(ticket);
  if (it == S.requests.end()) return set_error(RB_ENOTFOUND, "rb_poll: unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second.get();
  if (!r->done) {
    if (timeout_us == 0) return RB_PENDING;
    if (timeout_us < 0) {
      S.cv.wait(lk, [&] { return r->done; });
    } else if (!S.cv.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
      return set_error(RB_ETIMEDOUT, "rb_poll: ticket %llu not done after %lld us", (unsigned long long)ticket,
                       (long long)timeout_us);
    }
  }
  const int status = r->status;
  if (status != RB_OK) set_error(status, "rb_poll: request failed: %s", r->msg);
  if (status == RB_OK) {
    if (logl_out) std::memcpy(logl_out, r->logl.data(), sizeof(double) * r->W);
    if (grad_out && r->want_grad) std::memcpy(grad_out, r->grad.data(), sizeof(double) * kNPar * r->W);
  }
  S.requests.erase(it);
  return status;
}

int rb_ticket_info(rb_server_t srv, uint64_t ticket, int64_t* W, int32_t* want_grad) {
  RB_NVTX("rb_ticket_info");
  if (!srv) return set_error(RB_EINVAL, "rb_ticket_info: NULL server");
  Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  auto it = S.requests.find(ticket);
  if (it == S.requests.end()) return set_error(RB_ENOTFOUND, "rb_ticket_info: unknown ticket %llu", (unsigned long long)ticket);
  if (W) *W = it->second->W;
  if (want_grad) *want_grad = it->second->want_grad ? 1 : 0;
  return RB_OK;
}

int rb_server_latency(rb_server_t srv, int part, int reset, int64_t* count, double* p50_ms, double* p99_ms,
                      double* max_ms) {
  RB_NVTX("rb_server_latency");
  if (!srv) return set_error(RB_EINVAL, "rb_server_latency: NULL server");
  if (part < 0 || part > 3) return set_error(RB_EINVAL, "rb_server_latency: part %d not in 0..3", part);
  Server& S = srv->s;
  std::vector<float> v;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    v = S.latency_us[part];
    if (reset)
      for (auto& x : S.latency_us) x.clear();
  }
  if (count) *count = (int64_t)v.size();
  double q[3] = {0.0, 0.0, 0.0};
  if (!v.empty()) {
    std::sort(v.begin(), v.end());
    const double fr[3] = {0.5, 0.99, 1.0};
    for (int i = 0; i < 3; ++i) {  // nearest rank
      size_t k = (size_t)std::ceil(fr[i] * (double)v.size());
      k = k < 1 ? 0 : k - 1;
      q[i] = v[k] / 1e3;
    }
  }
  if (p50_ms) *p50_ms = q[0];
  if (p99_ms) *p99_ms = q[1];
  if (max_ms) *max_ms = q[2];
  return RB_OK;
}

int rb_server_get_stats(rb_server_t srv, rb_server_stats* stats) {
  RB_NVTX("rb_server_get_stats");
  if (!srv || !stats) return set_error(RB_EINVAL, "rb_server_get_stats: NULL argument");
  Server& S = srv->s;
  std::lock_guard<std::mutex> lk(S.mu);
  *stats = S.stats;
  stats->in_flight = S.in_flight;
  stats->queued = (int32_t)S.pending.size();
  stats->hbm_in_use = S.hbm_in_use;
  return RB_OK;
}

}  // extern "C"
