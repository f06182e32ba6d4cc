// rb_server.cu -- continuous-batching request loop over resident events.
//
// Clients call rb_submit from any thread; a scheduler thread admits pending
// requests in arrival order whenever a slot (a CUDA stream with pinned and
// device staging buffers) is free and the request's device footprint fits in
// the remaining budget.  Admitted requests run concurrently on their slots'
// streams, so work that arrives while others are on the GPU starts as soon as
// resources free up.  Each launch replays a CUDA graph captured once per
// (slot, event, walker bucket, gradient flag): copy-in, per-walker set-up,
// likelihood kernel, copy-out and a host node that hands the results back.
// Requests are padded to a power-of-two walker bucket with copies of their
// first walker; every walker is computed independently by one warp, so each
// result is bit-identical to the same request evaluated alone.
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "rb.h"
#include "rb_api_internal.h"

namespace rb {

struct Request {
  uint64_t ticket = 0;
  const EventEntry* ev = nullptr;
  int64_t W = 0, bucket = 0;
  bool want_grad = false;
  size_t footprint = 0;
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
  Request* req = nullptr;
  std::map<std::tuple<uint64_t, int64_t, bool>, cudaGraphExec_t> graphs;
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
  std::thread thread;

  void run();
  int launch(Slot* s, Request* r);
  void complete(Slot* s);
};

static void CUDART_CB slot_done(void* p) {
  Slot* s = static_cast<Slot*>(p);
  s->srv->complete(s);
}

void Server::complete(Slot* s) {
  std::lock_guard<std::mutex> lk(mu);
  Request* r = s->req;
  if (r) {
    std::memcpy(r->logl.data(), s->h_logl, sizeof(double) * r->W);
    if (r->want_grad) std::memcpy(r->grad.data(), s->h_grad, sizeof(double) * kNPar * r->W);
    r->status = RB_OK;
    r->done = true;
    hbm_in_use -= r->footprint;
    --in_flight;
    ++stats.completed;
  }
  s->req = nullptr;
  free_slots.push_back(s);
  cv.notify_all();
}

// Issue copy-in, set-up + likelihood kernels, copy-out and the completion
// host node on the slot's stream (captured into a graph when enabled).
static int enqueue_work(Slot* s, const EventEntry* ev, int64_t bucket, bool grad, int mode) {
  cudaError_t err = cudaMemcpyAsync(s->d_theta, s->h_theta, sizeof(double) * kNPar * bucket, cudaMemcpyHostToDevice,
                                    s->stream);
  if (err != cudaSuccess) return cuda_fail(err, "server copy-in");
  int rc = run_batch(ev, s->d_theta, bucket, s->d_logl, grad ? s->d_grad : nullptr, mode, s->stream, s->d_ws);
  if (rc != RB_OK) return rc;
  if ((err = cudaMemcpyAsync(s->h_logl, s->d_logl, sizeof(double) * bucket, cudaMemcpyDeviceToHost, s->stream)) !=
      cudaSuccess)
    return cuda_fail(err, "server copy-out");
  if (grad && (err = cudaMemcpyAsync(s->h_grad, s->d_grad, sizeof(double) * kNPar * bucket, cudaMemcpyDeviceToHost,
                                     s->stream)) != cudaSuccess)
    return cuda_fail(err, "server copy-out grad");
  if ((err = cudaLaunchHostFunc(s->stream, slot_done, s)) != cudaSuccess) return cuda_fail(err, "server host node");
  return RB_OK;
}

int Server::launch(Slot* s, Request* r) {
  std::memcpy(s->h_theta, r->theta.data(), sizeof(double) * kNPar * r->W);
  for (int64_t w = r->W; w < r->bucket; ++w)  // pad with the first walker
    std::memcpy(s->h_theta + kNPar * w, r->theta.data(), sizeof(double) * kNPar);
  if (!opts.use_graphs) {
    ++stats.plain_launches;
    return enqueue_work(s, r->ev, r->bucket, r->want_grad, opts.mode);
  }
  const auto key = std::make_tuple(r->ev->uid, r->bucket, r->want_grad);
  auto it = s->graphs.find(key);
  cudaGraphExec_t exec = nullptr;
  if (it == s->graphs.end()) {
    cudaGraph_t graph = nullptr;
    cudaError_t err = cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeRelaxed);
    if (err != cudaSuccess) return cuda_fail(err, "begin capture");
    int rc = enqueue_work(s, r->ev, r->bucket, r->want_grad, opts.mode);
    err = cudaStreamEndCapture(s->stream, &graph);
    if (rc != RB_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (err != cudaSuccess) return cuda_fail(err, "end capture");
    err = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (err != cudaSuccess) return cuda_fail(err, "graph instantiate");
    s->graphs.emplace(key, exec);
    ++stats.graphs_captured;
  } else {
    exec = it->second;
  }
  cudaError_t err = cudaGraphLaunch(exec, s->stream);
  if (err != cudaSuccess) return cuda_fail(err, "graph launch");
  ++stats.graph_launches;
  count_launches(2);
  return RB_OK;
}

void Server::run() {
  std::unique_lock<std::mutex> lk(mu);
  for (;;) {
    cv.wait(lk, [&] {
      if (stopping) return true;
      if (pending.empty() || free_slots.empty()) return false;
      const Request* r = pending.front();
      return hbm_in_use + r->footprint <= opts.hbm_budget_bytes || in_flight == 0;
    });
    if (stopping) break;
    Request* r = pending.front();
    pending.pop_front();
    Slot* s = free_slots.back();
    free_slots.pop_back();
    s->req = r;
    hbm_in_use += r->footprint;
    ++in_flight;
    if (in_flight > stats.max_in_flight) stats.max_in_flight = in_flight;
    lk.unlock();
    const int rc = launch(s, r);
    lk.lock();
    if (rc != RB_OK) {
      // the host node never ran: release here
      std::snprintf(r->msg, sizeof(r->msg), "%s", rb_last_error());
      r->status = rc;
      r->done = true;
      hbm_in_use -= r->footprint;
      --in_flight;
      s->req = nullptr;
      free_slots.push_back(s);
      cv.notify_all();
    }
  }
  // wait for in-flight work, then fail whatever is still pending
  cv.wait(lk, [&] { return in_flight == 0; });
  for (Request* r : pending) {
    r->status = RB_ECLOSED;
    std::snprintf(r->msg, sizeof(r->msg), "server shut down before the request ran");
    r->done = true;
  }
  pending.clear();
  cv.notify_all();
}

static int64_t bucket_of(int64_t W, int64_t max_w) {
  int64_t b = 256;
  while (b < W) b <<= 1;
  return b < max_w ? b : max_w;
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
  // slot buffers hold the largest bucket
  const int64_t cap = bucket_of(o.max_walkers, (int64_t)1 << 40);
  o.max_walkers = cap;
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
  for (auto& sl : S.slots) {
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
  r->bucket = bucket_of(W, S.opts.max_walkers);
  r->want_grad = want_grad != 0;
  r->footprint = S.bytes_per_walker * r->bucket;
  r->theta.assign(theta_host, theta_host + kNPar * W);
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
