// rb_static.cu -- rb_loglike_grad_batch_static: the batched likelihood and
// gradient with its per-walker workspace in a fixed device array instead of
// memory taken from an allocator.
//
// Some callers cannot allocate device memory at the point where they need a
// likelihood: a host framework whose own allocator owns all device memory and
// forbids others from taking more, or a latency-critical sampler loop that
// must not pay for, or synchronise on, an allocation.  This entry point allocates nothing: the set-up kernel writes
// its per-walker records into g_static_ws, a file-scope __device__ array of
// RB_STATIC_MAX_WALKERS records of the largest layout (about 7.5 MiB), which
// every GPU that loads the library holds until the process exits.
//
// Host code cannot use g_static_ws's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and keeps it; make that first call before any stream
// capture.  Calls share the array: two calls whose kernels overlap on the GPU
// (different streams, or different host threads) race on it and must be
// ordered by the caller.  Nothing in the array needs to start at zero -- the
// set-up kernel writes every record the likelihood kernel reads -- and the
// array keeps the last call's records.
#include <cstdint>
#include <mutex>

#include "rb.h"
#include "rb_api_internal.h"
#include "rb_internal.cuh"

namespace rb {

constexpr size_t kStaticRecordBytes =
    (sizeof(WalkerF64) + sizeof(WalkerTan<double>)) > (sizeof(WalkerMixed) + sizeof(WalkerTan<float>))
        ? (sizeof(WalkerF64) + sizeof(WalkerTan<double>))
        : (sizeof(WalkerMixed) + sizeof(WalkerTan<float>));

static __device__ __align__(256) unsigned char g_static_ws[(size_t)RB_STATIC_MAX_WALKERS * kStaticRecordBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void* g_static_ptr[kMaxDevices];

static int static_workspace(void** out) {
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return cuda_fail(err, "rb_loglike_grad_batch_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(RB_EINVAL, "rb_loglike_grad_batch_static: device %d", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_static_ws);
    if (err != cudaSuccess) return cuda_fail(err, "rb_loglike_grad_batch_static: cudaGetSymbolAddress");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return RB_OK;
}

}  // namespace rb

extern "C" int rb_loglike_grad_batch_static(rb_event_t ev, const double* theta_dev, int64_t W, double* logl_dev,
                                            double* grad_dev, int mode, void* stream) {
  RB_NVTX("rb_loglike_grad_batch_static");
  if (!ev) return rb::set_error(RB_EINVAL, "rb_loglike_grad_batch_static: NULL event");
  if (W < 0) return rb::set_error(RB_EINVAL, "rb_loglike_grad_batch_static: W < 0");
  if (W > RB_STATIC_MAX_WALKERS)
    return rb::set_error(RB_EINVAL,
                         "rb_loglike_grad_batch_static: W=%lld exceeds the static workspace (%d walkers); "
                         "split the batch or use rb_loglike_grad_batch",
                         (long long)W, RB_STATIC_MAX_WALKERS);
  if (W == 0) return RB_OK;
  void* ws = nullptr;
  const int rc = rb::static_workspace(&ws);
  if (rc != RB_OK) return rc;
  return rb::run_batch(rb::event_entry(ev), theta_dev, W, logl_dev, grad_dev, mode, (cudaStream_t)stream, ws);
}
