// rb_mala.cu -- the MALA local step of the sampler (Sec. II.D: flowMC's local
// sampler is the Metropolis-adjusted Langevin algorithm) for W chains, on the
// device, fused with the likelihood and its adjoint.
//
// Sampling coordinates (Table II): z = (Mc, q, chi1, chi2, Lambda1, Lambda2,
// d_L, t_c, phi_c, cos iota, psi, ra, sin dec) with the uniform prior of the
// table on an open box lo < z < hi, so log pi(z) = log L(theta(z)) (+ const)
// inside and -inf outside.  With step sizes eps_j and draws xi ~ N(0, 1), u ~ U(0, 1):
//   z'        = z + eps^2/2 grad log pi(z) + eps xi                (k_mala_propose)
//   log L(theta(z')) and d log L / d theta                         (set-up + batch kernel)
//   log alpha = log pi(z') - log pi(z) - 1/2 sum_j [(xi_j + eps_j (g_j + g'_j)/2)^2 - xi_j^2]
//   accept if log u < log alpha, state updated in place            (batch kernel epilogue)
// The draws are inputs, so the step is reproducible.
#include <cmath>
#include <cstdint>

#include "rb.h"
#include "rb_api_internal.h"
#include "rb_internal.cuh"

namespace rb {

struct MalaBox {
  double eps[kNPar], lo[kNPar], hi[kNPar];
};

// Proposal, box test, likelihood parameters theta(z') (theta(z) of the
// current state for a proposal outside the box: it is evaluated but
// rejected), log u and the Jacobian factors of the two angle coordinates at
// the proposal.  A block of four warps takes 32 chains, lane = chain, so every
// FP64 instruction runs on full warps (the FP64 pipe issues per warp):
// warp k forms the proposals of parameters k, k + 4, ...; after the box test,
// the four warps evaluate acos (warp 0), asin (1), the Jacobian factors (2)
// and log u (3) side by side.
constexpr int kProposeThreads = 128;
__global__ void __launch_bounds__(kProposeThreads) k_mala_propose(const double* __restrict__ z,
                                                                 const double* __restrict__ gz,
                                                                 const double* __restrict__ xi,
                                                                 const double* __restrict__ u, MalaBox box, int64_t W,
                                                                 int init, double* __restrict__ zp,
                                                                 double* __restrict__ theta, double* __restrict__ lu,
                                                                 double* __restrict__ jac, int* __restrict__ inside) {
  __shared__ double sp[kNPar][32], sc[kNPar][32];  // proposal and current state of the block's chains
  __shared__ int sok[kNPar][32];
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  const int64_t w = (int64_t)blockIdx.x * 32 + lane;
  const bool live = w < W;
  for (int j = k; j < kNPar; j += kProposeThreads / 32) {
    double c = 0.0, p = 0.0;
    bool ok = true;
    if (live) {
      const int64_t i = w * kNPar + j;
      c = z[i];
      p = init ? c : c + 0.5 * box.eps[j] * box.eps[j] * gz[i] + box.eps[j] * xi[i];
      ok = p > box.lo[j] && p < box.hi[j];
      zp[i] = p;
    }
    sp[j][lane] = p;
    sc[j][lane] = c;
    sok[j][lane] = ok ? 1 : 0;
  }
  __syncthreads();
  if (!live) return;
  bool in = true;
#pragma unroll
  for (int j = 0; j < kNPar; ++j) in = in && sok[j][lane];
  if (k == 0) {
    for (int j = 0; j < kNPar; ++j) {  // all but parameter 12 (warp 1)
      if (j == 12) continue;
      const double src = in ? sp[j][lane] : sc[j][lane];
      theta[w * kNPar + j] = j == 9 ? acos(src) : src;
    }
  } else if (k == 1) {
    theta[w * kNPar + 12] = asin(in ? sp[12][lane] : sc[12][lane]);
  } else if (k == 2) {
    // d iota / d cos iota = -1 / sin iota, d dec / d sin dec = 1 / cos dec
    // (1 - z^2 as (1 - z)(1 + z): no cancellation next to the box edges)
    const double p9 = sp[9][lane], p12 = sp[12][lane];
    jac[2 * w] = in ? -1.0 / sqrt((1.0 - p9) * (1.0 + p9)) : 0.0;
    jac[2 * w + 1] = in ? 1.0 / sqrt((1.0 - p12) * (1.0 + p12)) : 0.0;
  } else {
    lu[w] = init ? 0.0 : log(u[w]);
    inside[w] = in ? 1 : 0;
  }
}

// Per-chain workspace of a MALA call (bytes per chain, without the batch's).
static size_t mala_ws_bytes() { return sizeof(double) * (2 * kNPar + 1 + 2) + 2 * sizeof(int); }

static int mala_run(rb_event_t ev, double* z, double* logp, double* gz, int64_t W, const double* eps_host,
                    const double* lo_host, const double* hi_host, const double* xi, const double* u, int* accepted,
                    int mode, void* stream, bool init, const char* who) {
  if (!ev) return set_error(RB_EINVAL, "%s: NULL event", who);
  if (W < 0) return set_error(RB_EINVAL, "%s: W < 0", who);
  if (W == 0) return RB_OK;
  if (!z || !logp || !gz || !lo_host || !hi_host) return set_error(RB_EINVAL, "%s: NULL argument", who);
  if (!init && (!eps_host || !xi || !u)) return set_error(RB_EINVAL, "%s: NULL eps, xi or u", who);
  if (mode != RB_MIXED && mode != RB_FP64 && mode != RB_MIXED_F64PHASE) return set_error(RB_EINVAL, "%s: bad mode %d", who, mode);
  MalaBox box;
  for (int j = 0; j < kNPar; ++j) {
    box.eps[j] = init ? 0.0 : eps_host[j];
    box.lo[j] = lo_host[j];
    box.hi[j] = hi_host[j];
    if (!(box.lo[j] < box.hi[j])) return set_error(RB_EINVAL, "%s: empty prior interval for parameter %d", who, j);
    if (!init && !(box.eps[j] >= 0.0)) return set_error(RB_EINVAL, "%s: step size %d must be >= 0", who, j);
  }
  if (box.lo[9] < -1.0 || box.hi[9] > 1.0 || box.lo[12] < -1.0 || box.hi[12] > 1.0)
    return set_error(RB_EINVAL, "%s: cos iota and sin dec bounds must lie in [-1, 1]", who);
  const EventEntry* e = event_entry(ev);
  cudaStream_t s = (cudaStream_t)stream;
  char* buf = nullptr;
  const size_t per = mala_ws_bytes();
  cudaError_t err = ws_alloc(reinterpret_cast<void**>(&buf), per * W, s);
  if (err != cudaSuccess) return cuda_fail(err, "MALA workspace allocation");
  double* zp = reinterpret_cast<double*>(buf);
  double* theta = zp + kNPar * W;
  double* lu = theta + kNPar * W;
  double* jac = lu + W;
  int* inside = reinterpret_cast<int*>(jac + 2 * W);
  int* acc_scratch = inside + W;
  k_mala_propose<<<(unsigned)((W + 31) / 32), kProposeThreads, 0, s>>>(z, gz, xi, u, box, W, init ? 1 : 0, zp, theta,
                                                                       lu, jac, inside);
  err = cudaGetLastError();
  int rc = RB_OK;
  if (err != cudaSuccess) {
    rc = cuda_fail(err, "MALA proposal kernel");
  } else {
    count_launches(1);
    MalaArgs m{};
    m.z = z;
    m.zp = zp;
    m.logp = logp;
    m.gz = gz;
    m.xi = init ? zp : xi;  // unused terms when init (eps = 0)
    m.lu = lu;
    m.jac = jac;
    m.inside = inside;
    m.accepted = accepted ? accepted : acc_scratch;
    for (int j = 0; j < kNPar; ++j) m.eps[j] = box.eps[j];
    m.init = init ? 1 : 0;
    rc = run_batch(e, theta, W, nullptr, nullptr, mode, s, nullptr, &m);
  }
  cudaFreeAsync(buf, s);
  return rc;
}

}  // namespace rb

extern "C" int rb_mala_init(rb_event_t ev, const double* z_dev, int64_t W, const double* lo_host,
                            const double* hi_host, double* logp_dev, double* gz_dev, int mode, void* stream) {
  RB_NVTX("rb_mala_init");
  return rb::mala_run(ev, const_cast<double*>(z_dev), logp_dev, gz_dev, W, nullptr, lo_host, hi_host, nullptr,
                      nullptr, nullptr, mode, stream, true, "rb_mala_init");
}

extern "C" int rb_mala_step(rb_event_t ev, double* z_dev, double* logp_dev, double* gz_dev, int64_t W,
                            const double* eps_host, const double* lo_host, const double* hi_host, const double* xi_dev,
                            const double* u_dev, int* accepted_dev, int mode, void* stream) {
  RB_NVTX("rb_mala_step");
  return rb::mala_run(ev, z_dev, logp_dev, gz_dev, W, eps_host, lo_host, hi_host, xi_dev, u_dev, accepted_dev, mode,
                      stream, false, "rb_mala_step");
}
