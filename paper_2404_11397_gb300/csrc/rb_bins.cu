// rb_bins.cu -- bin placement without the PN ansatz (build time).
//
// The paper places the bin edges of relative binning (Sec. II.C) with a PN
// ansatz for the largest phase difference any waveform can have from the
// fiducial one, and its outlook (Sec. V) asks for bins built without prior
// assumptions about the waveform.  This placement takes the model's own
// phase directions instead of the ansatz's power laws:
//   w_j(f) = dPsi(f; theta_ref) / dtheta_j,  j = Mc, q, chi1, chi2, Lambda1,
//            Lambda2 (from the phase basis and the FP64 tangents at theta_ref)
//            and t_c (w = 2 pi f),
// gives each the same 2 pi of total variation across the band, and places the
// B + 1 edges uniformly in
//   M(f) = 2 pi sum_j V_j(f) / V_j(f_high),   V_j(f) = total variation of w_j on
//          [f_low, f] over the grid (sum of |w_j(f_k+1) - w_j(f_k)|),
// directions with no variation left out; epsilon = M(f_high) / B.  The edges
// are then snapped and made strictly increasing exactly as the PN placement's.
//
// Pipeline (one event build, FP64 throughout, every sum in a fixed order):
//   k_agn_increments  |w_j(f_k+1) - w_j(f_k)| per grid step and direction, the
//                     increments formed without cancellation (f^p expm1(p ln(f1/f0)))
//                     and per-block sums;
//   k_agn_totals      V_j(f_high) from the block sums;
//   k_agn_scan_local  dM_k = 2 pi sum_j inc_jk / V_j(f_high), scanned per block;
//   k_agn_scan_blocks exclusive scan of the block totals;
//   k_agn_measure     M on the grid;
//   k_agn_edges       the edges (as the PN placement), then the shared fix-up.
#include "rb_internal.cuh"

namespace rb {

constexpr int kAgnDirs = 7;  // Mc, q, chi1, chi2, Lambda1, Lambda2, t_c
constexpr int kAgnThreads = 256;

__device__ __forceinline__ double agn_f(int64_t kmin, int64_t k, double T) { return (double)(kmin + k) / T; }

// Block-wide sum of v over kAgnThreads threads in a fixed order (tree in
// shared memory); every thread returns the total.
__device__ double agn_block_sum(double v, double* red) {
  const int t = threadIdx.x;
  red[t] = v;
  __syncthreads();
  for (int s = kAgnThreads / 2; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kAgnThreads) k_agn_increments(int64_t kmin, int64_t N, double T,
                                                                const double* __restrict__ tng,
                                                                double* __restrict__ inc, double* __restrict__ part) {
  __shared__ double red[kAgnThreads];
  const int64_t k = (int64_t)blockIdx.x * kAgnThreads + threadIdx.x;
  const int64_t n_inc = N - 1;
  double a[kAgnDirs];
#pragma unroll
  for (int j = 0; j < kAgnDirs; ++j) a[j] = 0.0;
  if (k < n_inc) {
    const double f0 = agn_f(kmin, k, T), f1 = agn_f(kmin, k + 1, T);
    const double L1 = log1p((f1 - f0) / f0);  // ln(f1 / f0)
    const double lf = log(f0);
    const double c = cbrt(f0), ic = 1.0 / c, ic2 = ic * ic;
    // increments of the basis g = {f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3,
    // f^1/3 ln f, f^2/3, f^5/3, f^7/3} between f0 and f1: f0^p expm1(p L1)
    const double third = 1.0 / 3.0;
    const double d13 = c * expm1(third * L1);
    double dg[kNBasis];
    dg[0] = ic2 * ic2 * ic * expm1(-5.0 * third * L1);
    dg[1] = (1.0 / f0) * expm1(-L1);
    dg[2] = ic2 * expm1(-2.0 * third * L1);
    dg[3] = ic * expm1(-third * L1);
    dg[4] = L1;
    dg[5] = d13;
    dg[6] = d13 * (lf + L1) + c * L1;  // (a b)(f1) - (a b)(f0) with a = f^1/3, b = ln f
    dg[7] = c * c * expm1(2.0 * third * L1);
    dg[8] = f0 * c * c * expm1(5.0 * third * L1);
    dg[9] = f0 * f0 * c * expm1(7.0 * third * L1);
#pragma unroll
    for (int j = 0; j < kNTanIntr; ++j) {
      double w = 0.0;
#pragma unroll
      for (int q = 0; q < kNBasis; ++q) w = fma(tng[q * kNTanIntr + j], dg[q], w);
      a[j] = fabs(w);
    }
    a[6] = fabs(kTwoPi * f1 - kTwoPi * f0);
#pragma unroll
    for (int j = 0; j < kAgnDirs; ++j) inc[(size_t)j * n_inc + k] = a[j];
  }
#pragma unroll
  for (int j = 0; j < kAgnDirs; ++j) {
    const double s = agn_block_sum(a[j], red);
    if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = s;
  }
}

// V_j(f_high): warp j sums the block sums of direction j (lane-strided, then a
// fixed butterfly).
__global__ void k_agn_totals(int nblk, const double* __restrict__ part, double* __restrict__ vend) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j >= kAgnDirs) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(size_t)j * nblk + b];
  s = warp_sum_f64(s);
  if (lane == 0) vend[j] = s;
}

// dM_k = 2 pi sum_j inc_jk / V_j(f_high) and its inclusive scan within the block.
__global__ void __launch_bounds__(kAgnThreads) k_agn_scan_local(int64_t N, const double* __restrict__ inc,
                                                                const double* __restrict__ vend,
                                                                double* __restrict__ loc, double* __restrict__ bsum) {
  __shared__ double sc[kAgnThreads];
  const int t = threadIdx.x;
  const int64_t k = (int64_t)blockIdx.x * kAgnThreads + t;
  const int64_t n_inc = N - 1;
  double dm = 0.0;
  if (k < n_inc) {
#pragma unroll
    for (int j = 0; j < kAgnDirs; ++j) {
      const double v = vend[j];
      if (v > 0.0) dm += inc[(size_t)j * n_inc + k] / v;
    }
    dm *= kTwoPi;
  }
  sc[t] = dm;
  __syncthreads();
  for (int o = 1; o < kAgnThreads; o <<= 1) {  // Hillis-Steele: a fixed order of additions
    const double add = t >= o ? sc[t - o] : 0.0;
    __syncthreads();
    sc[t] += add;
    __syncthreads();
  }
  if (k < n_inc) loc[k] = sc[t];
  if (t == kAgnThreads - 1) bsum[blockIdx.x] = sc[t];
}

// Exclusive scan of the block totals, one block, in chunks of its size.
__global__ void __launch_bounds__(1024) k_agn_scan_blocks(int nblk, const double* __restrict__ bsum,
                                                          double* __restrict__ boff) {
  __shared__ double sc[1024];
  __shared__ double carry;
  const int t = threadIdx.x;
  if (t == 0) carry = 0.0;
  __syncthreads();
  for (int base = 0; base < nblk; base += 1024) {
    const int b = base + t;
    sc[t] = b < nblk ? bsum[b] : 0.0;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const double add = t >= o ? sc[t - o] : 0.0;
      __syncthreads();
      sc[t] += add;
      __syncthreads();
    }
    const double c0 = carry;
    if (b < nblk) boff[b] = c0 + (t > 0 ? sc[t - 1] : 0.0);
    __syncthreads();
    if (t == 1023) carry = c0 + sc[1023];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kAgnThreads) k_agn_measure(int64_t N, const double* __restrict__ loc,
                                                             const double* __restrict__ boff, double* __restrict__ M) {
  const int64_t k = (int64_t)blockIdx.x * kAgnThreads + threadIdx.x;
  if (k >= N) return;
  M[k] = k == 0 ? 0.0 : boff[(k - 1) / kAgnThreads] + loc[k - 1];
}

// Edge e at the target M[0] + (M[N-1] - M[0]) e / B: the largest k with
// M[k] <= target, linear interpolation to the next point, nearest of the two.
__global__ void k_agn_edges(int64_t N, int B, const double* __restrict__ M, int64_t* __restrict__ edges,
                            double* __restrict__ span) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > B) return;
  if (e == 0) {
    edges[0] = 0;
    *span = M[N - 1] - M[0];
    return;
  }
  if (e == B) { edges[B] = N - 1; return; }
  const double tau = M[0] + (M[N - 1] - M[0]) * (double)e / (double)B;
  int64_t lo = 0, hi = N;  // first index with M > tau lies in (lo - 1, hi]
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (M[mid] <= tau) lo = mid + 1; else hi = mid;
  }
  int64_t k = lo - 1;
  k = k < 0 ? 0 : (k > N - 2 ? N - 2 : k);
  const double frac = (tau - M[k]) / (M[k + 1] - M[k]);
  edges[e] = frac < 0.5 ? k : k + 1;
}

cudaError_t launch_ref_phase_tangents(const double* theta_ref_dev, double* out, cudaStream_t s);
cudaError_t launch_bin_edges_fix(int64_t N, int B, int64_t* edges, cudaStream_t s);

size_t bin_edges_agnostic_scratch_bytes(int64_t N) {
  const int64_t n_inc = N - 1;
  const int64_t nblk = (n_inc + kAgnThreads - 1) / kAgnThreads;
  return sizeof(double) * ((size_t)kAgnDirs * n_inc + n_inc + N + (size_t)kAgnDirs * nblk + 2 * nblk + kAgnDirs +
                           kNBasis * kNTanIntr);
}

// scratch: bin_edges_agnostic_scratch_bytes(N) of device memory, free after the
// stream reaches the end of these kernels; span: device double, M(f_high) - M(f_low).
cudaError_t launch_bin_edges_agnostic(const double* theta_ref_dev, double T, int64_t kmin, int64_t N, int B,
                                      int64_t* edges, double* span, void* scratch, cudaStream_t s) {
  const int64_t n_inc = N - 1;
  const int64_t nblk = (n_inc + kAgnThreads - 1) / kAgnThreads;
  double* inc = static_cast<double*>(scratch);
  double* loc = inc + (size_t)kAgnDirs * n_inc;
  double* M = loc + n_inc;
  double* part = M + N;
  double* bsum = part + (size_t)kAgnDirs * nblk;
  double* boff = bsum + nblk;
  double* vend = boff + nblk;
  double* tng = vend + kAgnDirs;
  cudaError_t err = launch_ref_phase_tangents(theta_ref_dev, tng, s);
  if (err != cudaSuccess) return err;
  k_agn_increments<<<(unsigned)nblk, kAgnThreads, 0, s>>>(kmin, N, T, tng, inc, part);
  k_agn_totals<<<1, kAgnDirs * 32, 0, s>>>((int)nblk, part, vend);
  k_agn_scan_local<<<(unsigned)nblk, kAgnThreads, 0, s>>>(N, inc, vend, loc, bsum);
  k_agn_scan_blocks<<<1, 1024, 0, s>>>((int)nblk, bsum, boff);
  k_agn_measure<<<(unsigned)((N + kAgnThreads - 1) / kAgnThreads), kAgnThreads, 0, s>>>(N, loc, boff, M);
  k_agn_edges<<<(B + 1 + 255) / 256, 256, 0, s>>>(N, B, M, edges, span);
  if ((err = cudaGetLastError()) != cudaSuccess) return err;
  return launch_bin_edges_fix(N, B, edges, s);
}

}  // namespace rb
