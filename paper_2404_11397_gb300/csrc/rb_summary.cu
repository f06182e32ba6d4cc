// rb_summary.cu -- per-event set-up (step a7): bin edges, the fiducial
// waveform h0 on the full frequency grid, the summary data and the
// device-resident tables of the batch kernels.
//
// Summary data (Sec. II.C): for detector d and bin b with midpoint f_m(b),
//   A0 = 4 df sum_{k in b} d_k h0_k* / S_k,   A1 = 4 df sum d h0* (f_k - f_m) / S,
//   B0 = 4 df sum |h0_k|^2 / S_k,             B1 = 4 df sum |h0|^2 (f_k - f_m) / S.
// Bin placement (Sec. II.C and the epsilon <-> bin-count statement of
// Sec. IV.B, after Zackay et al. 2018): edges equally spaced in the PN phase
// bound dPsi_max(f) = 2 pi sum_g sgn(g) (f/f*_g)^g, g in {-5/3,-2/3,1,5/3,7/3},
// f* = f_low for g < 0 and f_high otherwise.
#include <algorithm>

#include "rb_internal.cuh"

namespace rb {

__device__ __forceinline__ double grid_f(int64_t kmin, int64_t k, double T) { return (double)(kmin + k) / T; }

__device__ double dpsi_max(double f, double f_low, double f_high) {
  const double gam[5] = {-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0};
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const double g = gam[i];
    const double fs = g < 0.0 ? f_low : f_high;
    s += (g < 0.0 ? -1.0 : 1.0) * pow(f / fs, g);
  }
  return 2.0 * kPi * s;
}

// One thread per interior edge: largest k with P(k) <= tau_e by bisection,
// then snap to the nearer of k, k+1 by linear interpolation.
__global__ void k_bin_edges(double f_low, double f_high, double T, int64_t kmin, int64_t N, int B,
                            int64_t* __restrict__ edges) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > B) return;
  if (e == 0) { edges[0] = 0; return; }
  if (e == B) { edges[B] = N - 1; return; }
  const double P0 = dpsi_max(grid_f(kmin, 0, T), f_low, f_high);
  const double PN = dpsi_max(grid_f(kmin, N - 1, T), f_low, f_high);
  const double tau = P0 + (PN - P0) * (double)e / (double)B;
  int64_t lo = 0, hi = N - 1;  // invariant: P(lo) <= tau (or lo = 0), P(hi) > tau (or hi = N-1)
  if (dpsi_max(grid_f(kmin, hi, T), f_low, f_high) <= tau) {
    lo = hi;
  } else {
    while (hi - lo > 1) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (dpsi_max(grid_f(kmin, mid, T), f_low, f_high) <= tau) lo = mid; else hi = mid;
    }
  }
  int64_t k = lo < N - 2 ? lo : N - 2;
  const double pk = dpsi_max(grid_f(kmin, k, T), f_low, f_high);
  const double pk1 = dpsi_max(grid_f(kmin, k + 1, T), f_low, f_high);
  const double frac = (tau - pk) / (pk1 - pk);
  edges[e] = frac < 0.5 ? k : k + 1;
}

// At least one grid point per bin: clamp into [e, N-1-(B-e)], then make the
// sequence strictly increasing (a running maximum, written as e + prefix max
// of edges[j] - j, computed by one warp).
__global__ void k_bin_edges_fix(int64_t N, int B, int64_t* __restrict__ edges) {
  const int lane = threadIdx.x;
  int64_t carry = INT64_MIN;  // running max of (edges[j] - j)
  for (int base = 0; base <= B; base += 32) {
    const int e = base + lane;
    int64_t v = INT64_MIN;
    if (e <= B) {
      int64_t x = edges[e];
      const int64_t lo = e, hi = N - 1 - (B - e);
      x = x < lo ? lo : (x > hi ? hi : x);
      v = x - e;
    }
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v = v > t ? v : t;
    }
    v = v > carry ? v : carry;
    if (e <= B) edges[e] = e + v;
    carry = __shfl_sync(0xffffffffu, v, 31);
  }
}

// Fiducial strain h_d(f) in FP64 from absolute source values.
__device__ __forceinline__ void strain_f64(const Values& v, int d, double f, double& hr, double& hi) {
  const double lf = log(f);
  const double cf = cbrt(f);
  const double icf = 1.0 / cf;
  const double icf2 = icf * icf;
  const double g[kNBasis] = {icf2 * icf2 * icf, 1.0 / f, icf2, icf, lf, cf, cf * lf, cf * cf, f * cf * cf,
                             f * f * cf};
  double psi = v.phi0 + kTwoPi * f * v.tau[d];
#pragma unroll
  for (int k = 0; k < kNBasis; ++k) psi = fma(v.c[k], g[k], psi);
  // A f^{-7/6}, A = sqrt(5/24) pi^{-2/3} Mc^{5/6} / d_L with Mc, d_L in seconds:
  // sqrt(5/24) pi^{-2/3} (G Msun/c^3)^{5/6} = 8.035028173395984e-06 s^{5/6}
  const double kamp = 8.035028173395984e-06 / kMpcS;
  const double a = kamp * v.amp / (f * sqrt(cf));
  double s, c;
  sincos(psi, &s, &c);
  const double P = v.P64[d][0], Q = v.P64[d][1];
  // a (P + iQ)(c - i s)
  hr = a * (P * c + Q * s);
  hi = a * (Q * c - P * s);
}

// One block per (bin, detector): FP64 fiducial waveform generated inline,
// FP64 accumulation, fixed-order block reduction (deterministic).
constexpr int kSumThreads = 128;
__global__ void __launch_bounds__(kSumThreads) k_summary(DataPtrs in, int64_t kmin, int64_t N, double T, int B,
                                                         const int64_t* __restrict__ edges,
                                                         const RefValues* __restrict__ ref, double* __restrict__ out) {
  const int b = blockIdx.x, d = blockIdx.y;
  const Values& v = ref->v;
  const int64_t k0 = edges[b];
  const int64_t k1 = (b == B - 1) ? edges[b + 1] + 1 : edges[b + 1];
  const double fm = 0.5 * (grid_f(kmin, edges[b], T) + grid_f(kmin, edges[b + 1], T));
  const double w0 = 4.0 / T;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (int64_t k = k0 + threadIdx.x; k < k1; k += blockDim.x) {
    const double f = grid_f(kmin, k, T);
    double hr, hi;
    strain_f64(v, d, f, hr, hi);
    const double dr = in.data[d][2 * k], di = in.data[d][2 * k + 1];
    const double w = w0 / in.psd[d][k];
    const double xr = dr * hr + di * hi, xi = di * hr - dr * hi, hh = hr * hr + hi * hi;
    const double df = f - fm;
    acc[0] += w * xr;
    acc[1] += w * xi;
    acc[2] += w * xr * df;
    acc[3] += w * xi * df;
    acc[4] += w * hh;
    acc[5] += w * hh * df;
  }
  __shared__ double red[kSumThreads / 32][6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 6; ++j) acc[j] = warp_sum_f64(acc[j]);
  if (lane == 0)
    for (int j = 0; j < 6; ++j) red[wid][j] = acc[j];
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int i = 0; i < kSumThreads / 32; ++i) s += red[i][threadIdx.x];
    // out layout: [D][B][6] = A0r, A0i, A1r, A1i, B0, B1
    out[((size_t)d * B + b) * 6 + threadIdx.x] = s;
  }
}

// Edge and bin tables for the batch kernels, and the fiducial log-likelihood.
__global__ void k_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp, const int64_t* __restrict__ edges,
                         const double* __restrict__ summ, float* __restrict__ tab32, size_t edge32_floats,
                         double* __restrict__ tab64) {
  const int E = B + 1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const double inv2pi = 1.0 / kTwoPi;
  for (int e = tid; e < Ep; e += nth) {
    double g[kNBasis], f = 0.0;
    if (e < E) {
      f = grid_f(kmin, edges[e], T);
      const double lf = log(f), cf = cbrt(f), icf = 1.0 / cf, icf2 = icf * icf;
      const double gg[kNBasis] = {icf2 * icf2 * icf, 1.0 / f, icf2, icf, lf, cf, cf * lf, cf * cf, f * cf * cf,
                                  f * f * cf};
      for (int k = 0; k < kNBasis; ++k) g[k] = gg[k] * inv2pi;
    } else {
      for (int k = 0; k < kNBasis; ++k) g[k] = 0.0;
    }
    for (int k = 0; k < kNBasis; ++k) {
      tab64[(size_t)k * Ep + e] = g[k];
      const f2x p = f2x_from(g[k]);
      tab32[(size_t)k * Ep + e] = p.hi;
      tab32[(size_t)(kNBasis + k) * Ep + e] = p.lo;
    }
    tab64[(size_t)kNBasis * Ep + e] = f;
    const f2x fp = f2x_from(f);
    tab32[(size_t)2 * kNBasis * Ep + e] = fp.hi;
    tab32[(size_t)(2 * kNBasis + 1) * Ep + e] = fp.lo;
  }
  double* bin64 = tab64 + (size_t)(kNBasis + 1) * Ep;
  float* bin32 = tab32 + edge32_floats;
  for (int i = tid; i < D * Bp; i += nth) {
    const int d = i / Bp, b = i % Bp;
    double v[6] = {0, 0, 0, 0, 0, 0};
    if (b < B) {
      const double* s = summ + ((size_t)d * B + b) * 6;
      const double idf = 1.0 / (grid_f(kmin, edges[b + 1], T) - grid_f(kmin, edges[b], T));
      v[0] = 0.5 * s[0];
      v[1] = 0.5 * s[1];
      v[2] = s[2] * idf;
      v[3] = s[3] * idf;
      v[4] = 0.5 * s[4];
      v[5] = s[5] * idf;
    }
    for (int j = 0; j < 6; ++j) {
      bin64[((size_t)d * 6 + j) * Bp + b] = v[j];
      bin32[((size_t)d * 6 + j) * Bp + b] = (float)v[j];
    }
  }
}

// base = sum_d sum_b (Re A0 - B0/2), one warp, fixed summation order.
__global__ void k_base_logl(int D, int B, const double* __restrict__ summ, double* __restrict__ out) {
  double s = 0.0;
  for (int i = threadIdx.x; i < D * B; i += 32) s += summ[(size_t)i * 6 + 0] - 0.5 * summ[(size_t)i * 6 + 4];
  s = warp_sum_f64(s);
  if (threadIdx.x == 0) *out = s;
}

// Detector strain for one source on a grid (FP64).
__global__ void k_strain(const RefValues* __restrict__ src, int64_t kmin, int64_t N, double T,
                         double* __restrict__ h) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  const Values& v = src->v;
  if (!v.valid) {
    h[2 * k] = h[2 * k + 1] = nan("");
    return;
  }
  double hr, hi;
  strain_f64(v, 0, grid_f(kmin, k, T), hr, hi);
  h[2 * k] = hr;
  h[2 * k + 1] = hi;
}

// ---------------------------------------------------------------------------
cudaError_t launch_bin_edges(double f_low, double f_high, double T, int64_t kmin, int64_t N, int B, int64_t* edges,
                             cudaStream_t s) {
  const int bs = 32;
  k_bin_edges<<<(B + 1 + bs - 1) / bs, bs, 0, s>>>(f_low, f_high, T, kmin, N, B, edges);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_bin_edges_fix<<<1, 32, 0, s>>>(N, B, edges);
  return cudaGetLastError();
}

cudaError_t launch_summary(const DataPtrs& in, int64_t kmin, int64_t N, double T, int D, int B,
                           const int64_t* edges, const RefValues* ref, double* out, cudaStream_t s) {
  dim3 grid(B, D);
  k_summary<<<grid, kSumThreads, 0, s>>>(in, kmin, N, T, B, edges, ref, out);
  return cudaGetLastError();
}

cudaError_t launch_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp, const int64_t* edges,
                          const double* summ, float* tab32, size_t edge32_floats, double* tab64, double* base,
                          cudaStream_t s) {
  k_tables<<<64, 256, 0, s>>>(kmin, T, D, B, Ep, Bp, edges, summ, tab32, edge32_floats, tab64);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  k_base_logl<<<1, 32, 0, s>>>(D, B, summ, base);
  return cudaGetLastError();
}

cudaError_t launch_strain(const RefValues* src, int64_t kmin, int64_t N, double T, double* h, cudaStream_t s) {
  const int bs = 256;
  k_strain<<<(unsigned)((N + bs - 1) / bs), bs, 0, s>>>(src, kmin, N, T, h);
  return cudaGetLastError();
}

}  // namespace rb
