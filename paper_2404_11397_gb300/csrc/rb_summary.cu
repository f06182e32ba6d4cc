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


// ===========================================================================
// Fast summary build for the mixed-precision path.
//
// The fiducial phase in turns, x_d(f) = [Phi0 + sum_k c_k g_k(f)] / 2pi
// + f tau_d, is expanded around the centre f_c of every 32-point chunk of
// the grid, f = f_c (1 + j u) with u = df / f_c and j = k - k_c in [-16, 15]:
//   g_k(f_c (1 + j u)) = P_k(f_c) sum_n (alpha_kn + beta_kn ln f_c) (j u)^n,
// the binomial series of the PN power laws (alpha = binom(p_k, n)) and of
// ln(1 + j u) for the two logarithmic terms.  The coefficients X_n of j^n are
// formed once per chunk in FP64 (orders 0-3; orders 4-8 in FP32, where the
// terms are below 1e-5 turns), and each grid point then needs only FP32 and
// float-pair arithmetic: X0 + X1 j + X2 j^2 (float pairs) + j^3 (X3 + ... +
// X8 j^5) (FP32 Horner), reduction to [-1/2, 1/2] turns, the half-angle
// sin/cos, and the amplitude f^-7/6 = f_c^-7/6 (1 + j u)^-7/6 (FP32 series).
// With T f_low >= 1024 the truncated terms are below 1e-10 turns.  Strain
// and PSD are scaled by powers of two into FP32 range; per-thread partial
// sums are FP32, the block reduction is in float pairs, and the epilogue
// applies conj(K_d) = conj(A_ref P_d) and the scale factors in FP64.
// ===========================================================================
constexpr int kChunk = 32;
constexpr int kOrd = 8;

struct TaylorTables {
  double alpha[kNBasis][kOrd + 1];
  double beta6[kOrd + 1];  // ln f_c coefficient of the f^1/3 ln f term
  float amp[5];            // binom(-7/6, n)
};

struct ChunkCoef {
  float x0[kMaxDet][2];   // X0 + f_c tau_d, reduced to [-1/2, 1/2] turns, float pair
  float x1[kMaxDet][2];   // X1 + df tau_d, float pair
  float x2[2];            // float pair
  float xh[kOrd - 2];     // X3 .. X8
  float amp[5];           // f_c^-7/6, then binom(-7/6, n) u^n, n = 1..4
  float pad[7];
};
static_assert(sizeof(ChunkCoef) == 128, "chunk record is one 128-byte line");

__global__ void __launch_bounds__(128) k_chunk_coef(const RefValues* __restrict__ ref, int64_t kmin, double T, int D,
                                                    int64_t n_chunks, TaylorTables tt, ChunkCoef* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const Values& v = ref->v;
  const double nc = (double)(kmin + c * kChunk + kChunk / 2);
  const double fc = nc / T, u = 1.0 / nc;
  const double cf = cbrt(fc), lf = log(fc), icf = 1.0 / cf, icf2 = icf * icf;
  const double P[kNBasis] = {icf2 * icf2 * icf, 1.0 / fc, icf2, icf, 1.0, cf, cf, cf * cf, fc * cf * cf, fc * fc * cf};
  double vk[kNBasis];
#pragma unroll
  for (int k = 0; k < kNBasis; ++k) vk[k] = v.c[k] * (1.0 / kTwoPi) * P[k];
  double X[4];
  double un = 1.0;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    double s = lf * vk[6] * tt.beta6[n];
#pragma unroll
    for (int k = 0; k < kNBasis; ++k) s = fma(vk[k], tt.alpha[k][n], s);
    if (n == 0) s = fma(lf, vk[4], s);
    X[n] = s * un;
    un *= u;
  }
  ChunkCoef o;
  float vf[kNBasis];
#pragma unroll
  for (int k = 0; k < kNBasis; ++k) vf[k] = (float)vk[k];
  const float lff = (float)lf;
  float unf = (float)un;  // u^4
  const float uf = (float)u;
#pragma unroll
  for (int n = 4; n <= kOrd; ++n) {
    float s = lff * vf[6] * (float)tt.beta6[n];
#pragma unroll
    for (int k = 0; k < kNBasis; ++k) s = fmaf(vf[k], (float)tt.alpha[k][n], s);
    o.xh[n - 3] = s * unf;
    unf *= uf;
  }
  const double x0 = X[0] + v.phi0 * (1.0 / kTwoPi);
  for (int d = 0; d < kMaxDet; ++d) {
    if (d < D) {
      double a = fma(fc, v.tau[d], x0);
      a -= rint(a);
      const f2x p0 = f2x_from(a), p1 = f2x_from(X[1] + v.tau[d] / T);
      o.x0[d][0] = p0.hi;
      o.x0[d][1] = p0.lo;
      o.x1[d][0] = p1.hi;
      o.x1[d][1] = p1.lo;
    } else {
      o.x0[d][0] = o.x0[d][1] = o.x1[d][0] = o.x1[d][1] = 0.f;
    }
  }
  const f2x p2 = f2x_from(X[2]);
  o.x2[0] = p2.hi;
  o.x2[1] = p2.lo;
  o.xh[0] = (float)X[3];
  o.amp[0] = (float)(sqrt(icf) / fc);  // f_c^-7/6
  float ua = uf;
#pragma unroll
  for (int n = 1; n < 5; ++n) {
    o.amp[n] = tt.amp[n] * ua;
    ua *= uf;
  }
#pragma unroll
  for (int i = 0; i < 7; ++i) o.pad[i] = 0.f;
  out[c] = o;
}

// FP64 -> FP32 of x * 2^s with integer operations only (the FP64 -> FP32
// conversion instruction runs on the FP64 pipe, ~1/70 of the FP32 rate):
// shift the exponent, keep the top 23 mantissa bits and round on the next
// bit.  Zero and subnormal inputs give a signed zero, overflow gives inf.
__device__ __forceinline__ float scaled_float(double x, int s) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned sign = (unsigned)hi & 0x80000000u;
  const int e = ((hi >> 20) & 0x7FF) - 1023 + 127 + s;
  const unsigned m = (((unsigned)hi & 0xFFFFFu) << 3) | (lo >> 29);
  const unsigned bits = (sign | ((unsigned)e << 23) | m) + ((lo >> 28) & 1u);
  return __int_as_float((int)(e <= 0 ? sign : (e >= 255 ? (sign | 0x7f800000u) : bits)));
}

__device__ __forceinline__ void f2x_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fadd_rn(s, -hi);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bb)), __fadd_rn(v, -bb)));
  hi = s;
}

constexpr int kFastThreads = 128;
__global__ void __launch_bounds__(kFastThreads) k_summary_fast(DataPtrs in, const ChunkCoef* __restrict__ ch,
                                                               int64_t kmin, int64_t N, double T, int B,
                                                               const int64_t* __restrict__ edges,
                                                               const RefValues* __restrict__ ref,
                                                               double* __restrict__ out) {
  const int b = blockIdx.x, d = blockIdx.y;
  const int64_t e0 = edges[b], e1 = edges[b + 1];
  const int64_t k0 = e0;
  const int64_t k1 = (b == B - 1) ? e1 + 1 : e1;
  const double* __restrict__ dat = in.data[d];
  const double* __restrict__ psd = in.psd[d];
  // power-of-two scales from the first PSD sample: S' = S 2^sS ~ 1, d' = d 2^sd
  const int ex = ((__double2hiint(psd[0]) >> 20) & 0x7FF) - 1023;
  const int sS = -ex, sd = -(ex / 2);
  const float half_df = (float)(0.5 / T);
  float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (int64_t k = k0 + threadIdx.x; k < k1; k += kFastThreads) {
    const ChunkCoef& C = ch[k >> 5];
    const float jf = (float)((int)(k & (kChunk - 1)) - kChunk / 2);
    const double2 dv = *reinterpret_cast<const double2*>(dat + 2 * k);
    const float dre = scaled_float(dv.x, sd), dim = scaled_float(dv.y, sd);
    const float Sp = scaled_float(psd[k], sS);
    // phase in turns: float pairs for X0 + X1 j + X2 j^2, FP32 for the rest
    float t = C.xh[5];
#pragma unroll
    for (int n = 4; n >= 0; --n) t = fmaf(t, jf, C.xh[n]);
    const float j2 = jf * jf;
    const float t3 = t * (j2 * jf);
    const float p1 = __fmul_rn(C.x1[d][0], jf);
    float e1e = __fmaf_rn(C.x1[d][0], jf, -p1);
    e1e = __fmaf_rn(C.x1[d][1], jf, e1e);
    const float p2 = __fmul_rn(C.x2[0], j2);
    float e2e = __fmaf_rn(C.x2[0], j2, -p2);
    e2e = __fmaf_rn(C.x2[1], j2, e2e);
    float sh = C.x0[d][0], sl = C.x0[d][1];
    f2x_add(sh, sl, p1);
    f2x_add(sh, sl, p2);
    sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e1e, e2e), t3));
    const float y = frac_turns(sh, sl);
    float sn, cs;
    sincos_pi_half(y, sn, cs);
    const float Cc = fmaf(-2.f * sn, sn, 1.f), Ss = 2.f * sn * cs;  // exp(+2 pi i y)
    const float A = C.amp[0] * fmaf(jf, fmaf(jf, fmaf(jf, fmaf(jf, C.amp[4], C.amp[3]), C.amp[2]), C.amp[1]), 1.f);
    const float wA = A / Sp;
    const float dr = dre * wA, di = dim * wA;
    const float qr = fmaf(dr, Cc, -di * Ss), qi = fmaf(dr, Ss, di * Cc);
    const float dff = (float)(2 * k - e0 - e1) * half_df;  // f - f_m
    acc[0] += qr;
    acc[1] += qi;
    acc[2] = fmaf(qr, dff, acc[2]);
    acc[3] = fmaf(qi, dff, acc[3]);
    const float hh = wA * A;
    acc[4] += hh;
    acc[5] = fmaf(hh, dff, acc[5]);
  }
  // float-pair block reduction (fixed order)
  float lo[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      const float oh = __shfl_xor_sync(0xffffffffu, acc[j], o);
      const float ol = __shfl_xor_sync(0xffffffffu, lo[j], o);
      f2x_add(acc[j], lo[j], oh);
      lo[j] = __fadd_rn(lo[j], ol);
    }
  }
  __shared__ float red[kFastThreads / 32][6][2];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int j = 0; j < 6; ++j) {
      red[wid][j][0] = acc[j];
      red[wid][j][1] = lo[j];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s[6];
    for (int j = 0; j < 6; ++j) {
      double t = 0.0;
      for (int i = 0; i < kFastThreads / 32; ++i) t += (double)red[i][j][0] + (double)red[i][j][1];
      s[j] = t;
    }
    const Values& v = ref->v;
    const double kamp = 8.035028173395984e-06 / kMpcS;
    const double a = kamp * v.amp;
    const double Kr = a * v.P64[d][0], Ki = a * v.P64[d][1];
    const double w4 = 4.0 / T;
    const double sq = ldexp(w4, sS - sd), sb = ldexp(w4, sS);
    double* o = out + ((size_t)d * B + b) * 6;
    // conj(K) (s0 + i s1)
    o[0] = sq * (Kr * s[0] + Ki * s[1]);
    o[1] = sq * (Kr * s[1] - Ki * s[0]);
    o[2] = sq * (Kr * s[2] + Ki * s[3]);
    o[3] = sq * (Kr * s[3] - Ki * s[2]);
    const double K2 = Kr * Kr + Ki * Ki;
    o[4] = sb * K2 * s[4];
    o[5] = sb * K2 * s[5];
  }
}

static TaylorTables make_taylor_tables() {
  TaylorTables t{};
  const double p[kNBasis] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, 0.0, 1.0 / 3.0, 1.0 / 3.0, 2.0 / 3.0,
                             5.0 / 3.0, 7.0 / 3.0};
  for (int k = 0; k < kNBasis; ++k) {
    double b = 1.0;  // binom(p, n)
    for (int n = 0; n <= kOrd; ++n) {
      t.alpha[k][n] = b;
      b *= (p[k] - n) / (n + 1);
    }
  }
  // ln f = ln f_c + sum_{n>=1} (-1)^{n+1} (j u)^n / n
  for (int n = 0; n <= kOrd; ++n) t.alpha[4][n] = (n == 0) ? 0.0 : ((n % 2) ? 1.0 : -1.0) / n;
  // f^1/3 ln f = f_c^1/3 (1+ju)^1/3 (ln f_c + ln(1+ju))
  double b13[kOrd + 1];
  b13[0] = 1.0;
  for (int n = 1; n <= kOrd; ++n) b13[n] = b13[n - 1] * (1.0 / 3.0 - (n - 1)) / n;
  for (int n = 0; n <= kOrd; ++n) {
    double s = 0.0;
    for (int m = 1; m <= n; ++m) s += b13[n - m] * (((m % 2) ? 1.0 : -1.0) / m);
    t.alpha[6][n] = s;
    t.beta6[n] = b13[n];
  }
  double b = 1.0;
  for (int n = 0; n < 5; ++n) {
    t.amp[n] = (float)b;
    b *= (-7.0 / 6.0 - n) / (n + 1);
  }
  return t;
}

size_t chunk_scratch_bytes(int64_t N) { return sizeof(ChunkCoef) * (size_t)((N + kChunk - 1) / kChunk); }

cudaError_t launch_summary_fast(const DataPtrs& in, int64_t kmin, int64_t N, double T, int D, int B,
                                const int64_t* edges, const RefValues* ref, void* chunk_scratch, double* out,
                                cudaStream_t s) {
  static const TaylorTables tt = make_taylor_tables();
  const int64_t n_chunks = (N + kChunk - 1) / kChunk;
  ChunkCoef* ch = static_cast<ChunkCoef*>(chunk_scratch);
  k_chunk_coef<<<(unsigned)((n_chunks + 127) / 128), 128, 0, s>>>(ref, kmin, T, D, n_chunks, tt, ch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  dim3 grid(B, D);
  k_summary_fast<<<grid, kFastThreads, 0, s>>>(in, ch, kmin, N, T, B, edges, ref, out);
  return cudaGetLastError();
}

}  // namespace rb
