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

// ---------------------------------------------------------------------------
// Summary epilogue shared by the FP64 and fast kernels: from the six block
// sums (A0 re/im, A1 re/im, B0, B1 before the constant factors) lanes 0..5
// of warp 0 each finish one output (SIMT: the FP64 instructions are issued
// once for all six), write the FP64 summary entry and the bin tables
// (alpha0 = A0/2, alpha1 = A1/df_b, beta0 = B0/2, beta1 = B1/df_b), and the
// block's share Re A0 - B0/2 of log L(theta_ref).  The last block to finish
// sums the shares in a fixed order (deterministic).
// ---------------------------------------------------------------------------
__device__ void summary_epilogue(const SummaryOut& so, int b, int d, int B, int D, const double* sblock,
                                 const double* scale, bool scaled_form) {
  __shared__ bool last;
  if (threadIdx.x < 32) {
    const int j = threadIdx.x;
    double o = 0.0;
    if (j < 6) {
      o = sblock[j];
      if (scaled_form) {
        // A = conj(K) (s_re + i s_im) * scale[0];  B = |K|^2 s * scale[1]
        const double Kr = scale[2], Ki = scale[3];
        const double pr = sblock[j & ~1], pi = sblock[j | 1];
        if (j < 4) o = scale[0] * ((j & 1) ? (Kr * pi - Ki * pr) : (Kr * pr + Ki * pi));
        else o = scale[1] * (Kr * Kr + Ki * Ki) * o;
      }
      so.summ[((size_t)d * B + b) * 6 + j] = o;
      const double t = (j == 2 || j == 3 || j == 5) ? o * so.inv_df[b] : 0.5 * o;
      so.bin64[((size_t)d * 6 + j) * so.Bp + b] = t;
      so.bin32[((size_t)d * 6 + j) * so.Bp + b] = (float)t;
    }
    const double b0 = __shfl_sync(0xffffffffu, o, 4);
    if (j == 0) so.share[(size_t)d * B + b] = o - 0.5 * b0;
    if (j == 0) {
      __threadfence();
      const unsigned ticket = atomicAdd(so.counter, 1u);
      last = (ticket == (unsigned)(B * D) - 1u);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  __shared__ double part[32];
  const int n = B * D;
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += so.share[i];
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += part[i];
    *so.base = t;
    *so.counter = 0u;
  }
}

// One block per (bin, detector): FP64 fiducial waveform generated inline,
// FP64 accumulation, fixed-order block reduction (deterministic).
constexpr int kSumThreads = 128;
__global__ void __launch_bounds__(kSumThreads) k_summary(DataPtrs in, int64_t kmin, int64_t N, double T, int B, int D,
                                                         const int64_t* __restrict__ edges,
                                                         const RefValues* __restrict__ ref, SummaryOut so) {
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
  __shared__ double sblock[6];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 6; ++j) acc[j] = warp_sum_f64(acc[j]);
  if (lane == 0)
    for (int j = 0; j < 6; ++j) red[wid][j] = acc[j];
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int i = 0; i < kSumThreads / 32; ++i) t += red[i][threadIdx.x];
    sblock[threadIdx.x] = t;
  }
  __syncthreads();
  summary_epilogue(so, b, d, B, D, sblock, nullptr, false);
}

// ---------------------------------------------------------------------------
// Event-constant edge tables (built once per event): g_k(f_e) / 2pi as float
// pairs and FP64, f_e, and 1 / df_b per bin; pad entries are zero.
// ---------------------------------------------------------------------------
__global__ void k_edge_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp,
                              const int64_t* __restrict__ edges, float* __restrict__ tab32, size_t edge32_floats,
                              double* __restrict__ tab64, double* __restrict__ inv_df) {
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
  for (int b = tid; b < B; b += nth) inv_df[b] = T / (double)(edges[b + 1] - edges[b]);
  // bin tables: zero the padding once (the summary kernels write b < B)
  double* bin64 = tab64 + (size_t)(kNBasis + 1) * Ep;
  float* bin32 = tab32 + edge32_floats;
  for (int i = tid; i < D * 6 * Bp; i += nth) {
    bin64[i] = 0.0;
    bin32[i] = 0.f;
  }
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
                           const int64_t* edges, const RefValues* ref, const SummaryOut& so, cudaStream_t s) {
  dim3 grid(B, D);
  k_summary<<<grid, kSumThreads, 0, s>>>(in, kmin, N, T, B, D, edges, ref, so);
  return cudaGetLastError();
}

cudaError_t launch_edge_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp, const int64_t* edges,
                               float* tab32, size_t edge32_floats, double* tab64, double* inv_df, cudaStream_t s) {
  k_edge_tables<<<16, 256, 0, s>>>(kmin, T, D, B, Ep, Bp, edges, tab32, edge32_floats, tab64, inv_df);
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
// ln(1 + j u) for the two logarithmic terms.  The event-constant matrices
// Q_kn(c) = u^n P_k(f_c) (alpha_kn + beta_kn ln f_c) are built once per event
// in FP64 and stored as float pairs (orders 0-2) and floats (orders 3-8); a
// rebuild forms X_n(c) = sum_k (c_k / 2pi) Q_kn(c) with float-pair dot
// products on the FP32 pipe.  Each grid point then needs only FP32 and
// float-pair arithmetic: X0 + X1 j + X2 j^2 (float pairs) + j^3 (X3 + ... +
// X8 j^5) (FP32 Horner), reduction to [-1/2, 1/2] turns, the half-angle
// sin/cos, and the amplitude f^-7/6 = f_c^-7/6 (1 + j u)^-7/6 (FP32 series).
// With T f_low >= 1024 the truncated terms are below 1e-10 turns.  Strain
// and PSD are scaled by powers of two into FP32 range; per-thread partial
// sums are FP32, the block reduction is in float pairs, and the epilogue
// applies conj(K_d) and the scale factors in FP64.
// ===========================================================================
constexpr int kChunk = 32;
constexpr int kOrd = 8;

struct TaylorTables {
  double alpha[kNBasis][kOrd + 1];
  double beta6[kOrd + 1];  // ln f_c coefficient of the f^1/3 ln f term
  double amp[5];           // binom(-7/6, n)
};

// Event-constant per-chunk matrices, stored field-major ([field][chunk]) so
// that consecutive threads read consecutive chunks.  Fields:
constexpr int kQ01 = 0;                       // (k*2 + n)*2 + h: orders 0, 1 as float pairs
constexpr int kQ2 = kQ01 + kNBasis * 4;       // k*2 + h: order 2 as a float pair
constexpr int kQh = kQ2 + kNBasis * 2;        // (n-3)*10 + k: orders 3..8
constexpr int kQfc = kQh + (kOrd - 2) * kNBasis;  // f_c as a float pair
constexpr int kQamp = kQfc + 2;               // f_c^-7/6, binom(-7/6, n) u^n (n = 1..4)
constexpr int kQFields = kQamp + 5;
static_assert(kQFields <= 128, "chunk matrix fields");

// Per-rebuild chunk coefficients (128 bytes).
struct ChunkCoef {
  float x0[kMaxDet][2];   // X0 + f_c tau_d, reduced to [-1/2, 1/2] turns, float pair
  float x1[kMaxDet][2];   // X1 + df tau_d, float pair
  float x2[2];            // float pair
  float xh[kOrd - 2];     // X3 .. X8
  float amp[5];           // f_c^-7/6, then binom(-7/6, n) u^n, n = 1..4
  float pad[7];
};
static_assert(sizeof(ChunkCoef) == 128, "chunk record is one 128-byte line");

__global__ void __launch_bounds__(128) k_chunk_q(int64_t kmin, double T, int64_t n_chunks, TaylorTables tt,
                                                 float* __restrict__ q) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  auto put = [&](int f, float v) { q[(size_t)f * n_chunks + c] = v; };
  const double nc = (double)(kmin + c * kChunk + kChunk / 2);
  const double fc = nc / T, u = 1.0 / nc;
  const double cf = cbrt(fc), lf = log(fc), icf = 1.0 / cf, icf2 = icf * icf;
  const double P[kNBasis] = {icf2 * icf2 * icf, 1.0 / fc, icf2, icf, 1.0, cf, cf, cf * cf, fc * cf * cf, fc * fc * cf};
  double un = 1.0;
  for (int n = 0; n <= kOrd; ++n) {
    for (int k = 0; k < kNBasis; ++k) {
      double a = tt.alpha[k][n];
      if (k == 6) a += tt.beta6[n] * lf;
      if (k == 4 && n == 0) a = lf;
      const double v = un * P[k] * a;
      if (n < 2) {
        const f2x p = f2x_from(v);
        put(kQ01 + (k * 2 + n) * 2, p.hi);
        put(kQ01 + (k * 2 + n) * 2 + 1, p.lo);
      } else if (n == 2) {
        const f2x p = f2x_from(v);
        put(kQ2 + k * 2, p.hi);
        put(kQ2 + k * 2 + 1, p.lo);
      } else {
        put(kQh + (n - 3) * kNBasis + k, (float)v);
      }
    }
    un *= u;
  }
  const f2x fcp = f2x_from(fc);
  put(kQfc, fcp.hi);
  put(kQfc + 1, fcp.lo);
  put(kQamp, (float)(sqrt(icf) / fc));  // f_c^-7/6
  double ua = u;
  for (int n = 1; n < 5; ++n) {
    put(kQamp + n, (float)(tt.amp[n] * ua));
    ua *= u;
  }
}

__global__ void __launch_bounds__(128) k_chunk_coef(const RefValues* __restrict__ ref, const float* __restrict__ q,
                                                    float invT_hi, float invT_lo, int D, int64_t n_chunks,
                                                    ChunkCoef* __restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  const RefValues& r = *ref;
  auto get = [&](int f) { return q[(size_t)f * n_chunks + c]; };
  float x0h = r.phi0t[0], x0l = r.phi0t[1], x1h = 0.f, x1l = 0.f, x2h = 0.f, x2l = 0.f;
  float xh[kOrd - 2];
#pragma unroll
  for (int n = 0; n < kOrd - 2; ++n) xh[n] = 0.f;
#pragma unroll
  for (int k = 0; k < kNBasis; ++k) {
    const float ch = r.chat[k][0], cl = r.chat[k][1];
    f2x_fma_acc(ch, cl, get(kQ01 + k * 4), get(kQ01 + k * 4 + 1), x0h, x0l);
    f2x_fma_acc(ch, cl, get(kQ01 + k * 4 + 2), get(kQ01 + k * 4 + 3), x1h, x1l);
    f2x_fma_acc(ch, cl, get(kQ2 + k * 2), get(kQ2 + k * 2 + 1), x2h, x2l);
#pragma unroll
    for (int n = 0; n < kOrd - 2; ++n) xh[n] = fmaf(ch, get(kQh + n * kNBasis + k), xh[n]);
  }
  const float fch = get(kQfc), fcl = get(kQfc + 1);
  ChunkCoef o;
#pragma unroll
  for (int d = 0; d < kMaxDet; ++d) {
    if (d < D) {
      float ah = x0h, al = x0l;
      f2x_fma_acc(r.taut[d][0], r.taut[d][1], fch, fcl, ah, al);
      const float rh = __fadd_rn(ah, -round_fma_pipe(ah));  // exact: drop whole turns
      o.x0[d][0] = rh;
      o.x0[d][1] = al;
      float bh = x1h, bl = x1l;
      f2x_fma_acc(r.taut[d][0], r.taut[d][1], invT_hi, invT_lo, bh, bl);
      o.x1[d][0] = bh;
      o.x1[d][1] = bl;
    } else {
      o.x0[d][0] = o.x0[d][1] = o.x1[d][0] = o.x1[d][1] = 0.f;
    }
  }
  o.x2[0] = x2h;
  o.x2[1] = x2l;
#pragma unroll
  for (int n = 0; n < kOrd - 2; ++n) o.xh[n] = xh[n];
#pragma unroll
  for (int n = 0; n < 5; ++n) o.amp[n] = get(kQamp + n);
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

// One grid point of the fast summary sums.
__device__ __forceinline__ void fast_point(const ChunkCoef& C, int d, int64_t k, double2 dv, double psd, int sd,
                                           int sS, int64_t e01, float half_df, float* acc) {
  const float jf = (float)((int)(k & (kChunk - 1)) - kChunk / 2);
  const float dre = scaled_float(dv.x, sd), dim = scaled_float(dv.y, sd);
  const float Sp = scaled_float(psd, sS);
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
  const float dff = (float)(2 * k - e01) * half_df;  // f - f_m
  acc[0] += qr;
  acc[1] += qi;
  acc[2] = fmaf(qr, dff, acc[2]);
  acc[3] = fmaf(qi, dff, acc[3]);
  const float hh = wA * A;
  acc[4] += hh;
  acc[5] = fmaf(hh, dff, acc[5]);
}

constexpr int kFastThreads = 128;
constexpr int kFastUnroll = 4;
constexpr int kSeg = 1024;  // points per staged segment
__global__ void __launch_bounds__(kFastThreads) k_summary_fast(DataPtrs in, const ChunkCoef* __restrict__ ch,
                                                               double T, int B, int D,
                                                               const int64_t* __restrict__ edges,
                                                               const RefValues* __restrict__ ref, SummaryOut so) {
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
  // The bin is processed in segments of kSeg points; the segment's chunk
  // records are staged in shared memory first (coalesced 16-byte loads).
  __shared__ __align__(16) ChunkCoef sch[kSeg / kChunk + 1];
  for (int64_t s0 = k0; s0 < k1; s0 += kSeg) {
    const int64_t s1 = (s0 + kSeg < k1) ? s0 + kSeg : k1;
    const int64_t c0 = s0 >> 5, nch = ((s1 - 1) >> 5) - c0 + 1;
    {
      const float4* src = reinterpret_cast<const float4*>(ch + c0);
      float4* dst = reinterpret_cast<float4*>(sch);
      const int n4 = (int)nch * (int)(sizeof(ChunkCoef) / 16);
      for (int i = threadIdx.x; i < n4; i += kFastThreads) dst[i] = src[i];
    }
    __syncthreads();
    // issue the loads of kFastUnroll points before using any of them
    for (int64_t kb = s0 + threadIdx.x; kb < s1; kb += kFastThreads * kFastUnroll) {
      double2 dv[kFastUnroll];
      double pv[kFastUnroll];
#pragma unroll
      for (int u = 0; u < kFastUnroll; ++u) {
        const int64_t k = kb + (int64_t)u * kFastThreads;
        if (k < s1) {
          dv[u] = *reinterpret_cast<const double2*>(dat + 2 * k);
          pv[u] = psd[k];
        }
      }
#pragma unroll
      for (int u = 0; u < kFastUnroll; ++u) {
        const int64_t k = kb + (int64_t)u * kFastThreads;
        if (k < s1) fast_point(sch[(k >> 5) - c0], d, k, dv[u], pv[u], sd, sS, e0 + e1, half_df, acc);
      }
    }
    __syncthreads();
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
  __shared__ double sblock[6];
  __shared__ double scale[4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
    for (int j = 0; j < 6; ++j) {
      red[wid][j][0] = acc[j];
      red[wid][j][1] = lo[j];
    }
  __syncthreads();
  if (threadIdx.x < 6) {
    float h = red[0][threadIdx.x][0], l = red[0][threadIdx.x][1];
    for (int i = 1; i < kFastThreads / 32; ++i) {
      f2x_add(h, l, red[i][threadIdx.x][0]);
      l = __fadd_rn(l, red[i][threadIdx.x][1]);
    }
    sblock[threadIdx.x] = (double)h + (double)l;
  } else if (threadIdx.x >= 32 && threadIdx.x < 36) {
    const int j = threadIdx.x - 32;
    const double w4 = 4.0 / T;
    scale[j] = j == 0 ? ldexp(w4, sS - sd) : (j == 1 ? ldexp(w4, sS) : ref->K[d][j - 2]);
  }
  __syncthreads();
  summary_epilogue(so, b, d, B, D, sblock, scale, true);
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
    t.amp[n] = b;
    b *= (-7.0 / 6.0 - n) / (n + 1);
  }
  return t;
}

int64_t n_chunks_of(int64_t N) { return (N + kChunk - 1) / kChunk; }
size_t chunk_q_bytes(int64_t N) { return sizeof(float) * 128 * (size_t)n_chunks_of(N); }
size_t chunk_coef_bytes(int64_t N) { return sizeof(ChunkCoef) * (size_t)n_chunks_of(N); }

cudaError_t launch_chunk_q(int64_t kmin, double T, int64_t N, void* cq, cudaStream_t s) {
  static const TaylorTables tt = make_taylor_tables();
  const int64_t nc = n_chunks_of(N);
  k_chunk_q<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(kmin, T, nc, tt, static_cast<float*>(cq));
  return cudaGetLastError();
}

cudaError_t launch_summary_fast(const DataPtrs& in, int64_t N, double T, int D, int B, const int64_t* edges,
                                const RefValues* ref, const void* cq, void* chunk_coef, const SummaryOut& so,
                                cudaStream_t s) {
  const int64_t nc = n_chunks_of(N);
  ChunkCoef* ch = static_cast<ChunkCoef*>(chunk_coef);
  const double invT = 1.0 / T;
  const float ih = (float)invT, il = (float)(invT - (double)ih);
  k_chunk_coef<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(ref, static_cast<const float*>(cq), ih, il, D, nc, ch);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  dim3 grid(B, D);
  k_summary_fast<<<grid, kFastThreads, 0, s>>>(in, ch, T, B, D, edges, ref, so);
  return cudaGetLastError();
}

}  // namespace rb
