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
                            int64_t* __restrict__ edges, double* __restrict__ span) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > B) return;
  if (e == 0) {
    edges[0] = 0;
    if (span) *span = dpsi_max(grid_f(kmin, N - 1, T), f_low, f_high) - dpsi_max(grid_f(kmin, 0, T), f_low, f_high);
    return;
  }
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
// Summary epilogue shared by the FP64 and fast kernels: from the block sums
// of nd detectors d0 .. d0+nd-1 (six each: A0 re/im, A1 re/im, B0, B1 before
// the constant factors), lane j < 6 nd of warp 0 finishes output j % 6 of
// detector d0 + j / 6 (SIMT: the FP64 instructions are issued once for all),
// writes the FP64 summary entry and the bin tables (alpha0 = A0/2,
// alpha1 = A1/df_b, beta0 = B0/2, beta1 = B1/df_b), and each detector's share
// Re A0 - B0/2 of log L(theta_ref).  log L(theta_ref) is the sum of all
// shares, formed deterministically in one of two ways:
//   fixed_base = false: the last of the n_blocks blocks to finish sums the
//     D x B shares in a fixed order (FP64);
//   fixed_base = true: every block adds its bin's share (over the nd
//     detectors) to a 64-bit fixed-point accumulator (2^-32 units; integer
//     addition does not depend on the order) and the last block converts it;
//     if a share does not fit (|share| >= 2^31) the last block falls back to
//     the fixed-order FP64 sum;
//   fixed_base = true, ticket = false (fast build): no block waits to find the
//     last one: the accumulator (zeroed by the reference-value kernel at the
//     start of the build) is converted by its readers (event_base_logl).
// ---------------------------------------------------------------------------
__device__ void summary_epilogue(const SummaryOut& so, int b, int d0, int nd, int B, int D, const double* sblock,
                                 const double* scale, bool scaled_form, unsigned n_blocks, double inv_df_b,
                                 bool fixed_base, bool ticket = true) {
  __shared__ bool last;
  SummarySync* sy = so.sync;
  if (threadIdx.x < 32) {
    const int j = threadIdx.x;
    const int g = j / 6, f = j - 6 * g, d = d0 + g;
    const bool mine = j < 6 * nd;
    double o = 0.0, t = 0.0;
    if (mine) {
      o = sblock[j];
      if (scaled_form) {
        // A = conj(K) (s_re + i s_im) * scale[0];  B = |K|^2 s * scale[1]
        const double* sc = scale + 4 * g;
        const double Kr = sc[2], Ki = sc[3];
        const double pr = sblock[6 * g + (f & ~1)], pi = sblock[6 * g + (f | 1)];
        if (f < 4) o = sc[0] * ((f & 1) ? (Kr * pi - Ki * pr) : (Kr * pr + Ki * pi));
        else o = sc[1] * (Kr * Kr + Ki * Ki) * o;
      }
      so.summ[((size_t)d * B + b) * 6 + f] = o;
      t = (f == 2 || f == 3 || f == 5) ? o * inv_df_b : 0.5 * o;
      so.bin64[((size_t)d * 6 + f) * so.Bp + b] = t;
      // float image (layout in EventDev), with beta0 and beta1 negated
      const float t32 = (float)(f >= 4 ? -t : t);
      const size_t Bp = so.Bp;
      if (D >= 2 && d < 2)  // detector pair: quad f/2 holds {x_0, x_1, y_0, y_1} of fields (f&~1, f|1)
        so.bin32[((size_t)(f >> 1) * Bp + b) * 4 + (f & 1) * 2 + d] = t32;
      else {                // the single detector D - 1
        const size_t base = (D >= 2) ? 12 * Bp : 0;
        so.bin32[f < 4 ? base + (size_t)b * 4 + f : base + 4 * Bp + (size_t)b * 2 + (f - 4)] = t32;
      }
    }
    // slot image: bin b is half h of slot sl; lane 6 g + m (m < 6) of the
    // detector's six lanes writes entry m of {gmr, gpr, gmi, gpi, h, q}
    {
      double tv[5];
#pragma unroll
      for (int m = 0; m < 5; ++m) tv[m] = __shfl_sync(0xffffffffu, t, (6 * g + m) & 31);
      if (mine) {
        const double a0r = tv[0], a0i = tv[1], a1r = tv[2], a1i = tv[3], b0 = tv[4];
        const double val = f == 0 ? a0r - b0 - a1r : f == 1 ? a0r - b0 + a1r : f == 2 ? a0i - a1i
                         : f == 3 ? a0i + a1i : f == 4 ? -0.5 * b0 : -0.25 * b0;
        const int it = b / kSlotBins, r = b - kSlotBins * it, h = r & 1, sl = 32 * it + (r >> 1);
        const size_t NS = so.n_slots;
        float* sb = so.slot_bin32 + (size_t)d * kSlotBinFloats * NS;
        sb[((size_t)(f >> 1) * NS + sl) * 4 + (f & 1) * 2 + h] = (float)val;
      }
    }
    const double b0 = __shfl_sync(0xffffffffu, o, (6 * g + 4) & 31);
    const double sh = (mine && f == 0) ? o - 0.5 * b0 : 0.0;
    if (mine && f == 0) so.share[(size_t)d * B + b] = sh;
    if (fixed_base) {
      double tot = __shfl_sync(0xffffffffu, sh, 0);  // detectors in order
      for (int g2 = 1; g2 < nd; ++g2) tot += __shfl_sync(0xffffffffu, sh, 6 * g2);
      if (j == 0) {
        if (fabs(tot) < 2147483648.0)
          atomicAdd(&sy->base_acc, (unsigned long long)__double2ll_rn(tot * 4294967296.0));
        else
          atomicOr(&sy->overflow, 1u);
      }
    }
    if (!ticket) return;
    fence_acq_rel_gpu();
    __syncwarp();
    if (j == 0) {
      const unsigned done = atomicAdd(&sy->counter, 1u);
      last = (done == n_blocks - 1u);
    }
  }
  if (!ticket) return;
  __syncthreads();
  if (!last) return;
  fence_acq_rel_gpu();
  if (fixed_base && *reinterpret_cast<volatile unsigned*>(&sy->overflow) == 0u) {
    if (threadIdx.x == 0) {
      const unsigned long long acc = atomicExch(&sy->base_acc, 0ull);
      *so.base = (double)(long long)acc * (1.0 / 4294967296.0);
      sy->base_in_acc = 0u;
      sy->counter = 0u;
    }
    return;
  }
  __shared__ double part[32];
  const int n = B * D;
  // loads first (up to 8 per thread in flight), then a pairwise tree
  double acc = 0.0;
  for (int i0 = threadIdx.x; i0 < n; i0 += 8 * blockDim.x) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      v[u] = i < n ? __ldcg(so.share + i) : 0.0;
    }
    acc += ((v[0] + v[1]) + (v[2] + v[3])) + ((v[4] + v[5]) + (v[6] + v[7]));
  }
  acc = warp_sum_f64(acc);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = (int)(blockDim.x >> 5);
    double t = 0.0;
    for (int i = 0; i < nw; ++i) t += part[i];
    *so.base = t;
    sy->base_in_acc = 0u;
    sy->counter = 0u;
    sy->overflow = 0u;
    sy->base_acc = 0ull;
  }
}

// One block per (bin, detector): FP64 fiducial waveform generated inline,
// FP64 accumulation, fixed-order block reduction (deterministic).
constexpr int kSumThreads = 128;
__global__ void __launch_bounds__(kSumThreads) k_summary(DataPtrs in, int64_t kmin, int64_t N, double T, int B, int D,
                                                         const int64_t* __restrict__ edges,
                                                         const RefValues* __restrict__ ref, SummaryOut so,
                                                         double* __restrict__ h0_out) {
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
    if (h0_out) __stcs(reinterpret_cast<double2*>(h0_out) + (size_t)d * N + k, make_double2(hr, hi));
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
  summary_epilogue(so, b, d, 1, B, D, sblock, nullptr, false, (unsigned)(B * D), so.inv_df[b], false);
}

// ---------------------------------------------------------------------------
// Event-constant edge tables (built once per event): g_k(f_e) / 2pi as float
// pairs and FP64, f_e, and 1 / df_b per bin; pad entries are zero.  The same
// values go to the edge part of the slot image (layout in EventDev).
// ---------------------------------------------------------------------------
// g_k(f_e) / 2pi and f_e of edge e (zero past the last edge).
__device__ void edge_basis(int64_t kmin, double T, int E, const int64_t* __restrict__ edges, int e, double (&g)[kNBasis],
                           double& f) {
  f = 0.0;
  for (int k = 0; k < kNBasis; ++k) g[k] = 0.0;
  if (e >= E) return;
  f = grid_f(kmin, edges[e], T);
  const double lf = log(f), cf = cbrt(f), icf = 1.0 / cf, icf2 = icf * icf;
  const double gg[kNBasis] = {icf2 * icf2 * icf, 1.0 / f, icf2, icf, lf, cf, cf * lf, cf * cf, f * cf * cf, f * f * cf};
  const double inv2pi = 1.0 / kTwoPi;
  for (int k = 0; k < kNBasis; ++k) g[k] = gg[k] * inv2pi;
}

__global__ void k_edge_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp,
                              const int64_t* __restrict__ edges, float* __restrict__ tab32, size_t edge32_floats,
                              double* __restrict__ tab64, double* __restrict__ inv_df, float* __restrict__ slot32,
                              int NS) {
  const int E = B + 1;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int e = tid; e < Ep; e += nth) {
    double g[kNBasis], f;
    edge_basis(kmin, T, E, edges, e, g, f);
    float4* t4 = reinterpret_cast<float4*>(tab32);  // [kEdgeQuads][Ep]
    for (int q = 0; q < kNBasis / 2; ++q) {
      tab64[(size_t)(2 * q) * Ep + e] = g[2 * q];
      tab64[(size_t)(2 * q + 1) * Ep + e] = g[2 * q + 1];
      const f2x p0 = f2x_from(g[2 * q]), p1 = f2x_from(g[2 * q + 1]);
      t4[(size_t)q * Ep + e] = make_float4(p0.hi, p1.hi, p0.lo, p1.lo);
    }
    tab64[(size_t)kNBasis * Ep + e] = f;
    const f2x fp = f2x_from(f);
    t4[(size_t)(kEdgeQuads - 1) * Ep + e] = make_float4(fp.hi, fp.lo, 0.f, 0.f);
  }
  // slot image, edge part: slot s = 32 i + l, half h holds edge 63 i + 2 l + h
  for (int t = tid; t < 2 * NS; t += nth) {
    const int sl = t >> 1, h = t & 1;
    const int e = kSlotBins * (sl >> 5) + 2 * (sl & 31) + h;
    double g[kNBasis], f;
    edge_basis(kmin, T, E, edges, e, g, f);
    for (int k = 0; k <= kNBasis; ++k) {
      const f2x v = f2x_from(k < kNBasis ? g[k] : f);
      slot32[((size_t)k * NS + sl) * 4 + h] = v.hi;
      slot32[((size_t)k * NS + sl) * 4 + 2 + h] = v.lo;
    }
  }
  for (int b = tid; b < B; b += nth) inv_df[b] = T / (double)(edges[b + 1] - edges[b]);
  // bin tables: zero the padding once (the summary kernels write b < B)
  double* bin64 = tab64 + (size_t)(kNBasis + 1) * Ep;
  float* bin32 = tab32 + edge32_floats;
  for (int i = tid; i < D * 6 * Bp; i += nth) {
    bin64[i] = 0.0;
    bin32[i] = 0.f;
  }
  float* slot_bins = slot32 + (size_t)4 * (kNBasis + 1) * NS;
  for (int i = tid; i < D * kSlotBinFloats * NS; i += nth) slot_bins[i] = 0.f;
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
cudaError_t launch_bin_edges_fix(int64_t N, int B, int64_t* edges, cudaStream_t s) {
  k_bin_edges_fix<<<1, 32, 0, s>>>(N, B, edges);
  return cudaGetLastError();
}

// span (device, may be NULL): the phase bound's range over the band, so that
// epsilon = span / B.
cudaError_t launch_bin_edges(double f_low, double f_high, double T, int64_t kmin, int64_t N, int B, int64_t* edges,
                             double* span, cudaStream_t s) {
  const int bs = 32;
  k_bin_edges<<<(B + 1 + bs - 1) / bs, bs, 0, s>>>(f_low, f_high, T, kmin, N, B, edges, span);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  return launch_bin_edges_fix(N, B, edges, s);
}

cudaError_t launch_summary(const DataPtrs& in, int64_t kmin, int64_t N, double T, int D, int B,
                           const int64_t* edges, const RefValues* ref, const SummaryOut& so, double* h0_out,
                           cudaStream_t s) {
  dim3 grid(B, D);
  k_summary<<<grid, kSumThreads, 0, s>>>(in, kmin, N, T, B, D, edges, ref, so, h0_out);
  return cudaGetLastError();
}

// FP64 summary sums from the stored fiducial waveform h0_d(f) (written by
// k_summary for the current theta_ref): the build then streams the strain,
// the PSD and h0, 40 B per (point, detector), with no waveform arithmetic.
// One block of kStoredThreads per part of a bin (the fast build's parts), all
// detectors; the per-point terms are k_summary's, with f = (kmin + k) (1/T)
// and 1/S from rcp_newton in place of the two FP64 divisions (the FP64 pipe
// is the bound); block sums in a fixed order, the parts of a bin added in index order by the
// last of them to finish, which runs the FP64 epilogue (base log L by the
// fixed-point sum).  Several warps per part keep enough FP64 work in flight
// to cover the FP64 pipe's latency.
constexpr int kStoredThreads = 128;

// 1/S for a positive normal double by Newton-Raphson iteration for the
// reciprocal, r <- r + r (1 - S r), which doubles the correct bits per step:
// the seed is the FP32 reciprocal of S scaled to [1, 2) (built and moved back
// to FP64 with integer operations, ~23 correct bits), two steps give FP64
// accuracy (within 1 ulp).  Four FP64 FMAs in all; inputs outside
// [2^-1022, 2^1021) take the division.
__device__ __forceinline__ double rcp_newton(double S) {
  const unsigned hi = (unsigned)__double2hiint(S), lo = (unsigned)__double2loint(S);
  const int ef = (int)((hi >> 20) & 0x7FFu);
  // zero, subnormal, infinite or NaN, negative, or so large (>= 2^1021) that
  // 1/S is at the subnormal edge: the division
  if (ef == 0 || ef >= 0x7FC || (hi >> 31)) return 1.0 / S;
  const float s1 = __uint_as_float(0x3F800000u | ((hi & 0xFFFFFu) << 3) | (lo >> 29));  // S 2^-e, truncated
  const unsigned rb = __float_as_uint(__frcp_rn(s1));  // in (0.5, 1]
  const int er = (int)((rb >> 23) & 0xFFu) - 127;
  const unsigned m = rb & 0x7FFFFFu;
  double r = __hiloint2double((int)(((unsigned)(er + 1023 - (ef - 1023)) << 20) | (m >> 3)), (int)((m & 7u) << 29));
  r = fma(r, fma(-S, r, 1.0), r);
  r = fma(r, fma(-S, r, 1.0), r);
  return r;
}

template <int ND>
__global__ void __launch_bounds__(kStoredThreads) k_summary_stored(DataPtrs in, const double* __restrict__ h0,
                                                                   int64_t kmin, int64_t N, double T, int B,
                                                                   const int64_t* __restrict__ edges, SummaryOut so) {
  __shared__ double red[6 * ND][kStoredThreads];  // per-thread sums, one row per quantity
  __shared__ double qsum[6 * kMaxDet];
  __shared__ double sblock[6 * kMaxDet];
  __shared__ bool s_last;
  const int pid = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const PartDesc pd = so.parts[RB_IDX(pid, so.n_parts, 201)];
  const int b = pd.bin;
  const double fm = 0.5 * (grid_f(kmin, edges[b], T) + grid_f(kmin, edges[b + 1], T));
  const double inv_T = 1.0 / T;
  double acc[ND][6];
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int j = 0; j < 6; ++j) acc[d][j] = 0.0;
  // sums of the terms over S; the factor 4 df = 4 / T is applied to the sums
  for (int64_t k = pd.start + tid; k < pd.end; k += kStoredThreads) {
    const double f = (double)(kmin + k) * inv_T;
    const double df = f - fm;
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      const double2 dv = __ldcs(reinterpret_cast<const double2*>(in.data[d]) + RB_IDX(k, N, 222));
      const double2 hv = __ldcs(reinterpret_cast<const double2*>(h0) + (size_t)d * N + RB_IDX(k, N, 222));
      const double w = rcp_newton(__ldcs(in.psd[d] + k));
      const double hr = hv.x, hi = hv.y, dr = dv.x, di = dv.y;
      const double xr = dr * hr + di * hi, xi = di * hr - dr * hi, hh = hr * hr + hi * hi;
      acc[d][0] += w * xr;
      acc[d][1] += w * xi;
      acc[d][2] += w * xr * df;
      acc[d][3] += w * xi * df;
      acc[d][4] += w * hh;
      acc[d][5] += w * hh * df;
    }
  }
  // block sums in a fixed order: warp w takes quantities w, w + 4, ...; each
  // lane adds the 4 threads l, l + 32, l + 64, l + 96, then a shuffle tree
#pragma unroll
  for (int d = 0; d < ND; ++d)
#pragma unroll
    for (int j = 0; j < 6; ++j) red[6 * d + j][tid] = acc[d][j];
  __syncthreads();
  for (int q = wid; q < 6 * ND; q += kStoredThreads / 32) {
    double v = red[q][lane];
#pragma unroll
    for (int i = 1; i < kStoredThreads / 32; ++i) v += red[q][lane + 32 * i];
    v = warp_sum_f64(v);
    if (lane == 0) qsum[q] = 4.0 * inv_T * v;
  }
  __syncthreads();
  double mine = tid < 6 * ND ? qsum[tid] : 0.0;
  if (pd.n_parts > 1) {
    double* ps = reinterpret_cast<double*>(so.part_sums);  // [n_parts][kPartSlots] doubles
    if (tid < 6 * ND) ps[(size_t)pid * kPartSlots + tid] = mine;
    fence_acq_rel_gpu();
    __syncthreads();
    if (tid == 0) {
      const unsigned ticket = atomicAdd(&so.sync->bin_parts_done[b], 1u);
      s_last = (ticket == (unsigned)pd.n_parts - 1u);
      if (s_last) so.sync->bin_parts_done[b] = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    fence_acq_rel_gpu();
    if (tid < 6 * ND) {
      const double* p0 = ps + (size_t)pd.first * kPartSlots + tid;
      double t = __ldcg(p0);
      for (int p = 1; p < pd.n_parts; ++p) t += __ldcg(p0 + (size_t)p * kPartSlots);
      mine = t;
    }
  }
  if (tid < 6 * ND) sblock[tid] = mine;
  __syncthreads();
  summary_epilogue(so, b, 0, ND, B, ND, sblock, nullptr, false, (unsigned)B, so.inv_df[b], true);
}

cudaError_t launch_summary_stored(const DataPtrs& in, const double* h0, int64_t kmin, int64_t N, double T, int D, int B,
                                  const int64_t* edges, const SummaryOut& so, int n_parts, cudaStream_t s) {
  auto kf = D == 1 ? k_summary_stored<1> : D == 2 ? k_summary_stored<2> : k_summary_stored<3>;
  kf<<<(unsigned)n_parts, kStoredThreads, 0, s>>>(in, h0, kmin, N, T, B, edges, so);
  return cudaGetLastError();
}

cudaError_t launch_edge_tables(int64_t kmin, double T, int D, int B, int Ep, int Bp, const int64_t* edges,
                               float* tab32, size_t edge32_floats, double* tab64, double* inv_df, float* slot32,
                               int n_slots, cudaStream_t s) {
  k_edge_tables<<<16, 256, 0, s>>>(kmin, T, D, B, Ep, Bp, edges, tab32, edge32_floats, tab64, inv_df, slot32, n_slots);
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

struct TaylorTables {
  double alpha[kNBasis][kOrd + 1];
  double beta6[kOrd + 1];  // ln f_c coefficient of the f^1/3 ln f term
  double amp[5];           // binom(-7/6, n)
};


__global__ void __launch_bounds__(128) k_chunk_q(int64_t kmin, double T, int64_t n_chunks, TaylorTables tt,
                                                 float* __restrict__ q) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_chunks) return;
  auto put = [&](int f, float v) { q[(size_t)c * kQRow + f] = v; };
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

// FP64 -> FP32 of x * 2^s with integer operations only (the FP64 -> FP32
// conversion instruction issues on the FP64 pipe): subtract the exponent
// offset from the magnitude word, round the 64-bit magnitude on the first
// dropped bit, and shift the top 32 bits into FP32 position.  `bias` is
// (896 - s) << 20; zero and results below the FP32 normal range give a
// signed zero, results above it give inf.
__device__ __forceinline__ float scaled_float(double x, unsigned bias) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned mag = hi & 0x7FFFFFFFu;
  unsigned rlo, rhi;
  asm("add.cc.u32 %0, %2, 0x10000000;\n\taddc.u32 %1, %3, 0;" : "=r"(rlo), "=r"(rhi) : "r"(lo), "r"(mag));
  const unsigned bits = __funnelshift_l(rlo, rhi - bias, 3) | sign;
  const unsigned lo_lim = bias + (1u << 20), hi_lim = bias + (255u << 20);
  return __uint_as_float(mag < lo_lim ? sign : (mag >= hi_lim ? (sign | 0x7F800000u) : bits));
}

// Per-rebuild chunk coefficients (32 floats, 16-byte aligned groups):
//   [0 .. 3]    X0 (pair, whole turns dropped), X1 (pair): intrinsic phase
//   [4 .. 11]   X2 (pair), X3 .. X8
//   [12 .. 16]  f_c^-7/6, binom(-7/6, n) u^n (n = 1..4)
//   [18 .. 19]  exp(+2 pi i f_c tau_d) of the single detector D-1 (D odd)
//   [20 .. 23]  the same for detectors 0 and 1 (D >= 2): {re_0, re_1, im_0, im_1}
// The detector delay enters the fiducial phase linearly, x_d(f) = x(f) +
// f tau_d, so per grid point exp(2 pi i x_d) = exp(2 pi i x) exp(2 pi i f_c
// tau_d) exp(2 pi i j df tau_d): one sine/cosine per point, the chunk factor
// from this record and the offset factor from a 32-entry table per block.
constexpr int kRec = 32;

// The record of one chunk from its Taylor matrix row and the float-float
// reference values: X_n = sum_k (c_k / 2pi) Q_kn by float-pair dot products.
// task 0 forms orders 0 and 1 and the per-detector chunk factors, task 1
// order 2 and the amplitude series, task 2 orders 3..8; each reads its part
// of the 512-byte row with 16-byte loads issued before use.  rec: kRec floats,
// 16-byte aligned.
// WAIT: the reference values come from the preceding kernel of the stream and
// this grid was launched programmatically: the matrix row is loaded first,
// then the grid waits for that kernel before it reads them.
template <bool WAIT = false>
__device__ __forceinline__ void chunk_record(const RefValues* __restrict__ ref, const float4* __restrict__ row, int D,
                                             int task, float* __restrict__ rec) {
  if (task == 0) {
    float4 m[kNBasis];
#pragma unroll
    for (int k = 0; k < kNBasis; ++k) m[k] = __ldcs(row + (kQ01 / 4) + k);
    const float4 fc = __ldcs(row + kQfc / 4);
    if (WAIT) asm volatile("griddepcontrol.wait;" ::: "memory");
    float x0h = ref->phi0t[0], x0l = ref->phi0t[1], x1h = 0.f, x1l = 0.f;
#pragma unroll
    for (int k = 0; k < kNBasis; ++k) {
      const float ch = ref->chat[k][0], cl = ref->chat[k][1];
      f2x_fma_acc(ch, cl, m[k].x, m[k].y, x0h, x0l);
      f2x_fma_acc(ch, cl, m[k].z, m[k].w, x1h, x1l);
    }
    reinterpret_cast<float4*>(rec)[0] = make_float4(__fadd_rn(x0h, -round_fma_pipe(x0h)), x0l, x1h, x1l);
    float2 e[kMaxDet];
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      float ah = 0.f, al = 0.f;
      if (d < D) f2x_fma_acc(ref->taut[d][0], ref->taut[d][1], fc.x, fc.y, ah, al);
      e[d] = cis_turns(frac_turns(ah, al));
    }
    if (D >= 2) reinterpret_cast<float4*>(rec)[5] = make_float4(e[0].x, e[1].x, e[0].y, e[1].y);
    if (D & 1) reinterpret_cast<float2*>(rec)[9] = e[D - 1];
  } else if (task == 1) {
    float4 m[kNBasis / 2];
#pragma unroll
    for (int i = 0; i < kNBasis / 2; ++i) m[i] = __ldcs(row + kQ2 / 4 + i);
    const float4 a0 = __ldcs(row + kQfc / 4), a1 = __ldcs(row + kQfc / 4 + 1);
    if (WAIT) asm volatile("griddepcontrol.wait;" ::: "memory");
    float xh = 0.f, xl = 0.f;
#pragma unroll
    for (int i = 0; i < kNBasis / 2; ++i) {
      f2x_fma_acc(ref->chat[2 * i][0], ref->chat[2 * i][1], m[i].x, m[i].y, xh, xl);
      f2x_fma_acc(ref->chat[2 * i + 1][0], ref->chat[2 * i + 1][1], m[i].z, m[i].w, xh, xl);
    }
    reinterpret_cast<float2*>(rec)[2] = make_float2(xh, xl);
    reinterpret_cast<float4*>(rec)[3] = make_float4(a0.z, a0.w, a1.x, a1.y);
    rec[16] = a1.z;
  } else {
    float4 m[(kOrd - 2) * kNBasis / 4];
#pragma unroll
    for (int i = 0; i < (kOrd - 2) * kNBasis / 4; ++i) m[i] = __ldcs(row + kQh / 4 + i);
    if (WAIT) asm volatile("griddepcontrol.wait;" ::: "memory");
    const float* mf = reinterpret_cast<const float*>(m);
    float xn[kOrd - 2];
#pragma unroll
    for (int n = 0; n < kOrd - 2; ++n) {
      float t = 0.f;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) t = fmaf(ref->chat[k][0], mf[n * kNBasis + k], t);
      xn[n] = t;
    }
    reinterpret_cast<float2*>(rec)[3] = make_float2(xn[0], xn[1]);
    reinterpret_cast<float4*>(rec)[2] = make_float4(xn[2], xn[3], xn[4], xn[5]);
  }
}

// The chunk records of all chunks, to global memory (32 chunks per block,
// one task per warp).  The rebuild + batch step launches this ahead of the
// summary sums, where it overlaps the walkers' set-up on the other stream;
// a rebuild on its own forms the records inside the summary kernel instead.
__global__ void __launch_bounds__(96) k_chunk_coef(const RefValues* __restrict__ ref, const float* __restrict__ q,
                                                   int D, int n_chunks, float* __restrict__ out) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  if (c >= n_chunks) return;
  chunk_record<true>(ref, reinterpret_cast<const float4*>(q + (size_t)c * kQRow), D, threadIdx.x >> 5,
                     out + (size_t)c * kRec);
}

// Integer -> float on the FMA pipe (exact for |i| < 2^22; larger |i| < 2^31
// are split in two parts and rounded once).
__device__ __forceinline__ float int_float_fma(int i) {
  const int hi = i >> 21, lo = i & ((1 << 21) - 1);
  return __fmaf_rn(small_int_float(hi), 2097152.0f, small_int_float(lo));
}

// FP32 working copy of an event's data for the fast summary build, made
// when the data change (not on every rebuild):
//   w_d = d'_d / S'_d (complex) and is_d = 1 / S'_d,  d' = d 2^sd, S' = S 2^sS,
// with power-of-two scales from the detector's first PSD sample (S' ~ 1 and
// d' ~ sqrt(T/4)); exps[d] = {sd, sS}.  One thread per (point, detector);
// the FP64 -> FP32 conversion uses integer operations (scaled_float).
__global__ void __launch_bounds__(256) k_data32(DataPtrs in, int64_t N, int D, float2* __restrict__ w32,
                                                float* __restrict__ is32, int* __restrict__ exps) {
  const int d = blockIdx.y;
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ex = ((__double2hiint(__ldg(in.psd[d])) >> 20) & 0x7FF) - 1023;
  const int sS = -ex, sd = -(ex / 2);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    exps[2 * d] = sd;
    exps[2 * d + 1] = sS;
  }
  if (k >= N) return;
  const double2 dv = __ldcs(reinterpret_cast<const double2*>(in.data[d]) + k);
  const float Sp = scaled_float(__ldcs(in.psd[d] + k), (unsigned)(896 - sS) << 20);
  const float is = __frcp_rn(Sp);
  const unsigned bd = (unsigned)(896 - sd) << 20;
  w32[(size_t)d * N + k] = make_float2(scaled_float(dv.x, bd) * is, scaled_float(dv.y, bd) * is);
  is32[(size_t)d * N + k] = is;
}

// Host-buffer step: the strain and PSD read straight from pinned host memory
// mapped into the device address space (one pass over the host link), stored
// as the event's resident FP64 copies and converted to the FP32 working copy
// with the k_data32 arithmetic.  Block row d = detector; the blocks of a row
// stride over the points with two points in flight per thread.  Half a block
// per SM in all: the host link, not the SMs, sets the rate (2 blocks per SM
// read no faster), and the rebuild's data-independent kernels launched beside
// it find free SMs at once instead of ~55 us later.
__global__ void __launch_bounds__(256) k_pull32(DataPtrs src, int64_t N, double* __restrict__ data,
                                                double* __restrict__ psd, float2* __restrict__ w32,
                                                float* __restrict__ is32, int* __restrict__ exps) {
  const int d = blockIdx.y;
  const double2* __restrict__ sd2 = reinterpret_cast<const double2*>(src.data[d]);
  const double* __restrict__ sp = src.psd[d];
  const int ex = ((__double2hiint(__ldcs(sp)) >> 20) & 0x7FF) - 1023;
  const int sS = -ex, sdx = -(ex / 2);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    exps[2 * d] = sdx;
    exps[2 * d + 1] = sS;
  }
  const unsigned bS = (unsigned)(896 - sS) << 20, bd = (unsigned)(896 - sdx) << 20;
  double2* __restrict__ od = reinterpret_cast<double2*>(data) + (size_t)d * N;
  double* __restrict__ op = psd + (size_t)d * N;
  float2* __restrict__ ow = w32 + (size_t)d * N;
  float* __restrict__ oi = is32 + (size_t)d * N;
  auto put = [&](int64_t k, double2 dv, double pv) {
    k = RB_IDX(k, N, 211);
    const float is = __frcp_rn(scaled_float(pv, bS));
    __stcs(od + k, dv);
    __stcs(op + k, pv);
    ow[k] = make_float2(scaled_float(dv.x, bd) * is, scaled_float(dv.y, bd) * is);
    oi[k] = is;
  };
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; k + stride < N; k += 2 * stride) {
    const double2 a = __ldcs(sd2 + k), b = __ldcs(sd2 + k + stride);
    const double pa = __ldcs(sp + k), pb = __ldcs(sp + k + stride);
    put(k, a, pa);
    put(k + stride, b, pb);
  }
  if (k < N) put(k, __ldcs(sd2 + k), __ldcs(sp + k));
}

cudaError_t launch_pull32(const DataPtrs& src, int64_t N, int D, double* data, double* psd, void* w32, float* is32,
                          int* exps, int n_sm, cudaStream_t s) {
  dim3 grid((unsigned)std::max(1, (n_sm / 2 + D - 1) / D), (unsigned)D);
  k_pull32<<<grid, 256, 0, s>>>(src, N, data, psd, static_cast<float2*>(w32), is32, exps);
  return cudaGetLastError();
}

constexpr int kSumFastThreads = 128;
constexpr int kNQ = 7;  // per detector: A0 re/im, A1 re/im, B0, B1 as a float pair (hi, lo)
constexpr int kNAcc = kNQ * kMaxDet;
constexpr int kPartRecs = kPartPoints / kChunk + 1;  // chunk records a part can touch
static_assert(kPartPoints % kSumFastThreads == 0, "parts are whole rounds of the block");

// One block per part of a bin (at most kPartPoints grid points), all
// detectors, reading the FP32 data copy (w = d'/S', 1/S').  The records of
// the part's chunks go to shared memory: with INBLOCK formed there from the
// event's chunk matrices q and the reference values (three threads per
// chunk, while the first data loads are in flight), otherwise copied from
// the records k_chunk_coef wrote (q then points to them).  Each thread
// evaluates every 128th point, with the next point's data loads in flight
// while the current one is evaluated.  Per point: the
// intrinsic fiducial phase from the chunk's Taylor coefficients, one
// sine/cosine, the detector factors exp(2 pi i f_c tau_d) (record) and
// exp(2 pi i j df tau_d) (block table).  Per-thread sums are FP32 (B1, which
// nearly cancels within a bin, a float pair); block sums are float pairs in a
// fixed order; the parts of a bin are added in index order by the last of
// them to finish, which then runs the FP64 epilogue.
// Registers: with the records copied (the rebuild + batch step) the kernel
// is held to 64 per thread, so that six blocks still fit on an SM that also
// holds a block of the walkers' set-up, which runs beside it there: at 78,
// such SMs took five and the C2 build (868 parts) needed a second wave.
template <int ND, bool INBLOCK>
__global__ void __launch_bounds__(kSumFastThreads, INBLOCK ? 6 : 8)
    k_summary_fast(const float2* __restrict__ w32, const float* __restrict__ is32, const int* __restrict__ exps,
                   int N, const float* __restrict__ q, double T, float invT_hi, float invT_lo, int B, int D,
                   const int64_t* __restrict__ edges, const RefValues* __restrict__ ref, SummaryOut so, int p_off) {
  __shared__ __align__(16) float srec[kPartRecs * kRec];
  // exp(2 pi i j df tau_d), indexed by k mod 32: detectors 0 and 1 as
  // {re_0, re_1, im_0, im_1}, the single detector D-1 as {re, im}
  __shared__ float4 toffP[kChunk];
  __shared__ float2 toffS[kChunk];
  __shared__ float red[kSumFastThreads / 32][kNAcc * 33];  // per-thread partials, one row per quantity
  __shared__ float wsum[kSumFastThreads / 32][kNAcc][2];
  __shared__ float qsum[kNAcc][2];
  __shared__ double sblock[6 * kMaxDet];
  __shared__ double scale[kMaxDet][4];
  __shared__ double s_inv_df;
  __shared__ bool s_last;
  const int pid = (int)blockIdx.x + p_off;  // this block's part
  const PartDesc pd = so.parts[RB_IDX(pid, so.n_parts, 201)];
  const int b = pd.bin;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int e0 = (int)edges[b], e1 = (int)edges[b + 1];
  const int ks = pd.start, ke = pd.end;
  const int w = e1 - e0;
  const float half_df = 0.5f * invT_hi;  // (float)(0.5 / T): no FP64 divide per thread
  if (tid < kMaxDet * kChunk) {
    const int d = tid >> 5, j = lane - kChunk / 2;
    float sh = 0.f, sl = 0.f;
    if (d < D) f2x_fma_acc(ref->taut[d][0], ref->taut[d][1], invT_hi, invT_lo, sh, sl);  // tau_d df
    const float jf = small_int_float(j);
    const float p = __fmul_rn(sh, jf);
    const float e = __fmaf_rn(sl, jf, __fmaf_rn(sh, jf, -p));
    const float2 t = cis_turns(frac_turns(p, e));
    if (ND >= 2 && d < 2) {
      float* tp = reinterpret_cast<float*>(&toffP[lane]);
      tp[d] = t.x;
      tp[2 + d] = t.y;
    }
    if ((ND & 1) && d == ND - 1) toffS[lane] = t;
  } else if (tid >= 96 && tid < 96 + D) {
    // undo the power-of-two scales of the FP32 data copy (d 2^sd, S 2^sS)
    const int d = tid - 96;
    const int sd = __ldg(exps + 2 * d), sS = __ldg(exps + 2 * d + 1);
    // 2^n as the bit pattern of a double (|n| well inside the exponent range)
    const double w4 = 4.0 / T;
    scale[d][0] = w4 * __hiloint2double((1023 + sS - sd) << 20, 0);
    scale[d][1] = w4 * __hiloint2double((1023 + sS) << 20, 0);
    scale[d][2] = ref->K[d][0];
    scale[d][3] = ref->K[d][1];
  } else if (tid == 127) {
    s_inv_df = so.inv_df[b];
  }
  // per-thread sums, kNQ per detector: detectors 0 and 1 paired, D-1 single
  float2 accP[kNQ];
  float accS[kNQ];
#pragma unroll
  for (int i = 0; i < kNQ; ++i) {
    accP[i] = make_float2(0.f, 0.f);
    accS[i] = 0.f;
  }
  float2 dv[kMaxDet], dn[kMaxDet];  // w = d'/S'
  float isv[kMaxDet], pn[kMaxDet];  // 1/S'
  auto load_point = [&](int k, float2* dd, float* pp) {
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d)
      if (d < D) {
        dd[d] = __ldcs(w32 + (size_t)d * N + RB_IDX(k, N, 202));
        pp[d] = __ldcs(is32 + (size_t)d * N + RB_IDX(k, N, 202));
      }
  };
  int k = ks + tid;
  if (k < ke) load_point(k, dn, pn);  // in flight across the staging below
  const int c0 = ks >> 5, nrec = ((ke - 1) >> 5) - c0 + 1;
  if (INBLOCK) {
    if (tid < 3 * kPartRecs) {
      const int r = tid % kPartRecs, task = tid / kPartRecs;
      if (r < nrec)
        chunk_record(ref, reinterpret_cast<const float4*>(q + (size_t)(c0 + r) * kQRow), D, task,
                     srec + RB_IDX(r, kPartRecs, 204) * kRec);
    }
  } else {
    const float4* src = reinterpret_cast<const float4*>(q + (size_t)c0 * kRec);
    float4* dst = reinterpret_cast<float4*>(srec);
    for (int i = tid; i < nrec * (kRec / 4); i += kSumFastThreads) dst[RB_IDX(i, kPartRecs * kRec / 4, 204)] = __ldg(src + i);
  }
  __syncthreads();
  for (; k < ke; k += kSumFastThreads) {
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      dv[d] = dn[d];
      isv[d] = pn[d];
    }
    if (k + kSumFastThreads < ke) load_point(k + kSumFastThreads, dn, pn);
    const float4* rec = reinterpret_cast<const float4*>(srec + RB_IDX((k >> 5) - c0, kPartRecs, 203) * kRec);
    const float jf = small_int_float((k & (kChunk - 1)) - kChunk / 2);
    const float4 x01 = rec[0];  // X0 pair, X1 pair
    const float4 h0 = rec[1];   // X2 pair, X3, X4
    const float4 h1 = rec[2];   // X5 .. X8
    const float4 a0 = rec[3];   // amplitude series
    const float a4 = reinterpret_cast<const float*>(rec)[16];
    // intrinsic fiducial phase x = X0 + X1 j + X2 j^2 + j^3 (X3 + ... + X8 j^5)
    const float t = fmaf(fmaf(fmaf(fmaf(fmaf(h1.w, jf, h1.z), jf, h1.y), jf, h1.x), jf, h0.w), jf, h0.z);
    const float j2 = jf * jf;
    const float t3 = t * (j2 * jf);
    const float p1 = __fmul_rn(x01.z, jf);
    float e1r = __fmaf_rn(x01.z, jf, -p1);
    e1r = __fmaf_rn(x01.w, jf, e1r);
    const float p2 = __fmul_rn(h0.x, j2);
    float e2r = __fmaf_rn(h0.x, j2, -p2);
    e2r = __fmaf_rn(h0.y, j2, e2r);
    float sh = x01.x, sl = x01.y;
    f2x_add(sh, sl, p1);
    f2x_add(sh, sl, p2);
    sl = __fadd_rn(sl, __fadd_rn(__fadd_rn(e1r, e2r), t3));
    const float2 z = cis_turns(frac_turns(sh, sl));  // exp(+2 pi i x)
    const float A = a0.x * fmaf(jf, fmaf(jf, fmaf(jf, fmaf(jf, a4, a0.w), a0.z), a0.y), 1.f);
    const float A2 = A * A;
    const float dff = int_float_fma(2 * (k - e0) - w) * half_df;  // f - f_m
    if constexpr (ND >= 2) {  // detectors 0 and 1, paired
      const float4 ep = rec[5];                 // exp(2 pi i f_c tau_d)
      const float4 tp = toffP[k & (kChunk - 1)];  // exp(2 pi i j df tau_d)
      const float2 er = make_float2(ep.x, ep.y), ei = make_float2(ep.z, ep.w);
      const float2 tr = make_float2(tp.x, tp.y), ti = make_float2(tp.z, tp.w);
      const float2 fr = pv::fma(er, tr, pv::mul(pv::neg(ei), ti)), fi = pv::fma(er, ti, pv::mul(ei, tr));
      const float2 zx = make_float2(z.x, z.x), zy = make_float2(z.y, z.y);
      const float2 Cc = pv::fma(zx, fr, pv::mul(pv::neg(zy), fi)), Ss = pv::fma(zx, fi, pv::mul(zy, fr));
      const float2 AA = make_float2(A, A);
      const float2 dr = pv::mul(make_float2(dv[0].x, dv[1].x), AA), di = pv::mul(make_float2(dv[0].y, dv[1].y), AA);
      const float2 qr = pv::fma(dr, Cc, pv::mul(pv::neg(di), Ss)), qi = pv::fma(dr, Ss, pv::mul(di, Cc));
      const float2 D2 = make_float2(dff, dff);
      accP[0] = pv::add(accP[0], qr);
      accP[1] = pv::add(accP[1], qi);
      accP[2] = pv::fma(qr, D2, accP[2]);
      accP[3] = pv::fma(qi, D2, accP[3]);
      const float2 hh = pv::mul(make_float2(A2, A2), make_float2(isv[0], isv[1]));
      accP[4] = pv::add(accP[4], hh);
      // B1 (|h0|^2 / S weighted by f - f_m > 0 or < 0) nearly cancels within a
      // bin: its per-thread sum is a float pair (hi, lo)
      pv::add_acc(accP[5], accP[6], pv::mul(hh, D2));
    }
    if constexpr ((ND & 1) != 0) {  // the single detector D-1
      constexpr int d = ND - 1;
      const float2 ec = reinterpret_cast<const float2*>(rec)[9];  // exp(2 pi i f_c tau_d)
      const float2 eo = toffS[k & (kChunk - 1)];                  // exp(2 pi i j df tau_d)
      const float fr = fmaf(ec.x, eo.x, -ec.y * eo.y), fi = fmaf(ec.x, eo.y, ec.y * eo.x);
      const float Cc = fmaf(z.x, fr, -z.y * fi), Ss = fmaf(z.x, fi, z.y * fr);  // exp(+2 pi i x_d)
      const float dr = dv[d].x * A, di = dv[d].y * A;
      const float qr = fmaf(dr, Cc, -di * Ss), qi = fmaf(dr, Ss, di * Cc);
      accS[0] += qr;
      accS[1] += qi;
      accS[2] = fmaf(qr, dff, accS[2]);
      accS[3] = fmaf(qi, dff, accS[3]);
      const float hh = A2 * isv[d];
      accS[4] += hh;
      f2x_add(accS[5], accS[6], hh * dff);
    }
  }
  // ---- block sums in float pairs, fixed order: lanes 0..20 of each warp sum
  // one quantity over the warp's 32 threads, then 21 threads sum the warp
  // totals (A1 and B1 cancel strongly within a bin, so no stage of this sum
  // is plain FP32) ----
  float acc[kNAcc];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) acc[kNQ * d + q] = 0.f;
    if (ND >= 2) {
      acc[q] = accP[q].x;
      acc[kNQ + q] = accP[q].y;
    }
    if (ND & 1) acc[kNQ * (ND - 1) + q] = accS[q];
  }
  float* wr = red[wid];
#pragma unroll
  for (int i = 0; i < kNAcc; ++i) wr[i * 33 + lane] = acc[i];
  __syncwarp();
  if (lane < kNAcc) {
    float h = 0.f, l = 0.f;
    for (int m = 0; m < 32; ++m) f2x_add(h, l, wr[lane * 33 + m]);
    wsum[wid][lane][0] = h;
    wsum[wid][lane][1] = l;
  }
  __syncthreads();
  const bool multi = pd.n_parts > 1;
  if (tid < kNAcc) {
    float h = wsum[0][tid][0], l = wsum[0][tid][1];
#pragma unroll
    for (int i = 1; i < kSumFastThreads / 32; ++i) {
      f2x_add(h, l, wsum[i][tid][0]);
      l = __fadd_rn(l, wsum[i][tid][1]);
    }
    qsum[tid][0] = h;
    qsum[tid][1] = l;
    if (multi) {
      float* ps = so.part_sums + ((size_t)pid * kNAcc + tid) * 2;
      ps[0] = h;
      ps[1] = l;
      fence_acq_rel_gpu();
    }
  }
  if (multi) {
    // the last part of the bin to finish adds the parts in index order
    __syncthreads();
    if (tid == 0) {
      const unsigned ticket = atomicAdd(&so.sync->bin_parts_done[b], 1u);
      s_last = (ticket == (unsigned)pd.n_parts - 1u);
      if (s_last) so.sync->bin_parts_done[b] = 0u;
    }
    __syncthreads();
    if (!s_last) return;
    fence_acq_rel_gpu();
    if (tid < kNAcc) {
      const float* ps = so.part_sums + ((size_t)pd.first * kNAcc + tid) * 2;
      float h = __ldcg(ps), l = __ldcg(ps + 1);
      for (int p = 1; p < pd.n_parts; ++p) {
        f2x_add(h, l, __ldcg(ps + (size_t)p * kNAcc * 2));
        l = __fadd_rn(l, __ldcg(ps + (size_t)p * kNAcc * 2 + 1));
      }
      qsum[tid][0] = h;
      qsum[tid][1] = l;
    }
  }
  __syncthreads();
  if (tid < 6 * D) {
    const int d = tid / 6, f = tid - 6 * d, q = kNQ * d + f;
    float h = qsum[q][0], l = qsum[q][1];
    if (f == 5) {  // B1 = its hi and lo sums
      f2x_add(h, l, qsum[q + 1][0]);
      l = __fadd_rn(l, qsum[q + 1][1]);
    }
    sblock[tid] = (double)h + (double)l;
  }
  __syncthreads();
  summary_epilogue(so, b, 0, D, B, D, sblock, &scale[0][0], true, (unsigned)B, s_inv_df, true, false);
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
size_t chunk_coef_bytes(int64_t N) { return sizeof(float) * kRec * (size_t)n_chunks_of(N); }

cudaError_t launch_chunk_coef(int64_t N, int D, const RefValues* ref, const void* cq, void* chunk_coef, cudaStream_t s) {
  const int nc = (int)n_chunks_of(N);
  // programmatic launch: the blocks may start while the reference-value
  // kernel before them runs, load their matrix rows, then wait for it
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)((nc + 31) / 32));
  cfg.blockDim = dim3(96);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_chunk_coef, ref, static_cast<const float*>(cq), D, nc, static_cast<float*>(chunk_coef));
}

cudaError_t launch_chunk_q(int64_t kmin, double T, int64_t N, void* cq, cudaStream_t s) {
  static const TaylorTables tt = make_taylor_tables();
  const int64_t nc = n_chunks_of(N);
  k_chunk_q<<<(unsigned)((nc + 127) / 128), 128, 0, s>>>(kmin, T, nc, tt, static_cast<float*>(cq));
  return cudaGetLastError();
}

cudaError_t launch_data32(const DataPtrs& in, int64_t N, int D, void* w32, float* is32, int* exps, cudaStream_t s) {
  dim3 grid((unsigned)((N + 255) / 256), (unsigned)D);
  k_data32<<<grid, 256, 0, s>>>(in, N, D, static_cast<float2*>(w32), is32, exps);
  return cudaGetLastError();
}

// recs: the chunk records k_chunk_coef wrote, or NULL to form them in-block
// from the chunk matrices chunk_q.
cudaError_t launch_summary_parts(const void* w32, const float* is32, const int* exps, int64_t N, double T, int D, int B,
                                 const int64_t* edges, const RefValues* ref, const void* chunk_q, const void* recs,
                                 const SummaryOut& so, int p0, int p1, cudaStream_t s) {
  if (p0 < 0 || p1 <= p0) return cudaErrorInvalidValue;
  const double invT = 1.0 / T;
  const float ih = (float)invT, il = (float)(invT - (double)ih);
  const bool inblock = recs == nullptr;
  auto kf = inblock ? (D == 1 ? k_summary_fast<1, true> : D == 2 ? k_summary_fast<2, true> : k_summary_fast<3, true>)
                    : (D == 1 ? k_summary_fast<1, false> : D == 2 ? k_summary_fast<2, false> : k_summary_fast<3, false>);
  kf<<<(unsigned)(p1 - p0), kSumFastThreads, 0, s>>>(static_cast<const float2*>(w32), is32, exps, (int)N,
                                                      static_cast<const float*>(inblock ? chunk_q : recs), T, ih, il, B,
                                                      D, edges, ref, so, p0);
  return cudaGetLastError();
}

}  // namespace rb

RB_BOUNDS_READER(rb_bounds_read_summary)
