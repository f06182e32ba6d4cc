// rb_loglike.cu -- batched relative-binning log-likelihood and its adjoint
// (steps a3-a6): ratio at the bin edges, per-bin linearisation, contraction
// with the summary data, and the reverse sweep back to the 13 parameters.
//
// Relative binning (Sec. II.C, Eqs. 4-5): per detector d,
//   r(f_e) = rho_d exp(-2 pi i x_d(f_e)),   x_d = dPsi_d / (2 pi)  [turns]
//   r0(b) = (r_b + r_{b+1}) / 2,  r1(b) = (r_{b+1} - r_b) / (f_{b+1} - f_b)
//   <d|h> = Re sum_b [A0 r0* + A1 r1*],  <h|h> = sum_b [B0 |r0|^2 + 2 B1 Re(r0 r1*)].
// The kernels evaluate the deviation from the fiducial point: with
// r = 1 + delta, s = delta_b + delta_{b+1}, t = delta_{b+1} - delta_b,
//   log L = base + sum_{d,b} Re(alpha0 s*) + Re(alpha1 t*) - beta0 (Re s + |s|^2/4)
//                            - beta1 (Re t + Re(s t*)/2),
// alpha0 = A0/2, alpha1 = A1/df_b, beta0 = B0/2, beta1 = B1/df_b and the FP64
// constant base = sum_d (Re sum_b A0 - sum_b B0/2) = log L(theta_ref).  At the
// fiducial point delta = 0 exactly and the result is base, bit for bit.
// delta is formed without cancellation from the half angle:
//   exp(-2 pi i x) - 1 = -2 sin^2(pi x) - 2 i sin(pi x) cos(pi x),
//   delta = rho (exp(-2 pi i x) - 1) + (rho - 1).
//
// Mapping: one warp per walker (persistent: each block takes a contiguous,
// equal share of the walkers and its warps take them in turn);
// lane l handles edge 31 c + l of chunk c and bin 31 c + l (lanes 0..30), so
// each bin's right edge comes from the next lane by one shuffle and every
// chunk overlaps the next by one edge.  Edge and bin tables live in shared
// memory.  The adjoint reuses the same chunking: each lane's edge collects
// U - V from its own bin and U + V from the bin on its left (shuffle up); an
// edge shared by two chunks collects the two halves in two passes, which is
// exact because the adjoint is linear in the per-edge cotangent.
#include <algorithm>
#include <mutex>

#include "rb_internal.cuh"

namespace rb {

constexpr int kThreads = 512;
constexpr unsigned kFull = 0xffffffffu;

struct LaunchArgs {
  EventDev ev;
  const void* ws;    // WalkerMixed* or WalkerF64*
  const void* tan;   // WalkerTan<float>* or WalkerTan<double>*
  int64_t W;
  double* logl;
  double* grad;
  MalaArgs mala;     // MALA kernels only
};

// MALA accept/reject for walker w after its log L and d log L / d theta
// (lane j < 13 holds component j): gradient in sampling coordinates,
//   log alpha = log pi(z') - log pi(z) - 1/2 sum_j [(xi_j + eps_j (g_j + g'_j)/2)^2 - xi_j^2]
// (Sec. II.D, MALA; the sum over j is a warp reduction), accept when
// log u < log alpha, and the chain state updated in place.  The whole warp
// calls it (logl and inside are warp-uniform).
__device__ __forceinline__ void mala_finish(const MalaArgs& m, int64_t w, int lane, double logl, double gth) {
  const bool inside = m.inside[w] != 0;
  const double logpp = inside ? logl : -INFINITY;
  double gz = 0.0, term = 0.0;
  if (lane < kNPar) {
    gz = gth;
    if (lane == 9) gz = gth * m.jac[2 * w];
    else if (lane == 12) gz = gth * m.jac[2 * w + 1];
    if (!inside) gz = 0.0;
    const double xi = m.xi[w * kNPar + lane];
    const double t = xi + 0.5 * m.eps[lane] * (m.gz[w * kNPar + lane] + gz);
    term = t * t - xi * xi;
  }
  term = warp_sum_f64(term);
  if (m.init) {
    if (lane < kNPar) m.gz[w * kNPar + lane] = gz;
    if (lane == 0) {
      m.logp[w] = logpp;
      m.accepted[w] = inside ? 1 : 0;
    }
    return;
  }
  const double la = (logpp == -INFINITY) ? -INFINITY : logpp - m.logp[w] - 0.5 * term;
  const bool acc = m.lu[w] < la;
  if (acc) {
    if (lane < kNPar) {
      m.z[w * kNPar + lane] = m.zp[w * kNPar + lane];
      m.gz[w * kNPar + lane] = gz;
    }
    if (lane == 0) m.logp[w] = logpp;
  }
  if (lane == 0) m.accepted[w] = acc ? 1 : 0;
}

// Chain rule for one walker: lane j < 13 returns d log L / d theta_j from the
// reduced adjoints (adj_c over the basis coefficients, adj_tau per detector
// delay, adj_rho per detector prefactor) and the set-up tangents.
template <class T>
__device__ __forceinline__ double chain_rule(int j, int n_det, const T* adj_c, const T* adj_tau, const T (*adj_rho)[2],
                                             const T (*rho)[2], const WalkerTan<T>& tn) {
  T g = T(0);
  if (j < kNTanIntr)
    for (int k = 0; k < kNBasis; ++k) g += adj_c[k] * tn.dc[k][j];
  for (int d = 0; d < n_det; ++d) {
    if (j == 7) g += adj_tau[d];                                   // t_c
    if (j == 11 || j == 12) g += adj_tau[d] * tn.dtd[d][j - 11];  // ra, dec through the delay
    // prefactor: d log L = Re(conj(gbar_rho) rho dln rho), dln rho = lr + i li
    const T Gr = adj_rho[d][0] * rho[d][0] + adj_rho[d][1] * rho[d][1];
    const T Gi = adj_rho[d][0] * rho[d][1] - adj_rho[d][1] * rho[d][0];
    T lr = T(0), li = T(0);
    if (j == 0) { lr = tn.lnamp_Mc; li = -tn.dphi0[0]; }
    else if (j == 1) { li = -tn.dphi0[1]; }
    else if (j == 6) { lr = tn.lnamp_dL; }
    else if (j == 8) { li = T(1); }
    else if (j >= 9) { lr = tn.dlnP[d][j - 9][0]; li = tn.dlnP[d][j - 9][1]; }
    g += Gr * lr - Gi * li;
  }
  return (double)g;
}

// ---------------------------------------------------------------------------
// Mixed precision.  PHASE64 = false: phase as float pairs (FP32 pipe);
// PHASE64 = true: phase accumulated in native FP64.
// ---------------------------------------------------------------------------
template <bool GRAD, bool PHASE64, bool MALA = false>
__global__ void __launch_bounds__(kThreads) k_rb_mixed(LaunchArgs a) {
  static_assert(!MALA || GRAD, "the MALA step needs the gradient");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EventDev& ev = a.ev;
  const int Ep = ev.e_pad, Bp = ev.b_pad, D = ev.n_det, B = ev.n_bins, E = ev.n_edges;

  // Stage the tables (16-byte vector copies).
  const float* sbin;
  const float4* g4 = nullptr;  // [kEdgeQuads][Ep] basis pairs and f_e (float pairs)
  const double* g64 = nullptr;
  const double* f64 = nullptr;
  {
    const int tid = threadIdx.x;
    if (!PHASE64) {
      const float4* src = reinterpret_cast<const float4*>(ev.tab32);
      float4* dst = reinterpret_cast<float4*>(smem_raw);
      const size_t n4 = ev.tab32_floats / 4;
      for (size_t i = tid; i < n4; i += blockDim.x) dst[i] = src[i];
      const float* s = reinterpret_cast<const float*>(smem_raw);
      g4 = reinterpret_cast<const float4*>(s);
      sbin = s + ev.edge32_floats;
    } else {
      const size_t n_e64 = (size_t)(kNBasis + 1) * Ep;  // g[10][Ep], f[Ep]
      const double2* src = reinterpret_cast<const double2*>(ev.tab64);
      double2* dst = reinterpret_cast<double2*>(smem_raw);
      for (size_t i = tid; i < n_e64 / 2; i += blockDim.x) dst[i] = src[i];
      const size_t nb = ev.tab32_floats - ev.edge32_floats;
      const float4* bsrc = reinterpret_cast<const float4*>(ev.tab32 + ev.edge32_floats);
      float4* bdst = reinterpret_cast<float4*>(smem_raw + n_e64 * sizeof(double));
      for (size_t i = tid; i < nb / 4; i += blockDim.x) bdst[i] = bsrc[i];
      g64 = reinterpret_cast<const double*>(smem_raw);
      f64 = g64 + (size_t)kNBasis * Ep;
      sbin = reinterpret_cast<const float*>(smem_raw + n_e64 * sizeof(double));
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const float4* binA = reinterpret_cast<const float4*>(sbin);             // [D][Bp] a0r a0i a1r a1i
  const float2* binB = reinterpret_cast<const float2*>(sbin + 4 * D * Bp);  // [D][Bp] b0 b1
  // each block takes a contiguous, equal share of the walkers (so every SM
  // gets W / grid of them, +-1), its warps take them in turn
  const int64_t per_blk = a.W / gridDim.x, rem_blk = a.W % gridDim.x;
  const int64_t w_begin = (int64_t)blockIdx.x * per_blk + min((int64_t)blockIdx.x, rem_blk);
  const int64_t w_end = w_begin + per_blk + ((int64_t)blockIdx.x < rem_blk ? 1 : 0);
  const int64_t warp0 = w_begin + (threadIdx.x >> 5);
  const int64_t nwarps = blockDim.x >> 5;

  for (int64_t w = warp0; w < w_end; w += nwarps) {
    // ---- per-walker constants (uniform across the warp) ----
    float dch[kNBasis], dcl[kNBasis];
    double dc64[kNBasis];
    float tauh[kMaxDet], taul[kMaxDet];
    double tau64[kMaxDet];
    float rho[kMaxDet][2], sig[kMaxDet][2];
    int valid;
    if (!PHASE64) {
      const WalkerMixed* s = reinterpret_cast<const WalkerMixed*>(a.ws) + w;
      valid = s->valid;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) { dch[k] = s->dc_hi[k]; dcl[k] = s->dc_lo[k]; }
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        tauh[d] = s->tau_hi[d]; taul[d] = s->tau_lo[d];
        rho[d][0] = s->rho[d][0]; rho[d][1] = s->rho[d][1];
        sig[d][0] = s->sig[d][0]; sig[d][1] = s->sig[d][1];
      }
    } else {
      const WalkerF64* s = reinterpret_cast<const WalkerF64*>(a.ws) + w;
      valid = s->valid;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) dc64[k] = s->dc[k];
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        tau64[d] = s->tau[d];
        rho[d][0] = (float)s->rho[d][0]; rho[d][1] = (float)s->rho[d][1];
        sig[d][0] = (float)s->sig[d][0]; sig[d][1] = (float)s->sig[d][1];
      }
    }
    if (!valid) {
      if (MALA) {
        mala_finish(a.mala, w, lane, -INFINITY, 0.0);
      } else {
        if (lane == 0) a.logl[w] = -INFINITY;
        if (GRAD && lane < kNPar) a.grad[w * kNPar + lane] = 0.0;
      }
      continue;
    }

    // float-pair accumulator: for walkers far from the fiducial point the
    // per-bin terms add up to about -log L(theta_ref), so a single float would
    // lose ~1e-3 of absolute precision
    float acc = 0.f, acc_lo = 0.f;
    float adj_c[kNBasis], adj_tau[kMaxDet], adj_rho[kMaxDet][2];
    if (GRAD) {
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) adj_c[k] = 0.f;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) { adj_tau[d] = 0.f; adj_rho[d][0] = adj_rho[d][1] = 0.f; }
    }

    for (int c0 = 0; c0 < B; c0 += 31) {
      const int e = c0 + lane;
      const bool has_edge = e < E;
      const bool has_bin = (lane < 31) && (e < B);
      const int ee = has_edge ? e : E - 1;

      // detector-independent phase sum_k dc_k g_k(f_e) / 2pi  [turns]
      float xh = 0.f, xl = 0.f;
      double x64 = 0.0;
      float fe, fe_lo = 0.f;
      if (!PHASE64) {
#pragma unroll
        for (int q = 0; q < kNBasis / 2; ++q) {
          const float4 g = g4[q * Ep + ee];
          f2x_fma_acc(dch[2 * q], dcl[2 * q], g.x, g.y, xh, xl);
          f2x_fma_acc(dch[2 * q + 1], dcl[2 * q + 1], g.z, g.w, xh, xl);
        }
        const float2 f2 = *reinterpret_cast<const float2*>(g4 + (kEdgeQuads - 1) * Ep + ee);
        fe = f2.x;
        fe_lo = f2.y;
      } else {
#pragma unroll
        for (int k = 0; k < kNBasis; ++k) x64 = fma(dc64[k], g64[k * Ep + ee], x64);
        fe = (float)f64[ee];
      }
      float adj_x = 0.f;

#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        if (d < D) {
          float y;
          if (!PHASE64) {
            float yh = xh, yl = xl;
            f2x_fma_acc(tauh[d], taul[d], fe, fe_lo, yh, yl);
            y = frac_turns(yh, yl);
          } else {
            const double xd = fma(f64[ee], tau64[d], x64);
            y = (float)(xd - rint(xd));
          }
          float sn, cs;
          sincos_pi_half(y, sn, cs);
          const float em_r = -2.f * sn * sn, em_i = -2.f * sn * cs;
          const float dr = fmaf(rho[d][0], em_r, fmaf(-rho[d][1], em_i, sig[d][0]));
          const float di = fmaf(rho[d][0], em_i, fmaf(rho[d][1], em_r, sig[d][1]));
          const float nr = __shfl_down_sync(kFull, dr, 1);
          const float ni = __shfl_down_sync(kFull, di, 1);
          float Ur = 0.f, Ui = 0.f, Vr = 0.f, Vi = 0.f;
          if (has_bin) {
            const float4 ta = binA[d * Bp + e];
            const float2 tb = binB[d * Bp + e];
            const float a0r = ta.x, a0i = ta.y, a1r = ta.z, a1i = ta.w, b0 = tb.x, b1 = tb.y;
            const float sr = dr + nr, si = di + ni, tr = nr - dr, ti = ni - di;
            float v = a0r * sr;
            v = fmaf(a0i, si, v);
            v = fmaf(a1r, tr, v);
            v = fmaf(a1i, ti, v);
            v = fmaf(-b0, fmaf(0.25f, fmaf(sr, sr, si * si), sr), v);
            v = fmaf(-b1, fmaf(0.5f, fmaf(sr, tr, si * ti), tr), v);
            {  // two-sum into (acc, acc_lo)
              const float sum = __fadd_rn(acc, v);
              const float bb = __fadd_rn(sum, -acc);
              acc_lo = __fadd_rn(acc_lo, __fadd_rn(__fadd_rn(acc, -__fadd_rn(sum, -bb)), __fadd_rn(v, -bb)));
              acc = sum;
            }
            if (GRAD) {
              const float hs_r = fmaf(0.5f, sr, 1.f), hs_i = 0.5f * si;  // 1 + s/2
              Ur = fmaf(-b0, hs_r, fmaf(-0.5f * b1, tr, a0r));
              Ui = fmaf(-b0, hs_i, fmaf(-0.5f * b1, ti, a0i));
              Vr = fmaf(-b1, hs_r, a1r);
              Vi = fmaf(-b1, hs_i, a1i);
            }
          }
          if (GRAD) {
            float gr = Ur - Vr, gi = Ui - Vi;  // own bin (edge on its left)
            const float lr = __shfl_up_sync(kFull, Ur + Vr, 1);
            const float li = __shfl_up_sync(kFull, Ui + Vi, 1);
            if (lane > 0) { gr += lr; gi += li; }
            if (has_edge) {
              const float rr = 1.f + dr, ri = di;
              const float dldx = gr * ri - gi * rr;  // Im(conj(gbar) r); times 2 pi later
              adj_x += dldx;
              adj_tau[d] = fmaf(dldx, fe, adj_tau[d]);
              const float Er = 1.f + em_r, Ei = em_i;  // gbar_rho += gbar conj(E)
              adj_rho[d][0] += gr * Er + gi * Ei;
              adj_rho[d][1] += gi * Er - gr * Ei;
            }
          }
        }
      }
      if (GRAD && has_edge) {
        if (!PHASE64) {
#pragma unroll
          for (int q = 0; q < kNBasis / 2; ++q) {
            const float4 g = g4[q * Ep + ee];
            adj_c[2 * q] = fmaf(adj_x, g.x, adj_c[2 * q]);
            adj_c[2 * q + 1] = fmaf(adj_x, g.z, adj_c[2 * q + 1]);
          }
        } else {
#pragma unroll
          for (int k = 0; k < kNBasis; ++k) adj_c[k] = fmaf(adj_x, (float)g64[k * Ep + ee], adj_c[k]);
        }
      }
    }

    const double tot = warp_sum_f64((double)acc + (double)acc_lo);
    const double logl = *ev.base_logl + tot;
    if (!MALA && lane == 0) a.logl[w] = logl;
    if (GRAD) {
      const float two_pi = 6.28318530717958648f;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) adj_c[k] = two_pi * warp_sum_f32(adj_c[k]);
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        adj_tau[d] = two_pi * warp_sum_f32(adj_tau[d]);
        adj_rho[d][0] = warp_sum_f32(adj_rho[d][0]);
        adj_rho[d][1] = warp_sum_f32(adj_rho[d][1]);
      }
      double g = 0.0;
      if (lane < kNPar) {
        const WalkerTan<float>& tn = reinterpret_cast<const WalkerTan<float>*>(a.tan)[w];
        g = chain_rule<float>(lane, D, adj_c, adj_tau, adj_rho, rho, tn);
      }
      if (MALA) mala_finish(a.mala, w, lane, logl, g);
      else if (lane < kNPar) a.grad[w * kNPar + lane] = g;
    }
  }
}

// ---------------------------------------------------------------------------
// Plain FP64 comparison path: same mapping, everything in FP64, tables read
// through the cache from global memory.
// ---------------------------------------------------------------------------
template <bool GRAD, bool MALA = false>
__global__ void __launch_bounds__(256) k_rb_f64(LaunchArgs a) {
  static_assert(!MALA || GRAD, "the MALA step needs the gradient");
  const EventDev& ev = a.ev;
  const int Ep = ev.e_pad, Bp = ev.b_pad, D = ev.n_det, B = ev.n_bins, E = ev.n_edges;
  const double* __restrict__ g64 = ev.tab64;
  const double* __restrict__ f64 = ev.tab64 + (size_t)kNBasis * Ep;
  const double* __restrict__ bin64 = ev.tab64 + (size_t)(kNBasis + 1) * Ep;
  const int lane = threadIdx.x & 31;
  // each block takes a contiguous, equal share of the walkers (so every SM
  // gets W / grid of them, +-1), its warps take them in turn
  const int64_t per_blk = a.W / gridDim.x, rem_blk = a.W % gridDim.x;
  const int64_t w_begin = (int64_t)blockIdx.x * per_blk + min((int64_t)blockIdx.x, rem_blk);
  const int64_t w_end = w_begin + per_blk + ((int64_t)blockIdx.x < rem_blk ? 1 : 0);
  const int64_t warp0 = w_begin + (threadIdx.x >> 5);
  const int64_t nwarps = blockDim.x >> 5;
  for (int64_t w = warp0; w < w_end; w += nwarps) {
    const WalkerF64* s = reinterpret_cast<const WalkerF64*>(a.ws) + w;
    if (!s->valid) {
      if (MALA) {
        mala_finish(a.mala, w, lane, -INFINITY, 0.0);
      } else {
        if (lane == 0) a.logl[w] = -INFINITY;
        if (GRAD && lane < kNPar) a.grad[w * kNPar + lane] = 0.0;
      }
      continue;
    }
    double dc[kNBasis], tau[kMaxDet], rho[kMaxDet][2], sig[kMaxDet][2];
#pragma unroll
    for (int k = 0; k < kNBasis; ++k) dc[k] = s->dc[k];
#pragma unroll
    for (int d = 0; d < kMaxDet; ++d) {
      tau[d] = s->tau[d];
      rho[d][0] = s->rho[d][0]; rho[d][1] = s->rho[d][1];
      sig[d][0] = s->sig[d][0]; sig[d][1] = s->sig[d][1];
    }
    double acc = 0.0;
    double adj_c[kNBasis], adj_tau[kMaxDet], adj_rho[kMaxDet][2];
    if (GRAD) {
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) adj_c[k] = 0.0;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) { adj_tau[d] = 0.0; adj_rho[d][0] = adj_rho[d][1] = 0.0; }
    }
    for (int c0 = 0; c0 < B; c0 += 31) {
      const int e = c0 + lane;
      const bool has_edge = e < E;
      const bool has_bin = (lane < 31) && (e < B);
      const int ee = has_edge ? e : E - 1;
      double x = 0.0;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) x = fma(dc[k], g64[k * Ep + ee], x);
      const double fe = f64[ee];
      double adj_x = 0.0;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        if (d < D) {
          const double xd = fma(fe, tau[d], x);
          const double y = xd - rint(xd);
          double sn, cs;
          sincospi(y, &sn, &cs);
          const double em_r = -2.0 * sn * sn, em_i = -2.0 * sn * cs;
          const double dr = rho[d][0] * em_r - rho[d][1] * em_i + sig[d][0];
          const double di = rho[d][0] * em_i + rho[d][1] * em_r + sig[d][1];
          const double nr = __shfl_down_sync(kFull, dr, 1);
          const double ni = __shfl_down_sync(kFull, di, 1);
          double Ur = 0.0, Ui = 0.0, Vr = 0.0, Vi = 0.0;
          if (has_bin) {
            const double* bt = bin64 + (size_t)d * 6 * Bp;
            const double a0r = bt[e], a0i = bt[Bp + e], a1r = bt[2 * Bp + e], a1i = bt[3 * Bp + e];
            const double b0 = bt[4 * Bp + e], b1 = bt[5 * Bp + e];
            const double sr = dr + nr, si = di + ni, tr = nr - dr, ti = ni - di;
            acc += a0r * sr + a0i * si + a1r * tr + a1i * ti - b0 * (sr + 0.25 * (sr * sr + si * si)) -
                   b1 * (tr + 0.5 * (sr * tr + si * ti));
            if (GRAD) {
              const double hs_r = 1.0 + 0.5 * sr, hs_i = 0.5 * si;
              Ur = a0r - b0 * hs_r - 0.5 * b1 * tr;
              Ui = a0i - b0 * hs_i - 0.5 * b1 * ti;
              Vr = a1r - b1 * hs_r;
              Vi = a1i - b1 * hs_i;
            }
          }
          if (GRAD) {
            double gr = Ur - Vr, gi = Ui - Vi;
            const double lr = __shfl_up_sync(kFull, Ur + Vr, 1);
            const double li = __shfl_up_sync(kFull, Ui + Vi, 1);
            if (lane > 0) { gr += lr; gi += li; }
            if (has_edge) {
              const double rr = 1.0 + dr, ri = di;
              const double dldx = gr * ri - gi * rr;
              adj_x += dldx;
              adj_tau[d] += dldx * fe;
              const double Er = 1.0 + em_r, Ei = em_i;
              adj_rho[d][0] += gr * Er + gi * Ei;
              adj_rho[d][1] += gi * Er - gr * Ei;
            }
          }
        }
      }
      if (GRAD && has_edge) {
#pragma unroll
        for (int k = 0; k < kNBasis; ++k) adj_c[k] += adj_x * g64[k * Ep + ee];
      }
    }
    const double tot = warp_sum_f64(acc);
    const double logl = *ev.base_logl + tot;
    if (!MALA && lane == 0) a.logl[w] = logl;
    if (GRAD) {
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) adj_c[k] = kTwoPi * warp_sum_f64(adj_c[k]);
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        adj_tau[d] = kTwoPi * warp_sum_f64(adj_tau[d]);
        adj_rho[d][0] = warp_sum_f64(adj_rho[d][0]);
        adj_rho[d][1] = warp_sum_f64(adj_rho[d][1]);
      }
      double g = 0.0;
      if (lane < kNPar) {
        const WalkerTan<double>& tn = reinterpret_cast<const WalkerTan<double>*>(a.tan)[w];
        g = chain_rule<double>(lane, D, adj_c, adj_tau, adj_rho, rho, tn);
      }
      if (MALA) mala_finish(a.mala, w, lane, logl, g);
      else if (lane < kNPar) a.grad[w * kNPar + lane] = g;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
size_t mixed_smem_bytes(const EventDev& ev, bool phase64) {
  if (!phase64) return ev.tab32_floats * sizeof(float);
  return (size_t)(kNBasis + 1) * ev.e_pad * sizeof(double) + (ev.tab32_floats - ev.edge32_floats) * sizeof(float);
}

// Occupancy per (kernel, shared-memory size), cached in a fixed table (no
// heap allocation on the launch path): the query costs host time otherwise.
struct OccEntry {
  const void* fn;
  size_t smem;
  int blocks;
};
constexpr int kOccSlots = 256;
static std::mutex g_occ_mu;
static OccEntry g_occ[kOccSlots];
static int g_occ_n = 0;
static const void* g_smem_raised[16];
static int g_smem_raised_n = 0;

static cudaError_t blocks_per_sm(const void* fn, int threads, size_t smem, int* out) {
  std::lock_guard<std::mutex> lk(g_occ_mu);
  for (int i = 0; i < g_occ_n; ++i)
    if (g_occ[i].fn == fn && g_occ[i].smem == smem) {
      *out = g_occ[i].blocks;
      return cudaSuccess;
    }
  cudaError_t err = cudaSuccess;
  bool raised = false;
  for (int i = 0; i < g_smem_raised_n; ++i) raised = raised || g_smem_raised[i] == fn;
  if (!raised) {
    // allow any dynamic shared-memory size up to the device limit once, so
    // that launches for different events never shrink it for one another
    int dev = 0, smem_max = 0;
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err == cudaSuccess) err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (err != cudaSuccess) return err;
    if (g_smem_raised_n < 16) g_smem_raised[g_smem_raised_n++] = fn;
  }
  int n = 0;
  err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
  if (err != cudaSuccess) return err;
  if (g_occ_n < kOccSlots) g_occ[g_occ_n++] = OccEntry{fn, smem, n};
  *out = n;
  return cudaSuccess;
}

template <bool GRAD, bool PHASE64, bool MALA = false>
static cudaError_t launch_mixed_t(const LaunchArgs& a, cudaStream_t s, int n_sm) {
  const size_t smem = mixed_smem_bytes(a.ev, PHASE64);
  const void* fn = reinterpret_cast<const void*>(k_rb_mixed<GRAD, PHASE64, MALA>);
  int per_sm = 0;
  cudaError_t err = blocks_per_sm(fn, kThreads, smem, &per_sm);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t blocks_needed = (a.W * 32 + kThreads - 1) / kThreads;
  const int64_t grid = std::min<int64_t>(blocks_needed, (int64_t)per_sm * n_sm);
  k_rb_mixed<GRAD, PHASE64, MALA><<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_rb_mixed(const EventDev& ev, const void* ws, const void* tan, int64_t W, double* logl, double* grad,
                            bool phase64, cudaStream_t s, int n_sm, const MalaArgs* mala) {
  LaunchArgs a{ev, ws, tan, W, logl, grad, {}};
  if (mala) {
    a.mala = *mala;
    return phase64 ? launch_mixed_t<true, true, true>(a, s, n_sm) : launch_mixed_t<true, false, true>(a, s, n_sm);
  }
  if (grad) return phase64 ? launch_mixed_t<true, true>(a, s, n_sm) : launch_mixed_t<true, false>(a, s, n_sm);
  return phase64 ? launch_mixed_t<false, true>(a, s, n_sm) : launch_mixed_t<false, false>(a, s, n_sm);
}

cudaError_t launch_rb_f64(const EventDev& ev, const void* ws, const void* tan, int64_t W, double* logl, double* grad,
                          cudaStream_t s, int n_sm, const MalaArgs* mala) {
  LaunchArgs a{ev, ws, tan, W, logl, grad, {}};
  if (mala) a.mala = *mala;
  const int bs = 256;
  int per_sm = 0;
  const void* fn = mala ? reinterpret_cast<const void*>(k_rb_f64<true, true>)
                 : grad ? reinterpret_cast<const void*>(k_rb_f64<true>) : reinterpret_cast<const void*>(k_rb_f64<false>);
  cudaError_t err = blocks_per_sm(fn, bs, 0, &per_sm);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t blocks_needed = (W * 32 + bs - 1) / bs;
  const int64_t grid = std::min<int64_t>(blocks_needed, (int64_t)per_sm * n_sm);
  if (mala)
    k_rb_f64<true, true><<<(unsigned)grid, bs, 0, s>>>(a);
  else if (grad)
    k_rb_f64<true><<<(unsigned)grid, bs, 0, s>>>(a);
  else
    k_rb_f64<false><<<(unsigned)grid, bs, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace rb
