// rb_setup.cu -- per-walker set-up (steps a1/a2): theta -> phase-basis
// coefficients, constant phase, detector delays and complex prefactors, and
// (for the gradient) their tangents.  One thread per walker: this is the only
// FP64-heavy work of a batch, and on sm_103a the FP64 pipe is ~1/70 of the
// FP32 rate, so it is spread over as many lanes as there are walkers.
//
// Waveform (Sec. II.B; TaylorF2 from the PN literature cited there):
//   h+ = A f^-7/6 (1+cos^2 i)/2 e^{-i Psi},  hx = -i A f^-7/6 cos i e^{-i Psi},
//   A = sqrt(5/24) pi^-2/3 Mc^5/6 / d_L,
//   Psi = 2 pi f t_c - phi_c - pi/4 + 3/(128 eta v^5) sum_k phi_k v^k, v = (pi M f)^1/3,
// point-particle phi_k to 3.5PN, aligned-spin 1.5PN (beta) and 2PN (sigma,
// kappa = 1) terms, and 5PN/6PN tidal terms written per body (equivalent to
// the Lambda-tilde / delta-Lambda-tilde form of the paper's appendix).
// Detector response: h_d = (F+ h+ + Fx hx) e^{-2 pi i f dt_d}, dt_d = -n.r_d/c.
#include "rb_internal.cuh"

namespace rb {

// ---------------------------------------------------------------------------
// Absolute per-source values.  noinline: one instruction sequence for every
// caller, so theta == theta_ref reproduces the fiducial values bit for bit.
// ---------------------------------------------------------------------------
__device__ __noinline__ void walker_values(const double* th, const EventConst& ec, int need64, Values& out) {
  const double Mc = th[0], q = th[1], chi1 = th[2], chi2 = th[3], L1 = th[4], L2 = th[5];
  const double dL = th[6], tc = th[7], phic = th[8], iota = th[9], psi = th[10], ra = th[11], dec = th[12];
  bool ok = true;
  for (int j = 0; j < kNPar; ++j) ok = ok && isfinite(th[j]);
  ok = ok && Mc > 0.0 && q > 0.0 && q <= 1.0 && dL > 0.0;
  out.valid = ok ? 1 : 0;
  if (!ok) return;

  const double opq = 1.0 + q;
  const double eta = q / (opq * opq);
  const double X1 = 1.0 / opq, X2 = q / opq;
  const double X1_2 = X1 * X1, X2_2 = X2 * X2;
  const double X1_4 = X1_2 * X1_2, X2_4 = X2_2 * X2_2;

  // PN coefficients (normalisation of Psi above).
  const double beta = (chi1 * (113.0 * X1_2 + 75.0 * eta) + chi2 * (113.0 * X2_2 + 75.0 * eta)) / 12.0;
  const double sigma = eta * (474.0 / 48.0) * chi1 * chi2 + (486.0 / 96.0) * (X1_2 * chi1 * chi1 + X2_2 * chi2 * chi2);
  const double phi2 = 3715.0 / 756.0 + (55.0 / 9.0) * eta;
  const double phi3 = -16.0 * kPi + 4.0 * beta;
  const double phi4 = 15293365.0 / 508032.0 + (27145.0 / 504.0) * eta + (3085.0 / 72.0) * eta * eta - 10.0 * sigma;
  const double phi5p = kPi * (38645.0 / 756.0 - (65.0 / 9.0) * eta);
  const double phi6c = 11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kEulerGamma +
                       eta * (-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) +
                       (76055.0 / 1728.0) * eta * eta - (127825.0 / 1296.0) * eta * eta * eta;
  const double phi7 = kPi * (77096675.0 / 254016.0 + (378515.0 / 1512.0) * eta - (74045.0 / 756.0) * eta * eta);
  const double phi10 = (-288.0 + 264.0 * X1) * X1_4 * L1 + (-288.0 + 264.0 * X2) * X2_4 * L2;
  const double phi12 = X1_4 * L1 * (-15895.0 / 28.0 + 4595.0 / 28.0 * X1 + 5715.0 / 14.0 * X1_2 - 325.0 / 7.0 * X1_2 * X1) +
                       X2_4 * L2 * (-15895.0 / 28.0 + 4595.0 / 28.0 * X2 + 5715.0 / 14.0 * X2_2 - 325.0 / 7.0 * X2_2 * X2);

  // 3/(128 eta v^5) v^k = N0 (pi M)^{k/3} f^{(k-5)/3}, N0 = (3/128) (pi Mc)^{-5/3}
  const double lnMc = log(kPi * Mc * kMsunS);          // ln(pi Mc)
  const double u = lnMc - 0.6 * log(eta);              // ln(pi M)
  const double a = exp(u / 3.0);                        // (pi M)^{1/3}
  const double N0 = (3.0 / 128.0) * exp(-(5.0 / 3.0) * lnMc);
  const double a2 = a * a, a3 = a2 * a, a4 = a2 * a2, a5 = a4 * a, a6 = a3 * a3, a7 = a6 * a;
  const double a10 = a5 * a5, a12 = a6 * a6;
  out.c[0] = N0;
  out.c[1] = N0 * a2 * phi2;
  out.c[2] = N0 * a3 * phi3;
  out.c[3] = N0 * a4 * phi4;
  out.c[4] = N0 * a5 * phi5p;                                                 // ln f
  out.c[5] = N0 * a6 * (phi6c - (6848.0 / 21.0) * (log(4.0) + u / 3.0));      // f^1/3
  out.c[6] = N0 * a6 * (-6848.0 / 63.0);                                      // f^1/3 ln f
  out.c[7] = N0 * a7 * phi7;
  out.c[8] = N0 * a10 * phi10;
  out.c[9] = N0 * a12 * phi12;
  // constant: -phi_c - pi/4 + the v^0 part of the 2.5PN term, 1 - 3 ln v_lso + ln(pi M) (v_lso = 6^-1/2)
  out.phi0 = -phic - 0.25 * kPi + N0 * a5 * phi5p * (1.0 + 1.5 * log(6.0) + u);
  out.amp = exp((5.0 / 6.0) * log(Mc)) / dL;

  // Detector projection.
  double sd, cd, sa, ca;
  sincos(dec, &sd, &cd);
  sincos(ra - ec.gmst, &sa, &ca);
  const double n0 = cd * ca, n1 = cd * sa, n2 = sd;
  // antenna patterns in FP32 (angles are O(1); relative error ~1e-7)
  float sgf, cgf, sdf, cdf, spf, cpf;
  sincosf((float)(ec.gmst - ra), &sgf, &cgf);
  sincosf((float)dec, &sdf, &cdf);
  sincosf((float)psi, &spf, &cpf);
  const float cif = cosf((float)iota);
  const float Xf[3] = {-cpf * sgf - spf * cgf * sdf, -cpf * cgf + spf * sgf * sdf, spf * cdf};
  const float Yf[3] = {spf * sgf - cpf * cgf * sdf, spf * cgf + cpf * sgf * sdf, cpf * cdf};
  for (int d = 0; d < ec.n_det; ++d) {
    const DetGeom& g = ec.det[d];
    out.tau[d] = tc - (n0 * g.r[0] + n1 * g.r[1] + n2 * g.r[2]) / kClight;
    float fp = 0.f, fx = 0.f;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const float Dij = (float)g.D[i][j];
        fp += Dij * (Xf[i] * Xf[j] - Yf[i] * Yf[j]);
        fx += Dij * (Xf[i] * Yf[j] + Yf[i] * Xf[j]);
      }
    out.P32[d][0] = fp * (1.0f + cif * cif) * 0.5f;
    out.P32[d][1] = -fx * cif;
  }
  if (need64) {
    double sg, cg, sp, cp;
    sincos(ec.gmst - ra, &sg, &cg);
    sincos(psi, &sp, &cp);
    const double ci = cos(iota);
    const double X[3] = {-cp * sg - sp * cg * sd, -cp * cg + sp * sg * sd, sp * cd};
    const double Y[3] = {sp * sg - cp * cg * sd, sp * cg + cp * sg * sd, cp * cd};
    for (int d = 0; d < ec.n_det; ++d) {
      const DetGeom& g = ec.det[d];
      double fp = 0.0, fx = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          fp += g.D[i][j] * (X[i] * X[j] - Y[i] * Y[j]);
          fx += g.D[i][j] * (X[i] * Y[j] + Y[i] * X[j]);
        }
      out.P64[d][0] = fp * (1.0 + ci * ci) * 0.5;
      out.P64[d][1] = -fx * ci;
    }
  }
}

// ---------------------------------------------------------------------------
// Small forward-mode dual numbers for the tangents (T = float or double).
// ---------------------------------------------------------------------------
template <class T, int N>
struct Du {
  T v;
  T d[N];
};
template <class T, int N> __device__ __forceinline__ Du<T, N> du_const(T x) {
  Du<T, N> r; r.v = x;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = T(0);
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> du_var(T x, int k) {
  Du<T, N> r = du_const<T, N>(x); r.d[k] = T(1); return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator+(const Du<T, N>& a, const Du<T, N>& b) {
  Du<T, N> r; r.v = a.v + b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] + b.d[i];
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator-(const Du<T, N>& a, const Du<T, N>& b) {
  Du<T, N> r; r.v = a.v - b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] - b.d[i];
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator*(const Du<T, N>& a, const Du<T, N>& b) {
  Du<T, N> r; r.v = a.v * b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i];
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator/(const Du<T, N>& a, const Du<T, N>& b) {
  Du<T, N> r; r.v = a.v / b.v;
  const T ib = T(1) / b.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = (a.d[i] - r.v * b.d[i]) * ib;
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator*(T s, const Du<T, N>& a) {
  Du<T, N> r; r.v = s * a.v;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = s * a.d[i];
  return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> operator+(T s, const Du<T, N>& a) {
  Du<T, N> r = a; r.v = s + a.v; return r;
}
template <class T, int N> __device__ __forceinline__ Du<T, N> du_chain(const Du<T, N>& a, T fv, T dfv) {
  Du<T, N> r; r.v = fv;
#pragma unroll
  for (int i = 0; i < N; ++i) r.d[i] = dfv * a.d[i];
  return r;
}
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
template <class T, int N> __device__ __forceinline__ Du<T, N> du_log(const Du<T, N>& a) {
  return du_chain(a, m_log(a.v), T(1) / a.v);
}
template <class T, int N> __device__ __forceinline__ Du<T, N> du_exp(const Du<T, N>& a) {
  T e = m_exp(a.v); return du_chain(a, e, e);
}
template <class T, int N> __device__ __forceinline__ void du_sincos(const Du<T, N>& a, Du<T, N>& s, Du<T, N>& c) {
  T sv, cv; m_sincos(a.v, &sv, &cv);
  s = du_chain(a, sv, cv);
  c = du_chain(a, cv, -sv);
}

// Tangents of the phase coefficients and constant phase with respect to
// (Mc, q, chi1, chi2, Lambda1, Lambda2), and of the detector quantities with
// respect to (iota, psi, ra, dec).  Same formulas as walker_values, carried in
// precision T (FP32 suffices for the mixed paths: tangents need ~1e-6).
template <class T>
__device__ void walker_tangents(const double* th, const EventConst& ec, WalkerTan<T>& o) {
  using D6 = Du<T, kNTanIntr>;
  const D6 Mc = du_var<T, kNTanIntr>(T(th[0]), 0), q = du_var<T, kNTanIntr>(T(th[1]), 1);
  const D6 chi1 = du_var<T, kNTanIntr>(T(th[2]), 2), chi2 = du_var<T, kNTanIntr>(T(th[3]), 3);
  const D6 L1 = du_var<T, kNTanIntr>(T(th[4]), 4), L2 = du_var<T, kNTanIntr>(T(th[5]), 5);
  const D6 one = du_const<T, kNTanIntr>(T(1));
  const D6 opq = one + q;
  const D6 eta = q / (opq * opq);
  const D6 X1 = one / opq, X2 = q / opq;
  const D6 X1_2 = X1 * X1, X2_2 = X2 * X2, X1_4 = X1_2 * X1_2, X2_4 = X2_2 * X2_2;
  const D6 beta = T(1.0 / 12.0) * (chi1 * (T(113) * X1_2 + T(75) * eta) + chi2 * (T(113) * X2_2 + T(75) * eta));
  const D6 sigma = T(474.0 / 48.0) * (eta * chi1 * chi2) + T(486.0 / 96.0) * (X1_2 * chi1 * chi1 + X2_2 * chi2 * chi2);
  const D6 phi2 = T(3715.0 / 756.0) + T(55.0 / 9.0) * eta;
  const D6 phi3 = T(-16.0 * kPi) + T(4) * beta;
  const D6 phi4 = T(15293365.0 / 508032.0) + T(27145.0 / 504.0) * eta + T(3085.0 / 72.0) * (eta * eta) - T(10) * sigma;
  const D6 phi5p = T(kPi * 38645.0 / 756.0) + T(-kPi * 65.0 / 9.0) * eta;
  const D6 phi6c = T(11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kEulerGamma) +
                   T(-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) * eta +
                   T(76055.0 / 1728.0) * (eta * eta) + T(-127825.0 / 1296.0) * (eta * eta * eta);
  const D6 phi7 = T(kPi * 77096675.0 / 254016.0) + T(kPi * 378515.0 / 1512.0) * eta + T(-kPi * 74045.0 / 756.0) * (eta * eta);
  const D6 phi10 = (T(-288) + T(264) * X1) * X1_4 * L1 + (T(-288) + T(264) * X2) * X2_4 * L2;
  const D6 phi12 =
      X1_4 * L1 * (T(-15895.0 / 28.0) + T(4595.0 / 28.0) * X1 + T(5715.0 / 14.0) * X1_2 + T(-325.0 / 7.0) * (X1_2 * X1)) +
      X2_4 * L2 * (T(-15895.0 / 28.0) + T(4595.0 / 28.0) * X2 + T(5715.0 / 14.0) * X2_2 + T(-325.0 / 7.0) * (X2_2 * X2));
  const D6 lnMc = du_log(T(kPi * kMsunS) * Mc);
  const D6 u = lnMc + T(-0.6) * du_log(eta);
  const D6 a = du_exp(T(1.0 / 3.0) * u);
  const D6 N0 = T(3.0 / 128.0) * du_exp(T(-5.0 / 3.0) * lnMc);
  const D6 a2 = a * a, a3 = a2 * a, a4 = a2 * a2, a5 = a4 * a, a6 = a3 * a3, a7 = a6 * a, a10 = a5 * a5, a12 = a6 * a6;
  D6 c[kNBasis];
  c[0] = N0;
  c[1] = N0 * a2 * phi2;
  c[2] = N0 * a3 * phi3;
  c[3] = N0 * a4 * phi4;
  c[4] = N0 * a5 * phi5p;
  c[5] = N0 * a6 * (phi6c + T(-6848.0 / 21.0) * (T(1.3862943611198906) + T(1.0 / 3.0) * u));
  c[6] = T(-6848.0 / 63.0) * (N0 * a6);
  c[7] = N0 * a7 * phi7;
  c[8] = N0 * a10 * phi10;
  c[9] = N0 * a12 * phi12;
  const D6 phi0v = N0 * a5 * phi5p * (T(1.0 + 1.5 * 1.791759469228055) + u);  // ln 6 = 1.7917594692
  for (int k = 0; k < kNBasis; ++k)
    for (int j = 0; j < kNTanIntr; ++j) o.dc[k][j] = c[k].d[j];
  o.dphi0[0] = phi0v.d[0];
  o.dphi0[1] = phi0v.d[1];
  o.lnamp_Mc = T(5.0 / 6.0) / T(th[0]);
  o.lnamp_dL = T(-1) / T(th[6]);

  // detector tangents: variables (iota, psi, ra, dec)
  using D4 = Du<T, 4>;
  const D4 iota = du_var<T, 4>(T(th[9]), 0), psi = du_var<T, 4>(T(th[10]), 1);
  const D4 ra = du_var<T, 4>(T(th[11]), 2), dec = du_var<T, 4>(T(th[12]), 3);
  const D4 g = T(ec.gmst) + T(-1) * ra;
  D4 sg, cg, sd, cd, sp, cp, si, ci;
  du_sincos(g, sg, cg);
  du_sincos(dec, sd, cd);
  du_sincos(psi, sp, cp);
  du_sincos(iota, si, ci);
  const D4 X[3] = {T(-1) * (cp * sg) - sp * cg * sd, T(-1) * (cp * cg) + sp * sg * sd, sp * cd};
  const D4 Y[3] = {sp * sg - cp * cg * sd, sp * cg + cp * sg * sd, cp * cd};
  // sky direction n(ra - gmst, dec) = (cd cos(-g), cd sin(-g), sd) = (cd cg, -cd sg, sd)
  const D4 n[3] = {cd * cg, T(-1) * (cd * sg), sd};
  for (int d = 0; d < kMaxDet; ++d) {
    if (d >= ec.n_det) {
      for (int j = 0; j < 2; ++j) o.dtd[d][j] = T(0);
      for (int j = 0; j < 4; ++j) o.dlnP[d][j][0] = o.dlnP[d][j][1] = T(0);
      continue;
    }
    const DetGeom& G = ec.det[d];
    D4 fp = du_const<T, 4>(T(0)), fx = du_const<T, 4>(T(0));
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        const T Dij = T(G.D[i][j]);
        fp = fp + Dij * (X[i] * X[j] - Y[i] * Y[j]);
        fx = fx + Dij * (X[i] * Y[j] + Y[i] * X[j]);
      }
    const D4 Pr = T(0.5) * (fp * (T(1) + ci * ci));
    const D4 Pi = T(-1) * (fx * ci);
    const T den = Pr.v * Pr.v + Pi.v * Pi.v;
    for (int j = 0; j < 4; ++j) {
      // d ln P = dP / P = dP conj(P) / |P|^2
      o.dlnP[d][j][0] = (Pr.d[j] * Pr.v + Pi.d[j] * Pi.v) / den;
      o.dlnP[d][j][1] = (Pi.d[j] * Pr.v - Pr.d[j] * Pi.v) / den;
    }
    const D4 dt = T(-1.0 / kClight) * (T(G.r[0]) * n[0] + T(G.r[1]) * n[1] + T(G.r[2]) * n[2]);
    o.dtd[d][0] = dt.d[2];
    o.dtd[d][1] = dt.d[3];
  }
}

// ---------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------
__global__ void k_ref_values(const double* theta, EventConst ec, RefValues* out) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double th[kNPar];
    for (int j = 0; j < kNPar; ++j) th[j] = theta[j];
    walker_values(th, ec, 1, out->v);
  }
}

__device__ __forceinline__ void load_theta(const double* __restrict__ theta, int64_t w, double* th) {
#pragma unroll
  for (int j = 0; j < kNPar; ++j) th[j] = theta[w * kNPar + j];
}

__device__ __forceinline__ double wrap_pi(double x) { return x - kTwoPi * rint(x * (1.0 / kTwoPi)); }

template <bool GRAD>
__global__ void __launch_bounds__(128) k_setup_mixed(const double* __restrict__ theta, int64_t W, EventConst ec,
                                                     const RefValues* __restrict__ ref, WalkerMixed* __restrict__ ws,
                                                     WalkerTan<float>* __restrict__ tan) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double th[kNPar];
  load_theta(theta, w, th);
  Values v;
  walker_values(th, ec, 1, v);
  WalkerMixed o;
  o.valid = v.valid;
  o.pad[0] = o.pad[1] = o.pad[2] = 0;
  if (v.valid) {
    const Values& r = ref->v;
    for (int k = 0; k < kNBasis; ++k) {
      f2x c = f2x_from(v.c[k] - r.c[k]);
      o.dc_hi[k] = c.hi;
      o.dc_lo[k] = c.lo;
    }
    // The prefactor ratio is formed in FP64: F+ = D:(XX - YY) cancels, and
    // an FP32 antenna pattern can be off by ~1e-7 absolute, i.e. up to ~1e-5
    // relative, which moves log L by ~1e-3 at SNR ~ 100.
    double sp, cp;
    sincos(wrap_pi(v.phi0 - r.phi0), &sp, &cp);
    const double ampr = v.amp / r.amp;
    for (int d = 0; d < kMaxDet; ++d) {
      if (d < ec.n_det) {
        f2x t = f2x_from(v.tau[d] - r.tau[d]);
        o.tau_hi[d] = t.hi;
        o.tau_lo[d] = t.lo;
        // Q = ampr P e^{-i dphi0};  rho = Q / P_ref;  sig = (Q - P_ref) / P_ref
        const double pr = v.P64[d][0], pi = v.P64[d][1];
        const double qr = ampr * (pr * cp + pi * sp);
        const double qi = ampr * (pi * cp - pr * sp);
        const double rr = r.P64[d][0], ri = r.P64[d][1];
        const double den = rr * rr + ri * ri;
        o.rho[d][0] = (float)((qr * rr + qi * ri) / den);
        o.rho[d][1] = (float)((qi * rr - qr * ri) / den);
        const double er = qr - rr, ei = qi - ri;
        o.sig[d][0] = (float)((er * rr + ei * ri) / den);
        o.sig[d][1] = (float)((ei * rr - er * ri) / den);
      } else {
        o.tau_hi[d] = o.tau_lo[d] = 0.f;
        o.rho[d][0] = o.rho[d][1] = o.sig[d][0] = o.sig[d][1] = 0.f;
      }
    }
  }
  ws[w] = o;
  if (GRAD && v.valid) {
    WalkerTan<float> t;
    walker_tangents<float>(th, ec, t);
    tan[w] = t;
  }
}

template <bool GRAD, class TanT>
__global__ void __launch_bounds__(128) k_setup_f64(const double* __restrict__ theta, int64_t W, EventConst ec,
                                                   const RefValues* __restrict__ ref, WalkerF64* __restrict__ ws,
                                                   WalkerTan<TanT>* __restrict__ tan) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  double th[kNPar];
  load_theta(theta, w, th);
  Values v;
  walker_values(th, ec, 1, v);
  WalkerF64 o;
  o.valid = v.valid;
  o.pad = 0;
  if (v.valid) {
    const Values& r = ref->v;
    for (int k = 0; k < kNBasis; ++k) o.dc[k] = v.c[k] - r.c[k];
    double sp, cp;
    sincos(wrap_pi(v.phi0 - r.phi0), &sp, &cp);
    const double ampr = v.amp / r.amp;
    for (int d = 0; d < kMaxDet; ++d) {
      if (d < ec.n_det) {
        o.tau[d] = v.tau[d] - r.tau[d];
        const double pr = v.P64[d][0], pi = v.P64[d][1];
        const double qr = ampr * (pr * cp + pi * sp);
        const double qi = ampr * (pi * cp - pr * sp);
        const double rr = r.P64[d][0], ri = r.P64[d][1];
        const double den = rr * rr + ri * ri;
        o.rho[d][0] = (qr * rr + qi * ri) / den;
        o.rho[d][1] = (qi * rr - qr * ri) / den;
        const double er = qr - rr, ei = qi - ri;
        o.sig[d][0] = (er * rr + ei * ri) / den;
        o.sig[d][1] = (ei * rr - er * ri) / den;
      } else {
        o.tau[d] = 0.0;
        o.rho[d][0] = o.rho[d][1] = o.sig[d][0] = o.sig[d][1] = 0.0;
      }
    }
  } else {
    for (int k = 0; k < kNBasis; ++k) o.dc[k] = 0.0;
    for (int d = 0; d < kMaxDet; ++d) {
      o.tau[d] = 0.0;
      o.rho[d][0] = o.rho[d][1] = o.sig[d][0] = o.sig[d][1] = 0.0;
    }
  }
  ws[w] = o;
  if (GRAD && v.valid) {
    WalkerTan<TanT> t;
    walker_tangents<TanT>(th, ec, t);
    tan[w] = t;
  }
}

// Host-side launchers (declared in rb_launch.h).
cudaError_t launch_ref_values(const double* theta_ref_dev, const EventConst& ec, RefValues* out, cudaStream_t s) {
  k_ref_values<<<1, 32, 0, s>>>(theta_ref_dev, ec, out);
  return cudaGetLastError();
}

cudaError_t launch_setup_mixed(const double* theta, int64_t W, const EventConst& ec, const RefValues* ref,
                               WalkerMixed* ws, WalkerTan<float>* tan, bool grad, cudaStream_t s) {
  const int bs = 128;
  const unsigned grid = (unsigned)((W + bs - 1) / bs);
  if (grad)
    k_setup_mixed<true><<<grid, bs, 0, s>>>(theta, W, ec, ref, ws, tan);
  else
    k_setup_mixed<false><<<grid, bs, 0, s>>>(theta, W, ec, ref, ws, tan);
  return cudaGetLastError();
}

// tan: WalkerTan<double> (tan_f32 = false) or WalkerTan<float> (tan_f32 = true).
cudaError_t launch_setup_f64(const double* theta, int64_t W, const EventConst& ec, const RefValues* ref,
                             WalkerF64* ws, void* tan, bool grad, bool tan_f32, cudaStream_t s) {
  const int bs = 128;
  const unsigned grid = (unsigned)((W + bs - 1) / bs);
  if (!grad)
    k_setup_f64<false, double><<<grid, bs, 0, s>>>(theta, W, ec, ref, ws, nullptr);
  else if (tan_f32)
    k_setup_f64<true, float><<<grid, bs, 0, s>>>(theta, W, ec, ref, ws, static_cast<WalkerTan<float>*>(tan));
  else
    k_setup_f64<true, double><<<grid, bs, 0, s>>>(theta, W, ec, ref, ws, static_cast<WalkerTan<double>*>(tan));
  return cudaGetLastError();
}

}  // namespace rb
