// rb_setup.cu -- per-walker set-up (steps a1/a2): theta -> phase-basis
// coefficients, constant phase, detector delays and complex prefactors, and
// (for the gradient) their tangents.
//
// Waveform (Sec. II.B; TaylorF2 from the PN literature cited there):
//   h+ = A f^-7/6 (1+cos^2 i)/2 e^{-i Psi},  hx = -i A f^-7/6 cos i e^{-i Psi},
//   A = sqrt(5/24) pi^-2/3 Mc^5/6 / d_L,
//   Psi = 2 pi f t_c - phi_c - pi/4 + 3/(128 eta v^5) sum_k phi_k v^k, v = (pi M f)^1/3,
// point-particle phi_k to 3.5PN, aligned-spin 1.5PN (beta) and 2PN (sigma,
// kappa = 1) terms, and 5PN/6PN tidal terms written per body (equivalent to
// the Lambda-tilde / delta-Lambda-tilde form of the paper's appendix).
// Detector response: h_d = (F+ h+ + Fx hx) e^{-2 pi i f dt_d}, dt_d = -n.r_d/c.
//
// On sm_103a an FP64 warp instruction occupies its SM sub-partition's FP64
// unit for ~65 cycles whatever the number of active lanes, so what limits
// this step is the number of FP64 instructions each warp issues.  A block
// handles 32 walkers (one per lane) and splits each walker's FP64 work into
// roles run by different warps, exchanging results through shared memory:
//   phase 1  warp 0: ln(pi Mc), (pi Mc)^-5/3, (pi Mc)^1/3, Mc^5/6 / d_L
//            warp 1: eta, ln eta, eta^-1/5
//            warp 2: PN coefficients phi_k (polynomials in eta, X_i, chi_i, Lambda_i)
//            warp 3: sky direction, detector delays tau_d = t_c + dt_d
//            warp 4: polarisation and inclination sines/cosines
//   phase 2  warp 0: basis coefficients c_k, constant phase Phi0, their
//                    differences to the fiducial values, exp(-i dPhi0) - 1
//            warps 1-3: antenna factor P_d = F+ (1+cos^2 i)/2 - i Fx cos i (FP64,
//                    since F+ = D:(XX - YY) cancels)
//            warp 4: delay differences
//   phase 3  warps 1-3: prefactor ratio rho_d and rho_d - 1
//   (gradient) warps 5, 6: tangents in FP32 (mixed) or FP64 dual numbers.
// Every role is a noinline function, so a walker at theta_ref reproduces the
// fiducial values bit for bit (the reference kernel runs the same roles).
#include <type_traits>

#include "rb.h"
#include "rb_dd.cuh"
#include "rb_internal.cuh"

namespace rb {

constexpr int kSetupWalkers = 32;
constexpr int kRoleThreads = 5 * 32;  // warps 0-4 take part in the FP64 phases

// Barrier over the FP64-phase warps only (the tangent warps run on their own).
__device__ __forceinline__ void roles_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kRoleThreads) : "memory"); }

// ---------------------------------------------------------------------------
// Roles (FP64).  noinline: one instruction sequence for every caller.
// ---------------------------------------------------------------------------
__device__ __noinline__ void role_mass(double Mc, double dL, double* lnMc, double* N0, double* a1, double* amp) {
  const double l = log(kPi * Mc * kMsunS);
  *lnMc = l;
  *N0 = (3.0 / 128.0) * exp(-(5.0 / 3.0) * l);
  *a1 = exp(l * (1.0 / 3.0));
  // Mc^5/6 / d_L  (Msun^5/6 / Mpc):  Mc^5/6 = exp(5/6 l) / (pi G Msun / c^3)^5/6
  *amp = exp((5.0 / 6.0) * l) * (1.0 / 9.802409278970853e-05) / dL;
}

__device__ __noinline__ void role_eta(double q, double* eta, double* lneta, double* a2) {
  const double opq = 1.0 + q;
  const double e = q / (opq * opq);
  const double le = log(e);
  *eta = e;
  *lneta = le;
  *a2 = exp(-0.2 * le);  // eta^-1/5
}

// phi: phi2, phi3, phi4, phi5p, phi6c, phi7, phi10, phi12
__device__ __noinline__ void role_pn(double q, double chi1, double chi2, double L1, double L2, double* phi) {
  const double opq = 1.0 + q;
  const double eta = q / (opq * opq);
  const double X1 = 1.0 / opq, X2 = q / opq;
  const double X1_2 = X1 * X1, X2_2 = X2 * X2;
  const double X1_4 = X1_2 * X1_2, X2_4 = X2_2 * X2_2;
  const double beta = (chi1 * (113.0 * X1_2 + 75.0 * eta) + chi2 * (113.0 * X2_2 + 75.0 * eta)) / 12.0;
  const double sigma = eta * (474.0 / 48.0) * chi1 * chi2 + (486.0 / 96.0) * (X1_2 * chi1 * chi1 + X2_2 * chi2 * chi2);
  phi[0] = 3715.0 / 756.0 + (55.0 / 9.0) * eta;
  phi[1] = -16.0 * kPi + 4.0 * beta;
  phi[2] = 15293365.0 / 508032.0 + (27145.0 / 504.0) * eta + (3085.0 / 72.0) * eta * eta - 10.0 * sigma;
  phi[3] = kPi * (38645.0 / 756.0 - (65.0 / 9.0) * eta);
  phi[4] = 11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kEulerGamma +
           eta * (-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) + (76055.0 / 1728.0) * eta * eta -
           (127825.0 / 1296.0) * eta * eta * eta;
  phi[5] = kPi * (77096675.0 / 254016.0 + (378515.0 / 1512.0) * eta - (74045.0 / 756.0) * eta * eta);
  phi[6] = (-288.0 + 264.0 * X1) * X1_4 * L1 + (-288.0 + 264.0 * X2) * X2_4 * L2;
  phi[7] = X1_4 * L1 * (-15895.0 / 28.0 + 4595.0 / 28.0 * X1 + 5715.0 / 14.0 * X1_2 - 325.0 / 7.0 * X1_2 * X1) +
           X2_4 * L2 * (-15895.0 / 28.0 + 4595.0 / 28.0 * X2 + 5715.0 / 14.0 * X2_2 - 325.0 / 7.0 * X2_2 * X2);
}

// sky: sin/cos dec, sin/cos (ra - gmst); tau_d = t_c - n.r_d / c
__device__ __noinline__ void role_sky(double ra, double dec, double tc, const EventConst& ec, double* sky,
                                      double* tau) {
  double sd, cd, sa, ca;
  sincos(dec, &sd, &cd);
  sincos(ra - ec.gmst, &sa, &ca);
  sky[0] = sd;
  sky[1] = cd;
  sky[2] = sa;
  sky[3] = ca;
  const double n0 = cd * ca, n1 = cd * sa, n2 = sd;
  for (int d = 0; d < kMaxDet; ++d) {
    const DetGeom& g = ec.det[d];
    tau[d] = (d < ec.n_det) ? tc - (n0 * g.r[0] + n1 * g.r[1] + n2 * g.r[2]) / kClight : 0.0;
  }
}

__device__ __noinline__ void role_orient(double psi, double iota, double* o) {
  double sp, cp;
  sincos(psi, &sp, &cp);
  o[0] = sp;
  o[1] = cp;
  o[2] = cos(iota);
}

// c_k and Phi0 from the phase-1 results (see walker layout in rb_internal.cuh)
__device__ __noinline__ void role_coef(double lnMc, double N0, double a1, double a2, double lneta, const double* phi,
                                       double phic, double* c, double* phi0) {
  const double u = lnMc - 0.6 * lneta;  // ln(pi M)
  const double a = a1 * a2;             // (pi M)^1/3
  const double a2p = a * a, a3 = a2p * a, a4 = a2p * a2p, a5 = a4 * a, a6 = a3 * a3, a7 = a6 * a;
  const double a10 = a5 * a5, a12 = a6 * a6;
  c[0] = N0;
  c[1] = N0 * a2p * phi[0];
  c[2] = N0 * a3 * phi[1];
  c[3] = N0 * a4 * phi[2];
  c[4] = N0 * a5 * phi[3];                                                    // ln f
  c[5] = N0 * a6 * (phi[4] - (6848.0 / 21.0) * (1.3862943611198906 + u / 3.0));  // f^1/3 (ln 4 = 1.386...)
  c[6] = N0 * a6 * (-6848.0 / 63.0);                                          // f^1/3 ln f
  c[7] = N0 * a7 * phi[5];
  c[8] = N0 * a10 * phi[6];
  c[9] = N0 * a12 * phi[7];
  // -phi_c - pi/4 + the v^0 part of the 2.5PN term, 1 - 3 ln v_lso + ln(pi M), v_lso = 6^-1/2
  *phi0 = -phic - 0.25 * kPi + N0 * a5 * phi[3] * (1.0 + 1.5 * 1.791759469228055 + u);
}

// P_d = F+ (1 + cos^2 i)/2 - i Fx cos i,  F+ = X.DX - Y.DY,  Fx = X.DY + Y.DX
__device__ __noinline__ void role_antenna(const DetGeom& g, const double* sky, const double* ori, double* P) {
  const double sd = sky[0], cd = sky[1], sg = -sky[2], cg = sky[3];  // g = gmst - ra
  const double sp = ori[0], cp = ori[1], ci = ori[2];
  const double X[3] = {-cp * sg - sp * cg * sd, -cp * cg + sp * sg * sd, sp * cd};
  const double Y[3] = {sp * sg - cp * cg * sd, sp * cg + cp * sg * sd, cp * cd};
  double DX[3], DY[3];
  for (int i = 0; i < 3; ++i) {
    DX[i] = g.D[i][0] * X[0] + g.D[i][1] * X[1] + g.D[i][2] * X[2];
    DY[i] = g.D[i][0] * Y[0] + g.D[i][1] * Y[1] + g.D[i][2] * Y[2];
  }
  const double fp = (X[0] * DX[0] + X[1] * DX[1] + X[2] * DX[2]) - (Y[0] * DY[0] + Y[1] * DY[1] + Y[2] * DY[2]);
  const double fx = (X[0] * DY[0] + X[1] * DY[1] + X[2] * DY[2]) + (Y[0] * DX[0] + Y[1] * DX[1] + Y[2] * DX[2]);
  P[0] = fp * (1.0 + ci * ci) * 0.5;
  P[1] = -fx * ci;
}

__device__ __forceinline__ bool theta_valid(const double* th) {
  bool ok = true;
  for (int j = 0; j < kNPar; ++j) ok = ok && isfinite(th[j]);
  return ok && th[0] > 0.0 && th[1] > 0.0 && th[1] <= 1.0 && th[6] > 0.0;
}

__device__ __forceinline__ double wrap_pi(double x) { return x - kTwoPi * rint(x * (1.0 / kTwoPi)); }

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
// One warp computes the derivatives with respect to one pair of variables,
// part 0: (Mc, q), part 1: (chi1, chi2), part 2: (Lambda1, Lambda2).
template <class T>
__device__ void tangents_intrinsic(const double* th, int part, WalkerTan<T>& o) {
  using DI = Du<T, 2>;
  auto var = [&](int v) { return (v >> 1) == part ? du_var<T, 2>(T(th[v]), v & 1) : du_const<T, 2>(T(th[v])); };
  const DI Mc = var(0), q = var(1);
  const DI chi1 = var(2), chi2 = var(3);
  const DI L1 = var(4), L2 = var(5);
  const DI one = du_const<T, 2>(T(1));
  const DI opq = one + q;
  const DI eta = q / (opq * opq);
  const DI X1 = one / opq, X2 = q / opq;
  const DI X1_2 = X1 * X1, X2_2 = X2 * X2, X1_4 = X1_2 * X1_2, X2_4 = X2_2 * X2_2;
  const DI beta = T(1.0 / 12.0) * (chi1 * (T(113) * X1_2 + T(75) * eta) + chi2 * (T(113) * X2_2 + T(75) * eta));
  const DI sigma = T(474.0 / 48.0) * (eta * chi1 * chi2) + T(486.0 / 96.0) * (X1_2 * chi1 * chi1 + X2_2 * chi2 * chi2);
  const DI phi2 = T(3715.0 / 756.0) + T(55.0 / 9.0) * eta;
  const DI phi3 = T(-16.0 * kPi) + T(4) * beta;
  const DI phi4 = T(15293365.0 / 508032.0) + T(27145.0 / 504.0) * eta + T(3085.0 / 72.0) * (eta * eta) - T(10) * sigma;
  const DI phi5p = T(kPi * 38645.0 / 756.0) + T(-kPi * 65.0 / 9.0) * eta;
  const DI phi6c = T(11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kEulerGamma) +
                   T(-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi) * eta +
                   T(76055.0 / 1728.0) * (eta * eta) + T(-127825.0 / 1296.0) * (eta * eta * eta);
  const DI phi7 = T(kPi * 77096675.0 / 254016.0) + T(kPi * 378515.0 / 1512.0) * eta + T(-kPi * 74045.0 / 756.0) * (eta * eta);
  const DI phi10 = (T(-288) + T(264) * X1) * X1_4 * L1 + (T(-288) + T(264) * X2) * X2_4 * L2;
  const DI phi12 =
      X1_4 * L1 * (T(-15895.0 / 28.0) + T(4595.0 / 28.0) * X1 + T(5715.0 / 14.0) * X1_2 + T(-325.0 / 7.0) * (X1_2 * X1)) +
      X2_4 * L2 * (T(-15895.0 / 28.0) + T(4595.0 / 28.0) * X2 + T(5715.0 / 14.0) * X2_2 + T(-325.0 / 7.0) * (X2_2 * X2));
  const DI lnMc = du_log(T(kPi * kMsunS) * Mc);
  const DI u = lnMc + T(-0.6) * du_log(eta);
  const DI a = du_exp(T(1.0 / 3.0) * u);
  const DI N0 = T(3.0 / 128.0) * du_exp(T(-5.0 / 3.0) * lnMc);
  const DI a2 = a * a, a3 = a2 * a, a4 = a2 * a2, a5 = a4 * a, a6 = a3 * a3, a7 = a6 * a, a10 = a5 * a5, a12 = a6 * a6;
  DI c[kNBasis];
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
  const DI phi0v = N0 * a5 * phi5p * (T(1.0 + 1.5 * 1.791759469228055) + u);  // ln 6 = 1.7917594692
  for (int k = 0; k < kNBasis; ++k)
    for (int j = 0; j < 2; ++j) o.dc[k][2 * part + j] = c[k].d[j];
  if (part == 0) {
    o.dphi0[0] = phi0v.d[0];
    o.dphi0[1] = phi0v.d[1];
    o.lnamp_Mc = T(5.0 / 6.0) / T(th[0]);
    o.lnamp_dL = T(-1) / T(th[6]);
  }
}

template <class T>
__device__ void tangents_detector(const double* th, const EventConst& ec, int d, WalkerTan<T>& o) {
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
  {
    if (d >= ec.n_det) {
      for (int j = 0; j < 2; ++j) o.dtd[d][j] = T(0);
      for (int j = 0; j < 4; ++j) o.dlnP[d][j][0] = o.dlnP[d][j][1] = T(0);
      return;
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
// The block-level set-up: 32 walkers, phases 1-3 over warps 0-4 (+ tangents).
// ---------------------------------------------------------------------------
struct SetupSmem {
  double th[kNPar][kSetupWalkers];
  double lnMc[kSetupWalkers], N0[kSetupWalkers], a1[kSetupWalkers], amp[kSetupWalkers];
  double eta[kSetupWalkers], lneta[kSetupWalkers], a2[kSetupWalkers];
  double phi[8][kSetupWalkers];
  double sky[4][kSetupWalkers], tau[kMaxDet][kSetupWalkers];
  double ori[3][kSetupWalkers];
  double c[kNBasis][kSetupWalkers], phi0[kSetupWalkers];
  double P[kMaxDet][2][kSetupWalkers];
  double e64[2][kSetupWalkers];   // exp(-i dPhi0)
  int valid[kSetupWalkers];
};

// Runs phases 1 and 2 for the walkers of this block and leaves the absolute
// values in shared memory.  Warps 0-4 (and only they) must call it.
__device__ void setup_absolute(const double* __restrict__ theta, int64_t w0, int64_t W, const EventConst& ec,
                               SetupSmem& S) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kNPar * kSetupWalkers; i += kRoleThreads) {
    const int l = i / kNPar, j = i % kNPar;
    const int64_t w = (w0 + l < W) ? w0 + l : W - 1;  // pad with the last walker
    S.th[j][l] = theta[w * kNPar + j];
  }
  roles_sync();
  const int l = lane;
  if (warp == 0) {
    double th[kNPar];
    for (int j = 0; j < kNPar; ++j) th[j] = S.th[j][l];
    S.valid[l] = theta_valid(th) ? 1 : 0;
    role_mass(th[0], th[6], &S.lnMc[l], &S.N0[l], &S.a1[l], &S.amp[l]);
  } else if (warp == 1) {
    role_eta(S.th[1][l], &S.eta[l], &S.lneta[l], &S.a2[l]);
  } else if (warp == 2) {
    double phi[8];
    role_pn(S.th[1][l], S.th[2][l], S.th[3][l], S.th[4][l], S.th[5][l], phi);
    for (int k = 0; k < 8; ++k) S.phi[k][l] = phi[k];
  } else if (warp == 3) {
    double sky[4], tau[kMaxDet];
    role_sky(S.th[11][l], S.th[12][l], S.th[7][l], ec, sky, tau);
    for (int k = 0; k < 4; ++k) S.sky[k][l] = sky[k];
    for (int d = 0; d < kMaxDet; ++d) S.tau[d][l] = tau[d];
  } else if (warp == 4) {
    double o[3];
    role_orient(S.th[10][l], S.th[9][l], o);
    for (int k = 0; k < 3; ++k) S.ori[k][l] = o[k];
  }
  roles_sync();
  if (warp == 0) {
    double phi[8], c[kNBasis], phi0;
    for (int k = 0; k < 8; ++k) phi[k] = S.phi[k][l];
    role_coef(S.lnMc[l], S.N0[l], S.a1[l], S.a2[l], S.lneta[l], phi, S.th[8][l], c, &phi0);
    for (int k = 0; k < kNBasis; ++k) S.c[k][l] = c[k];
    S.phi0[l] = phi0;
  } else if (warp >= 1 && warp <= kMaxDet) {
    const int d = warp - 1;
    if (d < ec.n_det) {
      double sky[4], ori[3], P[2];
      for (int k = 0; k < 4; ++k) sky[k] = S.sky[k][l];
      for (int k = 0; k < 3; ++k) ori[k] = S.ori[k][l];
      role_antenna(ec.det[d], sky, ori, P);
      S.P[d][0][l] = P[0];
      S.P[d][1][l] = P[1];
    } else {
      S.P[d][0][l] = S.P[d][1][l] = 0.0;
    }
  }
  roles_sync();
}

// Tangent warps of the set-up kernels: which = 0..2 take the derivatives
// with respect to one pair of intrinsic parameters, which = 3..5 those of
// detector which - 3 (the work is split so that no warp's chain is long).
constexpr int kTanWarps = 3 + kMaxDet;
template <class TanT>
__device__ void tangent_warp(const double* __restrict__ theta, int64_t W, int64_t w0, const EventConst& ec,
                             void* __restrict__ tan_out, int which) {
  const int lane = threadIdx.x & 31;
  const int64_t w = w0 + lane;
  const bool mine = w < W;
  double th[kNPar];
  const int64_t wc = mine ? w : W - 1;
  for (int j = 0; j < kNPar; ++j) th[j] = theta[wc * kNPar + j];
  WalkerTan<TanT>* tan = static_cast<WalkerTan<TanT>*>(tan_out) + wc;
  WalkerTan<TanT> t;
  if (which < 3) {
    tangents_intrinsic<TanT>(th, which, t);
    if (mine) {
      for (int k = 0; k < kNBasis; ++k)
        for (int j = 2 * which; j < 2 * which + 2; ++j) tan->dc[k][j] = t.dc[k][j];
      if (which == 0) {
        tan->dphi0[0] = t.dphi0[0];
        tan->dphi0[1] = t.dphi0[1];
        tan->lnamp_Mc = t.lnamp_Mc;
        tan->lnamp_dL = t.lnamp_dL;
      }
    }
  } else {
    const int d = which - 3;
    tangents_detector<TanT>(th, ec, d, t);
    if (mine) {
      tan->dtd[d][0] = t.dtd[d][0];
      tan->dtd[d][1] = t.dtd[d][1];
      for (int j = 0; j < 4; ++j) {
        tan->dlnP[d][j][0] = t.dlnP[d][j][0];
        tan->dlnP[d][j][1] = t.dlnP[d][j][1];
      }
    }
  }
}

// FP64 reference kernel (FP64 and FP64-phase paths): one block; every lane
// evaluates theta_ref.
__global__ void __launch_bounds__(7 * 32) k_ref_values(const double* theta, EventConst ec, RefValues* out) {
  __shared__ SetupSmem S;
  setup_absolute(theta, 0, 1, ec, S);
  if (threadIdx.x == 0) {
    Values v;
    for (int k = 0; k < kNBasis; ++k) v.c[k] = S.c[k][0];
    v.phi0 = S.phi0[0];
    for (int d = 0; d < kMaxDet; ++d) {
      v.tau[d] = S.tau[d][0];
      v.P64[d][0] = S.P[d][0][0];
      v.P64[d][1] = S.P[d][1][0];
      v.P32[d][0] = (float)v.P64[d][0];
      v.P32[d][1] = (float)v.P64[d][1];
    }
    v.amp = S.amp[0];
    v.valid = S.valid[0];
    v.pad = 0;
    out->v = v;
  }
}

// Batch set-up in FP64 for the FP64 paths: RB_FP64 writes WalkerF64 (+
// double tangents), RB_MIXED_F64PHASE writes WalkerF64 (+ float tangents).
// (RB_MIXED uses the float-float set-up, k_setup_dd.)
template <int MODE, bool GRAD>
__global__ void __launch_bounds__((5 + kTanWarps) * 32) k_setup(const double* __restrict__ theta, int64_t W, EventConst ec,
                                                  const RefValues* __restrict__ ref, void* __restrict__ ws_out,
                                                  void* __restrict__ tan_out) {
  static_assert(MODE == RB_FP64 || MODE == RB_MIXED_F64PHASE, "RB_MIXED uses the float-float set-up");
  using TanT = typename std::conditional<MODE == RB_FP64, double, float>::type;
  __shared__ SetupSmem S;
  const int64_t w0 = (int64_t)blockIdx.x * kSetupWalkers;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w = w0 + lane;
  const bool mine = w < W;
  if (warp >= 5) {
    // tangents (gradient only) do not depend on the FP64 phases: these warps
    // run them alongside and take no part in the role barriers
    if (GRAD) tangent_warp<TanT>(theta, W, w0, ec, tan_out, warp - 5);
    return;
  }
  setup_absolute(theta, w0, W, ec, S);
  const Values& r = ref->v;
  const int l = lane;
  if (warp == 0) {
    // constant-phase factor exp(-i dPhi0) (FP64; from the half angle for the FP64-phase mode)
    const double dphi0 = wrap_pi(S.phi0[l] - r.phi0);
    if (MODE == RB_FP64) {
      double sp, cp;
      sincos(dphi0, &sp, &cp);
      S.e64[0][l] = cp;
      S.e64[1][l] = -sp;
    } else {
      // exp(-i dPhi0) - 1 = -2 sin^2(pi y) - 2i sin(pi y) cos(pi y), y = dPhi0 / 2pi as a float pair,
      // plus the first-order term of the low part: d/dy exp(-2 pi i y) = -2 pi i exp(-2 pi i y)
      const double y64 = dphi0 * (1.0 / kTwoPi);
      const float yh = (float)y64, yl = (float)(y64 - (double)yh);
      float sn, cs;
      sincos_pi_half(yh, sn, cs);
      const float er = -2.f * sn * sn, ei = -2.f * sn * cs;
      const float t = 6.28318530717958648f * yl;
      S.e64[0][l] = 1.0 + ((double)er + (double)(ei * t));
      S.e64[1][l] = (double)ei - (double)((1.f + er) * t);
    }
  } else if (warp == 4 && mine) {
    for (int d = 0; d < kMaxDet; ++d) {
      const double dt = (d < ec.n_det) ? S.tau[d][l] - r.tau[d] : 0.0;
      static_cast<WalkerF64*>(ws_out)[w].tau[d] = dt;
    }
  }
  roles_sync();
  // phase 3: coefficient differences (warp 0) and prefactor ratios per detector (warps 1-3), FP64
  if (warp == 0 && mine) {
    WalkerF64* o = static_cast<WalkerF64*>(ws_out) + w;
    for (int k = 0; k < kNBasis; ++k) o->dc[k] = S.c[k][l] - r.c[k];
    o->valid = S.valid[l];
    o->pad = 0;
  } else if (warp >= 1 && warp <= kMaxDet && mine) {
    const int d = warp - 1;
    double rho_r = 0.0, rho_i = 0.0, sig_r = 0.0, sig_i = 0.0;
    if (d < ec.n_det) {
      // Q = ampr P exp(-i dPhi0);  rho = Q / P_ref;  sig = (Q - P_ref) / P_ref
      const double ampr = S.amp[l] / r.amp;
      const double er = S.e64[0][l], ei = S.e64[1][l];
      const double pr = S.P[d][0][l], pi = S.P[d][1][l];
      const double qr = ampr * (pr * er - pi * ei), qi = ampr * (pr * ei + pi * er);
      const double rr = r.P64[d][0], ri = r.P64[d][1];
      const double den = rr * rr + ri * ri;
      rho_r = (qr * rr + qi * ri) / den;
      rho_i = (qi * rr - qr * ri) / den;
      const double xr = qr - rr, xi = qi - ri;
      sig_r = (xr * rr + xi * ri) / den;
      sig_i = (xi * rr - xr * ri) / den;
    }
    WalkerF64* o = static_cast<WalkerF64*>(ws_out) + w;
    o->rho[d][0] = rho_r;
    o->rho[d][1] = rho_i;
    o->sig[d][0] = sig_r;
    o->sig[d][1] = sig_i;
  }
}


// ===========================================================================
// Mixed path: the same set-up in float-float arithmetic on the FP32 pipe
// (rb_dd.cuh).  Values are float pairs (hi, lo) with ~48 bits; the phase
// coefficients need ~1e-12 relative and the delays ~1e-12 s, well inside.
// Powers of the masses come from Newton roots instead of exp/log:
//   x = pi Mc (G Msun/c^3),  a1 = x^1/3,  N0 = (3/128) a1^-5,
//   Mc^5/6 = a1^5/2 / (pi G Msun/c^3)^5/6,  a = (pi M)^1/3 = a1 eta^-1/5,
// and one logarithm ln a = ln(pi M) / 3 (2.5PN and 3PN logarithmic terms).
// The antenna factor uses the arm unit vectors, F+ = ((x.X)^2 - (y.X)^2 -
// (x.Y)^2 + (y.Y)^2) / 2, Fx = (x.X)(x.Y) - (y.X)(y.Y), the same as D:(XX-YY)
// and D:(XY+YX) with D = (x x^T - y y^T)/2.
// Float-float chains are latency-bound, so the work of a walker is split
// into short roles on eight warps (phase 1: masses, eta, two halves of the PN
// polynomials, the four sines/cosines; phase 2: the logarithmic and the power
// parts of the coefficients, three antenna factors, the delays).  The whole
// set-up is one noinline function, so a walker at theta_ref reproduces the
// reference values bit for bit.
// ===========================================================================
namespace fx = rb::ffx;
using fx::dd;

constexpr int kDdRoleWarps = 8;
constexpr int kDdRoleThreads = kDdRoleWarps * 32;
__device__ __forceinline__ void ddroles_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kDdRoleThreads) : "memory"); }

__device__ __forceinline__ dd ld2(const float2& v) { return {v.x, v.y}; }
__device__ __forceinline__ float2 st2(dd v) { return make_float2(v.h, v.l); }
__device__ __forceinline__ dd ldp(const float* p) { return {p[0], p[1]}; }
__device__ __forceinline__ dd inv2pi() {
  constexpr fx::cdd c(1.0 / kTwoPi);
  return fx::K(c);
}

struct DdSmem {
  double th[kNPar][kSetupWalkers];
  float2 thd[kNPar][kSetupWalkers];  // theta as float pairs
  float2 a1[kSetupWalkers], N0[kSetupWalkers], amp[kSetupWalkers], e15[kSetupWalkers];
  float2 phi[8][kSetupWalkers];
  float2 trig[8][kSetupWalkers];  // sin/cos of dec, (ra - gmst), psi, iota
  float2 tau[kMaxDet][kSetupWalkers];
  float2 c[kNBasis][kSetupWalkers], phi0[kSetupWalkers];
  float2 P[kMaxDet][2][kSetupWalkers];
  float2 E[2][kSetupWalkers];  // exp(-i dPhi0)
  int valid[kSetupWalkers];
};

// PN polynomials phi2, phi3, phi4, phi5p (part 0) or phi6c, phi7, phi10,
// phi12 (part 1) of the walker (see the FP64 role).
__device__ __forceinline__ void ddpn(int part, dd qd, dd c1, dd c2, dd l1, dd l2, dd* phi) {
  using fx::add;
  using fx::mul;
  using fx::K;
  const dd opq = add(qd, 1.f);
  const dd X1 = fx::div(1.f, opq), X2 = fx::div(qd, opq);
  const dd eta = mul(X1, X2);
  const dd eta2 = fx::sqr(eta);
  const dd X1_2 = fx::sqr(X1), X2_2 = fx::sqr(X2);
  if (part == 0) {
    const dd e75 = mul(eta, 75.f);
    // beta = (chi1 (113 X1^2 + 75 eta) + chi2 (113 X2^2 + 75 eta)) / 12
    constexpr fx::cdd k12(1.0 / 12.0);
    const dd beta = mul(add(mul(c1, add(mul(X1_2, 113.f), e75)), mul(c2, add(mul(X2_2, 113.f), e75))), K(k12));
    // sigma = eta (474/48) chi1 chi2 + (486/96) (X1^2 chi1^2 + X2^2 chi2^2)
    constexpr fx::cdd k474(474.0 / 48.0), k486(486.0 / 96.0);
    const dd sigma = add(mul(mul(mul(eta, c1), c2), K(k474)),
                         mul(add(mul(X1_2, fx::sqr(c1)), mul(X2_2, fx::sqr(c2))), K(k486)));
    constexpr fx::cdd p2a(3715.0 / 756.0), p2b(55.0 / 9.0);
    phi[0] = add(K(p2a), mul(eta, K(p2b)));
    constexpr fx::cdd p3a(-16.0 * kPi);
    phi[1] = add(K(p3a), mul(beta, 4.f));
    constexpr fx::cdd p4a(15293365.0 / 508032.0), p4b(27145.0 / 504.0), p4c(3085.0 / 72.0);
    phi[2] = add(add(add(K(p4a), mul(eta, K(p4b))), mul(eta2, K(p4c))), mul(sigma, -10.f));
    constexpr fx::cdd p5a(kPi * 38645.0 / 756.0), p5b(-kPi * 65.0 / 9.0);
    phi[3] = add(K(p5a), mul(eta, K(p5b)));
  } else {
    const dd eta3 = mul(eta2, eta);
    const dd X1_4 = fx::sqr(X1_2), X2_4 = fx::sqr(X2_2);
    constexpr fx::cdd p6a(11583231236531.0 / 4694215680.0 - (640.0 / 3.0) * kPi * kPi - (6848.0 / 21.0) * kEulerGamma);
    constexpr fx::cdd p6b(-15737765635.0 / 3048192.0 + (2255.0 / 12.0) * kPi * kPi), p6c(76055.0 / 1728.0),
        p6d(-127825.0 / 1296.0);
    phi[4] = add(add(add(K(p6a), mul(eta, K(p6b))), mul(eta2, K(p6c))), mul(eta3, K(p6d)));
    constexpr fx::cdd p7a(kPi * 77096675.0 / 254016.0), p7b(kPi * 378515.0 / 1512.0), p7c(-kPi * 74045.0 / 756.0);
    phi[5] = add(add(K(p7a), mul(eta, K(p7b))), mul(eta2, K(p7c)));
    // 5PN tidal: sum_i (-288 + 264 X_i) X_i^4 Lambda_i
    phi[6] = add(mul(mul(add(mul(X1, 264.f), -288.f), X1_4), l1), mul(mul(add(mul(X2, 264.f), -288.f), X2_4), l2));
    // 6PN tidal: sum_i X_i^4 Lambda_i (-15895/28 + 4595/28 X_i + 5715/14 X_i^2 - 325/7 X_i^3)
    constexpr fx::cdd t0(-15895.0 / 28.0), t1(4595.0 / 28.0), t2(5715.0 / 14.0), t3(-325.0 / 7.0);
    const dd q1 = add(add(add(K(t0), mul(X1, K(t1))), mul(X1_2, K(t2))), mul(mul(X1_2, X1), K(t3)));
    const dd q2 = add(add(add(K(t0), mul(X2, K(t1))), mul(X2_2, K(t2))), mul(mul(X2_2, X2), K(t3)));
    phi[7] = add(mul(mul(X1_4, l1), q1), mul(mul(X2_4, l2), q2));
  }
}

// P_d = F+ (1 + cos^2 i)/2 - i Fx cos i from the arm unit vectors;
// t = sin/cos of (dec, ra - gmst, psi, iota).
__device__ __forceinline__ void ddantenna(const DetGeom& g, const dd* t, dd* P) {
  using fx::add;
  using fx::mul;
  using fx::sub;
  const dd sd = t[0], cd = t[1], sg = fx::neg(t[2]), cg = t[3];  // g = gmst - ra
  const dd sp = t[4], cp = t[5], ci = t[7];
  const dd sdcg = mul(sd, cg), sdsg = mul(sd, sg);
  const dd X[3] = {fx::neg(add(mul(cp, sg), mul(sp, sdcg))), sub(mul(sp, sdsg), mul(cp, cg)), mul(sp, cd)};
  const dd Y[3] = {sub(mul(sp, sg), mul(cp, sdcg)), add(mul(sp, cg), mul(cp, sdsg)), mul(cp, cd)};
  auto dot = [&](const float (*v)[2], const dd* u) {
    return add(add(mul(ldp(v[0]), u[0]), mul(ldp(v[1]), u[1])), mul(ldp(v[2]), u[2]));
  };
  const dd xX = dot(g.xa, X), xY = dot(g.xa, Y), yX = dot(g.ya, X), yY = dot(g.ya, Y);
  const dd fp = mul(add(sub(fx::sqr(xX), fx::sqr(yX)), sub(fx::sqr(yY), fx::sqr(xY))), 0.5f);
  const dd fc = sub(mul(xX, xY), mul(yX, yY));
  P[0] = mul(mul(fp, add(fx::sqr(ci), 1.f)), 0.5f);
  P[1] = fx::neg(mul(fc, ci));
}

// Phases 1 and 2 of the float-float set-up for the block's walkers (the
// kDdRoleWarps role warps only), absolute values left in shared memory.
__device__ __noinline__ void setup_absolute_dd(const double* __restrict__ theta, int64_t w0, int64_t W,
                                               const EventConst& ec, DdSmem& S) {
  using fx::add;
  using fx::mul;
  using fx::K;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kNPar * kSetupWalkers; i += kDdRoleThreads) {
    const int l = i / kNPar, j = i % kNPar;
    const int64_t w = (w0 + l < W) ? w0 + l : W - 1;  // pad with the last walker
    const double v = theta[w * kNPar + j];
    S.th[j][l] = v;
    S.thd[j][l] = st2(fx::from_double(v));
  }
  ddroles_sync();
  const int l = lane;
  switch (warp) {
    case 0: {  // masses and amplitude
      double th[kNPar];
      for (int j = 0; j < kNPar; ++j) th[j] = S.th[j][l];
      S.valid[l] = theta_valid(th) ? 1 : 0;
      constexpr fx::cdd kPiMsunDD(kPi * kMsunS);
      constexpr fx::cdd kAmpInvDD(1.0 / 9.802409278970853e-05);  // (pi G Msun / c^3)^-5/6 [Msun^5/6]
      constexpr fx::cdd k3over128(3.0 / 128.0);
      const dd x = mul(K(kPiMsunDD), ld2(S.thd[0][l]));
      const dd r = fx::cbrt(x);
      const dd r2 = fx::sqr(r);
      S.a1[l] = st2(r);
      S.N0[l] = st2(fx::div(K(k3over128), mul(fx::sqr(r2), r)));
      S.amp[l] = st2(fx::div(mul(mul(r2, fx::sqrt(r)), K(kAmpInvDD)), ld2(S.thd[6][l])));
      break;
    }
    case 1: {  // eta^-1/5
      const dd qd = ld2(S.thd[1][l]);
      S.e15[l] = st2(fx::rroot5(fx::div(qd, fx::sqr(add(qd, 1.f)))));
      break;
    }
    case 2:
    case 3: {  // PN polynomials, two halves
      dd phi[8];
      const int part = warp - 2;
      ddpn(part, ld2(S.thd[1][l]), ld2(S.thd[2][l]), ld2(S.thd[3][l]), ld2(S.thd[4][l]), ld2(S.thd[5][l]), phi);
      for (int k = 4 * part; k < 4 * part + 4; ++k) S.phi[k][l] = st2(phi[k]);
      break;
    }
    case 4:
    case 5:
    case 6:
    case 7: {  // sin/cos of dec, ra - gmst, psi, iota
      const int i = warp - 4;
      const dd ang = (i == 0) ? ld2(S.thd[12][l])
                   : (i == 1) ? fx::sub(ld2(S.thd[11][l]), ldp(ec.gmst2))
                   : (i == 2) ? ld2(S.thd[10][l]) : ld2(S.thd[9][l]);
      dd sn, cs;
      fx::sincos(ang, &sn, &cs);
      S.trig[2 * i][l] = st2(sn);
      S.trig[2 * i + 1][l] = st2(cs);
      break;
    }
  }
  ddroles_sync();
  switch (warp) {
    case 0: {  // the two logarithmic coefficients and Phi0
      const dd a = mul(ld2(S.a1[l]), ld2(S.e15[l]));
      const dd la = fx::log(a);  // ln(pi M) / 3
      const dd a2 = fx::sqr(a), a5 = mul(fx::sqr(a2), a), a6 = fx::sqr(mul(a2, a));
      const dd N0 = ld2(S.N0[l]);
      const dd N5 = mul(N0, a5), N6 = mul(N0, a6);
      constexpr fx::cdd kLn4(1.3862943611198906), k6848(-6848.0 / 21.0);
      S.c[5][l] = st2(mul(N6, add(ld2(S.phi[4][l]), mul(add(K(kLn4), la), K(k6848)))));  // f^1/3
      // -phi_c - pi/4 + the v^0 part of the 2.5PN term, 1 + 1.5 ln 6 + ln(pi M)
      constexpr fx::cdd kPi4(0.25 * kPi), kC(1.0 + 1.5 * 1.791759469228055);
      const dd t = mul(N5, mul(ld2(S.phi[3][l]), add(K(kC), mul(la, 3.f))));
      S.phi0[l] = st2(add(fx::sub(fx::neg(ld2(S.thd[8][l])), K(kPi4)), t));
      break;
    }
    case 1: {  // the other coefficients
      const dd a = mul(ld2(S.a1[l]), ld2(S.e15[l]));
      const dd a2 = fx::sqr(a), a3 = mul(a2, a), a4 = fx::sqr(a2), a5 = mul(a4, a), a6 = fx::sqr(a3), a7 = mul(a6, a);
      const dd a10 = fx::sqr(a5), a12 = fx::sqr(a6);
      const dd N0 = ld2(S.N0[l]);
      constexpr fx::cdd k6848_63(-6848.0 / 63.0);
      S.c[0][l] = st2(N0);
      S.c[1][l] = st2(mul(mul(N0, a2), ld2(S.phi[0][l])));
      S.c[2][l] = st2(mul(mul(N0, a3), ld2(S.phi[1][l])));
      S.c[3][l] = st2(mul(mul(N0, a4), ld2(S.phi[2][l])));
      S.c[4][l] = st2(mul(mul(N0, a5), ld2(S.phi[3][l])));  // ln f
      S.c[6][l] = st2(mul(mul(N0, a6), K(k6848_63)));       // f^1/3 ln f
      S.c[7][l] = st2(mul(mul(N0, a7), ld2(S.phi[5][l])));
      S.c[8][l] = st2(mul(mul(N0, a10), ld2(S.phi[6][l])));
      S.c[9][l] = st2(mul(mul(N0, a12), ld2(S.phi[7][l])));
      break;
    }
    case 2:
    case 3:
    case 4: {  // antenna factor of one detector
      const int d = warp - 2;
      if (d < ec.n_det) {
        dd t[8], P[2];
        for (int k = 0; k < 8; ++k) t[k] = ld2(S.trig[k][l]);
        ddantenna(ec.det[d], t, P);
        S.P[d][0][l] = st2(P[0]);
        S.P[d][1][l] = st2(P[1]);
      } else {
        S.P[d][0][l] = S.P[d][1][l] = make_float2(0.f, 0.f);
      }
      break;
    }
    case 5: {  // tau_d = t_c - n.r_d / c, n = (cos dec cos(ra - gmst), cos dec sin(ra - gmst), sin dec)
      const dd sd = ld2(S.trig[0][l]), cd = ld2(S.trig[1][l]);
      const dd n0 = mul(cd, ld2(S.trig[3][l])), n1 = mul(cd, ld2(S.trig[2][l]));
      const dd tc = ld2(S.thd[7][l]);
      for (int d = 0; d < kMaxDet; ++d) {
        const DetGeom& g = ec.det[d];
        const dd nr = add(add(mul(n0, ldp(g.rc[0])), mul(n1, ldp(g.rc[1]))), mul(sd, ldp(g.rc[2])));
        S.tau[d][l] = st2((d < ec.n_det) ? fx::sub(tc, nr) : dd{0.f, 0.f});
      }
      break;
    }
    default:
      break;
  }
  ddroles_sync();
}

// Float-float reference kernel (mixed path and the fast summary build): one
// block, every lane evaluates theta_ref; also writes the reference copies
// used by the summary build (c/2pi, Phi0/2pi, tau as float pairs and the
// complex h0 prefactor K_d = A_ref P_d in FP64).
__global__ void __launch_bounds__(kDdRoleThreads) k_ref_dd(const double* theta, EventConst ec, RefValues* out,
                                                          SummarySync* base_reset) {
  __shared__ DdSmem S;
  // a fast summary build follows on the same stream: it leaves log L(theta_ref)
  // in the fixed-point accumulator, zeroed here
  if (base_reset && threadIdx.x == 0) {
    base_reset->base_acc = 0ull;
    base_reset->overflow = 0u;
    base_reset->base_in_acc = 1u;
  }
  // a kernel launched programmatically after this one (the chunk records of
  // the rebuild + batch step) may start and load its own inputs now; it waits
  // for this grid's completion before it reads the reference values
  asm volatile("griddepcontrol.launch_dependents;");
  setup_absolute_dd(theta, 0, 1, ec, S);
  const int j = threadIdx.x;
  RefDD& R = out->dd;
  auto put = [](float* p, dd v) { p[0] = v.h; p[1] = v.l; };
  if (j < kNBasis) {
    const dd c = ld2(S.c[j][0]);
    put(R.c[j], c);
    put(out->chat[j], fx::mul(c, inv2pi()));
  } else if (j == kNBasis) {
    const dd p = ld2(S.phi0[0]);
    put(R.phi0, p);
    put(out->phi0t, fx::mul(p, inv2pi()));
  } else if (j == kNBasis + 1) {
    put(R.amp, ld2(S.amp[0]));
  } else if (j >= 32 && j < 32 + kMaxDet) {
    const int d = j - 32;
    const bool on = d < ec.n_det;
    const dd t = on ? ld2(S.tau[d][0]) : dd{0.f, 0.f};
    put(R.tau[d], t);
    put(out->taut[d], t);
    const dd pr = on ? ld2(S.P[d][0][0]) : dd{0.f, 0.f}, pi = on ? ld2(S.P[d][1][0]) : dd{0.f, 0.f};
    put(R.P[d][0], pr);
    put(R.P[d][1], pi);
    // sqrt(5/24) pi^{-2/3} (G Msun/c^3)^{5/6} / (1 Mpc / c): h0 amplitude per Msun^{5/6}/Mpc
    constexpr fx::cdd kAmpH(8.035028173395984e-06 / kMpcS);
    const dd a = fx::mul(fx::K(kAmpH), ld2(S.amp[0]));
    out->K[d][0] = fx::to_double(fx::mul(a, pr));
    out->K[d][1] = fx::to_double(fx::mul(a, pi));
  }
}

// Mixed batch set-up: WalkerMixed (+ float tangents on the warps after the
// role warps).
template <bool GRAD>
__global__ void __launch_bounds__(kDdRoleThreads + kTanWarps * 32) k_setup_dd(const double* __restrict__ theta, int64_t W,
                                                                 EventConst ec, const RefValues* __restrict__ ref,
                                                                 void* __restrict__ ws_out,
                                                                 void* __restrict__ tan_out) {
  __shared__ DdSmem S;
  const int64_t w0 = (int64_t)blockIdx.x * kSetupWalkers;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w = w0 + lane;
  const bool mine = w < W;
  if (warp >= kDdRoleWarps) {
    if (GRAD) tangent_warp<float>(theta, W, w0, ec, tan_out, warp - kDdRoleWarps);
    return;
  }
  setup_absolute_dd(theta, w0, W, ec, S);
  const RefDD& r = ref->dd;
  const int l = lane;
  WalkerMixed* o = static_cast<WalkerMixed*>(ws_out) + w;
  if (warp == 0) {
    // exp(-i dPhi0): dPhi0 / 2pi = y in turns (float pair, whole turns
    // dropped); exp(-2 pi i y) - 1 = -2 sin^2(pi y) - 2i sin(pi y) cos(pi y)
    // from the high part, plus the first-order term of the low part
    const dd y = fx::mul(fx::sub(ld2(S.phi0[l]), ldp(r.phi0)), inv2pi());
    const float yh = __fadd_rn(y.h, -round_fma_pipe(y.h)), yl = y.l;
    float sn, cs;
    sincos_pi_half(yh, sn, cs);
    const float er = -2.f * sn * sn, ei = -2.f * sn * cs;
    const float t = 6.28318530717958648f * yl;
    S.E[0][l] = st2(fx::add(fx::two_sum(1.f, er), ei * t));
    S.E[1][l] = st2(fx::two_sum(ei, -(1.f + er) * t));
  } else if (warp == 4 && mine) {
    // delays: detectors 0, 1 into their pair slots, detector D - 1 (D odd) alone
    float* f = reinterpret_cast<float*>(o->q);
    const int ds = (ec.n_det & 1) ? ec.n_det - 1 : -1;
    f[kWmSingle] = f[kWmSingle + 1] = f[kWmSingle + 2] = f[kWmSingle + 3] = 0.f;
    if (ds < 0) f[kWmSingle + 4] = f[kWmSingle + 5] = f[kWmSingle + 6] = f[kWmSingle + 7] = 0.f;
    for (int d = 0; d < kMaxDet; ++d) {
      const dd dt = (d < ec.n_det) ? fx::sub(ld2(S.tau[d][l]), ldp(r.tau[d])) : dd{0.f, 0.f};
      if (d < 2) {
        f[kWmTauPair + d] = dt.h;
        f[kWmTauPair + 2 + d] = dt.l;
      }
      if (d == ds) {
        f[kWmSingle] = dt.h;
        f[kWmSingle + 1] = dt.l;
      }
    }
  } else if (warp == 5 && mine) {
    float* f = reinterpret_cast<float*>(o->q);
    for (int k = 0; k < kNBasis; ++k) {
      const dd c = fx::sub(ld2(S.c[k][l]), ldp(r.c[k]));
      f[wm_dc_hi(k)] = c.h;
      f[wm_dc_lo(k)] = c.l;
    }
    o->valid = S.valid[l];
    o->pad[0] = o->pad[1] = o->pad[2] = 0;
  }
  ddroles_sync();
  if (warp >= 1 && warp <= kMaxDet && mine) {
    const int d = warp - 1;
    float rho_r = 0.f, rho_i = 0.f, sig_r = 0.f, sig_i = 0.f;
    if (d < ec.n_det) {
      using fx::add;
      using fx::mul;
      using fx::sub;
      // Q = (amp / amp_ref) P exp(-i dPhi0);  rho = Q / P_ref;  sig = (Q - P_ref) / P_ref
      const dd ampr = fx::div(ld2(S.amp[l]), ldp(r.amp));
      const dd er = ld2(S.E[0][l]), ei = ld2(S.E[1][l]);
      const dd pr = ld2(S.P[d][0][l]), pi = ld2(S.P[d][1][l]);
      const dd qr = mul(ampr, sub(mul(pr, er), mul(pi, ei))), qi = mul(ampr, add(mul(pr, ei), mul(pi, er)));
      const dd rr = ldp(r.P[d][0]), ri = ldp(r.P[d][1]);
      const dd iden = fx::div(1.f, add(mul(rr, rr), mul(ri, ri)));
      const dd xr = sub(qr, rr), xi = sub(qi, ri);
      rho_r = mul(add(mul(qr, rr), mul(qi, ri)), iden).h;
      rho_i = mul(sub(mul(qi, rr), mul(qr, ri)), iden).h;
      sig_r = mul(add(mul(xr, rr), mul(xi, ri)), iden).h;
      sig_i = mul(sub(mul(xi, rr), mul(xr, ri)), iden).h;
    }
    float* f = reinterpret_cast<float*>(o->q);
    if (d < 2) {
      f[kWmRhoPair + d] = rho_r;
      f[kWmRhoPair + 2 + d] = rho_i;
      f[kWmSigPair + d] = sig_r;
      f[kWmSigPair + 2 + d] = sig_i;
    }
    if ((ec.n_det & 1) && d == ec.n_det - 1) {
      f[kWmSingle + 4] = rho_r;
      f[kWmSingle + 5] = rho_i;
      f[kWmSingle + 6] = sig_r;
      f[kWmSingle + 7] = sig_i;
    }
  }
}

// Host-side launchers.
cudaError_t launch_ref_values(const double* theta_ref_dev, const EventConst& ec, RefValues* out, cudaStream_t s) {
  k_ref_values<<<1, 5 * 32, 0, s>>>(theta_ref_dev, ec, out);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_setup_t(const double* theta, int64_t W, const EventConst& ec, const RefValues* ref, void* ws,
                                  void* tan, bool grad, cudaStream_t s) {
  const unsigned grid = (unsigned)((W + kSetupWalkers - 1) / kSetupWalkers);
  if (grad)
    k_setup<MODE, true><<<grid, (5 + kTanWarps) * 32, 0, s>>>(theta, W, ec, ref, ws, tan);
  else
    k_setup<MODE, false><<<grid, 5 * 32, 0, s>>>(theta, W, ec, ref, ws, tan);
  return cudaGetLastError();
}

// Absolute values of W walkers for the full-grid likelihood (32 walkers per
// block, the float-float set-up of the mixed path; lane l writes walker w0 + l).
__global__ void __launch_bounds__(kDdRoleThreads) k_setup_abs(const double* __restrict__ theta, int64_t W,
                                                             EventConst ec, WalkerAbs* __restrict__ out) {
  __shared__ DdSmem S;
  const int64_t w0 = (int64_t)blockIdx.x * kSetupWalkers;
  setup_absolute_dd(theta, w0, W, ec, S);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w = w0 + lane;
  if (w >= W) return;
  WalkerAbs& o = out[w];
  auto put = [](float* p, dd v) { p[0] = v.h; p[1] = v.l; };
  if (warp == 0) {
    for (int k = 0; k < kNBasis; ++k) put(o.chat[k], fx::mul(ld2(S.c[k][lane]), inv2pi()));
    put(o.phi0t, fx::mul(ld2(S.phi0[lane]), inv2pi()));
    o.valid = S.valid[lane];
    o.pad[0] = o.pad[1] = o.pad[2] = 0;
  } else if (warp >= 1 && warp <= kMaxDet) {
    const int d = warp - 1;
    const bool on = d < ec.n_det;
    put(o.taut[d], on ? ld2(S.tau[d][lane]) : dd{0.f, 0.f});
    constexpr fx::cdd kAmpH(8.035028173395984e-06 / kMpcS);
    const dd a = fx::mul(fx::K(kAmpH), ld2(S.amp[lane]));
    o.K[d][0] = on ? fx::to_double(fx::mul(a, ld2(S.P[d][0][lane]))) : 0.0;
    o.K[d][1] = on ? fx::to_double(fx::mul(a, ld2(S.P[d][1][lane]))) : 0.0;
  }
}

cudaError_t launch_setup_abs(const double* theta, int64_t W, const EventConst& ec, WalkerAbs* out, cudaStream_t s) {
  const unsigned grid = (unsigned)((W + kSetupWalkers - 1) / kSetupWalkers);
  k_setup_abs<<<grid, kDdRoleThreads, 0, s>>>(theta, W, ec, out);
  return cudaGetLastError();
}

// The FP32 tangents alone, one warp per tangent group and 32 walkers per
// block: they depend on theta only, so the combined rebuild + batch runs them
// on a stream of their own from the start of the call.
__global__ void __launch_bounds__(kTanWarps * 32) k_tangents(const double* __restrict__ theta, int64_t W, EventConst ec,
                                                             void* __restrict__ tan_out) {
  tangent_warp<float>(theta, W, (int64_t)blockIdx.x * kSetupWalkers, ec, tan_out, threadIdx.x >> 5);
}

cudaError_t launch_tangents(const double* theta, int64_t W, const EventConst& ec, void* tan, cudaStream_t s) {
  const unsigned grid = (unsigned)((W + kSetupWalkers - 1) / kSetupWalkers);
  k_tangents<<<grid, kTanWarps * 32, 0, s>>>(theta, W, ec, tan);
  return cudaGetLastError();
}

// Phase directions of the fiducial waveform for the bin placement without the
// PN ansatz: dc_k / dtheta_j at theta_ref (the FP64 dual numbers of the FP64
// set-up's tangents), out[k][j] for j = Mc, q, chi1, chi2, Lambda1, Lambda2.
// With the basis functions g_k they give dPsi(f) / dtheta_j = sum_k out[k][j] g_k(f);
// the constant phase does not vary with f and is not needed.
__global__ void k_ref_phase_tangents(const double* __restrict__ theta_ref, double* __restrict__ out) {
  const int part = threadIdx.x;
  if (part >= 3) return;
  WalkerTan<double> t;
  tangents_intrinsic<double>(theta_ref, part, t);
  for (int k = 0; k < kNBasis; ++k)
    for (int j = 2 * part; j < 2 * part + 2; ++j) out[k * kNTanIntr + j] = t.dc[k][j];
}

cudaError_t launch_ref_phase_tangents(const double* theta_ref_dev, double* out, cudaStream_t s) {
  k_ref_phase_tangents<<<1, 32, 0, s>>>(theta_ref_dev, out);
  return cudaGetLastError();
}

cudaError_t launch_ref_dd(const double* theta_ref_dev, const EventConst& ec, RefValues* out, SummarySync* base_reset,
                          cudaStream_t s) {
  k_ref_dd<<<1, kDdRoleThreads, 0, s>>>(theta_ref_dev, ec, out, base_reset);
  return cudaGetLastError();
}

cudaError_t launch_setup(int mode, const double* theta, int64_t W, const EventConst& ec, const RefValues* ref,
                         void* ws, void* tan, bool grad, cudaStream_t s) {
  if (mode == RB_MIXED) {
    const unsigned grid = (unsigned)((W + kSetupWalkers - 1) / kSetupWalkers);
    if (grad)
      k_setup_dd<true><<<grid, kDdRoleThreads + kTanWarps * 32, 0, s>>>(theta, W, ec, ref, ws, tan);
    else
      k_setup_dd<false><<<grid, kDdRoleThreads, 0, s>>>(theta, W, ec, ref, ws, tan);
    return cudaGetLastError();
  }
  if (mode == RB_FP64) return launch_setup_t<RB_FP64>(theta, W, ec, ref, ws, tan, grad, s);
  return launch_setup_t<RB_MIXED_F64PHASE>(theta, W, ec, ref, ws, tan, grad, s);
}

}  // namespace rb
