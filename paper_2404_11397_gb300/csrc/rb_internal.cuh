// rb_internal.cuh -- layouts and device helpers shared by the librb kernels.
//
// Method: relative-binning likelihood of arXiv:2404.11397, Sec. II.A-II.C
// (Eqs. 2-5), with TaylorF2 + tides (Sec. II.B) at the bin edges.
//
// Phase factorisation used by every kernel.  With v = (pi M f)^{1/3}, the
// TaylorF2 phase Psi(f) = 2 pi f t_c - phi_c - pi/4 + 3/(128 eta v^5) sum_k phi_k v^k
// is written as
//     Psi(f) = Phi0 + sum_{k<10} c_k g_k(f) + 2 pi f t_c,
// with the ten frequency functions (the PN powers v^{k-5}, the 2.5PN and 3PN
// logarithms split into ln f parts)
//     g = { f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f, f^2/3, f^5/3, f^7/3 }
// and per-source coefficients c_k(theta) and constant Phi0(theta).  The
// detector delay adds 2 pi f dt_d, so each detector's phase difference to the
// fiducial waveform at a bin edge is
//     dPsi_d(f_e) = sum_k (c_k - c_k,ref) g_k(f_e) + 2 pi f_e (tau_d - tau_d,ref),
// tau_d = t_c + dt_d.  The kernels work in turns: x = dPsi / (2 pi), and the
// edge tables hold g_k(f_e) / (2 pi).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace rb {

constexpr int kNPar = 13;
constexpr int kMaxDet = 3;
constexpr int kNBasis = 10;
constexpr int kEdgeQuads = kNBasis / 2 + 1;  // float4 groups per edge in the float tables
static_assert(kNBasis % 2 == 0, "basis pairs per float4 of the edge tables");
constexpr int kNTanIntr = 6;  // Mc, q, chi1, chi2, Lambda1, Lambda2

// Edge slots of the mixed likelihood kernel: in iteration i of a walker's
// loop, lane l holds two neighbouring bin edges, e_A = 63 i + 2 l and
// e_B = e_A + 1, each with the bin on its right (b = e; lane 31's e_B has no
// bin and is the next iteration's e_A of lane 0), as the two halves of one
// paired FP32 value.  Slot s = 32 i + l.
constexpr int kSlotBins = 63;        // bins per iteration
constexpr int kSlotBinFloats = 12;   // bin-table floats per slot and detector
__host__ __device__ constexpr int slot_count(int n_bins) { return 32 * ((n_bins + kSlotBins - 1) / kSlotBins); }

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kEulerGamma = 0.577215664901532860606512090082402431;
constexpr double kMsunS = 4.925490947641266978e-6;   // G M_sun / c^3 [s]
constexpr double kClight = 299792458.0;               // [m/s]
constexpr double kMpcS = 3.085677581491367e22 / 299792458.0;  // 1 Mpc / c [s]

// Per-detector constant geometry (built on the host from the site row).
struct DetGeom {
  double D[3][3];   // response tensor (x x^T - y y^T)/2
  double r[3];      // vertex [m], Earth-fixed
  // float pairs (hi, lo) for the float-float set-up of the mixed path
  float xa[3][2], ya[3][2];  // arm unit vectors
  float rc[3][2];            // vertex / c [s]
};

// Constant event data needed by the per-walker set-up kernel.
struct EventConst {
  int n_det;
  int pad;
  double gmst;
  float gmst2[2];  // gmst as a float pair
  DetGeom det[kMaxDet];
};

// Absolute per-source quantities (FP64).  Produced by one noinline device
// function so that theta and theta_ref go through identical instructions.
struct Values {
  double c[kNBasis];     // phase-basis coefficients [rad]
  double phi0;           // constant phase [rad]
  double tau[kMaxDet];   // t_c + dt_d [s]
  double amp;            // Mc^{5/6} / d_L (Msun^{5/6} / Mpc)
  double P64[kMaxDet][2];  // F+ (1+cos^2 i)/2 - i Fx cos i   (FP64, only if requested)
  float P32[kMaxDet][2];   // same, FP32 trigonometry
  int valid;
  int pad;
};

// Per-detector strain [N][2] and PSD [N] pointers (device).
struct DataPtrs {
  const double* data[kMaxDet];
  const double* psd[kMaxDet];
};

// Fiducial (theta_ref) values of an event, written by the reference kernel:
// the FP64 values plus float-pair copies used by the FP32-pipe kernels.
// MALA local step state for the fused accept in the batch kernels (device
// pointers, [W] or [W][13]; eps by value).  See rb_mala.cu.
struct MalaArgs {
  double* z;            // [W][13] chain state in sampling coordinates (updated on accept)
  const double* zp;     // [W][13] proposal
  double* logp;         // [W] log posterior of the state (updated on accept)
  double* gz;           // [W][13] its gradient in sampling coordinates (updated on accept)
  const double* xi;     // [W][13] standard normal draws of the proposal
  const double* lu;     // [W] log of the uniform draws
  const double* jac;    // [W][2] d iota / d cos iota, d dec / d sin dec at the proposal
  const int* inside;    // [W] proposal inside the prior box
  int* accepted;        // [W] output
  double eps[kNPar];    // step sizes
  int init;             // 1: adopt the proposal (= the state) unconditionally
};

// Fiducial values of the mixed path, float pairs (hi, lo) from the
// float-float set-up (the same instructions as a walker's set-up).
struct RefDD {
  float c[kNBasis][2];
  float phi0[2];
  float tau[kMaxDet][2];
  float P[kMaxDet][2][2];
  float amp[2];
};

struct RefValues {
  Values v;       // FP64 fiducial values (FP64 and FP64-phase paths)
  RefDD dd;       // float-float fiducial values (mixed path)
  float chat[kNBasis][2];   // c_k / 2pi (turns), float pair
  float phi0t[2];           // Phi0 / 2pi (turns), float pair
  float taut[kMaxDet][2];   // tau_d [s], float pair
  double K[kMaxDet][2];     // A_ref P_d: h0_d = K_d f^-7/6 exp(-2 pi i x_d(f))
};

// Per-walker set-up output for the mixed (float-float) path, laid out as the
// likelihood kernel's per-warp constants so that it is copied to shared
// memory as it is.  dc = c_k - c_k,ref and tau_d - tau_d,ref [s] as float
// pairs (hi, lo); rho_d = C_d(theta) / C_d(theta_ref), sig_d = rho_d - 1
// computed as (Q - Q_ref) / Q_ref (complex: r, i).  Detectors 0 and 1 side
// by side; detector s = D - 1 alone when the detector count D is odd:
//   q[0..4] {dc_hi[2k], dc_hi[2k+1], dc_lo[2k], dc_lo[2k+1]}
//   q[5] {tau_hi0, tau_hi1, tau_lo0, tau_lo1}
//   q[6] {rho_r0, rho_r1, rho_i0, rho_i1}    q[7] {sig_r0, sig_r1, sig_i0, sig_i1}
//   q[8] {tau_hi_s, tau_lo_s, 0, 0}          q[9] {rho_r_s, rho_i_s, sig_r_s, sig_i_s}
// (detector slots beyond D, and q[8], q[9] when D is even, are zero).
constexpr int kWalkerQuads = 10;
struct __align__(16) WalkerMixed {
  float4 q[kWalkerQuads];
  int valid;
  int pad[3];
};
// float offsets into WalkerMixed::q
__host__ __device__ constexpr int wm_dc_hi(int k) { return 4 * (k >> 1) + (k & 1); }
__host__ __device__ constexpr int wm_dc_lo(int k) { return 4 * (k >> 1) + 2 + (k & 1); }
constexpr int kWmTauPair = 20, kWmRhoPair = 24, kWmSigPair = 28, kWmSingle = 32;

// Per-walker set-up output for the FP64 and FP64-phase paths.
struct WalkerF64 {
  double dc[kNBasis];
  double tau[kMaxDet];
  double rho[kMaxDet][2];
  double sig[kMaxDet][2];
  int valid;
  int pad;
};

// Absolute per-walker values for the full-grid likelihood (float-float
// set-up): h_d(f) = K_d f^-7/6 exp(-2 pi i x_d(f)),
// x_d(f) = phi0t + sum_k chat_k g_k(f) + f taut_d (turns).
struct WalkerAbs {
  float chat[kNBasis][2];  // c_k / 2pi, float pair
  float phi0t[2];          // Phi0 / 2pi, float pair
  float taut[kMaxDet][2];  // tau_d [s], float pair
  double K[kMaxDet][2];    // A P_d
  int valid;
  int pad[3];
};

// Tangents for the chain rule (T = float for the mixed paths, double for FP64).
template <class T>
struct WalkerTan {
  T dc[kNBasis][kNTanIntr];      // d c_k / d(Mc, q, chi1, chi2, L1, L2)
  T dphi0[2];                    // d Phi0 / d(Mc, q)
  T dtd[kMaxDet][2];             // d dt_d / d(ra, dec)
  T dlnP[kMaxDet][4][2];         // d ln P_d / d(iota, psi, ra, dec), complex
  T lnamp_Mc, lnamp_dL;          // d ln(Mc^{5/6}/d_L) / d(Mc, dL)
};

// Device-side event tables.  Offsets are in elements of the table type.
struct SummarySync;

struct EventDev {
  int n_det, n_bins, n_edges, e_pad, b_pad;
  int64_t kmin, n_freq;
  double T;
  const double* base_logl;  // device: sum_d (Re sum_b A0 - sum_b B0 / 2) = log L(theta_ref) (event_base_logl)
  const SummarySync* sync;  // where the fast build leaves it
  const double* share;      // [D][B] the bins' shares
  // float image, laid out for 16-byte loads (lane l reads edge / bin c0 + l:
  // consecutive 16 B, no bank conflicts) whose halves are ready operands of
  // the paired FP32 instructions; the FP64-phase mixed kernel copies its bin
  // part to shared memory (the float-float kernel reads the slot image
  // below, and no kernel reads the edge part, written at event creation):
  //   edge part, float4 [kEdgeQuads][Ep]: quad q < 5 holds
  //     {g_hi[2q], g_hi[2q+1], g_lo[2q], g_lo[2q+1]}  (g_k(f_e)/2pi as float pairs),
  //     quad 5 holds {f_hi, f_lo, 0, 0};
  //   bin part, with alpha0 = A0/2, alpha1 = A1/df_b, beta0 = B0/2,
  //   beta1 = B1/df_b, the betas stored negated:
  //     if D >= 2, detectors 0 and 1 side by side, float4 [3][Bp]:
  //       {a0r_0, a0r_1, a0i_0, a0i_1}, {a1r_0, a1r_1, a1i_0, a1i_1},
  //       {-b0_0, -b0_1, -b1_0, -b1_1};
  //     if D is odd, detector D - 1 after that: float4 [Bp] {a0r, a0i, a1r, a1i},
  //       then float2 [Bp] {-b0, -b1}
  const float* tab32;
  size_t tab32_floats;   // multiple of 4
  size_t edge32_floats;  // length of the edge part (4*kEdgeQuads*Ep)
  // slot image of the float-float mixed kernel (NS = slot_count(B) slots;
  // halves A, B of a pair are the slot's edges e_A, e_B and their bins):
  //   edge part, float4 [kNBasis + 1][NS]: quad k < kNBasis holds
  //     {g_hi_k(e_A), g_hi_k(e_B), g_lo_k(e_A), g_lo_k(e_B)}, quad kNBasis
  //     {f_hi(e_A), f_hi(e_B), f_lo(e_A), f_lo(e_B)};
  //   bin part, per detector d (kSlotBinFloats * NS floats), the bin's
  //     coefficients of its left and right edge values: float4 [3][NS]
  //     {gmr_A, gmr_B, gpr_A, gpr_B}, {gmi_A, gmi_B, gpi_A, gpi_B},
  //     {h_A, h_B, q_A, q_B} with gmr = a0r - b0 - a1r, gpr = a0r - b0 + a1r,
  //     gmi = a0i - a1i, gpi = a0i + a1i, h = -b0/2, q = -b0/4 (a = alpha,
  //     b = beta of the float image above);
  //   zero for edges past the last and where an edge has no bin.
  const float* slot32;
  size_t slot32_floats;  // multiple of 4
  int n_slots;           // NS
  // upper bounds of |g_k(f) / 2pi| (k < kNBasis) and of f over the event's
  // grid: the mixed kernel's per-walker bound on its phase terms
  float gmax[kNBasis + 1];
  // FP64 tables: g[k][e] (10*Ep), f[e] (Ep), then per detector 6 rows of Bp
  const double* tab64;
  const RefValues* ref;
};

// Outputs of the summary kernels (see summary_epilogue).
// Fast (Taylor-chunk) evaluation of the fiducial phase: the grid is cut
// into chunks of kChunk points and the phase expanded to order kOrd about
// each chunk centre (rb_summary.cu).
constexpr int kChunk = 32;
constexpr int kOrd = 8;
// Event-constant per-chunk matrices, stored chunk-major ([chunk][128
// floats], one 512-byte row per chunk, read with 16-byte vector loads).
// Fields:
constexpr int kQ01 = 0;                       // 4k + 2n + h: orders 0, 1 of basis k as float pairs
constexpr int kQ2 = kQ01 + kNBasis * 4;       // 2k + h: order 2 as a float pair
constexpr int kQh = kQ2 + kNBasis * 2;        // (n-3)*10 + k: orders 3..8
constexpr int kQfc = kQh + (kOrd - 2) * kNBasis;  // f_c as a float pair
constexpr int kQamp = kQfc + 2;               // f_c^-7/6, binom(-7/6, n) u^n (n = 1..4)
constexpr int kQFields = kQamp + 5;
constexpr int kQRow = 128;
static_assert(kQFields <= kQRow && kQ2 % 4 == 0 && kQh % 4 == 0 && kQfc % 4 == 0, "chunk matrix fields");

constexpr int kPartPoints = 512;  // grid points per part of a bin (fast summary build)

// Part of a bin for the fast summary build (bins are split into parts of at
// most kPartPoints grid points; the last part of a bin to finish combines
// the parts' sums in index order).
struct PartDesc {
  int bin, start, end;  // grid points [start, end) of bin `bin`
  int first, n_parts;   // index of the bin's first part, parts in the bin
  int pad[3];
};

// Synchronisation words of an event's summary build (zero between builds).
struct SummarySync {
  unsigned counter;              // bins (or blocks) finished
  unsigned overflow;             // a bin's share did not fit the fixed-point sum
  unsigned long long base_acc;   // sum of the bins' shares, fixed point 2^-32
  unsigned base_in_acc;          // 1: log L(theta_ref) is left in base_acc (fast build), 0: in EventDev::base_logl
  unsigned pad;
  unsigned bin_parts_done[1];    // [B] parts finished per bin (allocated with B entries)
};

// log L(theta_ref) of the event's last summary build.  The fast build leaves
// it as the fixed-point sum of the bins' shares, converted here by each
// reader (no block of the build waits to convert it); the FP64 builds store
// the value.  A share too large for the fixed-point sum sends the readers of a
// fast build to the fixed-order FP64 sum of the D x B shares.
// The loads are split from the conversion so that a kernel can issue them at
// its start and use the value after its own staging.
struct BaseRead {
  unsigned in_acc, overflow;
  unsigned long long acc;
  double stored;
};
__device__ __forceinline__ BaseRead event_base_read(const EventDev& ev) {
  const SummarySync* sy = ev.sync;
  return BaseRead{sy->base_in_acc, sy->overflow, sy->base_acc, *ev.base_logl};
}
__device__ __forceinline__ double event_base_value(const EventDev& ev, const BaseRead& r) {
  if (r.in_acc == 0u) return r.stored;
  if (r.overflow == 0u) return (double)(long long)r.acc * (1.0 / 4294967296.0);
  double t = 0.0;
  const int n = ev.n_det * ev.n_bins;
  for (int i = 0; i < n; ++i) t += ev.share[i];
  return t;
}
__device__ __forceinline__ double event_base_logl(const EventDev& ev) { return event_base_value(ev, event_base_read(ev)); }

struct SummaryOut {
  double* summ;          // [D][B][6] FP64 summary: A0 re/im, A1 re/im, B0, B1
  float* bin32;          // [D][6][Bp] bin tables (float)
  double* bin64;         // [D][6][Bp] bin tables (FP64)
  const double* inv_df;  // [B] 1 / (f_{b+1} - f_b)
  double* share;         // [D][B] per-bin share of log L(theta_ref)
  SummarySync* sync;     // counters, zero between builds
  double* base;          // log L(theta_ref)
  int Bp;
  const PartDesc* parts;  // fast build: [n_parts]
  float* part_sums;       // fast builds: [n_parts][kPartSlots] doubles, or float pairs [n_parts][7 kMaxDet][2]
  int n_parts;
  float* slot_bin32;      // bin part of the slot image (EventDev::slot32)
  int n_slots;
};

// ---------------------------------------------------------------------------
// Bounds checks of the debug build (compiled with -DRB_BOUNDS_CHECK).  A
// checked index outside [0, n) is recorded -- the first one's site, index and
// limit, and a count -- and replaced by 0, so the access stays inside the
// buffer and every lane keeps taking part in the warp's shuffles.  The record
// is per translation unit (a static device variable); the host reads and
// clears all of them with rb_debug_bounds().  In the normal build RB_IDX(i,
// n, site) is i and the checks cost nothing.
// ---------------------------------------------------------------------------
struct BoundsRecord {
  unsigned count;
  int site;
  long long index, limit;
};
#ifdef RB_BOUNDS_CHECK
static __device__ BoundsRecord g_bounds_rec;
__device__ __forceinline__ long long checked_index(long long i, long long n, int site) {
  if (i >= 0 && i < n) return i;
  if (atomicAdd(&g_bounds_rec.count, 1u) == 0u) {
    g_bounds_rec.site = site;
    g_bounds_rec.index = i;
    g_bounds_rec.limit = n;
  }
  return 0;
}
#define RB_IDX(i, n, site) ((decltype(i))::rb::checked_index((long long)(i), (long long)(n), (site)))
// host side, one per translation unit that checks: copy the unit's record to
// *out and clear it
#define RB_BOUNDS_READER(fn)                                                          \
  extern "C" int fn(::rb::BoundsRecord* out) {                                        \
    ::rb::BoundsRecord zero{};                                                        \
    cudaError_t e = cudaMemcpyFromSymbol(out, ::rb::g_bounds_rec, sizeof(zero));     \
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(::rb::g_bounds_rec, &zero, sizeof(zero)); \
    return (int)e;                                                                    \
  }
#else
#define RB_IDX(i, n, site) (i)
#define RB_BOUNDS_READER(fn)
#endif
// per-part sums of the builds that split bins into parts: 7 kMaxDet float
// pairs (fast build) or 6 kMaxDet doubles (stored-waveform FP64 build)
constexpr int kPartSlots = 7 * kMaxDet;
static_assert(6 * kMaxDet <= kPartSlots, "the FP64 part sums fit the part slots");

// ---------------------------------------------------------------------------
// Float-float helpers (all operations rounded explicitly: no contraction or
// reassociation may touch the error-free transformations).
// ---------------------------------------------------------------------------
struct f2x {
  float hi, lo;
};

__device__ __forceinline__ f2x f2x_from(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(x - (double)h);
  return {h, l};
}

// s += a * b, with a, b float pairs; (s_hi, s_lo) is an unnormalised pair.
// Product: hi*hi exactly by FMA (Dekker), cross terms folded into the error;
// lo*lo (< 2^-48 relative) is dropped.  Sum: Knuth two-sum on the high parts.
__device__ __forceinline__ void f2x_fma_acc(float a_hi, float a_lo, float b_hi, float b_lo, float& s_hi,
                                            float& s_lo) {
  float p = __fmul_rn(a_hi, b_hi);
  float e = __fmaf_rn(a_hi, b_hi, -p);
  e = __fmaf_rn(a_hi, b_lo, e);
  e = __fmaf_rn(a_lo, b_hi, e);
  float s = __fadd_rn(s_hi, p);
  float bb = __fadd_rn(s, -s_hi);
  float err = __fadd_rn(__fadd_rn(s_hi, -__fadd_rn(s, -bb)), __fadd_rn(p, -bb));
  s_hi = s;
  s_lo = __fadd_rn(s_lo, __fadd_rn(err, e));
}

// Round to nearest integer on the FMA pipe (valid for |x| < 2^22; larger
// inputs still give an integer within 1 of x, which the second stage of
// frac_turns absorbs).
__device__ __forceinline__ float round_fma_pipe(float x) {
  const float magic = 12582912.0f;  // 1.5 * 2^23
  return __fadd_rn(__fadd_rn(x, magic), -magic);
}

// Fractional part in [-1/2, 1/2] (up to rounding) of the float pair (hi, lo), in turns.
__device__ __forceinline__ float frac_turns(float hi, float lo) {
  float r = __fadd_rn(hi, -round_fma_pipe(hi));  // exact
  float y = __fadd_rn(r, lo);
  return __fadd_rn(y, -round_fma_pipe(y));
}

// Half-angle sine and cosine: s = sin(pi y), c = cos(pi y) for |y| <= 1/2,
// as polynomials in w = y^2:
//   sin(pi y) = y (pi - pi^3/6 w + w^2 (S0 + S1 w + S2 w^2 + S3 w^3)),
//   cos(pi y) = 1 - pi^2/2 w + w^2 (C0 + C1 w + C2 w^2 + C3 w^3).
// The two leading coefficients of each are exact (pi, pi^3/6, pi^2/2 applied
// as float pairs), the remaining ones are near-minimax fits on [0, 1/2]
// (least squares with Lawson reweighting, computed for this code and
// rounded to float).  Fit error below 1.1e-9 relative for sin and 1.1e-9
// absolute for cos; the FP32 evaluation adds about an ulp.  s is exactly 0
// at y = 0, which keeps the delta form exact at the fiducial point.
__device__ __forceinline__ void sincos_pi_half(float y, float& s, float& c) {
  const float w = y * y;
  float ps = -0.007060864474624395f;
  ps = fmaf(ps, w, 0.08207154273986816f);
  ps = fmaf(ps, w, -0.5992570519447327f);
  ps = fmaf(ps, w, 2.550163745880127f);
  ps = fmaf(ps, w, -9.160392266949202e-08f);  // low part of -pi^3/6
  ps = fmaf(ps, w, -8.742277657347586e-08f);  // low part of pi
  ps = fmaf(w, -5.167712688446045f, ps);      // high part of -pi^3/6
  s = fmaf(y, 3.1415927410125732f, y * ps);   // high part of pi
  float pc = -0.024529997259378433f;
  pc = fmaf(pc, w, 0.2350243180990219f);
  pc = fmaf(pc, w, -1.3352320194244385f);
  pc = fmaf(pc, w, 4.058711051940918f);
  pc = fmaf(pc, w, -1.451857940537593e-07f);  // low part of -pi^2/2
  c = fmaf(w, -4.934802055358887f, fmaf(pc, w, 1.0f));  // high part of -pi^2/2
}

// Small integer -> float on the FMA pipe (|i| < 2^22).
__device__ __forceinline__ float small_int_float(int i) {
  return __fadd_rn(__int_as_float(0x4B400000 + i), -12582912.0f);
}

__device__ __forceinline__ void f2x_add(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bb = __fadd_rn(s, -hi);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bb)), __fadd_rn(v, -bb)));
  hi = s;
}

// sin, cos of 2 pi y from the half-angle series (|y| <= 1/2 turns).
__device__ __forceinline__ float2 cis_turns(float y) {
  float sn, cs;
  sincos_pi_half(y, sn, cs);
  return make_float2(fmaf(-2.f * sn, sn, 1.f), 2.f * sn * cs);
}

// ---------------------------------------------------------------------------
// Paired FP32 arithmetic.  V = float evaluates one detector; V = float2
// evaluates detectors 0 and 1 side by side with the sm_100+ paired
// instructions (FFMA2 / FADD2 / FMUL2: one issue slot for two lanes of work,
// each component rounded exactly as the scalar instruction).
// ---------------------------------------------------------------------------
namespace pv {
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float neg(float a) { return -a; }
__device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub(float2 a, float2 b) {
  float2 r;
  asm("{.reg .b64 x, y, z;\n\tmov.b64 x, {%2, %3};\n\tmov.b64 y, {%4, %5};\n\tsub.rn.f32x2 z, x, y;\n\tmov.b64 {%0, %1}, z;}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }  // folded into the consumer
template <class V> __device__ __forceinline__ V splat(float x);
template <> __device__ __forceinline__ float splat<float>(float x) { return x; }
template <> __device__ __forceinline__ float2 splat<float2>(float x) { return make_float2(x, x); }
__device__ __forceinline__ float shfl_down(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float2 shfl_down(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float shfl_up(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float2 shfl_up(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}

// s_hi + s_lo += (a_hi + a_lo)(b_hi + b_lo): Dekker product, Knuth sum
// (the same steps as f2x_fma_acc).
template <class V>
__device__ __forceinline__ void fma_acc(V a_hi, V a_lo, V b_hi, V b_lo, V& s_hi, V& s_lo) {
  const V p = mul(a_hi, b_hi);
  V e = fma(a_hi, b_hi, neg(p));
  e = fma(a_hi, b_lo, e);
  e = fma(a_lo, b_hi, e);
  const V s = add(s_hi, p);
  const V bb = sub(s, s_hi);
  const V err = add(sub(s_hi, sub(s, bb)), sub(p, bb));
  s_hi = s;
  s_lo = add(s_lo, add(err, e));
}

// H + L += (a_hi + a_lo)(b_hi + b_lo) with H kept exact: m = 1.5 * 2^23 q for a
// power of two q, and |a_hi b_hi| < 2^22 q.  One FMA against m rounds the
// product's high part to a multiple h of q (the sum lands in m's binade, whose
// ulp is q); the multiples add exactly while |H| < 2^24 q.  The remainder
// a_hi b_hi - h (|.| <= q/2, rounded once) and the cross terms go to L.  The
// low-by-low term (~2^-48 of the product) is dropped.
template <class V>
__device__ __forceinline__ void split_acc(V a_hi, V a_lo, V b_hi, V b_lo, V m, V& H, V& L) {
  const V h = sub(fma(a_hi, b_hi, m), m);
  H = add(H, h);
  L = add(L, fma(a_hi, b_hi, neg(h)));
  L = fma(a_hi, b_lo, L);
  L = fma(a_lo, b_hi, L);
}

// hi + lo in turns with the whole turns of hi removed: hi - rint(hi) is
// exact, so the result is within |lo| (below an ulp of hi, at most a few
// 1e-3 turns for |hi| ~ 1e4) of [-1/2, 1/2].  The half-angle sine and cosine
// that take it are accurate slightly beyond +-1/2 and periodic in the result,
// so the sum is not reduced a second time.
template <class V>
__device__ __forceinline__ V frac(V hi, V lo) {
  const V m = splat<V>(12582912.0f);  // 1.5 * 2^23: round to nearest on the FMA pipe
  const V r = sub(hi, sub(add(hi, m), m));
  return add(r, lo);
}

// x with its whole turns removed (|x| < 2^22).
template <class V>
__device__ __forceinline__ V frac1(V x) {
  const V m = splat<V>(12582912.0f);
  return sub(x, sub(add(x, m), m));
}

// sin(pi y), cos(pi y) for |y| <= 1/2 (the polynomials of sincos_pi_half).
template <class V>
__device__ __forceinline__ void sincos_half(V y, V& s, V& c) {
  const V w = mul(y, y);
  V ps = splat<V>(-0.007060864474624395f);
  ps = fma(ps, w, splat<V>(0.08207154273986816f));
  ps = fma(ps, w, splat<V>(-0.5992570519447327f));
  ps = fma(ps, w, splat<V>(2.550163745880127f));
  ps = fma(ps, w, splat<V>(-9.160392266949202e-08f));  // low part of -pi^3/6
  ps = fma(ps, w, splat<V>(-8.742277657347586e-08f));  // low part of pi
  ps = fma(w, splat<V>(-5.167712688446045f), ps);      // high part of -pi^3/6
  s = fma(y, splat<V>(3.1415927410125732f), mul(y, ps));  // high part of pi
  V pc = splat<V>(-0.024529997259378433f);
  pc = fma(pc, w, splat<V>(0.2350243180990219f));
  pc = fma(pc, w, splat<V>(-1.3352320194244385f));
  pc = fma(pc, w, splat<V>(4.058711051940918f));
  pc = fma(pc, w, splat<V>(-1.451857940537593e-07f));  // low part of -pi^2/2
  c = fma(w, splat<V>(-4.934802055358887f), fma(pc, w, splat<V>(1.0f)));  // high part of -pi^2/2
}

// hi + lo += v (Knuth two-sum, as f2x_add).
template <class V>
__device__ __forceinline__ void add_acc(V& hi, V& lo, V v) {
  const V s = add(hi, v);
  const V bb = sub(s, hi);
  lo = add(lo, add(sub(hi, sub(s, bb)), sub(v, bb)));
  hi = s;
}
}  // namespace pv

// Device-scope release/acquire fence.  The summary builds publish per-part
// and per-bin results and then take a ticket with a relaxed atomic; the
// block that draws the last ticket fences again and reads the others'
// results.  That publish-then-flag pattern needs release/acquire ordering
// only, not the sequentially consistent fence of __threadfence().
__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// Sum a float over the warp in FP64 (all lanes get the total).
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f32(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace rb
