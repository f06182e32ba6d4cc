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
// With the Newtonian amplitude the ratio has the same modulus |rho_d| at every
// edge, so Re(r0 r1*) = (|r_{b+1}|^2 - |r_b|^2) / (2 df_b) = 0: the beta1 term
// (Re t + Re(s t*)/2 = (|1 + delta_{b+1}|^2 - |1 + delta_b|^2) / 2) and its
// derivatives vanish identically.  The mixed kernel leaves it out (in FP32 it
// is rounding noise about zero); the plain FP64 kernel keeps the general form.
// delta is formed without cancellation from the half angle:
//   exp(-2 pi i x) - 1 = -2 sin^2(pi x) - 2 i sin(pi x) cos(pi x),
//   delta = rho (exp(-2 pi i x) - 1) + (rho - 1).
//
// Mapping: one warp per walker (persistent: each block takes a contiguous,
// equal share of the walkers and its warps take them in turn).  Float-float
// path: in iteration i lane l holds edges 63 i + 2 l and 63 i + 2 l + 1 and
// the bins on their right as the two halves of paired FP32 values (the slot
// image, EventDev::slot32); FP64-phase path: lane l handles edge 31 c + l of
// chunk c and bin 31 c + l (lanes 0..30).  Either way a bin's right edge is
// at most one shuffle away and consecutive iterations overlap by one edge.
// Edge and bin tables live in shared memory.  The adjoint reuses the same
// mapping: each edge collects the cotangent from its own bin and from the
// bin on its left; an edge shared by two iterations collects the two halves
// in two passes, which is exact because the adjoint is linear in the per-edge
// cotangent.
#include <algorithm>
#include <mutex>
#include <type_traits>

#include "rb_internal.cuh"

namespace rb {

#ifndef RB_MIXED_THREADS
#define RB_MIXED_THREADS 512
#endif
constexpr int kThreads = RB_MIXED_THREADS;  // threads per block of the mixed likelihood kernel
constexpr unsigned kFull = 0xffffffffu;
// The current walker's constants sit in shared memory (read by broadcast
// loads in every iteration instead of held in registers): as the set-up wrote
// them (WalkerMixed: float4 quads, detectors 0 and 1 paired, detector D - 1
// alone when D is odd), and for the float-float loop expanded into {x, x, y, y}
// quads (WarpSlot::dup).

// Shared-memory load that the compiler may not hoist out of a loop.
__device__ __forceinline__ float4 lds4(const float4* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"((unsigned)__cvta_generic_to_shared(p)));
  return v;
}

// Asynchronous global -> shared copies (cp.async): the copies of a thread
// complete, in issue order, by its next cp_async_wait_all().
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Per-warp shared-memory slot after the tables: two buffers for a walker's
// set-up record (its constants, WalkerMixed) and tangents, so that the next
// walker's are fetched while this one runs.
constexpr int kTanBytes = 384;
struct __align__(16) WarpSlot {
  WalkerMixed rec[2];
  unsigned char tan[2][kTanBytes];
  float red[32];  // the walker's adjoint sums
  // the current walker's constants, each value in both halves of a pair
  // (float-float path): {hi, hi, lo, lo} of dc_k (k < kNBasis), then per
  // detector {tau_hi, tau_hi, tau_lo, tau_lo}, {rho_r, rho_r, rho_i, rho_i},
  // {sig_r, sig_r, sig_i, sig_i}, and last the walker's rounding constant m
  // of the phase sums (split_acc) in all four
  float4 dup[kNBasis + 3 * kMaxDet + 1];
  // per lane: the bound on |g_k| or f that the lane's phase term takes in the
  // record expansion (constant over the launch)
  float lane_gmax[32];
};
static_assert(sizeof(WalkerMixed) % 16 == 0, "record copied in 16-byte pieces");
static_assert(sizeof(WalkerTan<float>) <= kTanBytes && sizeof(WalkerTan<float>) % 8 == 0, "tangent buffer");

// Issue (the whole warp) the copies of one walker's record (unless PHASE64,
// whose FP64 record is read directly) and tangents into buffer buf, as one
// cp.async group.  Global addresses: records 16-byte, tangents 8-byte
// aligned (checked by the launcher).
template <bool GRAD, bool PHASE64>
__device__ __forceinline__ void prefetch_walker(WarpSlot* slot, int buf, const void* rec, const void* tan, int lane) {
  if (!PHASE64 && lane < (int)(sizeof(WalkerMixed) / 16))
    cp_async16(reinterpret_cast<unsigned char*>(&slot->rec[buf]) + 16 * lane, static_cast<const unsigned char*>(rec) + 16 * lane);
  if (GRAD) {
    constexpr int n = (int)(sizeof(WalkerTan<float>) / 8);
#pragma unroll
    for (int i = lane; i < n; i += 32) cp_async8(slot->tan[buf] + 8 * i, static_cast<const unsigned char*>(tan) + 8 * i);
  }
  cp_async_commit();
}

// Exact float -> double conversion on the integer pipe: an SMSP's FP64 unit
// takes ~65 clocks per warp instruction, conversions included, and the warps
// of a block reach their epilogues together.  Normal numbers: the exponent
// rebiased by 1023 - 127 and the mantissa moved up 29 bits; zero, subnormals,
// infinities and NaN take the regular conversion.
__device__ __forceinline__ double f2d_int(float x) {
  const unsigned u = __float_as_uint(x), m = u & 0x7fffffffu;
  if (m - 0x00800000u < 0x7f000000u)
    return __hiloint2double((int)((u & 0x80000000u) | ((m >> 3) + 0x38000000u)), (int)(m << 29));
  return (double)x;
}

// Float-pair warp sum: (h, l) on entry is a lane's value as an unevaluated
// sum; every lane returns the warp total (two-sum of the high parts, the low
// parts added, renormalised at each step), all on the FP32 pipe.
__device__ __forceinline__ void warp_sum_ff(float& h, float& l) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    const float s = __fadd_rn(h, oh);
    const float bb = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(oh, bb));
    const float lo = __fadd_rn(__fadd_rn(l, ol), e);
    h = __fadd_rn(s, lo);
    l = __fsub_rn(lo, __fsub_rn(h, s));
  }
}

// One level of a transposed warp sum: lanes whose bit o is clear keep values
// [0, M) of `in` and send [M, N), lanes whose bit is set keep [M, N) (zero
// beyond N) and send [0, M); each adds what its partner sent.
template <int N, int M>
__device__ __forceinline__ void tsum_level(const float (&in)[N], float (&out)[M], int lane, int o) {
  const bool up = (lane & o) != 0;
#pragma unroll
  for (int i = 0; i < M; ++i) {
    const float lo = in[i], hi = (M + i < N) ? in[M + i] : 0.f;
    const float keep = up ? hi : lo, send = up ? lo : hi;
    out[i] = __fadd_rn(keep, __shfl_xor_sync(0xffffffffu, send, o));
  }
}

// Warp sums of NV <= 32 values per lane, each a fixed-order five-level tree:
// after five halving levels every lane holds the total of one value, which
// it writes to out[index] (shared memory); 31 shuffles for 32 values against
// 5 NV for NV separate butterflies.
template <int NV>
__device__ __forceinline__ void warp_transposed_sums(const float (&v)[NV], int lane, float* out) {
  static_assert(NV >= 1 && NV <= 32, "up to 32 values");
  constexpr int m1 = (NV + 1) / 2, m2 = (m1 + 1) / 2, m3 = (m2 + 1) / 2, m4 = (m3 + 1) / 2, m5 = (m4 + 1) / 2;
  static_assert(m5 == 1, "five levels reduce to one value");
  float a[m1], b[m2], c[m3], d[m4], e[m5];
  tsum_level<NV, m1>(v, a, lane, 16);
  tsum_level<m1, m2>(a, b, lane, 8);
  tsum_level<m2, m3>(b, c, lane, 4);
  tsum_level<m3, m4>(c, d, lane, 2);
  tsum_level<m4, m5>(d, e, lane, 1);
  // the value's index: the positions this lane kept, from the last level back
  // (a lane whose kept half was padding at some level holds no value)
  int idx = (lane & 1) ? m5 : 0;
  bool ok = idx < m4;
  idx += (lane & 2) ? m4 : 0;
  ok = ok && idx < m3;
  idx += (lane & 4) ? m3 : 0;
  ok = ok && idx < m2;
  idx += (lane & 8) ? m2 : 0;
  ok = ok && idx < m1;
  idx += (lane & 16) ? m1 : 0;
  ok = ok && idx < NV;
  if (ok) out[idx] = e[0];
}

// Adds the float pair (bh, bl) to (h, l) (two-sum of the high parts).
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float lo = __fadd_rn(__fadd_rn(l, bl), e);
  h = __fadd_rn(s, lo);
  l = __fsub_rn(lo, __fsub_rn(h, s));
}

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

// The same chain rule for the mixed kernel, with the tangents in shared
// memory: every lane runs one instruction stream (the lane's tangent entries
// picked by index and select, no divergent branches).  G_d = conj(gbar_rho_d)
// rho_d, the prefactor's adjoint in the form d log L = Re(G_d dln rho_d).
template <int D>
__device__ __forceinline__ float chain_rule_lanes(int j, const float* adj_c, const float* adj_tau, const float (*G)[2],
                                                  const WalkerTan<float>& tn) {
  const float* t = reinterpret_cast<const float*>(&tn);
  constexpr int oDc = offsetof(WalkerTan<float>, dc) / 4, oPhi = offsetof(WalkerTan<float>, dphi0) / 4;
  constexpr int oDtd = offsetof(WalkerTan<float>, dtd) / 4, oLnP = offsetof(WalkerTan<float>, dlnP) / 4;
  constexpr int oMc = offsetof(WalkerTan<float>, lnamp_Mc) / 4, oDl = offsetof(WalkerTan<float>, lnamp_dL) / 4;
  const bool intr = j < kNTanIntr, radec = j == 11 || j == 12, ext = j >= 9;
  const int ji = intr ? j : 0, jr = radec ? j - 11 : 0, je = ext ? j - 9 : 0;
  float g = 0.f;
#pragma unroll
  for (int k = 0; k < kNBasis; ++k) {
    const float v = t[oDc + k * kNTanIntr + ji];
    g = fmaf(adj_c[k], intr ? v : 0.f, g);
  }
  // d ln rho_d = lr + i li: ln amplitude (Mc, dL), -dPhi0 (Mc, q), phi_c, antenna (iota, psi, ra, dec)
  const int ir = j == 0 ? oMc : (j == 6 ? oDl : oMc);
  const float lr_own = (j == 0 || j == 6) ? t[ir] : 0.f;
  const int ii = j == 1 ? oPhi + 1 : oPhi;
  const float li_own = (j == 0 || j == 1) ? -t[ii] : (j == 8 ? 1.f : 0.f);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const float td = t[oDtd + 2 * d + jr];
    g = fmaf(adj_tau[d], radec ? td : (j == 7 ? 1.f : 0.f), g);
    const float pr = t[oLnP + 8 * d + 2 * je], pi = t[oLnP + 8 * d + 2 * je + 1];
    const float lr = ext ? pr : lr_own, li = ext ? pi : li_own;
    g += G[d][0] * lr - G[d][1] * li;  // Re(G_d dln rho_d)
  }
  return g;
}

namespace pv {
// Per-walker detector constants and adjoint accumulators of one detector
// (V = float) or of the detector pair 0, 1 (V = float2).
template <class V>
struct DetState {
  V tau_h, tau_l;          // delta tau [s] as a float pair
  V rho_r, rho_i, sig_r, sig_i;
  V acc, acc_lo;           // log L terms, float-pair accumulator
  V adj_tau, adj_rr, adj_ri;
};

// One bin edge (and the bin on its right) for one detector or a detector
// pair: half-angle sin/cos, delta = rho (e^{-2 pi i y} - 1) + sigma, the
// neighbour edge by a shuffle, the bin's contraction with the tables (bins
// of lanes 0..30) and, with GRAD, the edge cotangent.  Returns d log L / dy
// per detector (times 1/2pi) for the basis adjoint.  The whole warp calls it.
template <bool GRAD, class V>
__device__ __forceinline__ V det_edge(V y, DetState<V>& st, const V* bt, bool has_bin, bool has_edge, int lane, V fe) {
  V sn, cs;
  sincos_half(y, sn, cs);
  const V t2 = mul(splat<V>(-2.f), sn);
  const V em_r = mul(t2, sn), em_i = mul(t2, cs);  // e^{-2 pi i y} - 1
  const V dr = fma(st.rho_r, em_r, fma(neg(st.rho_i), em_i, st.sig_r));
  const V di = fma(st.rho_r, em_i, fma(st.rho_i, em_r, st.sig_i));
  const V nr = shfl_down(dr), ni = shfl_down(di);
  V Ur = splat<V>(0.f), Ui = Ur, Vr = Ur, Vi = Ur;
  if (has_bin) {
    // bt: alpha0 (re, im), alpha1 (re, im), -beta0 (the -beta1 entry is not
    // needed: the beta1 term vanishes for a ratio of constant modulus)
    const V sr = add(dr, nr), si = add(di, ni), tr = sub(nr, dr), ti = sub(ni, di);
    V v = mul(bt[0], sr);
    v = fma(bt[1], si, v);
    v = fma(bt[2], tr, v);
    v = fma(bt[3], ti, v);
    v = fma(bt[4], fma(splat<V>(0.25f), fma(sr, sr, mul(si, si)), sr), v);
    const V s = add(st.acc, v);  // two-sum into (acc, acc_lo)
    const V bb = sub(s, st.acc);
    st.acc_lo = add(st.acc_lo, add(sub(st.acc, sub(s, bb)), sub(v, bb)));
    st.acc = s;
    if (GRAD) {
      const V hs_r = fma(splat<V>(0.5f), sr, splat<V>(1.f)), hs_i = mul(splat<V>(0.5f), si);  // 1 + s/2
      Ur = fma(bt[4], hs_r, bt[0]);
      Ui = fma(bt[4], hs_i, bt[1]);
      Vr = bt[2];
      Vi = bt[3];
    }
  }
  V dldx = splat<V>(0.f);
  if (GRAD) {
    V gr = sub(Ur, Vr), gi = sub(Ui, Vi);  // own bin (edge on its left)
    const V lr = shfl_up(add(Ur, Vr)), li = shfl_up(add(Ui, Vi));
    if (lane > 0) {
      gr = add(gr, lr);
      gi = add(gi, li);
    }
    if (has_edge) {
      const V rr = add(splat<V>(1.f), dr);
      dldx = fma(gr, di, mul(neg(gi), rr));  // Im(conj(gbar) r); times 2 pi later
      st.adj_tau = fma(dldx, fe, st.adj_tau);
      const V Er = add(splat<V>(1.f), em_r);  // gbar_rho += gbar conj(E)
      st.adj_rr = fma(gr, Er, fma(gi, em_i, st.adj_rr));
      st.adj_ri = fma(gi, Er, fma(neg(gr), em_i, st.adj_ri));
    }
  }
  return dldx;
}
// The same for the two edges of a slot (halves A and B: edges e_A = 63 i + 2 l
// and e_B = e_A + 1 of lane l) and one detector: e_A's right neighbour is
// the lane's own e_B, e_B's is lane l + 1's e_A (one shuffle); e_B's left
// bin is the lane's own A bin, e_A's is lane l - 1's B bin, none for lane 0
// (its e_A is lane 31's e_B of the previous iteration, which collected it).
// Edges without a bin, and slots past the last edge, have zero tables, so
// they add nothing.  vsum collects the bin terms of log L, adj_x
// d log L / dy (times 1/2pi) for the basis adjoint, (adj_rr, adj_ri) the sum
// of conj(gbar) r over the edges (the prefactor's adjoint times rho: G_d).
// The bin's term in the coefficients of its edge values (q0 = {gmr, gpr},
// q1 = {gmi, gpi}, q2 = {h, q} of the slot image): with d = delta at the
// left edge and n at the right one,
//   Re(alpha0 s*) + Re(alpha1 t*) - beta0 (Re s + |s|^2/4)
//     = gmr dr + gpr nr + gmi di + gpi ni + q |s|^2,
// and the cotangents of the left and right edge values are
//   (gmr + h sr, gmi + h si) and (gpr + h sr, gpi + h si).
template <bool GRAD>
__device__ __forceinline__ void det_edge_slot(float2 y, float4 rho, float4 sig, const float2 (&bt)[6], int lane,
                                              float2 fe, float2& vsum, float2& adj_x, float& adj_tau, float& adj_rr,
                                              float& adj_ri) {
  const float2 rho_r = make_float2(rho.x, rho.y), rho_i = make_float2(rho.z, rho.w);
  const float2 sig_r = make_float2(sig.x, sig.y), sig_i = make_float2(sig.z, sig.w);
  float2 sn, cs;
  sincos_half(y, sn, cs);
  const float2 t2 = mul(splat<float2>(-2.f), sn);
  const float2 em_r = mul(t2, sn), em_i = mul(t2, cs);  // e^{-2 pi i y} - 1
  const float2 dr = fma(rho_r, em_r, fma(neg(rho_i), em_i, sig_r));
  const float2 di = fma(rho_r, em_i, fma(rho_i, em_r, sig_i));
  const float2 nr = make_float2(dr.y, __shfl_down_sync(0xffffffffu, dr.x, 1));
  const float2 ni = make_float2(di.y, __shfl_down_sync(0xffffffffu, di.x, 1));
  // bt: gmr, gpr, gmi, gpi, h, q (the beta1 term vanishes for a ratio of
  // constant modulus)
  const float2 sr = add(dr, nr), si = add(di, ni);
  float2 v = mul(bt[0], dr);
  v = fma(bt[1], nr, v);
  v = fma(bt[2], di, v);
  v = fma(bt[3], ni, v);
  v = fma(bt[5], fma(sr, sr, mul(si, si)), v);
  vsum = add(vsum, v);
  if (GRAD) {
    float2 gr = fma(bt[4], sr, bt[0]), gi = fma(bt[4], si, bt[2]);  // own bin (edge on its left)
    const float2 pr = fma(bt[4], sr, bt[1]), pi = fma(bt[4], si, bt[3]);  // the bin's right edge
    const float lr = __shfl_up_sync(0xffffffffu, pr.y, 1), li = __shfl_up_sync(0xffffffffu, pi.y, 1);
    gr = add(gr, make_float2(lane == 0 ? 0.f : lr, pr.x));
    gi = add(gi, make_float2(lane == 0 ? 0.f : li, pi.x));
    const float2 rr = add(splat<float2>(1.f), dr);
    const float2 dldx = fma(gr, di, mul(neg(gi), rr));  // Im(conj(gbar) r); times 2 pi later
    adj_x = add(adj_x, dldx);
    adj_tau = __fmaf_rn(dldx.x, fe.x, __fmaf_rn(dldx.y, fe.y, adj_tau));
    // the prefactor: r = rho E, so conj(gbar_rho) rho = sum conj(gbar) r, whose
    // imaginary part is the sum of dldx
    adj_rr = __fmaf_rn(gr.x, rr.x, __fmaf_rn(gr.y, rr.y, __fmaf_rn(gi.x, di.x, __fmaf_rn(gi.y, di.y, adj_rr))));
    adj_ri = __fadd_rn(adj_ri, __fadd_rn(dldx.x, dldx.y));
  }
}
}  // namespace pv

// ---------------------------------------------------------------------------
// Mixed precision.  PHASE64 = false: phase as float pairs (FP32 pipe);
// PHASE64 = true: phase accumulated in native FP64.  ND = number of
// detectors, a compile-time constant so that the independent chains of the
// detector pair and the single detector interleave in one instruction stream.
// ---------------------------------------------------------------------------
template <int ND, bool GRAD, bool PHASE64, bool MALA = false>
__global__ void __launch_bounds__(kThreads) k_rb_mixed(LaunchArgs a) {
  static_assert(!MALA || GRAD, "the MALA step needs the gradient");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EventDev& ev = a.ev;
  constexpr int D = ND;
  const int Ep = ev.e_pad, Bp = ev.b_pad, B = ev.n_bins, E = ev.n_edges;
  const BaseRead base_read = event_base_read(ev);  // in flight across the staging

  // Stage the tables (16-byte asynchronous copies, all in flight at once).
  const float* sbin;
#ifdef RB_BOUNDS_CHECK
  unsigned smem_bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(smem_bytes));
  const size_t smem16 = smem_bytes / 16;
#else
  constexpr size_t smem16 = 0;  // unused
#endif
  const float4* g4 = nullptr;  // slot image: [kNBasis + 1][NS] basis values and f_e of the slots' edge pairs
  const double* g64 = nullptr;
  const double* f64 = nullptr;
  {
    const int tid = threadIdx.x;
    if (!PHASE64) {
      const float4* src = reinterpret_cast<const float4*>(ev.slot32);
      float4* dst = reinterpret_cast<float4*>(smem_raw);
      const size_t n4 = ev.slot32_floats / 4;
      for (size_t i = tid; i < n4; i += blockDim.x) cp_async16(&dst[RB_IDX(i, smem16, 104)], &src[i]);
      const float* s = reinterpret_cast<const float*>(smem_raw);
      g4 = reinterpret_cast<const float4*>(s);
      sbin = s + (size_t)4 * (kNBasis + 1) * ev.n_slots;
    } else {
      const size_t n_e64 = (size_t)(kNBasis + 1) * Ep;  // g[10][Ep], f[Ep]
      const double2* src = reinterpret_cast<const double2*>(ev.tab64);
      double2* dst = reinterpret_cast<double2*>(smem_raw);
      for (size_t i = tid; i < n_e64 / 2; i += blockDim.x) cp_async16(&dst[RB_IDX(i, smem16, 104)], &src[i]);
      const size_t nb = ev.tab32_floats - ev.edge32_floats;
      const float4* bsrc = reinterpret_cast<const float4*>(ev.tab32 + ev.edge32_floats);
      float4* bdst = reinterpret_cast<float4*>(smem_raw + n_e64 * sizeof(double));
      for (size_t i = tid; i < nb / 4; i += blockDim.x) cp_async16(&bdst[RB_IDX(i, smem16 - n_e64 / 2, 104)], &bsrc[i]);
      g64 = reinterpret_cast<const double*>(smem_raw);
      f64 = g64 + (size_t)kNBasis * Ep;
      sbin = reinterpret_cast<const float*>(smem_raw + n_e64 * sizeof(double));
    }
  }
  cp_async_commit();

  const int lane = threadIdx.x & 31;
  WarpSlot* slot;  // this warp's slot, after the tables
  {
    const size_t tab_bytes = !PHASE64 ? ev.slot32_floats * sizeof(float)
                                      : (size_t)(kNBasis + 1) * Ep * sizeof(double) +
                                            (ev.tab32_floats - ev.edge32_floats) * sizeof(float);
    slot = reinterpret_cast<WarpSlot*>(smem_raw + tab_bytes) + (threadIdx.x >> 5);
  }
  // detectors 0 and 1 form a pair when D >= 2; an odd detector count leaves
  // detector D - 1 single (bin table layout in EventDev)
  constexpr bool paired = D >= 2;
  constexpr int ds = (D & 1) ? D - 1 : -1;
  constexpr int dss = ds < 0 ? 0 : ds;
  const float4* binP = reinterpret_cast<const float4*>(sbin);                                // [3][Bp]
  const float4* binS4 = reinterpret_cast<const float4*>(sbin + (paired ? 12 * Bp : 0));      // [Bp]
  const float2* binS2 = reinterpret_cast<const float2*>(sbin + (paired ? 12 * Bp : 0) + 4 * Bp);  // [Bp]
  // each block takes a contiguous, equal share of the walkers (so every SM
  // gets W / grid of them, +-1), its warps take them in turn
  const int64_t per_blk = a.W / gridDim.x, rem_blk = a.W % gridDim.x;
  const int64_t w_begin = (int64_t)blockIdx.x * per_blk + min((int64_t)blockIdx.x, rem_blk);
  const int64_t w_end = w_begin + per_blk + ((int64_t)blockIdx.x < rem_blk ? 1 : 0);
  const int64_t warp0 = w_begin + (threadIdx.x >> 5);
  const int64_t nwarps = blockDim.x >> 5;
  const unsigned char* rec_g = static_cast<const unsigned char*>(a.ws);
  const unsigned char* tan_g = static_cast<const unsigned char*>(a.tan);
  // the first walker's record and tangents travel with the tables
  if (warp0 < w_end)
    prefetch_walker<GRAD, PHASE64>(slot, 0, PHASE64 ? nullptr : rec_g + sizeof(WalkerMixed) * RB_IDX(warp0, a.W, 101),
                                   GRAD ? tan_g + sizeof(WalkerTan<float>) * RB_IDX(warp0, a.W, 107) : nullptr, lane);
  cp_async_wait_all();
  __syncthreads();
  const double base_logl = event_base_value(ev, base_read);

  // the bound on |g_k| or f that this lane's phase term takes (the record
  // expansion below: lane k < kNBasis basis k, lane kNBasis + 3 d detector d's
  // delay), read once into the warp's slot: indexed by lane, a constant-bank
  // load serialises
  if (!PHASE64) {
    const int j = lane - kNBasis;
    const int gk = lane < kNBasis ? lane : (j < 3 * D && j % 3 == 0 ? kNBasis : -1);
    slot->lane_gmax[lane] = gk >= 0 ? ev.gmax[gk] : 0.f;
  }

  int buf = 0;
  for (int64_t w = warp0; w < w_end; w += nwarps, buf ^= 1) {
    cp_async_wait_all();  // this walker's record and tangents
    __syncwarp();         // ... visible to the warp; the previous walker's reads of wc and of buffer buf ^ 1 done
    // ---- per-walker constants (uniform across the warp), in shared memory ----
    float4* const wc = slot->rec[buf].q;
    double dc64[kNBasis];
    double tau64[kMaxDet];
    pv::DetState<float2> P;  // detectors 0, 1: accumulators (constants come from wc)
    pv::DetState<float> S;   // detector ds
    int valid;
    unsigned walker_ex = 0;  // float-float path: exponent field of the walker's phase-term bound
    if (!PHASE64) {
      valid = slot->rec[buf].valid;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) dc64[k] = 0.0;
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) tau64[d] = 0.0;
      // each constant in both halves of a pair (the slot loop's operands):
      // lane k < kNBasis takes dc_k, lane kNBasis + 3 d + m the delay (m = 0),
      // prefactor ratio (1) or its difference from 1 (2) of detector d
      float mag = 0.f;  // the lane's bound on |its phase term| [turns]
      if (lane < kNBasis + 3 * D) {
        const float* f = reinterpret_cast<const float*>(wc);
        int iu, iv;
        if (lane < kNBasis) {
          iu = wm_dc_hi(lane);
          iv = wm_dc_lo(lane);
        } else {
          const int j = lane - kNBasis, d = j / 3, m = j - 3 * d;
          if (d == ds) {
            iu = kWmSingle + (m == 0 ? 0 : 2 + 2 * m);
          } else {
            iu = (m == 0 ? kWmTauPair : (m == 1 ? kWmRhoPair : kWmSigPair)) + d;
          }
          iv = iu + (d == ds ? 1 : 2);
        }
        const float u = f[iu], v = f[iv];
        slot->dup[lane] = make_float4(u, u, v, v);
        mag = fabsf(u) * slot->lane_gmax[lane];
      }
      // the walker's rounding constant m = 1.5 * 2^23 q with q = 2^-20 of a
      // power of two above every phase term (at least 2^-62 turns): then each
      // product's high part is below 2^22 q, and the eleven of a detector's
      // phase (ten basis terms and the delay) add to less than 2^24 q
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mag = fmaxf(mag, __shfl_xor_sync(0xffffffffu, mag, o));
      const unsigned ex = min(max((__float_as_uint(mag) >> 23) & 0xffu, 64u), 250u);  // mag < 2^(ex - 126)
      walker_ex = ex;
      if (lane == 0) {
        const float m = __uint_as_float(((ex + 4u) << 23) | 0x400000u);  // 1.5 * 2^(ex - 123)
        slot->dup[kNBasis + 3 * kMaxDet] = make_float4(m, m, m, m);
      }
    } else {
      float rho[kMaxDet][2], sg[kMaxDet][2];
      const WalkerF64* s = reinterpret_cast<const WalkerF64*>(a.ws) + w;
      valid = s->valid;
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) dc64[k] = s->dc[k];
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        tau64[d] = s->tau[d];
        rho[d][0] = (float)s->rho[d][0]; rho[d][1] = (float)s->rho[d][1];
        sg[d][0] = (float)s->sig[d][0]; sg[d][1] = (float)s->sig[d][1];
      }
      __syncwarp();  // the previous walker's reads of this buffer are done
      if (lane == 0) {
        // the phase and delay quads are not read on this path
#pragma unroll
        for (int q = 0; q < 6; ++q) wc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        wc[6] = make_float4(rho[0][0], rho[1][0], rho[0][1], rho[1][1]);
        wc[7] = make_float4(sg[0][0], sg[1][0], sg[0][1], sg[1][1]);
        wc[8] = make_float4(0.f, 0.f, 0.f, 0.f);
        wc[9] = make_float4(rho[dss][0], rho[dss][1], sg[dss][0], sg[dss][1]);
      }
    }
    __syncwarp();
    {
      // the next walker's record and tangents, into the other buffer (issued
      // after this walker's shared-memory reads above)
      const int64_t wn = w + nwarps;
      if (wn < w_end)
        prefetch_walker<GRAD, PHASE64>(slot, buf ^ 1, PHASE64 ? nullptr : rec_g + sizeof(WalkerMixed) * RB_IDX(wn, a.W, 101),
                                       GRAD ? tan_g + sizeof(WalkerTan<float>) * RB_IDX(wn, a.W, 107) : nullptr, lane);
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
    if (!PHASE64 && walker_ex > 126u + 18u) {
      // a phase term beyond 2^18 turns (~1.6e6 rad): past the range of the
      // float-pair phase sums' whole-turn reductions; not evaluated (NaN,
      // rejected by the MALA step)
      if (MALA) {
        mala_finish(a.mala, w, lane, -INFINITY, 0.0);
      } else {
        if (lane == 0) a.logl[w] = __longlong_as_double(0x7ff8000000000000ll);
        if (GRAD && lane < kNPar) a.grad[w * kNPar + lane] = __longlong_as_double(0x7ff8000000000000ll);
      }
      continue;
    }

    // float-pair accumulators: for walkers far from the fiducial point the
    // per-bin terms add up to about -log L(theta_ref), so a single float would
    // lose ~1e-3 of absolute precision
    constexpr int kNV = kNBasis + 3 * D;
    float lh, ll;   // the lane's share of log L - log L(theta_ref), a float pair
    float v[kNV];   // the lane's adjoint sums: basis coefficients, then per detector the delay and the ratio re/im
    if constexpr (!PHASE64) {
      // slot loop: both halves of every paired value are edges of this walker
      const int NS = ev.n_slots;
      const float4* const wd = slot->dup;
      float2 acc = make_float2(0.f, 0.f), acc_lo = acc;
      // the adjoint sums of a lane's two edges in one float each (as pairs,
      // the extra registers spilled)
      float adj_c[kNBasis];
      float adj_tau[D], adj_rr[D], adj_ri[D];
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) adj_c[k] = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) adj_tau[d] = adj_rr[d] = adj_ri[d] = 0.f;
      // walkers whose phase terms reach beyond 2^12 turns take a second
      // whole-turn reduction of the phase (the low sum can then carry it past
      // the half-angle polynomials' range): a second copy of the loop, so
      // that the others pay nothing for it
      auto slot_loop = [&](auto wide_c) {
      constexpr bool WIDE = decltype(wide_c)::value;
      for (int s0 = 0; s0 < NS; s0 += 32) {
        const int sl = RB_IDX(s0 + lane, NS, 102);
        // detector-independent phase sum_k dc_k g_k(f_e) / 2pi [turns] of the
        // two edges, as an exact sum of multiples of the walker's q (sh) and a
        // small remainder (sl_lo)
        const float4 mq = lds4(wd + kNBasis + 3 * kMaxDet);
        const float2 m2 = make_float2(mq.x, mq.y);
        float2 sh = make_float2(0.f, 0.f), sl_lo = sh;
#pragma unroll
        for (int k = 0; k < kNBasis; ++k) {
          const float4 g = g4[k * NS + sl];  // {g_hi(e_A), g_hi(e_B), g_lo(e_A), g_lo(e_B)}
          const float4 c = lds4(wd + k);     // {dc_hi, dc_hi, dc_lo, dc_lo}
          pv::split_acc(make_float2(c.x, c.y), make_float2(c.z, c.w), make_float2(g.x, g.y), make_float2(g.z, g.w), m2, sh,
                        sl_lo);
        }
        const float4 f4 = g4[kNBasis * NS + sl];
        const float2 fe = make_float2(f4.x, f4.y), fe_lo = make_float2(f4.z, f4.w);
        float2 vsum = make_float2(0.f, 0.f), adj_x = vsum;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const float4 tt = lds4(wd + kNBasis + 3 * d);
          float2 yh = sh, yl = sl_lo;
          pv::split_acc(make_float2(tt.x, tt.y), make_float2(tt.z, tt.w), fe, fe_lo, m2, yh, yl);
          float2 y = pv::frac(yh, yl);
          if constexpr (WIDE) y = pv::frac1(y);
          const float4* sb = reinterpret_cast<const float4*>(sbin + (size_t)d * kSlotBinFloats * NS);
          const float4 q0 = sb[sl], q1 = sb[NS + sl], q2 = sb[2 * NS + sl];
          const float2 bt[6] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                                make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
          pv::det_edge_slot<GRAD>(y, lds4(wd + kNBasis + 3 * d + 1), lds4(wd + kNBasis + 3 * d + 2), bt, lane, fe, vsum,
                                  adj_x, adj_tau[d], adj_rr[d], adj_ri[d]);
        }
        pv::add_acc(acc, acc_lo, vsum);
        if (GRAD) {
          // the high halves only: 8-byte loads (shared-memory bandwidth is
          // about as busy as the FMA pipe in this loop)
          const float2* g2 = reinterpret_cast<const float2*>(g4);
#pragma unroll
          for (int k = 0; k < kNBasis; ++k) {
            const float2 g = g2[2 * (k * NS + sl)];
            adj_c[k] = __fmaf_rn(adj_x.x, g.x, __fmaf_rn(adj_x.y, g.y, adj_c[k]));
          }
        }
      }
      };
      if (walker_ex > 126u + 12u) slot_loop(std::true_type{});
      else slot_loop(std::false_type{});
      lh = acc.x;
      ll = acc_lo.x;
      ff_add(lh, ll, acc.y, acc_lo.y);
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) v[k] = adj_c[k];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        v[kNBasis + d] = adj_tau[d];
        v[kNBasis + D + d] = adj_rr[d];
        v[kNBasis + 2 * D + d] = adj_ri[d];
      }
    } else {
      // FP64 phase: one edge per lane, lane l of chunk c at edge 31 c + l
      P.acc = P.acc_lo = P.adj_tau = P.adj_rr = P.adj_ri = make_float2(0.f, 0.f);
      S.acc = S.acc_lo = S.adj_tau = S.adj_rr = S.adj_ri = 0.f;
      float2 adj_c[kNBasis / 2];
#pragma unroll
      for (int q = 0; q < kNBasis / 2; ++q) adj_c[q] = make_float2(0.f, 0.f);

      for (int c0 = 0; c0 < B; c0 += 31) {
        const int e = c0 + lane;
        const bool has_edge = e < E;
        const bool has_bin = (lane < 31) && (e < B);
        const int ee = RB_IDX(has_edge ? e : E - 1, Ep, 102);
        const int eb = RB_IDX(has_bin ? e : 0, Bp, 103);
        double x64 = 0.0;
#pragma unroll
        for (int k = 0; k < kNBasis; ++k) x64 = ::fma(dc64[k], g64[k * Ep + ee], x64);
        const float fe = (float)f64[ee];

        float adj_x = 0.f;
        if constexpr (paired) {
          const float4 rr = lds4(wc + 6), ss = lds4(wc + 7);
          P.rho_r = make_float2(rr.x, rr.y); P.rho_i = make_float2(rr.z, rr.w);
          P.sig_r = make_float2(ss.x, ss.y); P.sig_i = make_float2(ss.z, ss.w);
          const double x0 = ::fma(f64[ee], tau64[0], x64), x1 = ::fma(f64[ee], tau64[1], x64);
          const float2 y = make_float2((float)(x0 - rint(x0)), (float)(x1 - rint(x1)));
          const float4 q0 = binP[eb], q1 = binP[Bp + eb], q2 = binP[2 * Bp + eb];
          const float2 bt[6] = {make_float2(q0.x, q0.y), make_float2(q0.z, q0.w), make_float2(q1.x, q1.y),
                                make_float2(q1.z, q1.w), make_float2(q2.x, q2.y), make_float2(q2.z, q2.w)};
          const float2 g = pv::det_edge<GRAD>(y, P, bt, has_bin, has_edge, lane, make_float2(fe, fe));
          adj_x = __fadd_rn(g.x, g.y);
        }
        if constexpr (ds >= 0) {
          const float4 rs = lds4(wc + 9);
          S.rho_r = rs.x; S.rho_i = rs.y; S.sig_r = rs.z; S.sig_i = rs.w;
          const double xd = ::fma(f64[ee], tau64[ds], x64);
          const float y = (float)(xd - rint(xd));
          const float4 q0 = binS4[eb];
          const float2 q1 = binS2[eb];
          const float bt[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
          adj_x = __fadd_rn(adj_x, pv::det_edge<GRAD>(y, S, bt, has_bin, has_edge, lane, fe));
        }
        if (GRAD && has_edge) {
          const float2 ax = make_float2(adj_x, adj_x);
#pragma unroll
          for (int q = 0; q < kNBasis / 2; ++q)
            adj_c[q] = pv::fma(ax, make_float2((float)g64[2 * q * Ep + ee], (float)g64[(2 * q + 1) * Ep + ee]),
                               adj_c[q]);
        }
      }
      lh = S.acc;
      ll = S.acc_lo;
      if constexpr (paired) {
        ff_add(lh, ll, P.acc.x, P.acc_lo.x);
        ff_add(lh, ll, P.acc.y, P.acc_lo.y);
      }
#pragma unroll
      for (int q = 0; q < kNBasis / 2; ++q) {
        v[2 * q] = adj_c[q].x;
        v[2 * q + 1] = adj_c[q].y;
      }
      if constexpr (paired) {
        v[kNBasis + 0] = P.adj_tau.x;
        v[kNBasis + 1] = P.adj_tau.y;
        v[kNBasis + D + 0] = P.adj_rr.x;
        v[kNBasis + D + 1] = P.adj_rr.y;
        v[kNBasis + 2 * D + 0] = P.adj_ri.x;
        v[kNBasis + 2 * D + 1] = P.adj_ri.y;
      }
      if constexpr (ds >= 0) {
        v[kNBasis + ds] = S.adj_tau;
        v[kNBasis + D + ds] = S.adj_rr;
        v[kNBasis + 2 * D + ds] = S.adj_ri;
      }
    }

    // the walker's sum as a float pair (FP32 pipe); FP64 only for the result
    warp_sum_ff(lh, ll);
    const double logl = base_logl + (f2d_int(lh) + f2d_int(ll));
    if (!MALA && lane == 0) a.logl[RB_IDX(w, a.W, 105)] = logl;
    if (GRAD) {
      const float two_pi = 6.28318530717958648f;
      // the walker's adjoint sums (basis coefficients, then per detector the
      // delay and the prefactor ratio re/im) by one transposed warp sum
      warp_transposed_sums<kNV>(v, lane, slot->red);
      __syncwarp();
      float ac[kNBasis], at[kMaxDet], ar[kMaxDet][2];
#pragma unroll
      for (int k = 0; k < kNBasis; ++k) ac[k] = two_pi * slot->red[k];
#pragma unroll
      for (int d = 0; d < kMaxDet; ++d) {
        at[d] = d < D ? two_pi * slot->red[kNBasis + d] : 0.f;
        ar[d][0] = d < D ? slot->red[kNBasis + D + d] : 0.f;
        ar[d][1] = d < D ? slot->red[kNBasis + 2 * D + d] : 0.f;
      }
      if constexpr (PHASE64) {
        // this path sums gbar conj(E) = gbar_rho: G_d = conj(gbar_rho) rho
        float rho[kMaxDet][2];
        const float4 r01 = lds4(wc + 6), rs = lds4(wc + 9);
        rho[0][0] = r01.x; rho[1][0] = r01.y; rho[0][1] = r01.z; rho[1][1] = r01.w;
        if (ds >= 0) { rho[dss][0] = rs.x; rho[dss][1] = rs.y; }
        if (D < kMaxDet) rho[kMaxDet - 1][0] = rho[kMaxDet - 1][1] = 0.f;
#pragma unroll
        for (int d = 0; d < kMaxDet; ++d) {
          const float a_r = ar[d][0], a_i = ar[d][1];
          ar[d][0] = a_r * rho[d][0] + a_i * rho[d][1];
          ar[d][1] = a_r * rho[d][1] - a_i * rho[d][0];
        }
      }
      double g = 0.0;
      if (lane < kNPar) {
        const WalkerTan<float>& tn = *reinterpret_cast<const WalkerTan<float>*>(slot->tan[buf]);  // prefetched
        g = f2d_int(chain_rule_lanes<D>(lane, ac, at, ar, tn));
      }
      if (MALA) mala_finish(a.mala, w, lane, logl, g);
      else if (lane < kNPar) a.grad[RB_IDX(w * kNPar + lane, a.W * kNPar, 106)] = g;
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
  const double base_logl = event_base_logl(ev);
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
    const double logl = base_logl + tot;
    if (!MALA && lane == 0) a.logl[RB_IDX(w, a.W, 105)] = logl;
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
      else if (lane < kNPar) a.grad[RB_IDX(w * kNPar + lane, a.W * kNPar, 106)] = g;
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
size_t mixed_smem_slot_bytes() { return (size_t)(kThreads / 32) * sizeof(WarpSlot); }

size_t mixed_smem_bytes(const EventDev& ev, bool phase64) {
  const size_t wc = (size_t)(kThreads / 32) * sizeof(WarpSlot);
  if (!phase64) return ev.slot32_floats * sizeof(float) + wc;
  return (size_t)(kNBasis + 1) * ev.e_pad * sizeof(double) + (ev.tab32_floats - ev.edge32_floats) * sizeof(float) + wc;
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
    // allow any dynamic shared-memory size up to the device limit (less the
    // kernel's static shared memory) once, so that launches for different
    // events never shrink it for one another
    int dev = 0, smem_max = 0;
    cudaFuncAttributes fa{};
    err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (err == cudaSuccess) err = cudaFuncGetAttributes(&fa, fn);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max - (int)fa.sharedSizeBytes);
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

template <int ND, bool GRAD, bool PHASE64, bool MALA>
static cudaError_t launch_mixed_nd(const LaunchArgs& a, cudaStream_t s, int n_sm) {
  // the kernel copies records in 16-byte and tangents in 8-byte asynchronous copies
  if (reinterpret_cast<uintptr_t>(a.ws) % 16 != 0 || (GRAD && reinterpret_cast<uintptr_t>(a.tan) % 8 != 0))
    return cudaErrorMisalignedAddress;
  const size_t smem = mixed_smem_bytes(a.ev, PHASE64);
  const void* fn = reinterpret_cast<const void*>(k_rb_mixed<ND, GRAD, PHASE64, MALA>);
  int per_sm = 0;
  cudaError_t err = blocks_per_sm(fn, kThreads, smem, &per_sm);
  if (err != cudaSuccess) return err;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t blocks_needed = (a.W * 32 + kThreads - 1) / kThreads;
  const int64_t grid = std::min<int64_t>(blocks_needed, (int64_t)per_sm * n_sm);
  k_rb_mixed<ND, GRAD, PHASE64, MALA><<<(unsigned)grid, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool GRAD, bool PHASE64, bool MALA = false>
static cudaError_t launch_mixed_t(const LaunchArgs& a, cudaStream_t s, int n_sm) {
  switch (a.ev.n_det) {
    case 1: return launch_mixed_nd<1, GRAD, PHASE64, MALA>(a, s, n_sm);
    case 2: return launch_mixed_nd<2, GRAD, PHASE64, MALA>(a, s, n_sm);
    case 3: return launch_mixed_nd<3, GRAD, PHASE64, MALA>(a, s, n_sm);
    default: return cudaErrorInvalidValue;
  }
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

RB_BOUNDS_READER(rb_bounds_read_loglike)
