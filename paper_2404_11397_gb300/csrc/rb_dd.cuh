// rb_dd.cuh -- float-float ("dd") arithmetic on the FP32 pipe for the
// per-walker set-up of the mixed-precision path.
//
// A value is an unevaluated sum h + l of two floats with |l| <= ulp(h) / 2,
// about 48 significant bits.  On sm_103a an FP64 instruction costs roughly 64
// times an FP32 one, so a dd operation of 10-25 FP32 instructions is several
// times cheaper than the FP64 operation it replaces, and its latency chain is
// shorter (FP32 dependent latency ~4 cycles against ~70).
//
// Error-free transformations: Knuth's two-sum, Dekker's fast two-sum and the
// FMA form of Dekker's two-product; dd add/multiply/divide/square root follow
// the classical double-double algorithms (Dekker 1971; Bailey's QD library
// description, Hida, Li & Bailey 2001) with float in place of double.
// Elementary functions, written for this code from their series:
//   log    atanh series  ln m = 2 s (1 + s^2/3 + s^4/5 + ...), s = (m-1)/(m+1),
//          after m = x 2^-e in [1/sqrt2, sqrt2)
//   sincos Taylor series about 0 after reduction by multiples of pi/2
//   x^(1/3), x^(-1/5), sqrt x   one Newton step in dd from the FP32 value
// Every rounding is explicit (__fadd_rn / __fmul_rn / __fmaf_rn on the
// device), so the compiler can neither contract nor reassociate them.  The
// header also compiles for the host (plain float operations, which round the
// same way when built without FP contraction) so the algorithms can be
// checked on the CPU.
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define RB_DD __host__ __device__ __forceinline__
#define RB_DD_CTOR __host__ __device__
// the longer routines are kept out of line: the set-up kernels run many
// warps on different code at once and are otherwise instruction-fetch bound
#define RB_DD_CALL __host__ __device__ __noinline__
#else
#define RB_DD inline
#define RB_DD_CTOR
#define RB_DD_CALL inline
#endif

namespace rb {
namespace ffx {

struct dd {
  float h, l;
};

RB_DD float add(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
RB_DD float mul(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
RB_DD float fma(float a, float b, float c) {
#if defined(__CUDA_ARCH__)
  return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
RB_DD float div(float a, float b) {
#if defined(__CUDA_ARCH__)
  return __fdiv_rn(a, b);
#else
  return a / b;
#endif
}
RB_DD float sqrt_rn(float a) {
#if defined(__CUDA_ARCH__)
  return __fsqrt_rn(a);
#else
  return std::sqrt(a);
#endif
}

// --- error-free transformations ---------------------------------------------
RB_DD dd two_sum(float a, float b) {
  const float s = add(a, b);
  const float bb = add(s, -a);
  const float e = add(add(a, -add(s, -bb)), add(b, -bb));
  return {s, e};
}
RB_DD dd fast_two_sum(float a, float b) {  // |a| >= |b| (or a == 0)
  const float s = add(a, b);
  return {s, add(b, -add(s, -a))};
}
RB_DD dd two_prod(float a, float b) {
  const float p = mul(a, b);
  return {p, fma(a, b, -p)};
}

// --- construction -------------------------------------------------------------
RB_DD dd from_float(float a) { return {a, 0.f}; }
// Exact split of a double into h + l (a double has 53 bits, a dd 48: the
// remainder below the 48th bit is rounded).
RB_DD dd from_double(double x) {
  const float h = (float)x;
  return {h, (float)(x - (double)h)};
}
RB_DD double to_double(dd a) { return (double)a.h + (double)a.l; }

// Compile-time split of a double constant.
struct cdd {
  float h, l;
  RB_DD_CTOR constexpr cdd(double x) : h((float)x), l((float)(x - (double)(float)x)) {}
};
RB_DD dd K(const cdd& c) { return {c.h, c.l}; }

// --- arithmetic ----------------------------------------------------------------
RB_DD dd neg(dd a) { return {-a.h, -a.l}; }

RB_DD dd add(dd a, dd b) {  // accurate (IEEE-style) dd addition
  dd s = two_sum(a.h, b.h);
  const dd t = two_sum(a.l, b.l);
  s.l = add(s.l, t.h);
  s = fast_two_sum(s.h, s.l);
  s.l = add(s.l, t.l);
  return fast_two_sum(s.h, s.l);
}
RB_DD dd sub(dd a, dd b) { return add(a, neg(b)); }
RB_DD dd add(dd a, float b) {
  dd s = two_sum(a.h, b);
  s.l = add(s.l, a.l);
  return fast_two_sum(s.h, s.l);
}
RB_DD dd mul(dd a, dd b) {
  dd p = two_prod(a.h, b.h);
  p.l = fma(a.h, b.l, p.l);
  p.l = fma(a.l, b.h, p.l);
  return fast_two_sum(p.h, p.l);
}
RB_DD dd mul(dd a, float b) {
  dd p = two_prod(a.h, b);
  p.l = fma(a.l, b, p.l);
  return fast_two_sum(p.h, p.l);
}
RB_DD dd sqr(dd a) {
  dd p = two_prod(a.h, a.h);
  p.l = fma(mul(2.f, a.h), a.l, p.l);
  return fast_two_sum(p.h, p.l);
}
// Approximate reciprocal (~1 ulp): the quotient digits below are corrected
// by exact remainders, so they need not be correctly rounded.
RB_DD float rcp_approx(float b) {
#if defined(__CUDA_ARCH__)
  return __fdividef(1.f, b);
#else
  return 1.f / b;
#endif
}
// a / b: quotient digit, exact remainder, second digit, one more correction.
RB_DD_CALL dd div(dd a, dd b) {
  const float rb = rcp_approx(b.h);
  const float q1 = mul(a.h, rb);
  dd r = sub(a, mul(b, q1));
  const float q2 = mul(r.h, rb);
  r = sub(r, mul(b, q2));
  const float q3 = mul(r.h, rb);
  return add(fast_two_sum(q1, q2), q3);
}
RB_DD dd div(float a, dd b) { return div(dd{a, 0.f}, b); }

// sqrt: FP32 root s, then s + (a - s^2) / (2 s).
RB_DD_CALL dd sqrt(dd a) {
  if (!(a.h > 0.f)) return {0.f, 0.f};
  const float s = sqrt_rn(a.h);
  const dd r = sub(a, two_prod(s, s));
  return fast_two_sum(s, mul(r.h, rcp_approx(mul(2.f, s))));
}

// x^(1/3) for x > 0: one Newton step y - (y^3 - x) / (3 y^2) from the FP32 root.
RB_DD_CALL dd cbrt(dd x) {
  const float y = std::cbrt(x.h);
  const dd y3 = mul(two_prod(y, y), y);
  const dd r = sub(y3, x);
  return fast_two_sum(y, -mul(r.h, rcp_approx(mul(3.f, mul(y, y)))));
}

// x^(-1/5) for x > 0: Newton on x y^5 = 1 from the FP32 value,
// y <- y + y (1 - x y^5) / 5.
RB_DD_CALL dd rroot5(dd x) {
  const float y = std::pow(x.h, -0.2f);
  const dd y2 = two_prod(y, y);
  const dd y5 = mul(sqr(y2), y);
  const dd r = sub(dd{1.f, 0.f}, mul(x, y5));
  return fast_two_sum(y, mul(y, mul(r.h, 0.2f)));
}

// Natural logarithm for x > 0.
RB_DD_CALL dd log(dd x) {
  constexpr cdd kLn2(0.69314718055994530942);
  int e;
  float m = std::frexp(x.h, &e);  // x.h = m 2^e, m in [1/2, 1)
  if (m < 0.70710678f) {
    m = mul(m, 2.f);
    --e;
  }
  // exact scaling of both parts by 2^-e
  const float sc = std::ldexp(1.f, -e);
  const dd xm{m, mul(x.l, sc)};
  const dd s = div(add(xm, -1.f), add(xm, 1.f));
  const dd z = sqr(s);
  // tail 1/7 + z/9 + ... + z^7/21 in FP32 (it is below 3e-5 z^3 of the sum)
  const float zf = z.h;
  float t = 1.f / 21.f;
  t = fma(t, zf, 1.f / 19.f);
  t = fma(t, zf, 1.f / 17.f);
  t = fma(t, zf, 1.f / 15.f);
  t = fma(t, zf, 1.f / 13.f);
  t = fma(t, zf, 1.f / 11.f);
  t = fma(t, zf, 1.f / 9.f);
  t = fma(t, zf, 1.f / 7.f);
  constexpr cdd c5(1.0 / 5.0), c3(1.0 / 3.0);
  dd p = add(mul(z, t), K(c5));
  p = add(mul(p, z), K(c3));
  p = add(mul(p, z), 1.f);
  const dd ln_m = mul(mul(s, p), 2.f);
  return add(mul(K(kLn2), (float)e), ln_m);
}

// sin and cos of x for |x| <= 2^13 (the angles of the set-up are within a
// few turns).  Reduction r = x - k pi/2 in dd with pi/2 to three floats
// (k pi/2 is formed without error in the leading parts), then the Taylor
// series of sin and cos for |r| <= pi/4: dd for the leading terms, FP32 for
// the tail (terms below z^4/9!).
RB_DD_CALL void sincos(dd x, dd* s, dd* c) {
  // pi/2 = P1 + P2 + P3: P1 has 8 bits (k P1 is exact), P2 is the next float,
  // P3 the remainder (k P2 is taken as an exact two-product)
  constexpr float kP1 = 1.5703125f;
  constexpr float kP2 = 4.838267923332751e-4f;
  constexpr cdd kP3(2.563344151594519e-12);
  // k = nearest integer to x 2/pi, rounded on the FMA pipe (|x| < 2^21)
  const float k = add(add(mul(x.h, 0.63661977236758134f), 12582912.0f), -12582912.0f);
  dd r = add(x, -mul(k, kP1));
  r = sub(r, two_prod(k, kP2));
  r = sub(r, mul(K(kP3), k));
  const dd z = sqr(r);
  const float zf = z.h;
  // sin r = r (1 - z/3! + z^2/5! - z^3/7! + z^4/9! - ...)
  float ts = 1.6059043836821613e-10f;       // 1/13!
  ts = fma(ts, zf, -2.5052108385441720e-08f);  // -1/11!
  ts = fma(ts, zf, 2.7557319223985893e-06f);   // 1/9!
  constexpr cdd s7(-1.0 / 5040.0), s5(1.0 / 120.0), s3(-1.0 / 6.0);
  dd ps = add(mul(z, ts), K(s7));
  ps = add(mul(ps, z), K(s5));
  ps = add(mul(ps, z), K(s3));
  const dd sr = add(mul(mul(ps, z), r), r);
  // cos r = 1 - z/2! + z^2/4! - z^3/6! + z^4/8! - ...
  float tc = -1.1470745597729725e-11f;        // -1/14!
  tc = fma(tc, zf, 2.0876756987868099e-09f);   // 1/12!
  tc = fma(tc, zf, -2.7557319223985891e-07f);  // -1/10!
  tc = fma(tc, zf, 2.4801587301587302e-05f);   // 1/8!
  constexpr cdd c6(-1.0 / 720.0), c4(1.0 / 24.0);
  dd pc = add(mul(z, tc), K(c6));
  pc = add(mul(pc, z), K(c4));
  pc = add(mul(pc, z), -0.5f);
  const dd cr = add(mul(pc, z), 1.f);
  const int q = ((int)k) & 3;
  const dd ss = (q & 1) ? cr : sr, cc = (q & 1) ? sr : cr;
  *s = (q & 2) ? neg(ss) : ss;
  *c = (q == 1 || q == 2) ? neg(cc) : cc;
}

}  // namespace ffx
}  // namespace rb
