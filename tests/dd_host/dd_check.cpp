// Host build of the float-float header (rb_dd.cuh) for a CPU accuracy check:
// prints the largest error of each routine over seeded inputs, measured
// against long double arithmetic and the C library.
#include <cmath>
#include <cstdio>
#include <random>

#include "rb_dd.cuh"

using namespace rb::ffx;

static long double val(dd a) { return (long double)a.h + (long double)a.l; }

int main() {
  std::mt19937_64 g(20240417);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  double e_add = 0, e_mul = 0, e_div = 0, e_sqrt = 0, e_cbrt = 0, e_r5 = 0, e_log = 0, e_sin = 0, e_cos = 0;
  for (int i = 0; i < 100000; ++i) {
    const double x = std::exp(std::log(1e-8) + U(g) * (std::log(1e8) - std::log(1e-8)));
    const double y = (U(g) - 0.5) * 30.0;
    const dd X = from_double(x), Y = from_double(y);
    const long double xr = val(X), yr = val(Y);
    e_add = std::fmax(e_add, (double)(fabsl(val(add(X, Y)) - (xr + yr)) / (fabsl(xr) + fabsl(yr))));
    e_mul = std::fmax(e_mul, (double)fabsl(val(mul(X, Y)) / (xr * yr) - 1));
    e_div = std::fmax(e_div, (double)fabsl(val(div(X, Y)) / (xr / yr) - 1));
    e_sqrt = std::fmax(e_sqrt, (double)fabsl(val(sqrt(X)) / sqrtl(xr) - 1));
    e_cbrt = std::fmax(e_cbrt, (double)fabsl(val(cbrt(X)) / cbrtl(xr) - 1));
    e_r5 = std::fmax(e_r5, (double)fabsl(val(rroot5(X)) / powl(xr, -0.2L) - 1));
    e_log = std::fmax(e_log, (double)(fabsl(val(log(X)) - logl(xr)) / fmaxl(1.0L, fabsl(logl(xr)))));
    dd s, c;
    sincos(Y, &s, &c);
    e_sin = std::fmax(e_sin, (double)fabsl(val(s) - sinl(yr)));
    e_cos = std::fmax(e_cos, (double)fabsl(val(c) - cosl(yr)));
  }
  std::printf("add %.3e\nmul %.3e\ndiv %.3e\nsqrt %.3e\ncbrt %.3e\nrroot5 %.3e\nlog %.3e\nsin %.3e\ncos %.3e\n", e_add, e_mul,
              e_div, e_sqrt, e_cbrt, e_r5, e_log, e_sin, e_cos);
  return 0;
}
