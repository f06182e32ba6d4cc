"""The FP64 reciprocal of the stored-waveform summary build (rcp_newton in
rb_summary.cu), emulated step by step on the CPU.

The device routine seeds 1/S with an FP32 reciprocal of S scaled to [1, 2),
built from and moved back to FP64 bits with integer operations.  It then takes
two Newton-Raphson steps r <- r + r (1 - S r) with fused multiply-adds.  Each
step doubles the correct bits (~23 -> ~46 -> beyond FP64).  The emulation
follows the same integer and floating-point operations (fma exact via rationals,
the FP32 reciprocal correctly rounded as the device's rcp.rn.f32); the result
must be within 1 ulp of 1/S over the PSD's range and at the edge cases."""
import math
from fractions import Fraction

import numpy as np


def _fma(a: float, b: float, c: float) -> float:
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _rcp_newton(S: float):
    bits = int(np.float64(S).view(np.uint64))
    hi, lo = bits >> 32, bits & 0xFFFFFFFF
    ef = (hi >> 20) & 0x7FF
    if ef == 0 or ef >= 0x7FC or S <= 0:  # the device routine divides there
        return 1.0 / S, 1.0 / S
    s1 = np.uint32(0x3F800000 | ((hi & 0xFFFFF) << 3) | (lo >> 29)).view(np.float32)  # S 2^-e, truncated
    rb = int(np.float32(np.float32(1.0) / s1).view(np.uint32))  # correctly rounded FP32 reciprocal
    er = ((rb >> 23) & 0xFF) - 127
    m = rb & 0x7FFFFF
    dhi = ((er + 1023 - (ef - 1023)) << 20) | (m >> 3)
    r = float(np.uint64((dhi << 32) | ((m & 7) << 29)).view(np.float64))
    r0 = r
    for _ in range(2):
        r = _fma(r, _fma(-S, r, 1.0), r)
    return r0, r


def test_newton_reciprocal_within_one_ulp():
    rng = np.random.default_rng(3)
    values = list(10.0 ** rng.uniform(-49, -38, 2000))  # one-sided PSD values of the synthetic curves
    values += list(10.0 ** rng.uniform(-300, 300, 500))
    values += [1.0, 1.5, 2.0, 3.0, 0.75, float(np.nextafter(2.0, 0.0)), float(np.nextafter(1.0, 2.0)), 1e-300, 1e300,
               2.0 ** -1022, 2.0 ** 1020, float(np.nextafter(2.0 ** 1021, 0.0)), 2.0 ** 1021, 1.7e308]
    worst_seed = worst = 0.0
    for S in values:
        r0, r = _rcp_newton(float(S))
        exact = Fraction(1) / Fraction(float(S))
        worst_seed = max(worst_seed, float(abs(Fraction(r0) - exact) / exact))
        worst = max(worst, float(abs(Fraction(r) - exact)) / math.ulp(float(exact)))
    assert worst_seed < 2.0 ** -22  # the seed: ~23 correct bits
    assert worst <= 1.0
