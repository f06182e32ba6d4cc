"""The mixed kernel's phase sums (split_acc in rb_internal.cuh and the
per-walker rounding constant of k_rb_mixed), emulated step by step on the CPU.

A walker's phase at an edge is sum_k dc_k g_k(f_e) + tau_d f_e (turns), every
factor a float pair.  The kernel picks, per walker, a power of two q = 2^-20
of a power of two above every term, and m = 1.5 * 2^23 q.  For each term one
FMA against m rounds the high product a_hi b_hi to a multiple h of q, the h
add exactly into H, and the remainder a_hi b_hi - h and the cross terms
a_hi b_lo + a_lo b_hi go to the low sum L.  The emulation follows the same
FP32 operations, each correctly rounded (exact rationals, then rounding to
nearest even on 24 bits), and checks that

* every h is a multiple of q and every addition into H is exact;
* H + L is the exact sum of the float-pair products to within 2^-32 of the
  terms' bound, far below the FP32 rounding of the reduced phase that follows
  (2^-25 turns at |y| = 1/2);
* the rounding constant built from the bound's exponent bits is 1.5 * 2^23 q.
"""
import struct
from fractions import Fraction

import numpy as np


def _f32(x: Fraction) -> Fraction:
    """x rounded to the nearest FP32 value (ties to even; normal range)."""
    if x == 0:
        return Fraction(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (23 - e)  # a * scale in [2^23, 2^24)
    m = a * scale
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return s * Fraction(n) / scale


def _bits(x: float) -> int:
    return struct.unpack("<I", struct.pack("<f", x))[0]


def _from_bits(u: int) -> float:
    return struct.unpack("<f", struct.pack("<I", u))[0]


def _split_acc(a_hi, a_lo, b_hi, b_lo, m, H, L):
    """One step of split_acc, every operation rounded to FP32 as on the device."""
    h = _f32(_f32(a_hi * b_hi + m) - m)
    H_new = _f32(H + h)
    exact_H = H_new == H + h
    L = _f32(L + _f32(a_hi * b_hi - h))
    L = _f32(a_hi * b_lo + L)
    L = _f32(a_lo * b_hi + L)
    return h, H_new, L, exact_H


def _rounding_constant(mag: float) -> float:
    ex = min(max((_bits(mag) >> 23) & 0xFF, 64), 250)
    return _from_bits(((ex + 4) << 23) | 0x400000)


def _pair(v):
    hi = np.float32(v)
    lo = np.float32(v - float(hi))
    return Fraction(float(hi)), Fraction(float(lo))


def test_rounding_constant():
    for mag in (0.0, 1e-30, 3.7e-5, 0.49, 1.0, 1.5, 700.0, 2047.9, 1.9e5):
        m = _rounding_constant(np.float32(mag))
        ex = (_bits(np.float32(mag)) >> 23) & 0xFF
        ex = min(max(ex, 64), 250)
        q = 2.0 ** (ex - 146)
        assert m == 1.5 * 2 ** 23 * q
        assert np.float32(mag) < 2.0 ** (ex - 126)  # the bound the kernel assumes


def test_split_acc_exact_high_sum_and_error():
    rng = np.random.default_rng(2404)
    worst = 0.0
    for trial in range(300):
        # eleven terms (ten basis terms and a delay) with magnitudes spread over
        # up to 40 binades below the largest, which ranges from 1e-6 to 4e3 turns
        top = 10.0 ** rng.uniform(-6, 3.6)
        if trial % 4 == 0:  # all eleven near the bound, one sign: the largest |H|
            mags = top * rng.uniform(0.9, 1.0, size=11)
            sgn = np.ones(11)
        else:
            mags = top * 2.0 ** -rng.uniform(0, 40, size=11)
            mags[rng.integers(11)] = top
            sgn = rng.choice([-1, 1], size=11)
        a = rng.uniform(0.5, 2.0, size=11)
        b = mags / a * sgn
        pairs = [(_pair(x), _pair(y)) for x, y in zip(a, b)]
        bound = max(abs(float(ah) * float(bh)) for (ah, _), (bh, _) in pairs) * 1.01
        m = Fraction(_rounding_constant(np.float32(bound)))
        q = m / (Fraction(3, 2) * 2 ** 23)
        H = L = Fraction(0)
        exact = Fraction(0)
        for (ah, al), (bh, bl) in pairs:
            h, H, L, ok = _split_acc(ah, al, bh, bl, m, H, L)
            assert ok, (trial, float(H), float(h))
            assert (h / q).denominator == 1
            exact += (ah + al) * (bh + bl)
        U = 2.0 ** (((_bits(np.float32(bound)) >> 23) & 0xFF) - 126)
        err = abs(float(H + L - exact))
        worst = max(worst, err / U)
        assert err <= 2.0 ** -32 * U, (trial, err, U)
    assert worst > 0.0


def test_split_acc_zero_walker():
    # the fiducial point: every phase offset is zero, the sums are exactly zero
    m = Fraction(_rounding_constant(np.float32(0.0)))
    H = L = Fraction(0)
    for _ in range(11):
        _, H, L, ok = _split_acc(Fraction(0), Fraction(0), Fraction(0.123), Fraction(1e-9), m, H, L)
        assert ok
    assert H == 0 and L == 0
