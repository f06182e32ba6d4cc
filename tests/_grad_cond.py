"""Conditioning of the relative-binning gradient, from the oracle (test helper).

The gradient of the binned likelihood is a sum over detectors d and bin edges e of
per-edge terms t_{d,e,j} = Re(conj(gbar_{d,e}) dr_{d,e}/dtheta_j), where r is the
ratio h(f_e; theta) / h(f_e; theta_ref) of Eq. 4 and gbar its cotangent, i.e. the
derivative of the Eq. 5 contraction with respect to Re r + i Im r.  Evaluated with
per-term relative rounding u, such a sum carries an error of order u K_j with

    K_j = sum_{d,e} |t_{d,e,j}|,

whatever order it is summed in.  For walkers far from the posterior the ratio
oscillates across the band and |g_j| can be 1e3-1e4 times smaller than K_j, so
u32 K_j (u32 = 2^-24) is the floor of any evaluation whose per-edge values are
FP32.  Everything here is FP64 on the CPU: the ratio from the oracle's strain,
its parameter derivatives by central differences (relative accuracy ~1e-8, ample
for a bound), and gbar from the oracle's summary data.
"""
from __future__ import annotations

import numpy as np

import oracle
import synth


def ratio_at_edges(ev, theta, fe):
    D = ev["geom"].shape[0]
    h0 = [oracle.strain(ev["theta_inj"], ev["geom"][d], ev["gmst"], fe) for d in range(D)]
    return np.stack([oracle.strain(theta, ev["geom"][d], ev["gmst"], fe) / h0[d] for d in range(D)])


def cotangent(s, r, fe):
    """gbar = dL/dRe r + i dL/dIm r at the edges, for L = sum_b Re(A0 r0* + A1 r1*)
    - B0 |r0|^2 / 2 - B1 Re(r0 r1*) with r0 the edge mean and r1 the edge slope."""
    A0, A1, B0, B1 = (np.asarray(s[k]) for k in ("A0", "A1", "B0", "B1"))
    df = fe[1:] - fe[:-1]
    r0 = 0.5 * (r[:, :-1] + r[:, 1:])
    r1 = (r[:, 1:] - r[:, :-1]) / df
    G0 = A0 - B0 * r0 - B1 * r1   # dL_b / d r0
    G1 = A1 - B1 * r0             # dL_b / d r1
    g = np.zeros_like(r)
    g[:, :-1] += 0.5 * G0 - G1 / df
    g[:, 1:] += 0.5 * G0 + G1 / df
    return g


def gradient_terms_abs(ev, s, edges, theta):
    """K [W][13]: the sum over detectors and edges of |t_{d,e,j}| per walker."""
    fe = ev["f"][np.asarray(edges)]
    th = np.atleast_2d(np.asarray(theta, dtype=np.float64))
    K = np.zeros_like(th)
    for w in range(th.shape[0]):
        r = ratio_at_edges(ev, th[w], fe)
        gbar = cotangent(s, r, fe)
        for j in range(th.shape[1]):
            h = 1e-6 * max(abs(th[w, j]), synth.PRIOR_WIDTH[j])
            tp, tm = th[w].copy(), th[w].copy()
            tp[j] += h
            tm[j] -= h
            if j == 1 and tp[1] > 1.0:  # q <= 1: one-sided at the edge of the box
                tp[1], tm[1] = th[w, 1], th[w, 1] - 2 * h
            dr = (ratio_at_edges(ev, tp, fe) - ratio_at_edges(ev, tm, fe)) / (tp[j] - tm[j])
            K[w, j] = np.sum(np.abs((np.conj(gbar) * dr).real))
    return K
