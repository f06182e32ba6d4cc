"""Pin of the oracle's amplitude normalisation and Fourier sign conventions.

A Newtonian quadrupole chirp h+ = a(t) (1 + cos^2 i)/2 cos Phi(t),
hx = a(t) cos i sin Phi(t), a = (4/D) Mc^{5/3} (pi f)^{2/3}, is built in the time
domain from the Newtonian frequency evolution, Fourier transformed with
h~(f) = int h(t) exp(-2 pi i f t) dt, and compared with the oracle's
polarisations: |h~+| = A f^{-7/6} (1 + cos^2 i)/2 with A = sqrt(5/24) pi^{-2/3}
Mc^{5/6} / D, h~x / h~+ = -i 2 cos i / (1 + cos^2 i), and the phase slope
d arg h~ / df = -2 pi t(f) (the e^{-i Psi} convention).  None of these numbers
come from the oracle's own formulas.
"""
import math

import numpy as np
import pytest

MSUN_S = 4.925490947641267e-6
MPC_S = 3.085677581491367e22 / 299792458.0


def _ramp(x):
    x = np.clip(x, 0.0, 1.0)
    return 0.5 - 0.5 * np.cos(np.pi * x)


def test_newtonian_chirp_fft_matches_oracle_polarisations(oracle_mod):
    mc_sun, dl_mpc, iota = 5.0, 100.0, 0.5
    mc, dist = mc_sun * MSUN_S, dl_mpc * MPC_S
    fs, tw, t_merge = 8192.0, 16.0, 12.0
    n = int(fs * tw)
    t = np.arange(n) / fs
    tau = t_merge - t
    f_lo, f_hi = 25.0, 600.0
    tau_lo = 5 / 256 * mc ** (-5 / 3) * (np.pi * f_lo) ** (-8 / 3)
    tau_hi = 5 / 256 * mc ** (-5 / 3) * (np.pi * f_hi) ** (-8 / 3)
    ok = (tau <= tau_lo) & (tau >= tau_hi)
    tt = np.where(ok, tau, 1.0)
    f = (1 / np.pi) * (5 / (256 * tt)) ** (3 / 8) * mc ** (-5 / 8)
    phi = -2 * (tt / (5 * mc)) ** (5 / 8)
    a = 4 / dist * mc ** (5 / 3) * (np.pi * f) ** (2 / 3)
    w = _ramp((f - f_lo) / 10.0) * _ramp((f_hi - f) / 100.0) * ok
    ci = math.cos(iota)
    hp = np.fft.rfft(w * a * (1 + ci * ci) / 2 * np.cos(phi)) / fs
    hc = np.fft.rfft(w * a * ci * np.sin(phi)) / fs
    fr = np.fft.rfftfreq(n, 1 / fs)
    sel = (fr > 60) & (fr < 300)
    theta = np.array([mc_sun, 1.0, 0, 0, 0, 0, dl_mpc, t_merge, 0.0, iota, 0, 0, 0])
    op, oc = oracle_mod.polarizations(theta, fr[sel])
    # amplitude normalisation (band-averaged: Fresnel ripples from the finite chirp average out)
    assert np.mean(np.abs(hp[sel]) / np.abs(op)) == pytest.approx(1.0, abs=0.02)
    assert np.mean(np.abs(hc[sel]) / np.abs(oc)) == pytest.approx(1.0, abs=0.02)
    # cross vs plus: relative phase -i in both
    rel = (hc[sel] / hp[sel]) / (oc / op)
    assert abs(np.mean(np.angle(rel))) < 0.02
    # e^{-i Psi}: same sign and size of the phase slope (PN terms change it by < 5 % here)
    slope_fft = np.diff(np.unwrap(np.angle(hp[sel])))
    slope_orc = np.diff(np.unwrap(np.angle(op)))
    assert np.median(slope_orc / slope_fft) == pytest.approx(1.0, abs=0.05)
