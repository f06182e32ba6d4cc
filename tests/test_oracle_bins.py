"""Pins of the oracle's bin placement without the PN ansatz (the outlook of the
paper's Sec. V asks for bins built without prior assumptions on the waveform).

The reading: each of the model's phase directions w_j(f) = dPsi(f; theta_ref)/dtheta_j
(Mc, q, chi1, chi2, Lambda1, Lambda2, t_c) is given 2 pi of total variation across
the band, and the edges are uniform in M(f) = 2 pi sum_j V_j(f) / V_j(f_high).
Each check compares the oracle with something it does not contain:

* the measure of power-law directions against its closed form;
* with the PN power laws of the ansatz as the directions, the paper's
  epsilon <-> bin-count pairs of Sec. IV.B (tests/golden/paper_bins_epsilon.json);
* the phase directions against central differences of the oracle's phase, and the
  t_c direction against 2 pi f exactly;
* invariances of the measure (scale and sign of a direction, duplicated directions);
* the edges against the targets they are placed at.
"""
import json
from pathlib import Path

import numpy as np
import pytest

import synth

GOLD = Path(__file__).resolve().parent / "golden"
PN_GAMMAS = (-5.0 / 3.0, -2.0 / 3.0, 1.0, 5.0 / 3.0, 7.0 / 3.0)


def test_measure_of_power_laws_matches_closed_form(oracle_mod):
    """Monotone directions f^gamma have total variation |f^gamma - f_low^gamma| on [f_low, f]."""
    ev = synth.make_event("C2", T=16.0)
    f = ev["f"]
    W = np.stack([f ** g for g in PN_GAMMAS])
    M = oracle_mod.direction_measure(W)
    closed = 2 * np.pi * sum(np.abs(f ** g - f[0] ** g) / abs(f[-1] ** g - f[0] ** g) for g in PN_GAMMAS)
    np.testing.assert_allclose(M, closed, rtol=1e-12, atol=1e-12)
    assert M[0] == 0.0 and M[-1] == pytest.approx(2 * np.pi * len(PN_GAMMAS), rel=1e-14)


def test_pn_power_law_directions_reproduce_paper_epsilon(oracle_mod):
    """With the ansatz's power laws as the directions the measure spans 5 x 2 pi over
    [20, 2048] Hz; bin counts M(f_high)/epsilon at the paper's epsilons land within 5 %
    of its bin counts (200 at 0.15, 1000 at 0.03), as the ansatz's own 31.06 rad does."""
    g = json.loads((GOLD / "paper_bins_epsilon.json").read_text())
    ev = synth.make_event("C2", T=8.0, f_low=g["f_low"], f_high=g["f_high"])
    f = ev["f"]
    M = oracle_mod.direction_measure(np.stack([f ** gm for gm in PN_GAMMAS]))
    for pair in g["pairs"]:
        assert M[-1] / pair["epsilon"] == pytest.approx(pair["n_bins"], rel=0.05)
    # the shape follows the ansatz bound to within its per-term normalisation (<= 5 %)
    P = np.array([oracle_mod.dpsi_max(x, g["f_low"], g["f_high"]) for x in f])
    P -= P[0]
    assert np.max(np.abs(M / M[-1] - P / P[-1])) < 0.02


def test_measure_invariances(oracle_mod):
    ev = synth.make_event("C1", T=8.0)
    W = oracle_mod.phase_directions(ev, ev["theta_inj"])
    M = oracle_mod.direction_measure(W)
    scaled = W * np.array([3.0, -0.5, 1e4, -2.0, 7.0, 1e-3, -1.0])[:, None]
    np.testing.assert_allclose(oracle_mod.direction_measure(scaled), M, rtol=1e-12)
    # a repeated direction counts twice; a constant direction (no variation) not at all
    M2 = oracle_mod.direction_measure(np.vstack([W, W[:1], np.full((1, W.shape[1]), 5.0)]))
    M1 = oracle_mod.direction_measure(W[:1])
    np.testing.assert_allclose(M2, M + M1, rtol=1e-12, atol=1e-12)
    assert np.all(np.diff(M) >= 0.0)


def test_phase_directions_match_central_differences(oracle_mod):
    th = synth.THETA_INJ.copy()
    f = np.array([20.0, 57.3, 200.0, 800.0, 2048.0])
    ev = synth.make_event("C2", T=0.5)
    W = np.zeros((7, f.size))
    for i, fi in enumerate(f):  # one-point grids at f
        W[:, i] = oracle_mod.phase_directions(dict(ev, T=1.0 / fi, kmin=1, N=1), th)[:, 0]
    params = (0, 1, 2, 3, 4, 5, 7)
    for j, p in enumerate(params):
        h = 1e-5 * max(abs(th[p]), synth.PRIOR_WIDTH[p])

        def cd(step):
            tp, tm = th.copy(), th.copy()
            tp[p] += step
            tm[p] -= step
            return (oracle_mod.tf2_phase(tp, f) - oracle_mod.tf2_phase(tm, f)) / (2 * step)
        fd = (4 * cd(h / 2) - cd(h)) / 3
        # the differences carry the phase's rounding (|Psi| ~ 1e4 rad at 20 Hz) divided by the step
        noise = 1e-14 * np.max(np.abs(oracle_mod.tf2_phase(th, f))) / h
        np.testing.assert_allclose(W[j], fd, rtol=1e-6, atol=noise), p
    np.testing.assert_array_equal(W[6], 2 * np.pi * f)  # t_c enters as 2 pi f t_c


def test_agnostic_edges_sit_at_their_targets(oracle_mod):
    ev = synth.make_event("C2", T=16.0)
    th = ev["theta_inj"]
    M = oracle_mod.direction_measure(oracle_mod.phase_directions(ev, th))
    for B in (1, 7, 100, 500):
        e, eps = oracle_mod.bin_edges_agnostic(ev, B)
        assert e[0] == 0 and e[-1] == ev["N"] - 1 and np.all(np.diff(e) >= 1)
        assert eps == pytest.approx(M[-1] / B, rel=1e-14)
        if B == 500:
            continue  # some bins are narrower than a grid step at the top of the band: clamped
        # each inner edge is the grid point nearest (in M) to its target e M(f_high) / B
        tgt = M[-1] * np.arange(1, B) / B
        k = e[1:-1]
        assert np.all(np.abs(M[k] - tgt) <= 0.5 * np.maximum(M[np.minimum(k + 1, ev["N"] - 1)] - M[k],
                                                                M[k] - M[np.maximum(k - 1, 0)]) + 1e-12)


def test_agnostic_epsilon_scale(oracle_mod):
    """Seven directions carry 7 x 2 pi = 14 pi across any band (all vary here)."""
    for cfg in ("C1", "C2", "C4"):
        ev = synth.make_event(cfg)
        _, eps = oracle_mod.bin_edges_agnostic(ev, ev["n_bins"])
        assert eps * ev["n_bins"] == pytest.approx(14 * np.pi, rel=1e-12), cfg
