"""Pins of the oracle's full and relative-binning likelihoods, summary data,
bin placement and gradient.

* exactness at the reference point (r = 1, r1 = 0): RB == full to 1e-10 relative;
* brute force: one grid point per bin (B = N - 1) makes the linear model exact,
  so RB with the B2 term == full likelihood;
* <h|h> proportional to 1/d_L^2 and <d|h> to 1/d_L;
* Eq. 2: log L = -<d-h|d-h>/2 + <d|d>/2 computed from independent inner products;
* bin count <-> epsilon pairs of Sec. IV.B (tests/golden/paper_bins_epsilon.json);
* forward-mode gradient == Richardson-extrapolated central differences.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import synth
from tests._events import event, inject, small_event

GOLD = Path(__file__).resolve().parent / "golden"


@pytest.fixture(scope="module")
def c1(oracle_mod):
    ev = event("C1")
    edges = oracle_mod.bin_edges(ev, ev["n_bins"])
    return ev, oracle_mod.summary(ev, ev["theta_inj"], edges)


@pytest.fixture(scope="module")
def net(oracle_mod):
    ev = small_event()
    edges = oracle_mod.bin_edges(ev, 60)
    return ev, oracle_mod.summary(ev, ev["theta_inj"], edges)


def test_rb_exact_at_reference(oracle_mod, c1, net):
    for ev, s in (c1, net):
        full = oracle_mod.loglike_full(ev, ev["theta_inj"])[0]
        rb = oracle_mod.loglike_rb(ev, s, ev["theta_inj"])[0]
        assert abs(rb - full) <= 1e-10 * abs(full)


def test_rb_one_point_per_bin_equals_full(oracle_mod):
    ev = inject(synth.make_event("C2", T=1.0, f_low=30.0, f_high=94.0))
    assert ev["N"] == 65
    B = ev["N"] - 1
    edges = oracle_mod.bin_edges(ev, B)
    np.testing.assert_array_equal(edges, np.arange(ev["N"]))
    s = oracle_mod.summary(ev, ev["theta_inj"], edges, with_b2=True)
    th = synth.draw_box(ev["theta_inj"], 16, seed=11, rel=0.05, abs_width=0.05 * synth.PRIOR_WIDTH)
    full = oracle_mod.loglike_full(ev, th)
    rb = oracle_mod.loglike_rb(ev, s, th, with_b2=True)
    np.testing.assert_allclose(rb, full, rtol=1e-11, atol=1e-11 * np.max(np.abs(full)))
    # without B2 the difference is exactly the dropped -(1/2) sum B2 |r1|^2 >= 0 term
    rb_std = oracle_mod.loglike_rb(ev, s, th)
    assert np.all(rb_std >= full - 1e-9 * np.abs(full))


def test_distance_scaling(oracle_mod, net):
    ev, _ = net
    quiet = dict(ev)
    quiet["data"] = np.zeros_like(ev["data"])  # log L = -<h|h>/2
    th = np.array(ev["theta_inj"])
    th2 = th.copy()
    th2[6] *= 2.0
    hh1 = -2 * oracle_mod.loglike_full(quiet, th)[0]
    hh2 = -2 * oracle_mod.loglike_full(quiet, th2)[0]
    assert hh1 / hh2 == pytest.approx(4.0, rel=1e-12)
    noisy = dict(ev)
    noisy["data"] = ev["noise"]
    dh1 = oracle_mod.loglike_full(noisy, th)[0] + 0.5 * hh1
    dh2 = oracle_mod.loglike_full(noisy, th2)[0] + 0.5 * hh2
    assert dh1 / dh2 == pytest.approx(2.0, rel=1e-10)


def test_likelihood_is_minus_half_residual_norm(oracle_mod, net):
    ev, _ = net
    th = synth.draw_box(ev["theta_inj"], 3, seed=12, rel=0.002, abs_width=1e-3 * synth.PRIOR_WIDTH)
    full = oracle_mod.loglike_full(ev, th)
    for w in range(3):
        res, dd = 0.0, 0.0
        for d in range(ev["geom"].shape[0]):
            h = oracle_mod.strain(th[w], ev["geom"][d], ev["gmst"], ev["f"])
            r = ev["data"][d] - h
            res += oracle_mod.inner(r, r, ev["psd"][d], ev["T"])
            dd += oracle_mod.inner(ev["data"][d], ev["data"][d], ev["psd"][d], ev["T"])
        assert full[w] == pytest.approx(-0.5 * res + 0.5 * dd, rel=1e-9, abs=1e-8 * dd)


def test_unphysical_walkers(oracle_mod, net):
    ev, s = net
    th = np.tile(ev["theta_inj"], (5, 1))
    th[0, 1] = 1.2      # q > 1
    th[1, 1] = 0.0      # q = 0
    th[2, 6] = -1.0     # d_L < 0
    th[3, 9] = np.nan   # NaN
    L, g = oracle_mod.loglike_rb(ev, s, th, grad=True)
    assert np.all(np.isneginf(L[:4])) and np.isfinite(L[4])
    assert np.all(g[:4] == 0.0)
    assert np.all(np.isneginf(oracle_mod.loglike_full(ev, th)[:4]))


def test_bin_count_matches_paper_epsilon(oracle_mod):
    g = json.loads((GOLD / "paper_bins_epsilon.json").read_text())
    span = oracle_mod.dpsi_max(g["f_high"], g["f_low"], g["f_high"]) - oracle_mod.dpsi_max(g["f_low"], g["f_low"],
                                                                                        g["f_high"])
    assert span == pytest.approx(31.06, abs=0.01)
    for pair in g["pairs"]:
        implied = span / pair["epsilon"]
        assert implied == pytest.approx(pair["n_bins"], rel=0.05)


def test_bin_edges_structure(oracle_mod):
    ev = synth.make_event("C2", T=16.0)
    for B in (1, 7, 100, 500):
        e = oracle_mod.bin_edges(ev, B)
        assert e[0] == 0 and e[-1] == ev["N"] - 1
        assert np.all(np.diff(e) >= 1)
    # equal spacing in the phase bound, to grid resolution
    e = oracle_mod.bin_edges(ev, 40)
    p = np.array([oracle_mod.dpsi_max(ev["f"][k], ev["f_low"], ev["f_high"]) for k in e])
    step = (p[-1] - p[0]) / 40
    dp = np.array([oracle_mod.dpsi_max(ev["f"][k + 1], ev["f_low"], ev["f_high"]) -
                   oracle_mod.dpsi_max(ev["f"][k], ev["f_low"], ev["f_high"]) for k in e[:-1]])
    assert np.all(np.abs(np.diff(p) - step) <= dp + 1e-12)
    with pytest.raises(ValueError):
        oracle_mod.bin_edges(ev, ev["N"])


def test_rb_accurate_near_reference(oracle_mod, c1):
    ev, s = c1
    th = synth.posterior_box(ev["theta_inj"], 32, seed=13)
    full = oracle_mod.loglike_full(ev, th)
    rb = oracle_mod.loglike_rb(ev, s, th)
    assert np.max(np.abs(rb - full)) < 0.1


def test_gradient_matches_finite_differences(oracle_mod, net):
    ev, s = net
    th = synth.draw_box(ev["theta_inj"], 3, seed=14, rel=0.003, abs_width=3e-3 * synth.PRIOR_WIDTH)
    L, g = oracle_mod.loglike_rb(ev, s, th, grad=True)
    for w in range(th.shape[0]):
        fd = np.zeros(13)
        for j in range(13):
            h = 1e-6 * max(abs(th[w, j]), synth.PRIOR_WIDTH[j])

            def cd(step):
                tp, tm = th[w].copy(), th[w].copy()
                tp[j] += step
                tm[j] -= step
                return (oracle_mod.loglike_rb(ev, s, tp)[0] - oracle_mod.loglike_rb(ev, s, tm)[0]) / (2 * step)
            fd[j] = (4 * cd(h / 2) - cd(h)) / 3  # Richardson: O(h^4)
        scale = np.maximum(np.abs(g[w]), 1e-2 * np.max(np.abs(g[w])))
        assert np.all(np.abs(fd - g[w]) <= 1e-6 * scale), (w, (fd - g[w]) / scale)
