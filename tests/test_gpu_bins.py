"""Bin placement without the PN ansatz (RB_BINS_AGNOSTIC) on the GPU vs the oracle.

* Edges: integer results, compared exactly.  Both sides evaluate the placement
  measure in FP64 along different routes (the oracle differences its phase
  derivatives at neighbouring grid points, the library forms each increment
  directly), so an edge whose target lies within FP64 noise of the midpoint
  between two grid points may legitimately go either way: such a near-tie
  (|frac - 1/2| < 1e-6 in the oracle's own measure) is the only difference allowed.
* epsilon: the measure's range over the band / B, to 1e-10.
* The likelihood on an event with agnostic bins: the parity tolerances of
  test_gpu_parity.py (the bins change the summary data, not the arithmetic).
* Accuracy of the placement: against the full likelihood at the same bin count,
  agnostic bins are no worse than the PN-ansatz bins on posterior-scale walkers.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from tests._events import inject

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2404_11397_gb300 as m
    m.load()
    return m


def _near_ties(ev, edges_gpu, edges_ref, B):
    """Indices where the two placements differ, each checked to be a near-tie."""
    diff = np.flatnonzero(edges_gpu != edges_ref)
    if diff.size == 0:
        return diff
    M = oracle.direction_measure(oracle.phase_directions(ev, ev["theta_inj"]))
    for e in diff:
        tau = M[0] + (M[-1] - M[0]) * e / B
        k = min(max(int(np.searchsorted(M, tau, side="right")) - 1, 0), M.size - 2)
        frac = (tau - M[k]) / (M[k + 1] - M[k])
        assert abs(frac - 0.5) < 1e-6 and abs(int(edges_gpu[e]) - int(edges_ref[e])) == 1, (e, frac)
    return diff


@pytest.mark.parametrize("cfg,n_bins,kw", [("C1", None, {}), ("C2", None, {}), ("C4", None, {}),
                                           ("C2", 45, dict(T=8.0, f_high=512.0)), ("C2", 1, dict(T=4.0, f_high=256.0)),
                                           ("C2", 1000, dict(T=16.0))])
def test_agnostic_edges_match_oracle(rb, cfg, n_bins, kw):
    ev = inject(synth.make_event(cfg, **kw))
    B = n_bins or ev["n_bins"]
    event = rb.Event.from_synth(ev, n_bins=B, bins="agnostic")
    ref, eps = oracle.bin_edges_agnostic(ev, B)
    got = event.summary()["edges"]
    assert _near_ties(ev, got, ref, B).size <= 1
    inf = event.info()
    assert inf["bin_scheme"] == rb.RB_BINS_AGNOSTIC
    assert inf["epsilon"] == pytest.approx(eps, rel=1e-10)
    event.free()


def test_agnostic_edges_one_point_per_bin(rb):
    ev = inject(synth.make_event("C2", T=1.0, f_low=30.0, f_high=94.0))
    event = rb.Event.from_synth(ev, n_bins=ev["N"] - 1, bins="agnostic")
    np.testing.assert_array_equal(event.summary()["edges"], np.arange(ev["N"]))
    event.free()


def test_pn_epsilon_reported(rb):
    ev = inject(synth.make_event("C2"))
    event = rb.Event.from_synth(ev)
    span = oracle.dpsi_max(ev["f"][-1], ev["f_low"], ev["f_high"]) - oracle.dpsi_max(ev["f"][0], ev["f_low"],
                                                                                      ev["f_high"])
    inf = event.info()
    assert inf["bin_scheme"] == rb.RB_BINS_PN
    assert inf["epsilon"] == pytest.approx(span / ev["n_bins"], rel=1e-12)
    event.free()


@pytest.mark.parametrize("mode", ["mixed", "mixed_f64phase", "fp64"])
def test_likelihood_on_agnostic_bins_matches_oracle(rb, mode):
    ev = inject(synth.make_event("C2"))
    B = ev["n_bins"]
    event = rb.Event.from_synth(ev, bins="agnostic")
    edges = event.summary()["edges"]
    s = oracle.summary(ev, ev["theta_inj"], edges)
    th = synth.posterior_box(ev["theta_inj"], 256, seed=41)
    L = rb.loglike(event, torch.tensor(th, device="cuda"), mode=mode)
    ref_L = oracle.loglike_rb(ev, s, th)
    tol = 1e-9 * np.abs(ref_L) + 1e-8 if mode == "fp64" else 1e-3
    assert np.all(np.abs(L.cpu().numpy() - ref_L) <= tol), mode
    # gradients on the +-0.3 % box of the main parity test (at posterior scale the
    # gradient is near zero and its FP64 error relative to it is not bounded by 1e-8)
    th = synth.draw_box(ev["theta_inj"], 64, seed=51, rel=3e-3, abs_width=3e-3 * synth.PRIOR_WIDTH)
    _, G = rb.loglike_grad(event, torch.tensor(th, device="cuda"), mode=mode)
    _, ref_G = oracle.loglike_rb(ev, s, th, grad=True)
    rel = 1e-8 if mode == "fp64" else 1e-4
    gtol = rel * np.maximum(np.abs(ref_G), 1e-2 * np.max(np.abs(ref_G), axis=1, keepdims=True))
    assert np.all(np.abs(G.cpu().numpy() - ref_G) <= gtol), mode
    assert B == len(edges) - 1
    event.free()


def test_agnostic_bins_no_less_accurate_than_pn_at_equal_bin_count(rb):
    """RB vs the full likelihood (the library's full-grid sum) at B = 200 on C2:
    the largest error over posterior-scale walkers with agnostic bins is no larger
    than with the PN-ansatz bins (oracle study: 0.056 vs 0.10)."""
    ev = inject(synth.make_event("C2"))
    th = torch.tensor(synth.posterior_box(ev["theta_inj"], 256, seed=43), device="cuda")
    err = {}
    for bins in ("pn", "agnostic"):
        event = rb.Event.from_synth(ev, n_bins=200, bins=bins)
        L = rb.loglike(event, th, mode="fp64").cpu().numpy()
        full = rb.loglike_full(event, th).cpu().numpy()
        err[bins] = np.max(np.abs(L - full))
        event.free()
    assert err["agnostic"] <= err["pn"], err
