"""MALA local step on the GPU (rb_mala_init / rb_mala_step, fused with the
likelihood and its adjoint) against the oracle's MALA step on the same
seeded draws (Sec. II.D; sampling coordinates and uniform priors of
Table II).

The proposals are plain FP64 arithmetic on both sides; log pi and its
gradient carry the likelihood tolerances of the batch tests; an accept
decision must agree wherever the oracle's margin |log u - log alpha|
exceeds that tolerance, and near ties must be valid (the chain either stays
or moves to its own proposal)."""
import math

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


def _box_z(prior):
    lo, hi = np.zeros(13), np.zeros(13)
    for j, name in enumerate(synth.PARAM_NAMES):
        spec = prior[name]
        lo[j], hi[j] = (-1.0, 1.0) if spec in ("cos", "sin") else spec
    return lo, hi


def _theta_to_z(th):
    z = np.array(th, dtype=np.float64)
    z[:, 9] = np.cos(z[:, 9])
    z[:, 12] = np.sin(z[:, 12])
    return z


@pytest.fixture(scope="module")
def setup(rb):
    ev = inject(synth.make_event("C2", T=16.0))
    B = 120
    event = rb.Event.from_synth(ev, n_bins=B)
    s = oracle.summary(ev, ev["theta_inj"], oracle.bin_edges(ev, B))
    lo, hi = _box_z(synth.PRIOR_GW170817)
    # the injection (Mc = 1.1744 from m1 = 1.40, m2 = 1.30) lies below the
    # GW170817 chirp-mass range: widen it so the chains start inside
    lo[0] = 1.16
    W = 700
    z0 = _theta_to_z(synth.posterior_box(ev["theta_inj"], W, seed=31))
    # step sizes from the curvature at the injection: eps_j = 0.5 / sqrt(F_jj),
    # F_jj = -d^2 log pi / dz_j^2 by central differences of the oracle gradient
    zi = _theta_to_z(np.array(ev["theta_inj"])[None])[0]
    eps = np.zeros(13)
    for j in range(13):
        h = 1e-7 * max(abs(zi[j]), 1e-2)
        zpl, zmi = zi.copy(), zi.copy()
        zpl[j] += h
        zmi[j] -= h
        gpl = oracle.mala_logpost(ev, s, zpl[None], lo, hi)[1][0, j]
        gmi = oracle.mala_logpost(ev, s, zmi[None], lo, hi)[1][0, j]
        F = max(-(gpl - gmi) / (2 * h), 1e-12)
        eps[j] = min(0.5 / np.sqrt(F), 0.05 * (hi[j] - lo[j]))
    z0[5, 9] = hi[9] - 1e-9  # at the cos iota bound
    rng = np.random.default_rng(2024)
    xi = rng.standard_normal((W, 13))
    xi[7, 0] = 1e6  # this chain's proposal leaves the box
    u = rng.uniform(size=W)
    yield dict(ev=ev, s=s, event=event, lo=lo, hi=hi, z0=z0, eps=eps, xi=xi, u=u)
    event.free()


def _tol(mode, lp):
    if mode == "fp64":
        return 1e-9 * np.abs(lp) + 1e-7
    return np.maximum(1e-3, 2e-6 * np.abs(lp) * 4)


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_f64phase"])
def test_mala_init_matches_oracle(rb, setup, mode):
    S = setup
    z = torch.tensor(S["z0"], device="cuda")
    lp, gz = rb.mala_init(S["event"], z, S["lo"], S["hi"], mode=mode)
    lp, gz = lp.cpu().numpy(), gz.cpu().numpy()
    lpo, gzo = oracle.mala_logpost(S["ev"], S["s"], S["z0"], S["lo"], S["hi"])
    assert np.all(np.isfinite(lpo))
    assert np.all(np.abs(lp - lpo) <= _tol(mode, lpo))
    # components near the likelihood peak are near-cancellations of large terms:
    # floor each component's scale at 1e-2 of its largest magnitude over the chains
    scale = np.maximum(np.abs(gzo), 1e-2 * np.max(np.abs(gzo), axis=0, keepdims=True))
    rel = 1e-8 if mode == "fp64" else 1e-4
    r = np.abs(gz - gzo) / (rel * scale)
    i, j = np.unravel_index(np.argmax(r), r.shape)
    assert r[i, j] <= 1.0, (i, j, gz[i, j], gzo[i, j], S["z0"][i, j])


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed_f64phase"])
def test_mala_step_matches_oracle(rb, setup, mode):
    S = setup
    lpo, gzo = oracle.mala_logpost(S["ev"], S["s"], S["z0"], S["lo"], S["hi"])
    # the same starting state on both sides (the oracle's log pi and gradient)
    z = torch.tensor(S["z0"], device="cuda")
    lp = torch.tensor(lpo, device="cuda")
    gz = torch.tensor(gzo, device="cuda")
    xi = torch.tensor(S["xi"], device="cuda")
    u = torch.tensor(S["u"], device="cuda")
    acc = rb.mala_step(S["event"], z, lp, gz, S["eps"], S["lo"], S["hi"], xi, u, mode=mode).cpu().numpy().astype(bool)
    z, lp, gz = z.cpu().numpy(), lp.cpu().numpy(), gz.cpu().numpy()
    zo, lpo2, gzo2, acco, la = oracle.mala_step(S["ev"], S["s"], S["z0"], lpo, gzo, S["eps"], S["xi"], S["u"],
                                                 S["lo"], S["hi"])
    zp, inside = oracle.mala_propose(S["z0"], gzo, S["eps"], S["xi"], S["lo"], S["hi"])
    assert not inside.all() and inside.any()
    assert not np.any(acc & ~inside)  # outside the box: never accepted
    margin = np.abs(np.log(S["u"]) - la)
    decided = margin > 2 * _tol(mode, lpo)
    assert decided.mean() > 0.8
    np.testing.assert_array_equal(acc[decided], acco[decided])
    # every chain is either unchanged or at its proposal
    np.testing.assert_allclose(np.where(acc[:, None], zp, S["z0"]), z, rtol=1e-13, atol=0)
    assert 0.05 < acc.mean() < 0.999
    # accepted chains carry log pi and gradient of the proposal
    both = acc & acco
    assert np.all(np.abs(lp[both] - lpo2[both]) <= _tol(mode, lpo2[both]))
    sc = np.maximum(np.abs(gzo2[both]), 1e-2 * np.max(np.abs(gzo2[both]), axis=0, keepdims=True))
    assert np.all(np.abs(gz[both] - gzo2[both]) <= (1e-8 if mode == "fp64" else 1e-4) * sc)
    # rejected chains keep theirs
    stay = ~acc
    np.testing.assert_array_equal(lp[stay], lpo[stay])
    np.testing.assert_array_equal(gz[stay], gzo[stay])


def test_mala_chain_runs(rb, setup):
    """Repeated steps in the mixed path: finite log pi, states inside the
    box, a useful acceptance rate, and log pi consistent with a fresh
    evaluation of the final states."""
    S = setup
    z = torch.tensor(S["z0"], device="cuda")
    lp, gz = rb.mala_init(S["event"], z, S["lo"], S["hi"], mode="mixed")
    g = torch.Generator(device="cuda").manual_seed(7)
    rates = []
    for _ in range(25):
        xi = torch.randn(z.shape, dtype=torch.float64, device="cuda", generator=g)
        u = torch.rand(z.shape[0], dtype=torch.float64, device="cuda", generator=g)
        rates.append(rb.mala_step(S["event"], z, lp, gz, S["eps"], S["lo"], S["hi"], xi, u).float().mean().item())
    zc = z.cpu().numpy()
    assert np.all((zc > S["lo"]) & (zc < S["hi"]))
    assert np.all(np.isfinite(lp.cpu().numpy()))
    assert 0.2 < np.mean(rates) < 0.999
    lp2, _ = rb.mala_init(S["event"], z, S["lo"], S["hi"], mode="mixed")
    np.testing.assert_allclose(lp.cpu().numpy(), lp2.cpu().numpy(), rtol=0, atol=1e-9)
    lpo, _ = oracle.mala_logpost(S["ev"], S["s"], zc, S["lo"], S["hi"])
    assert np.all(np.abs(lp.cpu().numpy() - lpo) <= _tol("mixed", lpo))
