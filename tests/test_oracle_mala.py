"""Pins of the oracle's MALA local step (Sec. II.D, the local sampler of
flowMC; the Metropolis-adjusted Langevin algorithm) in the sampling
coordinates of Table II (cos iota, sin dec; uniform prior on the box):

* MALA leaves its target invariant: chains started from a 13-dimensional
  correlated Gaussian keep its mean and covariance after many steps with a
  step size at which the unadjusted Langevin update visibly inflates them;
* as eps -> 0 the acceptance ratio tends to 1 (log alpha = O(eps^3));
* the chain rule to (cos iota, sin dec) matches central differences of the
  likelihood in z, and z -> theta inverts cos and sin.
"""
import numpy as np
import pytest

import oracle
from tests._events import small_event

NP = 13
BIG = 1e9


def _gauss_target(rng):
    # a random SPD precision matrix with variances spread over two decades
    A = rng.normal(size=(NP, NP)) / np.sqrt(NP)
    C = A @ A.T + np.diag(np.geomspace(0.05, 5.0, NP))
    P = np.linalg.inv(C)
    return C, P


def test_mala_leaves_gaussian_invariant(oracle_mod):
    rng = np.random.default_rng(11)
    C, P = _gauss_target(rng)
    L = np.linalg.cholesky(C)
    W, steps = 4000, 60
    eps = 0.9 * np.sqrt(np.diag(C))  # large steps: the Metropolis correction matters
    lo, hi = np.full(NP, -BIG), np.full(NP, BIG)
    logp = lambda z: -0.5 * np.einsum("wi,ij,wj->w", z, P, z)
    grad = lambda z: -z @ P
    z = rng.normal(size=(W, NP)) @ L.T  # start in the target
    zu = z.copy()                       # unadjusted Langevin from the same start, for contrast
    lp, g = logp(z), grad(z)
    acc_rate = []
    for _ in range(steps):
        xi = rng.normal(size=(W, NP))
        u = rng.uniform(size=W)
        zp, inside = oracle.mala_propose(z, g, eps, xi, lo, hi)
        assert inside.all()
        lpp, gp = logp(zp), grad(zp)
        la = oracle.mala_log_alpha(lp, lpp, g, gp, eps, xi)
        acc = np.log(u) < la
        z[acc], lp[acc], g[acc] = zp[acc], lpp[acc], gp[acc]
        acc_rate.append(acc.mean())
        zu, _ = oracle.mala_propose(zu, grad(zu), eps, rng.normal(size=(W, NP)), lo, hi)
    assert 0.2 < np.mean(acc_rate) < 0.95
    var, var_u = z.var(axis=0), zu.var(axis=0)
    # MALA keeps the variances (statistical error ~ sqrt(2/W) ~ 2.2 %)
    assert np.all(np.abs(var / np.diag(C) - 1) < 0.12), var / np.diag(C)
    assert np.all(np.abs(z.mean(axis=0)) < 6 * np.sqrt(np.diag(C) / W))
    cov = np.cov(z.T)
    assert np.max(np.abs(cov - C)) < 0.15 * np.max(np.diag(C))
    # the unadjusted chain does not (its stationary law differs at this step size)
    assert np.max(np.abs(var_u / np.diag(C) - 1)) > 0.3


def test_log_alpha_small_steps(oracle_mod):
    rng = np.random.default_rng(12)
    C, P = _gauss_target(rng)
    W = 200
    z = rng.normal(size=(W, NP))
    for scale, bound in [(1e-2, 5e-4), (1e-3, 5e-7), (1e-4, 5e-10)]:
        eps = scale * np.sqrt(np.diag(C))
        xi = rng.normal(size=(W, NP))
        zp, _ = oracle.mala_propose(z, -z @ P, eps, xi, np.full(NP, -BIG), np.full(NP, BIG))
        la = oracle.mala_log_alpha(-0.5 * np.einsum("wi,ij,wj->w", z, P, z),
                                   -0.5 * np.einsum("wi,ij,wj->w", zp, P, zp), -z @ P, -zp @ P, eps, xi)
        assert np.max(np.abs(la)) < bound  # O(eps^3)


def test_coordinates_and_chain_rule(oracle_mod):
    ev = small_event()
    s = oracle.summary(ev, ev["theta_inj"], oracle.bin_edges(ev, 20))
    th0 = np.array(ev["theta_inj"], dtype=float)
    z0 = th0.copy()
    z0[9], z0[12] = np.cos(th0[9]), np.sin(th0[12])
    np.testing.assert_allclose(oracle.z_to_theta(z0)[0], th0, rtol=0, atol=1e-12)
    lo = np.full(NP, -BIG)
    hi = np.full(NP, BIG)
    lo[9] = lo[12] = -1.0
    hi[9] = hi[12] = 1.0
    lp, gz = oracle.mala_logpost(ev, s, z0[None], lo, hi)
    for j in (6, 9, 12):  # d_L (unchanged coordinate), cos iota, sin dec
        h = 1e-6 * max(abs(z0[j]), 1e-2)
        zpl, zmi = z0.copy(), z0.copy()
        zpl[j] += h
        zmi[j] -= h
        fd = (oracle.mala_logpost(ev, s, zpl[None], lo, hi)[0][0] - oracle.mala_logpost(ev, s, zmi[None], lo, hi)[0][0]) / (2 * h)
        assert abs(fd - gz[0, j]) <= 1e-5 * max(1.0, abs(gz[0, j])), (j, fd, gz[0, j])
    # outside the box: -inf
    zo = z0.copy()
    zo[9] = 1.5
    assert oracle.mala_logpost(ev, s, zo[None], lo, hi)[0][0] == -np.inf
