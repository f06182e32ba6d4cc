"""Pins of the oracle's TaylorF2 phase coefficients and tidal combinations.

Each check compares the oracle with something it does not contain:

* the point-particle coefficients phi2..phi7 against a symbolic stationary-phase
  derivation from the PN binding energy E(v) and flux F(v) (Blanchet, Living Rev.
  Relativ. 2014, Eqs. 233 and 314): Psi(f) = 2 pi f t_c - 2 phi_c - pi/4 +
  (2/M) int_{v_f} (v_f^3 - u^3) E'(u)/F(u) du, re-expanded in v;
* Lambda-tilde / delta-Lambda-tilde (paper appendix) against the eta-polynomial
  forms of Wade et al. 2014 and the per-body 5PN/6PN forms;
* the spin-orbit part of phi3 against the same derivation with the leading
  spin-orbit terms of E(v) and F(v);
* the 2PN spin-spin sigma (and its weight -10 in phi4) against a derivation from
  the circular orbit with the spin-spin and spin-induced quadrupole couplings and
  the quadrupole plus current-quadrupole flux;
* the chirp time of the phase against the Newtonian time-to-coalescence.
"""
import math

import numpy as np
import pytest


def _theta(q, chi1=0.0, chi2=0.0, L1=0.0, L2=0.0, Mc=1.2):
    return np.array([Mc, q, chi1, chi2, L1, L2, 40.0, 0.0, 0.0, 0.3, 0.2, 1.0, 0.1])


@pytest.fixture(scope="module")
def energy_flux_coeffs():
    sp = pytest.importorskip("sympy")
    v, eta, lv = sp.symbols("v eta lv")
    pi, gE, R = sp.pi, sp.EulerGamma, sp.Rational
    # E(v) = -(1/2) M eta v^2 (1 + e2 v^2 + e4 v^4 + e6 v^6)
    e2 = -(R(3, 4) + eta / 12)
    e4 = -(R(27, 8) - R(19, 8) * eta + eta ** 2 / 24)
    e6 = -(R(675, 64) - (R(34445, 576) - R(205, 96) * pi ** 2) * eta + R(155, 96) * eta ** 2
           + R(35, 5184) * eta ** 3)
    # F(v) = (32/5) eta^2 v^10 (1 + f2 v^2 + ... + (f6 + f6l ln v) v^6 + f7 v^7)
    f2 = -R(1247, 336) - R(35, 12) * eta
    f3 = 4 * pi
    f4 = -R(44711, 9072) + R(9271, 504) * eta + R(65, 18) * eta ** 2
    f5 = -(R(8191, 672) + R(583, 24) * eta) * pi
    f6 = (R(6643739519, 69854400) + R(16, 3) * pi ** 2 - R(1712, 105) * gE - R(856, 105) * sp.log(16)
          + (-R(134543, 7776) + R(41, 48) * pi ** 2) * eta - R(94403, 3024) * eta ** 2 - R(775, 324) * eta ** 3)
    f6l = -R(1712, 105)
    f7 = (-R(16285, 504) + R(214745, 1728) * eta + R(193385, 3024) * eta ** 2) * pi
    # E'(v)/F(v) = -(5 M / (32 eta)) v^-9 * a(v)
    num = 1 + 2 * e2 * v ** 2 + 3 * e4 * v ** 4 + 4 * e6 * v ** 6
    den = 1 + f2 * v ** 2 + f3 * v ** 3 + f4 * v ** 4 + f5 * v ** 5 + (f6 + f6l * lv) * v ** 6 + f7 * v ** 7
    ser = sp.series(num / den, v, 0, 8).removeO()
    a = [sp.expand(ser.coeff(v, j)) for j in range(8)]
    # Term by term: int (v^3 - u^3) u^(j-9) du gives phi_j = 40 a_j / ((j-5)(j-8)) in the
    # 3/(128 eta v^5) normalisation; j = 5 gives a log (phi5 = phi5p (1 + 3 ln(v/v_lso)),
    # whose ln v coefficient 3 phi5p = -(40/3) a5); j = 6 carries ln v from the flux.
    a6c, a6l = a[6].coeff(lv, 0), a[6].coeff(lv, 1)
    out = {
        "phi0": 40 * a[0] / 40,
        "phi1": a[1],
        "phi2": 40 * a[2] / 18,
        "phi3": 4 * a[3],
        "phi4": 10 * a[4],
        "phi5p": -R(40, 9) * a[5],
        "phi6_lnv": -20 * a6l,
        # oracle: phi6 = phi6c - (6848/21) ln(4 v)  ->  non-log part phi6c - (6848/21) ln 4
        "phi6c": -20 * a6c + 10 * a6l + R(6848, 21) * sp.log(4),
        "phi7": -20 * a[7],
    }
    return eta, out


def test_point_particle_coefficients_match_energy_flux_derivation(oracle_mod, energy_flux_coeffs):
    eta_sym, coeff = energy_flux_coeffs
    assert coeff["phi0"] == 1 and coeff["phi1"] == 0
    # the flux's ln v term must give exactly the -(6848/21) ln(4v) 3PN log of the oracle
    assert float(coeff["phi6_lnv"]) == pytest.approx(-6848.0 / 21.0, rel=1e-15)
    for q in (1.0, 0.93, 0.6, 0.3, 0.125):
        o = oracle_mod.intrinsic(_theta(q))
        for name in ("phi2", "phi3", "phi4", "phi5p", "phi6c", "phi7"):
            expect = float(coeff[name].subs(eta_sym, o["eta"]))
            assert o[name] == pytest.approx(expect, rel=1e-13, abs=1e-12), (q, name)


def test_mass_parametrisation(oracle_mod):
    for Mc, q in ((1.1745, 0.93), (1.44, 0.125), (2.0, 1.0)):
        o = oracle_mod.intrinsic(_theta(q, Mc=Mc))
        m1, m2 = o["m1"], o["m2"]
        assert (m1 * m2) ** 0.6 / (m1 + m2) ** 0.2 == pytest.approx(Mc, rel=1e-14)
        assert m2 / m1 == pytest.approx(q, rel=1e-14)
        assert o["eta"] == pytest.approx(m1 * m2 / (m1 + m2) ** 2, rel=1e-14)
        assert o["eta"] <= 0.25


def test_lambda_tilde_matches_wade_eta_polynomials(oracle_mod):
    """Paper appendix definitions == Wade et al. 2014 Eqs. 5-6 (independent forms)."""
    for q, L1, L2 in ((1.0, 300.0, 300.0), (0.93, 300.0, 400.0), (0.6, 1200.0, 150.0), (0.125, 4000.0, 10.0)):
        o = oracle_mod.intrinsic(_theta(q, L1=L1, L2=L2))
        e = o["eta"]
        s = math.sqrt(1.0 - 4.0 * e)
        lt = 8.0 / 13.0 * ((1 + 7 * e - 31 * e ** 2) * (L1 + L2) + s * (1 + 9 * e - 11 * e ** 2) * (L1 - L2))
        dlt = 0.5 * (s * (1 - 13272.0 / 1319 * e + 8944.0 / 1319 * e ** 2) * (L1 + L2)
                     + (1 - 15910.0 / 1319 * e + 32850.0 / 1319 * e ** 2 + 3380.0 / 1319 * e ** 3) * (L1 - L2))
        assert o["Lt"] == pytest.approx(lt, rel=1e-12)
        assert o["dLt"] == pytest.approx(dlt, rel=1e-9, abs=1e-9 * (L1 + L2))


def test_lambda_tilde_equal_mass_limit(oracle_mod):
    o = oracle_mod.intrinsic(_theta(1.0, L1=700.0, L2=700.0))
    assert o["Lt"] == pytest.approx(700.0, rel=1e-14)
    assert abs(o["dLt"]) < 1e-12
    # swapping the deformabilities at equal mass flips delta-Lambda-tilde only
    a = oracle_mod.intrinsic(_theta(1.0, L1=200.0, L2=900.0))
    b = oracle_mod.intrinsic(_theta(1.0, L1=900.0, L2=200.0))
    assert a["Lt"] == pytest.approx(b["Lt"], rel=1e-14)
    assert a["dLt"] == pytest.approx(-b["dLt"], rel=1e-13)


def test_tidal_phase_per_body_identity(oracle_mod):
    """5PN/6PN tidal coefficients in the Lambda-tilde form == the per-body forms
    phi10 = sum_i (-288 + 264 X_i) X_i^4 Lambda_i and
    phi12 = sum_i X_i^4 Lambda_i (-15895/28 + 4595 X_i/28 + 5715 X_i^2/14 - 325 X_i^3/7)."""
    for q, L1, L2 in ((1.0, 300.0, 400.0), (0.8, 50.0, 3000.0), (0.45, 2000.0, 20.0), (0.125, 5000.0, 0.0)):
        o = oracle_mod.intrinsic(_theta(q, L1=L1, L2=L2))
        body = ((o["X1"], L1), (o["X2"], L2))
        p10 = sum((-288 + 264 * X) * X ** 4 * L for X, L in body)
        p12 = sum(X ** 4 * L * (-15895 / 28 + 4595 * X / 28 + 5715 * X ** 2 / 14 - 325 * X ** 3 / 7) for X, L in body)
        assert o["phi10"] == pytest.approx(p10, rel=1e-12)
        assert o["phi12"] == pytest.approx(p12, rel=1e-12)


def test_spin_orbit_term_matches_energy_flux_derivation(oracle_mod):
    """The 1.5PN spin-orbit part of phi3 (= 4 beta) from the leading spin-orbit terms
    of the binding energy and the flux for aligned spins (Kidder 1995; Blanchet,
    Living Rev. Relativ. 2014, spin-orbit section), in units M = 1:
    E gains v^3 [(14/3) S + 2 delta Sigma] and F gains v^3 [-4 S - (5/4) delta Sigma],
    with S = X1^2 chi1 + X2^2 chi2, Sigma = X2 chi2 - X1 chi1, delta = X1 - X2.
    The same stationary-phase step as the point-particle pin gives phi3 = 4 a3."""
    sp = pytest.importorskip("sympy")
    v, X1, c1, c2 = sp.symbols("v X1 c1 c2")
    pi, R = sp.pi, sp.Rational
    X2 = 1 - X1
    eta = X1 * X2
    S, Sig, dl = X1 ** 2 * c1 + X2 ** 2 * c2, X2 * c2 - X1 * c1, X1 - X2
    e2 = -(R(3, 4) + eta / 12)
    e3 = R(14, 3) * S + 2 * dl * Sig
    f2 = -R(1247, 336) - R(35, 12) * eta
    f3 = 4 * pi - 4 * S - R(5, 4) * dl * Sig
    # d/dv [v^2 (1 + e_k v^k)] / (2 v) = 1 + (k + 2)/2 e_k v^k
    num = 1 + 2 * e2 * v ** 2 + R(5, 2) * e3 * v ** 3
    den = 1 + f2 * v ** 2 + f3 * v ** 3
    a3 = sp.expand(sp.series(num / den, v, 0, 4).removeO().coeff(v, 3))
    phi3 = sp.lambdify((X1, c1, c2), 4 * a3)
    for q, x1, x2 in ((1.0, 0.03, -0.01), (0.8, 0.05, 0.05), (0.6, -0.04, 0.02), (0.3, 0.5, -0.7), (0.125, 0.9, 0.2)):
        o = oracle_mod.intrinsic(_theta(q, chi1=x1, chi2=x2))
        assert o["phi3"] == pytest.approx(phi3(1.0 / (1.0 + q), x1, x2), rel=1e-13, abs=1e-12), q


@pytest.fixture(scope="module")
def spin_spin_sigma():
    """The 2PN aligned-spin phase term sigma, derived here from the dynamics and the
    radiation of a circular orbit (units G = c = M = 1, so mu = eta = X1 X2), with
    spins S_i = X_i^2 chi_i normal to the orbital plane:

    * orbit: the Newtonian potential plus the leading spin-spin (dipole-dipole)
      coupling [3 (n.S1)(n.S2) - S1.S2] / r^3 (Barker & O'Connell 1975; Kidder 1995)
      and each body's spin-induced quadrupole Q_i = -kappa_i S_i^2 / m_i (Poisson
      1998), seen in its equatorial plane, -kappa_i m_j S_i^2 / (2 m_i r^3);
      a circular orbit has mu w^2 r = dU/dr and E = mu w^2 r^2 / 2 + U;
    * flux: the quadrupole formula (32/5) mu^2 r^4 w^6 on that orbit, plus the
      current quadrupole (16/45) <J'''_ij J'''_ij>, whose spin part is
      (3/2) sum_i [x_i^i S_i^j]^STF (Kidder 1995); for aligned spins both parts of J
      are multiples of [n^i z^j]^STF, whose square averages to 1/2;
    * both as series in v = (M w)^{1/3}; the spin-quadratic v^4 coefficients e4 of
      E / (-mu v^2 / 2) and f4 of F / ((32/5) eta^2 v^10) then enter the same
      stationary-phase step as the point-particle pin, a4 = 3 e4 - f4, and
      phi4 picks up 10 a4 = -10 sigma.

    Returns sigma(X1, chi1, chi2, kappa1, kappa2), and the current-quadrupole part
    of the 1PN flux coefficient as a check of the J normalisation."""
    sp = pytest.importorskip("sympy")
    v, a, X1, c1, c2, k1, k2 = sp.symbols("v a X1 c1 c2 k1 k2")
    r = sp.symbols("r", positive=True)
    X2 = 1 - X1
    mu = X1 * X2
    S1, S2 = X1 ** 2 * c1, X2 ** 2 * c2
    U = (-X1 * X2 / r - S1 * S2 / r ** 3
         - k1 * X2 * S1 ** 2 / (2 * X1 * r ** 3) - k2 * X1 * S2 ** 2 / (2 * X2 * r ** 3))
    w2 = sp.diff(U, r) / (mu * r)
    E = mu * w2 * r ** 2 / 2 + U
    # invert v^6 = w^2(r) for x = 1/r = v^2 (1 + a v^4 + ...)
    resid = sp.expand(sp.series(w2.subs(r, 1 / (v ** 2 * (1 + a * v ** 4))), v, 0, 12).removeO() - v ** 6)
    a_sol = sp.solve(resid.coeff(v, 10), a)[0]
    r_v = 1 / (v ** 2 * (1 + a_sol * v ** 4))
    e_ser = sp.expand(sp.series(E.subs(r, r_v) / (-mu * v ** 2 / 2), v, 0, 6).removeO())
    w = v ** 3
    F_I = sp.Rational(32, 5) * mu ** 2 * r_v ** 4 * w ** 6
    CJ = -mu * (X1 - X2) * r_v ** 3 * w + sp.Rational(3, 2) * r_v * (X2 * S1 - X1 * S2)
    F_J = sp.Rational(16, 45) * sp.Rational(1, 2) * w ** 6 * CJ ** 2
    f_ser = sp.expand(sp.series((F_I + F_J) / (sp.Rational(32, 5) * mu ** 2 * v ** 10), v, 0, 6).removeO())
    e4, f4 = e_ser.coeff(v, 4), f_ser.coeff(v, 4)
    sigma = sp.expand(sp.cancel(sp.together(f4 - 3 * e4)))
    # no spin-independent or spin-linear piece may leak into the 2PN spin-spin term
    assert sp.expand(sigma.subs({c1: 0, c2: 0})) == 0
    return (sp.lambdify((X1, c1, c2, k1, k2), sigma), sp.simplify(f_ser.coeff(v, 2) - (1 - 4 * mu) / 36))


def test_spin_spin_term_matches_orbit_and_flux_derivation(oracle_mod, spin_spin_sigma):
    """The oracle's 2PN spin-spin sigma (kappa_i = 1), and its weight -10 in phi4, equal
    the derivation of the spin_spin_sigma fixture.  Swapping the two S1 S2 coefficients
    (721/48, 247/48) or changing a self-spin factor ((720 kappa - 1), (240 kappa - 7))
    moves sigma by 2 eta chi1 chi2 or more, far outside these tolerances."""
    sigma, j_check = spin_spin_sigma
    # the current-quadrupole normalisation reproduces its known share (1 - 4 eta)/36 of
    # the 1PN flux coefficient -1247/336 - 35 eta/12 (Blanchet, Living Rev. Relativ. 2014)
    assert j_check == 0
    for q, x1, x2 in ((1.0, 0.6, -0.4), (0.8, 0.05, 0.05), (0.6, -0.9, 0.3), (0.3, 0.5, 0.8), (0.125, 0.9, -0.7)):
        o = oracle_mod.intrinsic(_theta(q, chi1=x1, chi2=x2))
        z = oracle_mod.intrinsic(_theta(q))
        expect = sigma(1.0 / (1.0 + q), x1, x2, 1.0, 1.0)
        assert o["sigma"] == pytest.approx(expect, rel=1e-13, abs=1e-15), q
        assert o["phi4"] - z["phi4"] == pytest.approx(-10.0 * expect, rel=1e-10), q


def test_spin_terms_limits(oracle_mod):
    o = oracle_mod.intrinsic(_theta(0.7))
    assert o["beta"] == 0.0 and o["sigma"] == 0.0
    # exchange symmetry at equal mass; linear (beta) and quadratic (sigma) scaling in the spins
    a = oracle_mod.intrinsic(_theta(1.0, chi1=0.03, chi2=-0.01))
    b = oracle_mod.intrinsic(_theta(1.0, chi1=-0.01, chi2=0.03))
    assert a["beta"] == pytest.approx(b["beta"], rel=1e-14)
    assert a["sigma"] == pytest.approx(b["sigma"], rel=1e-14)
    c = oracle_mod.intrinsic(_theta(0.6, chi1=0.02, chi2=0.04))
    d = oracle_mod.intrinsic(_theta(0.6, chi1=0.04, chi2=0.08))
    assert d["beta"] == pytest.approx(2 * c["beta"], rel=1e-13)
    assert d["sigma"] == pytest.approx(4 * c["sigma"], rel=1e-13)
    # phi3 and phi4 carry the spin terms with weights +4 and -10
    z = oracle_mod.intrinsic(_theta(0.6))
    assert c["phi3"] - z["phi3"] == pytest.approx(4 * c["beta"], rel=1e-9)
    assert c["phi4"] - z["phi4"] == pytest.approx(-10 * c["sigma"], rel=1e-6)


def test_phase_time_frequency_relation_is_newtonian_chirp(oracle_mod):
    """Psi'(f) / (2 pi) = t_c - tau(f); tau -> (5/256) Mc^{-5/3} (pi f)^{-8/3} at low f."""
    msun_s = 4.925490947641267e-6
    th = _theta(0.93, L1=300.0, L2=400.0, Mc=1.1745)
    th[7] = 0.05  # t_c
    for f0 in (20.0, 30.0, 50.0):
        h = f0 * 1e-6
        psi = oracle_mod.tf2_phase(th, np.array([f0 - h, f0 + h]))
        t_of_f = (psi[1] - psi[0]) / (2 * h) / (2 * math.pi)
        tau_n = 5.0 / 256.0 * (th[0] * msun_s) ** (-5.0 / 3.0) * (math.pi * f0) ** (-8.0 / 3.0)
        tau = th[7] - t_of_f
        assert tau > 0
        # PN corrections to the Newtonian chirp time are a few percent in this band
        assert tau / tau_n == pytest.approx(1.0, abs=0.08), f0
