"""The mixed kernel's form of the detector prefactor's adjoint, checked on the
CPU in FP64 against a finite difference.

At an edge the ratio is r = rho E with E = exp(-2 pi i y), written as
r = 1 + delta, delta = rho (E - 1) + sigma and sigma = rho - 1.  For a log L
whose dependence on r is Re(sum_e conj(gbar_e) r_e) to first order (gbar the
edge cotangent), a change dln rho of ln rho changes log L by Re(G dln rho) with

    G = conj(gbar_rho) rho = sum_e conj(gbar_e) r_e,
    Re G = sum_e (gbar_r r_r + gbar_i r_i),  Im G = sum_e (gbar_r r_i - gbar_i r_r),

gbar_rho = sum_e gbar_e conj(E_e) the adjoint of rho itself.  The kernel sums
Re G and Im G (the latter is the sum of the edge's d log L / dy term that the
basis adjoint also takes); the FP64 paths sum gbar_rho and form G from rho.
"""
import numpy as np


def _edges(rng, n):
    y = rng.uniform(-0.5, 0.5, n)
    E = np.exp(-2j * np.pi * y)
    g = rng.normal(size=n) + 1j * rng.normal(size=n)
    return E, g


def test_kernel_sums_equal_adjoint_times_rho():
    rng = np.random.default_rng(2404)
    for _ in range(50):
        E, g = _edges(rng, 257)
        rho = complex(rng.uniform(0.2, 3.0) * np.exp(1j * rng.uniform(-np.pi, np.pi)))
        sigma = rho - 1.0
        delta = rho * (E - 1.0) + sigma
        r = 1.0 + delta
        # the kernel's sums
        re_G = np.sum(g.real * r.real + g.imag * r.imag)
        dldx = g.real * r.imag - g.imag * r.real
        im_G = np.sum(dldx)
        # the adjoint of rho, then conj(gbar_rho) rho
        gbar_rho = np.sum(g * np.conj(E))
        G = np.conj(gbar_rho) * rho
        assert abs(re_G - G.real) <= 1e-12 * np.sum(np.abs(g))
        assert abs(im_G - G.imag) <= 1e-12 * np.sum(np.abs(g))


def test_adjoint_form_matches_finite_difference():
    rng = np.random.default_rng(11397)
    for _ in range(20):
        E, g = _edges(rng, 101)
        rho = complex(rng.uniform(0.5, 2.0) * np.exp(1j * rng.uniform(-np.pi, np.pi)))

        def L(rh):
            return float(np.sum((np.conj(g) * (rh * E)).real))

        G = np.sum(np.conj(g) * (rho * E))
        for dln in (1.0, 1j, 0.3 - 0.7j):
            h = 1e-6
            fd = (L(rho * np.exp(h * dln)) - L(rho * np.exp(-h * dln))) / (2 * h)
            assert abs(fd - (G * dln).real) <= 1e-7 * max(1.0, abs(fd))
