"""Checks of the seeded input generators (no method arithmetic involved)."""
import numpy as np
import pytest

import synth


def test_grid_inclusive_both_ends():
    kmin, N, f = synth.grid(128.0, 20.0, 2048.0)
    assert kmin == 2560 and N == 259585
    assert f[0] == 20.0 and f[-1] == 2048.0
    assert synth.grid(64.0, 20.0, 1024.0)[1] == 64257
    assert synth.grid(256.0, 20.0, 2048.0)[1] == 519169


def test_noise_normalisation():
    """Re, Im ~ N(0, S/(4 df)) gives E<n|n> = 2N with <a|b> = 4 df Re sum a b*/S."""
    T = 16.0
    _, N, f = synth.grid(T, 20.0, 2048.0)
    psd = synth.psd_aligo(f)
    n = synth.noise(psd, T, seed=3)
    nn = 4.0 / T * np.sum(np.abs(n) ** 2 / psd)
    # <n|n> = sum of 2N unit-variance chi^2 terms: mean 2N, sd 2 sqrt(N)
    assert abs(nn - 2 * N) < 5 * 2 * np.sqrt(N)


def test_generators_are_seeded_and_stable():
    a = synth.uniforms(7, 1000)
    b = synth.uniforms(7, 1000)
    np.testing.assert_array_equal(a, b)
    assert np.all((a > 0) & (a < 1))
    z = synth.normals(9, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_prior_draws_inside_table_boxes():
    w = synth.draw_prior(synth.PRIOR_GW170817, 4096, seed=2)
    for j, name in enumerate(synth.PARAM_NAMES):
        spec = synth.PRIOR_GW170817[name]
        if spec == "cos":
            assert np.all((w[:, j] >= 0) & (w[:, j] <= np.pi))
        elif spec == "sin":
            assert np.all(np.abs(w[:, j]) <= np.pi / 2)
        else:
            assert np.all((w[:, j] >= spec[0]) & (w[:, j] <= spec[1]))


def test_psd_positive_in_band():
    f = np.linspace(10, 4096, 1000)
    assert np.all(synth.psd_aligo(f) > 0)
    # minimum of the zero-detuned high-power curve sits near 200-300 Hz, ~(4e-24)^2
    fm = f[np.argmin(synth.psd_aligo(f))]
    assert 150 < fm < 350
    assert 1e-48 < synth.psd_aligo(np.array([fm]))[0] < 1e-46
