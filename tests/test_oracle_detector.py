"""Pins of the oracle's detector projection (antenna patterns, delays, site vertices).

* WGS-84 vertex positions against the published LIGO/Virgo site constants
  (tests/golden/detector_vertices.json);
* the textbook response of an interferometer with arms along x and y to a
  source at polar angle theta, azimuth phi:
  F+^2 + Fx^2 = (1 + cos^2 theta)^2 cos^2(2 phi) / 4 + cos^2 theta sin^2(2 phi);
* the overhead special case F+ = -cos 2(psi + g), Fx = sin 2(psi + g), g = GMST - ra
  (worked by hand from the polarisation vectors);
* invariance of F+^2 + Fx^2 under psi and the sign flip under psi -> psi + pi/2;
* geometric delays: -|r|/c for a source along the vertex direction and the
  H1-L1 light travel time (~10.0 ms).
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

GOLD = Path(__file__).resolve().parent / "golden"
C = 299792458.0


def _dms(d, m, s):
    sign = -1.0 if d < 0 else 1.0
    return sign * (abs(d) + m / 60.0 + s / 3600.0)


def _site_geom(entry, xaz=0.0, yaz=math.pi / 2):
    lat = math.radians(_dms(*entry["lat_dms"]))
    lon = math.radians(_dms(*entry["lon_dms"]))
    return np.array([lat, lon, entry["elev_m"], xaz, yaz])


def test_vertex_matches_published_site_positions(oracle_mod):
    sites = json.loads((GOLD / "detector_vertices.json").read_text())["sites"]
    for name, entry in sites.items():
        _, r = oracle_mod.detector_tensor(_site_geom(entry))
        assert np.linalg.norm(r - np.array(entry["vertex_m"])) < 0.01, name


def test_h1_l1_light_travel_time(oracle_mod):
    sites = json.loads((GOLD / "detector_vertices.json").read_text())["sites"]
    _, rh = oracle_mod.detector_tensor(_site_geom(sites["LHO"]))
    _, rl = oracle_mod.detector_tensor(_site_geom(sites["LLO"]))
    assert np.linalg.norm(rh - rl) / C == pytest.approx(10.01e-3, abs=0.05e-3)


def _polar_detector():
    # vertex at the north pole, x-arm along +x (azimuth pi from North at lon 0),
    # y-arm along +y (azimuth pi/2): D = (x x - y y) / 2
    return np.array([math.pi / 2, 0.0, 0.0, math.pi, math.pi / 2])


def test_detector_tensor_polar_frame(oracle_mod):
    D, _ = oracle_mod.detector_tensor(_polar_detector())
    np.testing.assert_allclose(D, np.diag([0.5, -0.5, 0.0]), atol=1e-15)
    # traceless and symmetric for any site
    D2, _ = oracle_mod.detector_tensor(np.array([0.81, -2.08, 142.0, 2.2, 3.77]))
    assert abs(np.trace(D2)) < 1e-15
    np.testing.assert_allclose(D2, D2.T, atol=1e-15)


def test_antenna_overhead_special_case(oracle_mod):
    g = _polar_detector()
    rng = np.random.default_rng(5)
    for _ in range(20):
        gmst, ra, psi = rng.uniform(0, 2 * math.pi, 3)
        fp, fx = oracle_mod.antenna(g, gmst, ra, math.pi / 2, psi)
        gg = gmst - ra
        assert fp == pytest.approx(-math.cos(2 * (psi + gg)), abs=1e-14)
        assert fx == pytest.approx(math.sin(2 * (psi + gg)), abs=1e-14)


def test_antenna_textbook_power(oracle_mod):
    g = _polar_detector()
    rng = np.random.default_rng(6)
    for _ in range(50):
        gmst, ra, psi = rng.uniform(0, 2 * math.pi, 3)
        dec = math.asin(rng.uniform(-1, 1))
        fp, fx = oracle_mod.antenna(g, gmst, ra, dec, psi)
        theta = math.pi / 2 - dec
        phi = ra - gmst
        expect = 0.25 * (1 + math.cos(theta) ** 2) ** 2 * math.cos(2 * phi) ** 2 + \
            math.cos(theta) ** 2 * math.sin(2 * phi) ** 2
        assert fp * fp + fx * fx == pytest.approx(expect, abs=1e-13)


def test_antenna_psi_invariance(oracle_mod):
    import synth
    geom = synth.site_geometry(["H1", "L1", "V1"])
    rng = np.random.default_rng(7)
    for d in range(3):
        for _ in range(10):
            ra, psi = rng.uniform(0, 2 * math.pi, 2)
            dec = math.asin(rng.uniform(-1, 1))
            fp, fx = oracle_mod.antenna(geom[d], 1.0, ra, dec, psi)
            fp2, fx2 = oracle_mod.antenna(geom[d], 1.0, ra, dec, psi + 0.77)
            fp3, fx3 = oracle_mod.antenna(geom[d], 1.0, ra, dec, psi + math.pi / 2)
            assert fp * fp + fx * fx == pytest.approx(fp2 * fp2 + fx2 * fx2, abs=1e-14)
            assert fp3 == pytest.approx(-fp, abs=1e-14)
            assert fx3 == pytest.approx(-fx, abs=1e-14)


def test_time_delay_along_vertex(oracle_mod):
    import synth
    geom = synth.site_geometry(["H1", "V1"])
    gmst = 1.0
    for d in range(2):
        _, r = oracle_mod.detector_tensor(geom[d])
        n = r / np.linalg.norm(r)
        dec = math.asin(n[2])
        ra = math.atan2(n[1], n[0]) + gmst
        assert oracle_mod.time_delay(geom[d], gmst, ra, dec) == pytest.approx(-np.linalg.norm(r) / C, rel=1e-13)
        # antipodal source: +|r|/c
        assert oracle_mod.time_delay(geom[d], gmst, ra + math.pi, -dec) == pytest.approx(np.linalg.norm(r) / C,
                                                                                          rel=1e-13)
