"""FP64 CPU oracle for the relative-binning likelihood -- TEST INFRASTRUCTURE ONLY.

This package wraps ``rb_oracle.cpp`` (plain C++17, FP64, no CUDA) with ctypes and
numpy.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The GPU library
(``paper_2404_11397_gb300``) never imports, links or calls anything here, and the
two share no code: the only module both sides use is ``synth`` (seeded inputs,
none of the method's arithmetic).

What each function follows (arXiv:2404.11397 and the works it cites):

* ``loglike_full``  -- Eq. 2 with the inner product of Eq. 3 (constant dropped).
* ``loglike_rb``    -- Eqs. 4-5 (ratio and piecewise-linear form, Sec. II.C),
  contracted with the summary data; gradient by forward-mode dual numbers.
* ``summary``       -- A0, A1, B0, B1 (and B2) sums implied by Sec. II.C.
* ``bin_edges``     -- PN-ansatz phase-bound bin placement (Sec. II.C and the
  epsilon <-> bin-count statement of Sec. IV.B).
* ``bin_edges_agnostic`` / ``phase_directions`` / ``direction_measure`` -- bin
  placement without the PN ansatz (the outlook of Sec. V asks for one): the
  model's own phase derivatives, each given 2 pi of total variation.
* ``strain`` / ``polarizations`` / ``tf2_phase`` / ``intrinsic`` -- TaylorF2 with
  tides (Sec. II.B; coefficients from the cited PN literature); Lambda-tilde and
  delta-Lambda-tilde from the appendix.
* ``antenna`` / ``time_delay`` / ``detector_tensor`` -- detector projection for
  the parameters of Table III.

Pins: see ``tests/test_oracle_*.py``.  Waveform parity with LALSuite/ripple is
unpinned (neither is available); the spin-orbit and spin-spin coefficients are
pinned by energy-flux derivations (tests/test_oracle_pn.py).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "rb_oracle.cpp"
_LIB_PATH = _HERE / "liborc.so"
_lib = None

NPAR = 13
PARAM_NAMES = ("Mc", "q", "chi1", "chi2", "Lambda1", "Lambda2", "dL", "tc", "phic", "iota", "psi", "ra", "dec")
INTRINSIC_NAMES = ("m1", "m2", "M", "eta", "X1", "X2", "beta", "sigma", "Lt", "dLt",
                   "phi2", "phi3", "phi4", "phi5p", "phi6c", "phi7", "phi10", "phi12")


def build(force: bool = False) -> Path:
    """Compile the oracle shared library with g++ (plain host code, no CUDA)."""
    if _LIB_PATH.exists() and not force and _LIB_PATH.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB_PATH
    tmp = _LIB_PATH.with_suffix(f".{os.getpid()}.tmp.so")
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
           str(_SRC), "-o", str(tmp)]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(str(_LIB_PATH))
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int64)
    i64 = ctypes.c_int64
    d = ctypes.c_double
    c_int = ctypes.c_int
    lib.orc_abi_version.restype = c_int
    lib.orc_intrinsic.argtypes = [dp, dp]
    lib.orc_tf2_phase.argtypes = [dp, dp, i64, dp]
    lib.orc_polarizations.argtypes = [dp, dp, i64, dp, dp]
    lib.orc_detector_tensor.argtypes = [dp, dp, dp]
    lib.orc_antenna.argtypes = [dp, d, d, d, d, dp]
    lib.orc_time_delay.argtypes = [dp, d, d, d]
    lib.orc_time_delay.restype = d
    lib.orc_strain.argtypes = [dp, dp, d, dp, i64, dp]
    lib.orc_inner.argtypes = [dp, dp, dp, i64, d]
    lib.orc_inner.restype = d
    lib.orc_loglike_full.argtypes = [c_int, dp, d, d, i64, i64, dp, dp, dp, i64, dp, c_int]
    lib.orc_loglike_full.restype = c_int
    lib.orc_bin_edges.argtypes = [d, d, d, i64, i64, c_int, ip]
    lib.orc_bin_edges.restype = c_int
    lib.orc_dpsi_max.argtypes = [d, d, d]
    lib.orc_dpsi_max.restype = d
    lib.orc_bin_edges_agnostic.argtypes = [d, i64, i64, dp, c_int, ip, dp]
    lib.orc_bin_edges_agnostic.restype = c_int
    lib.orc_phase_directions.argtypes = [d, i64, i64, dp, dp]
    lib.orc_direction_measure.argtypes = [c_int, i64, dp, dp]
    lib.orc_summary.argtypes = [c_int, dp, d, d, i64, i64, dp, dp, dp, c_int, ip, dp, dp, dp, dp, dp]
    lib.orc_summary.restype = c_int
    lib.orc_loglike_rb.argtypes = [c_int, dp, d, d, i64, i64, c_int, ip, dp, dp, dp, dp, dp, dp, dp, i64, dp,
                                   dp, c_int]
    lib.orc_loglike_rb.restype = c_int
    lib.orc_z_to_theta.argtypes = [dp, i64, dp]
    lib.orc_grad_theta_to_z.argtypes = [dp, dp, i64, dp]
    lib.orc_mala_propose.argtypes = [dp, dp, dp, dp, dp, dp, i64, dp, ctypes.c_void_p]
    lib.orc_mala_log_alpha.argtypes = [dp, dp, dp, dp, dp, dp, i64, c_int, dp]
    _lib = lib
    return lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a: np.ndarray | None):
    if a is None:
        return None
    if a.dtype == np.int64:
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def default_threads() -> int:
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# Waveform and detector pieces
# ---------------------------------------------------------------------------
def intrinsic(theta) -> dict:
    lib = _load()
    th = _f64(theta).reshape(NPAR)
    out = np.zeros(len(INTRINSIC_NAMES))
    lib.orc_intrinsic(_p(th), _p(out))
    return dict(zip(INTRINSIC_NAMES, out.tolist()))


def tf2_phase(theta, f) -> np.ndarray:
    lib = _load()
    th = _f64(theta).reshape(NPAR)
    f = _f64(f)
    out = np.zeros_like(f)
    lib.orc_tf2_phase(_p(th), _p(f), f.size, _p(out))
    return out


def polarizations(theta, f):
    lib = _load()
    th = _f64(theta).reshape(NPAR)
    f = _f64(f)
    hp = np.zeros((f.size, 2))
    hc = np.zeros((f.size, 2))
    lib.orc_polarizations(_p(th), _p(f), f.size, _p(hp), _p(hc))
    return hp[:, 0] + 1j * hp[:, 1], hc[:, 0] + 1j * hc[:, 1]


def detector_tensor(geom):
    lib = _load()
    g = _f64(geom).reshape(5)
    D = np.zeros(9)
    r = np.zeros(3)
    lib.orc_detector_tensor(_p(g), _p(D), _p(r))
    return D.reshape(3, 3), r


def antenna(geom, gmst, ra, dec, psi):
    lib = _load()
    g = _f64(geom).reshape(5)
    F = np.zeros(2)
    lib.orc_antenna(_p(g), gmst, ra, dec, psi, _p(F))
    return float(F[0]), float(F[1])


def time_delay(geom, gmst, ra, dec) -> float:
    lib = _load()
    g = _f64(geom).reshape(5)
    return float(lib.orc_time_delay(_p(g), gmst, ra, dec))


def strain(theta, geom, gmst, f) -> np.ndarray:
    """Complex detector strain h_d(f) for one source."""
    lib = _load()
    th = _f64(theta).reshape(NPAR)
    g = _f64(geom).reshape(5)
    f = _f64(f)
    h = np.zeros((f.size, 2))
    lib.orc_strain(_p(th), _p(g), gmst, _p(f), f.size, _p(h))
    return h[:, 0] + 1j * h[:, 1]


def inner(a, b, psd, T) -> float:
    """<a|b> = 4 df Re sum a conj(b) / S on the grid."""
    lib = _load()
    a2 = _f64(np.stack([np.real(a), np.imag(a)], axis=-1))
    b2 = _f64(np.stack([np.real(b), np.imag(b)], axis=-1))
    s = _f64(psd)
    return float(lib.orc_inner(_p(a2), _p(b2), _p(s), s.size, T))


# ---------------------------------------------------------------------------
# Event-level functions.  An "event" is a dict with keys
#   geom [D][5], gmst, T, kmin, N, f_low, f_high, data [D][N] complex, psd [D][N]
# (see synth.make_event).
# ---------------------------------------------------------------------------
def _data_ri(ev) -> np.ndarray:
    d = np.asarray(ev["data"])
    return _f64(np.stack([d.real, d.imag], axis=-1))


def loglike_full(ev, theta, nthreads: int | None = None) -> np.ndarray:
    lib = _load()
    th = _f64(theta).reshape(-1, NPAR)
    out = np.zeros(th.shape[0])
    geom = _f64(ev["geom"])
    psd = _f64(ev["psd"])
    rc = lib.orc_loglike_full(geom.shape[0], _p(geom), ev["gmst"], ev["T"], ev["kmin"], ev["N"], _p(_data_ri(ev)),
                              _p(psd), _p(th), th.shape[0], _p(out), nthreads or default_threads())
    assert rc == 0
    return out


def dpsi_max(f, f_low, f_high) -> float:
    return float(_load().orc_dpsi_max(float(f), float(f_low), float(f_high)))


def bin_edges(ev, n_bins: int) -> np.ndarray:
    lib = _load()
    edges = np.zeros(n_bins + 1, dtype=np.int64)
    rc = lib.orc_bin_edges(ev["f_low"], ev["f_high"], ev["T"], ev["kmin"], ev["N"], n_bins, _p(edges))
    if rc != 0:
        raise ValueError("invalid bin count")
    return edges


PHASE_DIRECTIONS = ("Mc", "q", "chi1", "chi2", "Lambda1", "Lambda2", "tc")


def phase_directions(ev, theta_ref) -> np.ndarray:
    """[7][N] dPsi(f; theta_ref) / dtheta_j on the grid (j: PHASE_DIRECTIONS)."""
    lib = _load()
    W = np.zeros((len(PHASE_DIRECTIONS), ev["N"]))
    lib.orc_phase_directions(ev["T"], ev["kmin"], ev["N"], _p(_f64(theta_ref)), _p(W))
    return W


def direction_measure(W) -> np.ndarray:
    """M [N] = 2 pi sum_j V_j / V_j(end) for direction functions W [n][N] (V_j: total variation)."""
    lib = _load()
    W = _f64(np.atleast_2d(W))
    M = np.zeros(W.shape[1])
    lib.orc_direction_measure(W.shape[0], W.shape[1], _p(W), _p(M))
    return M


def bin_edges_agnostic(ev, n_bins: int, theta_ref=None):
    """Edges uniform in the direction measure of the model's phase at theta_ref
    (default: the event's injection); returns (edges, epsilon = M(f_high) / B)."""
    lib = _load()
    edges = np.zeros(n_bins + 1, dtype=np.int64)
    eps = ctypes.c_double(0.0)
    th = ev["theta_inj"] if theta_ref is None else theta_ref
    rc = lib.orc_bin_edges_agnostic(ev["T"], ev["kmin"], ev["N"], _p(_f64(th)), n_bins, _p(edges), ctypes.byref(eps))
    if rc != 0:
        raise ValueError("invalid bin count")
    return edges, eps.value


def summary(ev, theta_ref, edges, with_b2: bool = False) -> dict:
    lib = _load()
    geom = _f64(ev["geom"])
    D = geom.shape[0]
    B = len(edges) - 1
    edges = np.ascontiguousarray(edges, dtype=np.int64)
    A0 = np.zeros((D, B, 2))
    A1 = np.zeros((D, B, 2))
    B0 = np.zeros((D, B))
    B1 = np.zeros((D, B))
    B2 = np.zeros((D, B)) if with_b2 else None
    rc = lib.orc_summary(D, _p(geom), ev["gmst"], ev["T"], ev["kmin"], ev["N"], _p(_data_ri(ev)),
                         _p(_f64(ev["psd"])), _p(_f64(theta_ref)), B, _p(edges), _p(A0), _p(A1), _p(B0), _p(B1),
                         _p(B2))
    assert rc == 0
    out = {"edges": edges, "A0": A0[..., 0] + 1j * A0[..., 1], "A1": A1[..., 0] + 1j * A1[..., 1], "B0": B0,
           "B1": B1, "theta_ref": _f64(theta_ref)}
    if with_b2:
        out["B2"] = B2
    return out


def loglike_rb(ev, summ, theta, grad: bool = False, with_b2: bool = False, nthreads: int | None = None):
    """RB log-likelihood [W] (and gradient [W][13] if grad)."""
    lib = _load()
    geom = _f64(ev["geom"])
    D = geom.shape[0]
    th = _f64(theta).reshape(-1, NPAR)
    W = th.shape[0]
    edges = np.ascontiguousarray(summ["edges"], dtype=np.int64)
    B = len(edges) - 1
    A0 = _f64(np.stack([summ["A0"].real, summ["A0"].imag], axis=-1))
    A1 = _f64(np.stack([summ["A1"].real, summ["A1"].imag], axis=-1))
    B0 = _f64(summ["B0"])
    B1 = _f64(summ["B1"])
    B2 = _f64(summ["B2"]) if with_b2 else None
    logl = np.zeros(W)
    g = np.zeros((W, NPAR)) if grad else None
    rc = lib.orc_loglike_rb(D, _p(geom), ev["gmst"], ev["T"], ev["kmin"], ev["N"], B, _p(edges), _p(A0), _p(A1),
                            _p(B0), _p(B1), _p(B2), _p(_f64(summ["theta_ref"])), _p(th), W, _p(logl), _p(g),
                            nthreads or default_threads())
    assert rc == 0
    return (logl, g) if grad else logl



# ---------------------------------------------------------------------------
# MALA local step (Sec. II.D), sampling coordinates of Table II:
# z = (Mc, q, chi1, chi2, L1, L2, dL, tc, phic, cos iota, psi, ra, sin dec)
# ---------------------------------------------------------------------------
def z_to_theta(z):
    lib = _load()
    z = _f64(z).reshape(-1, NPAR)
    th = np.zeros_like(z)
    lib.orc_z_to_theta(_p(z), z.shape[0], _p(th))
    return th


def grad_theta_to_z(z, g_theta):
    lib = _load()
    z = _f64(z).reshape(-1, NPAR)
    g = _f64(g_theta).reshape(-1, NPAR)
    out = np.zeros_like(z)
    lib.orc_grad_theta_to_z(_p(z), _p(g), z.shape[0], _p(out))
    return out


def mala_log_alpha(logp, logp_prop, g, g_prop, eps, xi):
    """log alpha of the MALA acceptance for states of any dimension n."""
    lib = _load()
    g = _f64(g)
    W, n = g.shape
    out = np.zeros(W)
    lib.orc_mala_log_alpha(_p(_f64(logp)), _p(_f64(logp_prop)), _p(g), _p(_f64(g_prop)), _p(_f64(eps)),
                           _p(_f64(xi)), W, n, _p(out))
    return out


def mala_propose(z, g_z, eps, xi, lo, hi):
    lib = _load()
    z = _f64(z).reshape(-1, NPAR)
    zp = np.zeros_like(z)
    inside = np.zeros(z.shape[0], dtype=np.int32)
    lib.orc_mala_propose(_p(z), _p(_f64(g_z)), _p(_f64(eps)), _p(_f64(xi)), _p(_f64(lo)), _p(_f64(hi)),
                         z.shape[0], _p(zp), inside.ctypes.data_as(ctypes.c_void_p))
    return zp, inside.astype(bool)


def mala_logpost(ev, summ, z, lo, hi, nthreads=None):
    """log pi(z) = log L(theta(z)) (uniform prior: constant inside the open box,
    -inf outside) and d log pi / dz."""
    z = _f64(z).reshape(-1, NPAR)
    inside = np.all((z > np.asarray(lo)) & (z < np.asarray(hi)), axis=1)
    zc = np.where(inside[:, None], z, np.clip(z, np.asarray(lo) + 1e-12, np.asarray(hi) - 1e-12))
    th = z_to_theta(zc)
    logl, g = loglike_rb(ev, summ, th, grad=True, nthreads=nthreads)
    gz = grad_theta_to_z(zc, g)
    return np.where(inside, logl, -np.inf), np.where(inside[:, None], gz, 0.0)


def mala_step(ev, summ, z, logp, g_z, eps, xi, u, lo, hi, nthreads=None):
    """One MALA step for every chain; returns (z, logp, g_z, accepted, log_alpha)."""
    zp, inside = mala_propose(z, g_z, eps, xi, lo, hi)
    logpp, gzp = mala_logpost(ev, summ, zp, lo, hi, nthreads)
    la = mala_log_alpha(logp, logpp, g_z, gzp, eps, xi)
    acc = inside & (np.log(_f64(u)) < la)
    z = np.where(acc[:, None], zp, z)
    logp = np.where(acc, logpp, logp)
    g_z = np.where(acc[:, None], gzp, g_z)
    return z, logp, g_z, acc, la
