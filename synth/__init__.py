"""Seeded synthetic inputs for the relative-binning likelihood workloads.

This module holds no arithmetic of the method itself: it makes the frequency
grid, an analytic detector noise curve, seeded Gaussian noise, detector site
geometry and seeded walker draws.  Both the oracle tests and the GPU path take
their inputs from here; neither side imports the other.  The injected signal
is added by the caller (the oracle's waveform in tests, the library's own
waveform kernel in the benchmark), because a waveform is the method's
arithmetic.

Stand-ins for the paper's data (which are not available here):

* GWOSC strain (Sec. IV) and design-sensitivity PSDs (Sec. III) are replaced
  by an analytic aLIGO zero-detuned high-power fit (Ajith 2011) used for every
  detector, and seeded Gaussian noise with Re, Im ~ N(0, S_n / (4 df)) so that
  E<n|n> = 2N.
* Priors follow Table III (GW170817 column for the 3-detector configuration)
  with cos(iota) and sin(dec) uniform.

Random numbers: numpy's Philox-4x64 counter-based generator (raw 64-bit
stream, stable across numpy versions), uniforms from the top 53 bits, normals
by the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NPAR = 13
PARAM_NAMES = ("Mc", "q", "chi1", "chi2", "Lambda1", "Lambda2", "dL", "tc", "phic", "iota", "psi", "ra", "dec")
GMST = 1.0  # rad, per-event constant

# Site geometry rows: lat [deg], lon [deg], elevation [m], x-arm and y-arm
# azimuth [deg clockwise from North].  Rounded LIGO/Virgo-like values.
SITES_DEG = {
    "H1": (46.455, -119.408, 142.554, 126.0, 216.0),
    "L1": (30.563, -90.774, -6.574, 197.7, 287.7),
    "V1": (43.631, 10.505, 51.884, 70.6, 160.6),
}


def site_geometry(names) -> np.ndarray:
    """[D][5] rows (lat, lon [rad], elevation [m], x-arm az, y-arm az [rad])."""
    rows = []
    for n in names:
        lat, lon, elev, xa, ya = SITES_DEG[n]
        rows.append([math.radians(lat), math.radians(lon), elev, math.radians(xa), math.radians(ya)])
    return np.asarray(rows, dtype=np.float64)


def grid(T: float, f_low: float, f_high: float):
    """Grid f_k = k / T for k = ceil(f_low T) .. floor(f_high T), both ends included."""
    kmin = int(math.ceil(f_low * T - 1e-9))
    kmax = int(math.floor(f_high * T + 1e-9))
    N = kmax - kmin + 1
    f = (kmin + np.arange(N, dtype=np.float64)) / T
    return kmin, N, f


def psd_aligo(f) -> np.ndarray:
    """Analytic aLIGO zero-detuned high-power fit: S(f) = 1e-49 [x^-4.14 - 5 x^-2 +
    111 (1 - x^2 + x^4/2) / (1 + x^2/2)], x = f / 245.4 Hz."""
    x = np.asarray(f, dtype=np.float64) / 245.4
    return 1e-49 * (x ** -4.14 - 5.0 * x ** -2 + 111.0 * (1.0 - x ** 2 + 0.5 * x ** 4) / (1.0 + 0.5 * x ** 2))


def uniforms(seed: int, n: int) -> np.ndarray:
    """n uniforms in (0, 1) from the Philox raw stream keyed by ``seed``."""
    raw = np.random.Philox(seed).random_raw(n).astype(np.uint64)
    return ((raw >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53


def normals(seed: int, n: int) -> np.ndarray:
    """n standard normals (Box-Muller on pairs of uniforms)."""
    m = (n + 1) // 2
    u = uniforms(seed, 2 * m)
    r = np.sqrt(-2.0 * np.log(u[0::2]))
    t = 2.0 * np.pi * u[1::2]
    return np.concatenate([r * np.cos(t), r * np.sin(t)])[:n]


def noise(psd: np.ndarray, T: float, seed: int) -> np.ndarray:
    """Complex coloured noise with Re, Im ~ N(0, S / (4 df)) independently, df = 1/T."""
    n = psd.size
    z = normals(seed, 2 * n)
    sigma = np.sqrt(psd * T / 4.0)
    return sigma * (z[:n] + 1j * z[n:])


def masses_to_mc_q(m1: float, m2: float):
    M = m1 + m2
    return (m1 * m2) ** 0.6 / M ** 0.2, m2 / m1


# Injection of the 1- and 3-detector configurations: m1 = 1.40, m2 = 1.30 Msun,
# chi = 0.02 / 0.02, Lambda = 300 / 400, d_L = 40 Mpc; sky and orientation angles
# are fixed values chosen here.
_MC0, _Q0 = masses_to_mc_q(1.40, 1.30)
THETA_INJ = np.array([_MC0, _Q0, 0.02, 0.02, 300.0, 400.0, 40.0, 0.0, 1.0, 0.4, 0.6, 3.45, -0.41])
# Heavier system: the centre of its chirp-mass box.
THETA_INJ_HEAVY = np.array([1.44, 0.8, 0.02, 0.02, 800.0, 900.0, 40.0, 0.0, 1.0, 0.4, 0.6, 3.45, -0.41])

# Uniform prior boxes (Table III): (lo, hi) per parameter; iota and dec are
# drawn through cos(iota), sin(dec) uniform on [-1, 1].
PRIOR_GW170817 = {
    "Mc": (1.18, 1.21), "q": (0.125, 1.0), "chi1": (-0.05, 0.05), "chi2": (-0.05, 0.05),
    "Lambda1": (0.0, 5000.0), "Lambda2": (0.0, 5000.0), "dL": (1.0, 75.0), "tc": (-0.1, 0.1),
    "phic": (0.0, 2 * math.pi), "iota": "cos", "psi": (0.0, math.pi), "ra": (0.0, 2 * math.pi), "dec": "sin",
}
PRIOR_HEAVY = dict(PRIOR_GW170817, Mc=(1.42, 1.46), Lambda1=(0.0, 3000.0), Lambda2=(0.0, 3000.0))

# Widths used for finite-difference steps and posterior-scale boxes.
PRIOR_WIDTH = np.array([0.03, 0.875, 0.1, 0.1, 5000.0, 5000.0, 74.0, 0.2, 2 * math.pi, math.pi, math.pi,
                        2 * math.pi, math.pi])


def draw_prior(prior: dict, W: int, seed: int) -> np.ndarray:
    """W walkers [W][13] drawn uniformly from a prior box."""
    u = uniforms(seed, W * NPAR).reshape(NPAR, W)
    out = np.empty((W, NPAR))
    for j, name in enumerate(PARAM_NAMES):
        spec = prior[name]
        if spec == "cos":
            out[:, j] = np.arccos(2.0 * u[j] - 1.0)
        elif spec == "sin":
            out[:, j] = np.arcsin(2.0 * u[j] - 1.0)
        else:
            lo, hi = spec
            out[:, j] = lo + (hi - lo) * u[j]
    return out


def draw_box(center, W: int, seed: int, rel: float = 0.01, abs_width=None) -> np.ndarray:
    """W walkers uniform in center * (1 +/- rel) per parameter (plus/minus abs_width
    where given, for parameters whose centre is zero)."""
    c = np.asarray(center, dtype=np.float64)
    half = np.abs(c) * rel
    if abs_width is not None:
        half = np.maximum(half, np.asarray(abs_width, dtype=np.float64))
    u = uniforms(seed, W * NPAR).reshape(W, NPAR)
    out = c + (2.0 * u - 1.0) * half
    out[:, 1] = np.minimum(out[:, 1], 1.0)  # keep q <= 1
    return out


def posterior_box(center, W: int, seed: int) -> np.ndarray:
    """Posterior-scale box: +/-1e-5 relative in Mc, +/-1e-3 relative in the others
    (absolute 1e-3 x prior width for parameters centred at zero)."""
    c = np.asarray(center, dtype=np.float64)
    half = np.abs(c) * 1e-3
    half[0] = abs(c[0]) * 1e-5
    half = np.maximum(half, 1e-3 * PRIOR_WIDTH * (c == 0.0))
    u = uniforms(seed, W * NPAR).reshape(W, NPAR)
    out = c + (2.0 * u - 1.0) * half
    out[:, 1] = np.minimum(out[:, 1], 1.0)
    return out


@dataclass
class Config:
    name: str
    sites: tuple
    T: float
    f_low: float
    f_high: float
    n_bins: int
    n_walkers: int
    theta_inj: np.ndarray
    walkers: str  # "box" (+/-1 % around the injection) or "prior"
    prior: dict = field(default_factory=dict)
    seed_walkers: int = 1


CONFIGS = {
    # 1 detector, T = 64 s, 20-1024 Hz, 100 bins, 1000 walkers in a +/-1 % box.
    "C1": Config("C1", ("H1",), 64.0, 20.0, 1024.0, 100, 1000, THETA_INJ, "box", seed_walkers=1),
    # 3 detectors, T = 128 s, 20-2048 Hz, 500 bins, 4096 prior draws.
    "C2": Config("C2", ("H1", "L1", "V1"), 128.0, 20.0, 2048.0, 500, 4096, THETA_INJ, "prior", PRIOR_GW170817,
                 seed_walkers=2),
    # the 1-detector event with 4096 walkers and the gradient.
    "C3": Config("C3", ("H1",), 64.0, 20.0, 1024.0, 100, 4096, THETA_INJ, "box", seed_walkers=3),
    # 3 detectors, T = 256 s, 1000 bins, 16384 walkers, heavier chirp-mass box.
    "C4": Config("C4", ("H1", "L1", "V1"), 256.0, 20.0, 2048.0, 1000, 16384, THETA_INJ_HEAVY, "prior",
                 PRIOR_HEAVY, seed_walkers=4),
}


def noise_seed(det_index: int) -> int:
    return 20240417 + det_index


def make_event(cfg: Config | str, *, T=None, f_low=None, f_high=None, sites=None, gmst: float = GMST,
               noise_scale: float = 1.0) -> dict:
    """Grid, PSD, seeded noise and geometry of one event (no signal yet).

    Returns a dict with keys geom [D][5], gmst, T, kmin, N, f_low, f_high, f [N],
    psd [D][N], noise [D][N] complex, theta_inj [13].  The caller sets
    ``ev["data"] = ev["noise"] + injected signal``.
    """
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    T = cfg.T if T is None else T
    f_low = cfg.f_low if f_low is None else f_low
    f_high = cfg.f_high if f_high is None else f_high
    sites = cfg.sites if sites is None else tuple(sites)
    kmin, N, f = grid(T, f_low, f_high)
    psd1 = psd_aligo(f)
    D = len(sites)
    psd = np.tile(psd1, (D, 1))
    nz = np.stack([noise(psd1, T, noise_seed(i)) for i in range(D)]) * noise_scale
    return {"geom": site_geometry(sites), "gmst": float(gmst), "T": float(T), "kmin": int(kmin), "N": int(N),
            "f_low": float(f_low), "f_high": float(f_high), "f": f, "psd": psd, "noise": nz,
            "theta_inj": np.array(cfg.theta_inj, dtype=np.float64), "n_bins": cfg.n_bins, "sites": sites}


def walkers(cfg: Config | str, W: int | None = None) -> np.ndarray:
    if isinstance(cfg, str):
        cfg = CONFIGS[cfg]
    W = cfg.n_walkers if W is None else W
    if cfg.walkers == "prior":
        return draw_prior(cfg.prior, W, cfg.seed_walkers)
    return draw_box(cfg.theta_inj, W, cfg.seed_walkers, rel=0.01, abs_width=1e-2 * PRIOR_WIDTH)
