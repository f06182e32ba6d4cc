"""GPU path (librb, through the C ABI) vs the FP64 oracle on the same seeded inputs.

Tolerances (stated in the library's design notes):
* bin edges: bit-exact (integer work);
* summary data A0, A1, B0, B1 (FP64 on both sides): 1e-9 of the largest |entry| per detector;
* log L, mixed precision: |dlogL| <= 1e-3 absolute on C1 and C3 (the +-1 % box of the
  1-detector event) and on posterior-scale boxes; for draws from the whole prior box (C2,
  C4) and the other synthetic test events |dlogL| <= max(1e-3, 2e-6 (|<d|h>| + <h|h>/2)),
  since <h|h> reaches ~1e7 at d_L ~ 1 Mpc and FP32 products carry ~1e-7 of it; FP64 path:
  1e-9 of that scale (plus 1e-8 absolute);
* gradient: |dg_j| <= 1e-4 max(|g_j|, 1e-2 max_j |g_j|) (mixed), 1e-8 (FP64).  For prior
  draws a walker over that bound must still be within the FP32 floor of its sum,
  |dg_j| <= 1e-4 max(...) + 8 u32 K_j (K_j = sum over detectors and edges of the absolute
  per-edge terms of g_j, tests/_grad_cond.py; u32 = 2^-24), and every walker within
  max_j |dg_j| <= 1e-4 max_j |g_j|;
* at the fiducial point every mode returns the FP64 constant exactly.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from tests import _grad_cond
from tests._events import inject

pytestmark = pytest.mark.gpu

MODES = ("mixed", "mixed_f64phase", "fp64")


@pytest.fixture(scope="module")
def rb():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2404_11397_gb300 as m
    m.load()
    return m


def _terms(ev, s, theta):
    """Oracle RB log L, <d|h> and <h|h> (the latter from the data-free summary)."""
    zero = dict(s)
    zero["A0"] = np.zeros_like(s["A0"])
    zero["A1"] = np.zeros_like(s["A1"])
    hh = -2.0 * oracle.loglike_rb(ev, zero, theta)
    L = oracle.loglike_rb(ev, s, theta)
    return L, L + 0.5 * hh, hh


U32 = 2.0 ** -24


def _tol(mode, dh, hh, near=False):
    """near: walkers near the posterior, held to 1e-3 absolute in the mixed modes."""
    scale = np.abs(dh) + 0.5 * hh
    if mode == "fp64":
        return 1e-9 * scale + 1e-8
    if near:
        return np.full_like(scale, 1e-3)
    return np.maximum(1e-3, 2e-6 * scale)


def _gtol(mode, g):
    rel = 1e-8 if mode == "fp64" else 1e-4
    return rel * np.maximum(np.abs(g), 1e-2 * np.max(np.abs(g), axis=1, keepdims=True))


def _check_prior_gradients(ev, s, edges, th, G, ref_G, mode):
    """Every walker within the component bound, or (mixed modes only) within it plus
    the FP32 floor 8 u32 K_j of its sum; every walker within 1e-4 norm-wise.
    Returns the number of walkers that needed the floor."""
    err = np.abs(G - ref_G)
    flat = _gtol(mode, ref_G)
    over = np.unique(np.argwhere(err > flat)[:, 0])
    if mode == "fp64":
        assert over.size == 0, (mode, over[:5])
        return 0
    assert np.all(err.max(axis=1) <= 1e-4 * np.abs(ref_G).max(axis=1)), mode
    if over.size:
        K = _grad_cond.gradient_terms_abs(ev, s, edges, th[over])
        ratio = (err[over] - flat[over]) / (U32 * K)
        assert np.all(ratio <= 8.0), (mode, over, ratio.max())
    return over.size


class Case:
    def __init__(self, rb, cfg, n_bins=None, **kw):
        self.ev = inject(synth.make_event(cfg, **kw))
        self.n_bins = n_bins or self.ev["n_bins"]
        self.edges = oracle.bin_edges(self.ev, self.n_bins)
        self.s = oracle.summary(self.ev, self.ev["theta_inj"], self.edges)
        self.event = rb.Event.from_synth(self.ev, n_bins=self.n_bins)


@pytest.fixture(scope="module")
def c1(rb):
    return Case(rb, "C1")


@pytest.fixture(scope="module")
def c2(rb):
    return Case(rb, "C2")


@pytest.fixture(scope="module")
def small(rb):
    # a few thousand grid points, 3 detectors, 45 bins (one ragged 63-bin iteration of the
    # float-float kernel, two 31-bin chunks of the FP64-phase kernel)
    return Case(rb, "C2", n_bins=45, T=8.0, f_low=20.0, f_high=512.0)


@pytest.fixture(scope="module")
def two(rb):
    # two detectors: no odd detector (the FP64-phase kernel's pair-only bin tables)
    return Case(rb, "C2", n_bins=150, T=32.0, sites=("H1", "L1"))


@pytest.mark.parametrize("mode", MODES)
def test_two_detectors(rb, two, mode):
    th = synth.draw_box(two.ev["theta_inj"], 300, seed=23, rel=0.01, abs_width=1e-2 * synth.PRIOR_WIDTH)
    L, G = rb.loglike_grad(two.event, torch.tensor(th, device="cuda"), mode=mode)
    ref, dh, hh = _terms(two.ev, two.s, th)
    assert np.all(np.abs(L.cpu().numpy() - ref) <= _tol(mode, dh, hh, near=True))
    _, ref_G = oracle.loglike_rb(two.ev, two.s, th[:24], grad=True)
    assert np.all(np.abs(G.cpu().numpy()[:24] - ref_G) <= _gtol(mode, ref_G))


def test_grid_and_info(rb, c1, c2):
    for c in (c1, c2):
        inf = c.event.info()
        assert inf["n_freq"] == c.ev["N"] and inf["kmin"] == c.ev["kmin"]
        assert inf["n_bins"] == c.n_bins and inf["n_det"] == c.ev["geom"].shape[0]


@pytest.mark.parametrize("cfg,n_bins,kw", [("C1", None, {}), ("C2", None, {}), ("C2", 45, dict(T=8.0, f_high=512.0)),
                                           ("C4", None, {}), ("C2", 1, dict(T=4.0, f_high=256.0)),
                                           ("C2", 1000, dict(T=16.0))])
def test_bin_edges_bit_exact(rb, cfg, n_bins, kw):
    ev = inject(synth.make_event(cfg, **kw))
    B = n_bins or ev["n_bins"]
    event = rb.Event.from_synth(ev, n_bins=B)
    np.testing.assert_array_equal(event.summary()["edges"], oracle.bin_edges(ev, B))
    event.free()


def test_bin_edges_one_point_per_bin(rb):
    ev = inject(synth.make_event("C2", T=1.0, f_low=30.0, f_high=94.0))
    event = rb.Event.from_synth(ev, n_bins=ev["N"] - 1)
    np.testing.assert_array_equal(event.summary()["edges"], np.arange(ev["N"]))


def test_summary_data_matches_oracle(rb, c1, c2, small):
    for c in (c1, c2, small):
        g = c.event.summary()
        for key in ("A0", "A1", "B0", "B1"):
            ref = c.s[key]
            scale = np.max(np.abs(ref), axis=1, keepdims=True)
            assert np.all(np.abs(g[key] - ref) <= 1e-9 * scale), key


def test_strain_kernel_matches_oracle(rb, c2):
    ev = c2.ev
    th = synth.draw_prior(synth.PRIOR_GW170817, 3, seed=21)
    for w in range(3):
        for d in range(3):
            h = rb.strain(ev["geom"][d], ev["gmst"], th[w], ev["T"], ev["kmin"], ev["N"]).cpu().numpy()
            ref = oracle.strain(th[w], ev["geom"][d], ev["gmst"], ev["f"])
            assert np.max(np.abs(h - ref)) <= 1e-9 * np.max(np.abs(ref))


@pytest.mark.parametrize("mode", MODES)
def test_exact_at_reference(rb, c1, c2, small, mode):
    for c in (c1, c2, small):
        th = torch.tensor(np.tile(c.ev["theta_inj"], (33, 1)), device="cuda")
        L = rb.loglike(c.event, th, mode=mode).cpu().numpy()
        Lg, G = rb.loglike_grad(c.event, th, mode=mode)
        base = c.event.info()["base_logl"]
        assert np.all(L == base) and np.all(Lg.cpu().numpy() == base)
        full = oracle.loglike_full(c.ev, c.ev["theta_inj"])[0]
        assert abs(base - full) <= 1e-9 * abs(full)


@pytest.mark.parametrize("mode", MODES)
def test_loglike_box_walkers(rb, c1, small, mode):
    for c, W in ((c1, 1000), (small, 777)):
        th = synth.walkers("C1", W) if c is c1 else synth.draw_box(c.ev["theta_inj"], W, seed=31, rel=0.01,
                                                                   abs_width=1e-2 * synth.PRIOR_WIDTH)
        L = rb.loglike(c.event, torch.tensor(th, device="cuda"), mode=mode).cpu().numpy()
        ref, dh, hh = _terms(c.ev, c.s, th)
        err = np.abs(L - ref)
        assert np.all(err <= _tol(mode, dh, hh, near=c is c1)), (mode, err.max())


@pytest.mark.parametrize("mode", MODES)
def test_loglike_posterior_scale(rb, c1, c2, mode):
    for c in (c1, c2):
        th = synth.posterior_box(c.ev["theta_inj"], 256, seed=41)
        L = rb.loglike(c.event, torch.tensor(th, device="cuda"), mode=mode).cpu().numpy()
        ref, dh, hh = _terms(c.ev, c.s, th)
        assert np.all(np.abs(L - ref) <= _tol(mode, dh, hh, near=True))


@pytest.mark.parametrize("mode", MODES)
def test_loglike_prior_draws_full_batch(rb, c2, mode):
    """C2 at its full size (4096 prior draws, the benchmark's launch), every walker checked."""
    th = synth.walkers("C2")
    L = rb.loglike(c2.event, torch.tensor(th, device="cuda"), mode=mode).cpu().numpy()
    ref, dh, hh = _terms(c2.ev, c2.s, th)
    err = np.abs(L - ref)
    assert np.all(err <= _tol(mode, dh, hh)), (mode, err.max())


@pytest.mark.parametrize("mode", MODES)
def test_gradient_matches_oracle(rb, c1, small, mode):
    for c, W in ((c1, 64), (small, 40)):
        th = synth.draw_box(c.ev["theta_inj"], W, seed=51, rel=3e-3, abs_width=3e-3 * synth.PRIOR_WIDTH)
        L, G = rb.loglike_grad(c.event, torch.tensor(th, device="cuda"), mode=mode)
        ref_L, ref_G = oracle.loglike_rb(c.ev, c.s, th, grad=True)
        _, dh, hh = _terms(c.ev, c.s, th)
        assert np.all(np.abs(L.cpu().numpy() - ref_L) <= _tol(mode, dh, hh, near=c is c1))
        G = G.cpu().numpy()
        bad = np.abs(G - ref_G) > _gtol(mode, ref_G)
        assert not bad.any(), (mode, np.argwhere(bad)[:5], (np.abs(G - ref_G) / _gtol(mode, ref_G) * 1e-4).max())


@pytest.mark.parametrize("mode", MODES)
def test_gradient_prior_draws(rb, c2, mode):
    """C2's 4096 prior draws, every gradient against the oracle's."""
    th = synth.walkers("C2")
    _, G = rb.loglike_grad(c2.event, torch.tensor(th, device="cuda"), mode=mode)
    _, ref_G = oracle.loglike_rb(c2.ev, c2.s, th, grad=True)
    n_floor = _check_prior_gradients(c2.ev, c2.s, c2.edges, th, G.cpu().numpy(), ref_G, mode)
    assert n_floor <= 16, n_floor


@pytest.mark.parametrize("mode", ("mixed", "mixed_f64phase"))
def test_wide_phase_walkers(rb, c1, c2, mode):
    """Walkers far from the fiducial point (chirp mass x 0.5 ... 0.1: phase terms of
    2^13 to 2^17 turns), which take the mixed kernel's second whole-turn reduction:
    log L within the prior-draw bound, gradients within 1e-4 norm-wise."""
    for c in (c1, c2):
        th = np.repeat(c.ev["theta_inj"][None, :], 5, 0)
        th[:, 0] *= np.array([0.5, 0.4, 0.3, 0.2, 0.1])
        L, G = rb.loglike_grad(c.event, torch.tensor(th, device="cuda"), mode=mode)
        ref, dh, hh = _terms(c.ev, c.s, th)
        assert np.all(np.abs(L.cpu().numpy() - ref) <= _tol(mode, dh, hh)), (mode, np.abs(L.cpu().numpy() - ref))
        _, ref_G = oracle.loglike_rb(c.ev, c.s, th, grad=True)
        nw = np.max(np.abs(G.cpu().numpy() - ref_G), axis=1) / np.max(np.abs(ref_G), axis=1)
        assert np.all(nw <= 1e-4), (mode, nw)


def test_phase_terms_beyond_range_are_nan(rb, c1):
    """A walker whose phase terms reach past 2^18 turns (chirp mass x 0.05) is not
    evaluated by the float-pair phase sums: NaN log L and gradient in RB_MIXED; the
    FP64 path still evaluates it."""
    th = c1.ev["theta_inj"][None, :].copy()
    th[0, 0] *= 0.05
    th = np.concatenate([th, c1.ev["theta_inj"][None, :]])
    L, G = rb.loglike_grad(c1.event, torch.tensor(th, device="cuda"), mode="mixed")
    L, G = L.cpu().numpy(), G.cpu().numpy()
    assert np.isnan(L[0]) and np.all(np.isnan(G[0]))
    assert np.isfinite(L[1]) and np.all(np.isfinite(G[1]))
    L64, _ = rb.loglike_grad(c1.event, torch.tensor(th, device="cuda"), mode="fp64")
    ref = oracle.loglike_rb(c1.ev, c1.s, th)
    assert np.all(np.abs(L64.cpu().numpy() - ref) <= 1e-8 + 1e-9 * np.abs(ref))


def test_c3_box_walkers_with_gradient(rb, c1):
    """C3: C1's event, 4096 walkers in the +-1 % box, log L + gradient in one launch;
    every log L within 1e-3 absolute, 64 gradients against the oracle's."""
    th = synth.walkers("C3")
    assert th.shape == (4096, 13)
    for mode in MODES:
        L, G = rb.loglike_grad(c1.event, torch.tensor(th, device="cuda"), mode=mode)
        ref, dh, hh = _terms(c1.ev, c1.s, th)
        assert np.all(np.abs(L.cpu().numpy() - ref) <= _tol(mode, dh, hh, near=True)), mode
        idx = np.linspace(0, 4095, 64).astype(int)
        _, ref_G = oracle.loglike_rb(c1.ev, c1.s, th[idx], grad=True)
        assert np.all(np.abs(G.cpu().numpy()[idx] - ref_G) <= _gtol(mode, ref_G)), mode


def test_fp64_gradient_vs_finite_differences(rb, small):
    th0 = synth.draw_box(small.ev["theta_inj"], 4, seed=61, rel=3e-3, abs_width=3e-3 * synth.PRIOR_WIDTH)
    _, G = rb.loglike_grad(small.event, torch.tensor(th0, device="cuda"), mode="fp64")
    G = G.cpu().numpy()
    for j in range(13):
        h = 1e-6 * np.maximum(np.abs(th0[:, j]), synth.PRIOR_WIDTH[j])

        def cd(step):
            tp, tm = th0.copy(), th0.copy()
            tp[:, j] += step
            tm[:, j] -= step
            Lp = rb.loglike(small.event, torch.tensor(tp, device="cuda"), mode="fp64").cpu().numpy()
            Lm = rb.loglike(small.event, torch.tensor(tm, device="cuda"), mode="fp64").cpu().numpy()
            return (Lp - Lm) / (2 * step)
        fd = (4 * cd(h / 2) - cd(h)) / 3
        scale = np.maximum(np.abs(G[:, j]), 1e-2 * np.max(np.abs(G), axis=1))
        assert np.all(np.abs(fd - G[:, j]) <= 1e-6 * scale), j


def test_unphysical_walkers(rb, small):
    th = np.tile(small.ev["theta_inj"], (6, 1))
    th[0, 1] = 1.5
    th[1, 1] = -0.1
    th[2, 6] = 0.0
    th[3, 0] = np.nan
    th[4, 11] = np.inf
    for mode in MODES:
        L, G = rb.loglike_grad(small.event, torch.tensor(th, device="cuda"), mode=mode)
        L, G = L.cpu().numpy(), G.cpu().numpy()
        assert np.all(np.isneginf(L[:5])) and np.isfinite(L[5])
        assert np.all(G[:5] == 0.0)


def test_edge_cases_batch_shapes(rb, small):
    th = synth.draw_box(small.ev["theta_inj"], 70, seed=71, rel=1e-3, abs_width=1e-3 * synth.PRIOR_WIDTH)
    full = rb.loglike(small.event, torch.tensor(th, device="cuda")).cpu().numpy()
    # W = 0 is a no-op; W = 1 and ragged W give the same per-walker values (warp per walker)
    empty = rb.loglike(small.event, torch.zeros(0, 13, dtype=torch.float64, device="cuda"))
    assert empty.numel() == 0
    one = rb.loglike(small.event, torch.tensor(th[5:6], device="cuda")).cpu().numpy()
    assert one[0] == full[5]
    part = rb.loglike(small.event, torch.tensor(th[3:40], device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(part, full[3:40])


@pytest.mark.parametrize("mode", MODES)
def test_large_batch_many_walkers_per_warp(rb, small, mode):
    """150,000 walkers in one call: the grid is capped by occupancy and every
    warp takes many walkers in turn.  Each walker's values are those it gets in
    a small batch, bit for bit (one warp per walker, no cross-walker sums), and
    sampled walkers agree with the oracle."""
    W = 150_000
    th = synth.draw_box(small.ev["theta_inj"], W, seed=161, rel=0.01, abs_width=1e-2 * synth.PRIOR_WIDTH)
    L, G = rb.loglike_grad(small.event, torch.tensor(th, device="cuda"), mode=mode)
    L, G = L.cpu().numpy(), G.cpu().numpy()
    assert L.shape == (W,) and G.shape == (W, 13) and np.all(np.isfinite(L))
    idx = np.array([0, 1, 2431, 2432, 4863, 77_777, W - 2, W - 1])
    Ls, Gs = rb.loglike_grad(small.event, torch.tensor(th[idx], device="cuda"), mode=mode)
    np.testing.assert_array_equal(L[idx], Ls.cpu().numpy())
    np.testing.assert_array_equal(G[idx], Gs.cpu().numpy())
    ref, dh, hh = _terms(small.ev, small.s, th[idx])
    assert np.all(np.abs(L[idx] - ref) <= _tol(mode, dh, hh))


def test_one_bin_and_one_point_per_bin(rb):
    for n_bins, kw in ((1, dict(T=4.0, f_high=256.0)), (None, dict(T=1.0, f_low=30.0, f_high=94.0))):
        ev = inject(synth.make_event("C2", **kw))
        B = n_bins or ev["N"] - 1
        edges = oracle.bin_edges(ev, B)
        s = oracle.summary(ev, ev["theta_inj"], edges)
        event = rb.Event.from_synth(ev, n_bins=B)
        th = synth.draw_box(ev["theta_inj"], 50, seed=81, rel=0.01, abs_width=1e-2 * synth.PRIOR_WIDTH)
        for mode in MODES:
            L = rb.loglike(event, torch.tensor(th, device="cuda"), mode=mode).cpu().numpy()
            ref, dh, hh = _terms(ev, s, th)
            assert np.all(np.abs(L - ref) <= _tol(mode, dh, hh)), (B, mode)
        event.free()


def test_heavy_config_full_size_sampled(rb):
    """C4 (T = 256 s, 1000 bins, 16384 walkers) in one launch; 1024 sampled walkers vs
    the oracle (log L and gradient)."""
    ev = inject(synth.make_event("C4"))
    edges = oracle.bin_edges(ev, 1000)
    event = rb.Event.from_synth(ev, n_bins=1000)
    np.testing.assert_array_equal(event.summary()["edges"], edges)
    s = oracle.summary(ev, ev["theta_inj"], edges)
    th = synth.walkers("C4")
    L, G = rb.loglike_grad(event, torch.tensor(th, device="cuda"), mode="mixed")
    idx = np.linspace(0, th.shape[0] - 1, 1024).astype(int)
    ref, dh, hh = _terms(ev, s, th[idx])
    assert np.all(np.abs(L.cpu().numpy()[idx] - ref) <= _tol("mixed", dh, hh))
    _, ref_G = oracle.loglike_rb(ev, s, th[idx], grad=True)
    n_floor = _check_prior_gradients(ev, s, edges, th[idx], G.cpu().numpy()[idx], ref_G, "mixed")
    assert n_floor <= 8, n_floor
    event.free()


def test_autograd_function(rb, small):
    th = torch.tensor(synth.draw_box(small.ev["theta_inj"], 16, seed=91, rel=1e-3,
                                     abs_width=1e-3 * synth.PRIOR_WIDTH), device="cuda", requires_grad=True)
    L = rb.rb_loglike(th, small.event, "mixed")
    w = torch.linspace(0.5, 2.0, 16, dtype=torch.float64, device="cuda")
    (L * w).sum().backward()
    _, G = rb.loglike_grad(small.event, th.detach(), mode="mixed")
    torch.testing.assert_close(th.grad, w[:, None] * G, rtol=0, atol=0)


def test_host_entry_point_matches_device(rb, small):
    th = synth.draw_box(small.ev["theta_inj"], 100, seed=101, rel=1e-3, abs_width=1e-3 * synth.PRIOR_WIDTH)
    Ld, Gd = rb.loglike_grad(small.event, torch.tensor(th, device="cuda"), mode="mixed")
    Lh = np.zeros(100)
    Gh = np.zeros((100, 13))
    rb.loglike_grad_host(small.event, th, Lh, Gh, mode="mixed")
    np.testing.assert_array_equal(Lh, Ld.cpu().numpy())
    np.testing.assert_array_equal(Gh, Gd.cpu().numpy())
    # pinned walkers and outputs: read and written by the kernels over the host link
    th_p = torch.tensor(th).pin_memory()
    Lp = torch.zeros(100, dtype=torch.float64).pin_memory()
    Gp = torch.zeros(100, 13, dtype=torch.float64).pin_memory()
    for mode in ("mixed", "fp64", "mixed"):
        Ld, Gd = rb.loglike_grad(small.event, torch.tensor(th, device="cuda"), mode=mode)
        for _ in range(3):  # launched directly, then replayed from the graph captured for these buffers
            Lp.zero_()
            Gp.zero_()
            rb.loglike_grad_host(small.event, th_p, Lp, Gp, mode=mode)
            np.testing.assert_array_equal(Lp.numpy(), Ld.cpu().numpy())
            np.testing.assert_array_equal(Gp.numpy(), Gd.cpu().numpy())
    # new walkers in the same pinned buffer: the replay reads them
    th2 = synth.draw_box(small.ev["theta_inj"], 100, seed=103, rel=1e-3, abs_width=1e-3 * synth.PRIOR_WIDTH)
    th_p.copy_(torch.tensor(th2))
    Ld, Gd = rb.loglike_grad(small.event, torch.tensor(th2, device="cuda"), mode="mixed")
    rb.loglike_grad_host(small.event, th_p, Lp, Gp, mode="mixed")
    np.testing.assert_array_equal(Lp.numpy(), Ld.cpu().numpy())
    np.testing.assert_array_equal(Gp.numpy(), Gd.cpu().numpy())


def test_library_errors(rb, small):
    with pytest.raises(rb.RBError) as e:
        rb.loglike(small.event, torch.zeros(4, 13, dtype=torch.float64, device="cuda"), mode=7)
    assert e.value.status == rb.RB_EINVAL
    ev = dict(small.ev)
    with pytest.raises(rb.RBError):
        rb.Event.from_synth(ev, n_bins=ev["N"])  # more bins than grid intervals
    bad = np.array(ev["theta_inj"])
    bad[1] = 2.0
    with pytest.raises(rb.RBError):
        rb.Event.from_synth(ev, n_bins=10, theta_ref=bad)


def test_reference_loglike_across_build_kinds(rb, c2):
    """log L(theta_ref) through a sequence of builds of every kind (the fast
    build leaves it as a fixed-point sum that its readers convert, the FP64
    builds store it): after each, rb_event_get_info and a batch of walkers at
    theta_ref agree bit for bit in every mode, and the value matches the full
    likelihood at theta_ref (FP64 builds: 1e-9 relative; fast build: the
    FP32 summary's 2e-6 of the shares' scale)."""
    ev = c2.ev
    event = rb.Event.from_synth(ev)
    full = oracle.loglike_full(ev, ev["theta_inj"])[0]
    th = torch.tensor(np.tile(ev["theta_inj"], (40, 1)), device="cuda")
    scale = abs(full) + np.sum(np.abs(c2.s["B0"]))
    steps = [dict(mode="mixed"), dict(mode="fp64", theta_ref=ev["theta_inj"]), dict(mode="fp64"),
             dict(mode="mixed"), dict(mode="mixed"), dict(mode="fp64")]
    for kw in steps:
        event.rebuild(**kw)
        base = event.info()["base_logl"]
        tol = 1e-9 * abs(full) if kw["mode"] == "fp64" else 2e-6 * scale
        assert abs(base - full) <= tol, (kw, base, full)
        for mode in MODES:
            L = rb.loglike(event, th, mode=mode).cpu().numpy()
            assert np.all(L == base), (kw, mode)
    event.free()


# ---------------------------------------------------------------------------
# In-place rebuild (rb_event_rebuild): FP64 and fast (Taylor-chunk) summary
# ---------------------------------------------------------------------------
def _summary_close(g, ref, rel, b1_cond=None):
    """Every entry within rel of the largest entry of its detector.  With
    b1_cond (the FP32 fast build), B1 = 4 df sum |h0|^2 / S (f - f_m), whose
    terms change sign inside every bin, may instead be off by rel times the
    sum of the absolute values of its terms (its condition number: rounding
    of the terms, not of the sum, sets the error)."""
    for key in ("A0", "A1", "B0", "B1"):
        scale = np.max(np.abs(ref[key]), axis=1, keepdims=True)
        if key == "B1" and b1_cond is not None:
            scale = np.maximum(scale, b1_cond)
        err = np.max(np.abs(g[key] - ref[key]) / scale)
        assert err <= rel, (key, err)


def _b1_condition(ev, theta_ref, edges):
    """[D][B] sum over each bin of |4 df |h0|^2 / S (f - f_m)| (oracle waveform)."""
    f, T = ev["f"], ev["T"]
    D, B = ev["geom"].shape[0], len(edges) - 1
    out = np.zeros((D, B))
    for d in range(D):
        h0 = oracle.strain(theta_ref, ev["geom"][d], ev["gmst"], f)
        w = 4.0 / T * np.abs(h0) ** 2 / ev["psd"][d]
        for b in range(B):
            k0, k1 = edges[b], (edges[b + 1] + 1 if b == B - 1 else edges[b + 1])
            fm = 0.5 * (f[edges[b]] + f[edges[b + 1]])
            out[d, b] = np.sum(w[k0:k1] * np.abs(f[k0:k1] - fm))
    return out


def test_rebuild_fp64_is_bitwise_reproducible(rb, c2):
    def twice(**kw):
        c2.event.rebuild(mode="fp64", **kw)
        first = c2.event.summary()
        c2.event.rebuild(mode="fp64", **kw)
        return first, c2.event.summary()

    # streamed from the stored waveform, then generated inline (a theta_ref
    # argument discards the stored waveform)
    for before, after in (twice(), twice(theta_ref=c2.event.theta_ref)):
        for key in ("A0", "A1", "B0", "B1"):
            np.testing.assert_array_equal(before[key], after[key])


@pytest.mark.parametrize("cfg", ["C1", "C2", "C4"])
def test_fast_rebuild_summary_matches_oracle(rb, cfg):
    ev = inject(synth.make_event(cfg))
    B = ev["n_bins"]
    event = rb.Event.from_synth(ev, n_bins=B)
    edges = oracle.bin_edges(ev, B)
    s = oracle.summary(ev, ev["theta_inj"], edges)
    event.rebuild(mode="mixed")
    _summary_close(event.summary(), s, 2e-6, _b1_condition(ev, ev["theta_inj"], edges))
    th = synth.walkers(cfg, 512) if cfg != "C1" else synth.walkers("C1", 512)
    L = rb.loglike(event, torch.tensor(th, device="cuda"), mode="mixed").cpu().numpy()
    ref, dh, hh = _terms(ev, s, th)
    assert np.all(np.abs(L - ref) <= _tol("mixed", dh, hh, near=cfg == "C1"))
    thp = synth.posterior_box(ev["theta_inj"], 128, seed=111)
    L = rb.loglike(event, torch.tensor(thp, device="cuda"), mode="mixed").cpu().numpy()
    ref, dh, hh = _terms(ev, s, thp)
    assert np.all(np.abs(L - ref) <= _tol("mixed", dh, hh, near=True))
    event.free()


def test_fp64_build_from_stored_waveform(rb):
    """An FP64 build that generates h0 inline stores it for its theta_ref; the
    next FP64 builds with the same theta_ref stream strain, PSD and h0 instead.
    Both match the oracle, agree to rounding, and a new theta_ref (or new data
    read in place) is handled."""
    ev = inject(synth.make_event("C2", T=16.0, f_high=1024.0))
    B = 120
    edges = oracle.bin_edges(ev, B)
    event = rb.Event.from_synth(ev, n_bins=B)  # inline FP64 build
    inline = event.summary()
    base_inline = event.info()["base_logl"]
    s = oracle.summary(ev, ev["theta_inj"], edges)
    _summary_close(inline, s, 1e-9)
    event.rebuild(mode="fp64")  # stored waveform
    stored = event.summary()
    _summary_close(stored, s, 1e-9)
    _summary_close(stored, inline, 1e-11)
    # the streamed build adds the bins' shares of log L(theta_ref) in fixed
    # point (2^-32 per bin), the inline one in FP64
    assert abs(event.info()["base_logl"] - base_inline) <= 1e-9 * abs(base_inline)
    th = synth.posterior_box(ev["theta_inj"], 64, seed=131)
    L = rb.loglike(event, torch.tensor(th, device="cuda"), mode="fp64").cpu().numpy()
    ref, dh, hh = _terms(ev, s, th)
    assert np.all(np.abs(L - ref) <= _tol("fp64", dh, hh))
    # a new reference point: generated inline again (and stored), then streamed
    new_ref = synth.posterior_box(ev["theta_inj"], 1, seed=133)[0]
    s2 = oracle.summary(ev, new_ref, edges)
    event.rebuild(theta_ref=new_ref, mode="fp64")
    _summary_close(event.summary(), s2, 1e-9)
    event.rebuild(mode="fp64")
    _summary_close(event.summary(), s2, 1e-9)
    assert abs(event.info()["base_logl"] - oracle.loglike_full(ev, new_ref)[0]) <= 1e-9 * abs(event.info()["base_logl"])
    # new data read in place by the streamed build
    D = ev["geom"].shape[0]
    new = ev["noise"] * 0.5 + ev["signal"]
    ev3 = dict(ev)
    ev3["data"] = new
    dd = [torch.tensor(np.stack([new[d].real, new[d].imag], -1), device="cuda") for d in range(D)]
    pp = [torch.tensor(ev["psd"][d], device="cuda") for d in range(D)]
    event.rebuild(data=dd, psd=pp, mode="fp64")
    torch.cuda.synchronize()
    _summary_close(event.summary(), oracle.summary(ev3, new_ref, edges), 1e-9)
    event.free()


def test_event_save_and_load_round_trip(rb, tmp_path):
    """A saved event loads as a bit-identical event: summary data, edges, base
    log L and every log L / gradient, including a theta_ref changed after the
    build; a truncated file is refused."""
    ev = inject(synth.make_event("C2", T=64.0, sites=("H1", "V1")))
    event = rb.Event.from_synth(ev, n_bins=140)
    new_ref = synth.posterior_box(ev["theta_inj"], 1, seed=151)[0]
    event.rebuild(theta_ref=new_ref, mode="mixed")
    path = tmp_path / "event.rbev"
    event.save(path)
    loaded = rb.Event.load(path)
    event.rebuild(mode="fp64")  # both from the FP64 build, as the loaded event's build
    a, b = event.summary(), loaded.summary()
    for k in ("A0", "A1", "B0", "B1", "edges"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    ia, ib = event.info(), loaded.info()
    assert ia["base_logl"] == ib["base_logl"] and ia["n_freq"] == ib["n_freq"] and ia["kmin"] == ib["kmin"]
    np.testing.assert_array_equal(ib["theta_ref"], new_ref)
    th = torch.tensor(synth.posterior_box(ev["theta_inj"], 200, seed=153), device="cuda")
    for mode in MODES:
        La, Ga = rb.loglike_grad(event, th, mode=mode)
        Lb, Gb = rb.loglike_grad(loaded, th, mode=mode)
        torch.testing.assert_close(La, Lb, rtol=0, atol=0)
        torch.testing.assert_close(Ga, Gb, rtol=0, atol=0)
    raw = path.read_bytes()
    cut = tmp_path / "cut.rbev"
    cut.write_bytes(raw[:-8])
    with pytest.raises(rb.RBError):
        rb.Event.load(cut)
    loaded.free()
    event.free()


def test_rebuild_new_reference_and_data(rb, c1):
    ev = c1.ev
    event = rb.Event.from_synth(ev)
    new_ref = synth.posterior_box(ev["theta_inj"], 1, seed=121)[0]
    new_data = ev["noise"] * 0.5 + ev["signal"]
    ev2 = dict(ev)
    ev2["data"] = new_data
    s = oracle.summary(ev2, new_ref, c1.edges)
    # host data (copied in), FP64 sums
    host = [np.ascontiguousarray(np.stack([new_data[d].real, new_data[d].imag], -1)) for d in range(1)]
    event.rebuild(theta_ref=new_ref, data=host, psd=[ev["psd"][0]], mode="fp64")
    _summary_close(event.summary(), s, 1e-9)
    assert abs(event.info()["base_logl"] - oracle.loglike_full(ev2, new_ref)[0]) <= 1e-9 * abs(event.info()["base_logl"])
    # device data read in place, fast sums
    dd = [torch.tensor(h, device="cuda") for h in host]
    pp = [torch.tensor(ev["psd"][0], device="cuda")]
    event.rebuild(data=dd, psd=pp, mode="mixed")
    torch.cuda.synchronize()
    _summary_close(event.summary(), s, 2e-6, _b1_condition(ev2, new_ref, c1.edges))
    event.free()


# ---------------------------------------------------------------------------
# Rebuild + batch in one call (rb_rebuild_loglike_grad): the walkers' set-up
# overlapped with the summary sums gives the results of the two calls
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mode", MODES)
def test_rebuild_and_batch_equals_two_calls(rb, c2, small, mode):
    for c in (c2, small):  # the chunk-expanded rebuild, and one that falls back to the FP64 sums
        th = torch.tensor(synth.posterior_box(c.ev["theta_inj"], 333, seed=91), device="cuda")
        c.event.rebuild(mode=mode)
        L1, G1 = rb.loglike_grad(c.event, th, mode=mode)
        L2, G2 = rb.rebuild_loglike_grad(c.event, th, mode=mode)
        torch.testing.assert_close(L2, L1, rtol=0, atol=0)
        torch.testing.assert_close(G2, G1, rtol=0, atol=0)
        L3 = rb.rebuild_loglike_grad(c.event, th, mode=mode, grad=False)
        torch.testing.assert_close(L3, rb.loglike(c.event, th, mode=mode), rtol=0, atol=0)


def test_rebuild_and_batch_in_a_cuda_graph(rb, c2):
    th = torch.tensor(synth.walkers("C2", 1000), device="cuda")
    L_ref, G_ref = rb.rebuild_loglike_grad(c2.event, th)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        out = rb.rebuild_loglike_grad(c2.event, th)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        L, G = rb.rebuild_loglike_grad(c2.event, th)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(L, L_ref, rtol=0, atol=0)
    torch.testing.assert_close(G, G_ref, rtol=0, atol=0)
    # empty batch: only the rebuild
    assert rb.rebuild_loglike_grad(c2.event, th[:0])[0].numel() == 0


@pytest.mark.parametrize("mode", MODES)
def test_rebuild_and_batch_host_equals_two_calls(rb, c2, mode):
    """Host-buffer step (data copied on the copy stream while the data-free
    kernels run) against rb_event_rebuild(host data) + rb_loglike_grad_host."""
    ev = c2.ev
    D = ev["geom"].shape[0]
    new = ev["noise"] * 0.5 + ev["signal"]
    data = [torch.tensor(np.stack([new[d].real, new[d].imag], -1)).pin_memory() for d in range(D)]
    psd = [torch.tensor(ev["psd"][d]).pin_memory() for d in range(D)]
    th = synth.posterior_box(ev["theta_inj"], 257, seed=97)
    L1, G1 = np.zeros(257), np.zeros((257, 13))
    c2.event.rebuild(data=[d.numpy() for d in data], psd=[p.numpy() for p in psd], mode=mode)
    rb.loglike_grad_host(c2.event, th, L1, G1, mode=mode)
    L2, G2 = np.zeros(257), np.zeros((257, 13))
    rb.rebuild_loglike_grad_host(c2.event, data, psd, th, L2, G2, mode=mode)
    np.testing.assert_array_equal(L2, L1)
    np.testing.assert_array_equal(G2, G1)
    # log L only, then back to the original data (the module's other tests use it)
    L3 = np.zeros(257)
    rb.rebuild_loglike_grad_host(c2.event, data, psd, th, L3, None, mode=mode)
    np.testing.assert_array_equal(L3, L1)
    orig = [np.ascontiguousarray(np.stack([ev["data"][d].real, ev["data"][d].imag], -1)) for d in range(D)]
    c2.event.rebuild(data=orig, psd=[ev["psd"][d] for d in range(D)], mode="fp64")


def _pinned(a, offset):
    """Pinned float64 copy of `a` that starts `offset` elements into its allocation."""
    flat = np.ascontiguousarray(a, dtype=np.float64).ravel()
    t = torch.empty(flat.size + 2, dtype=torch.float64).pin_memory()
    v = t[offset:offset + flat.size]
    v.copy_(torch.from_numpy(flat))
    return v


@pytest.fixture(scope="module")
def two64(rb):
    # two detectors on a grid long enough (T f_low >= 1024) for the chunk-expanded summary
    return Case(rb, "C2", n_bins=150, T=64.0, sites=("L1", "V1"))


@pytest.mark.parametrize("case", ["c2", "two64"])
def test_host_step_mapped_equals_copied(rb, case, request):
    """The host-buffer step reads 16-byte-aligned pinned buffers in the summary
    kernel itself (conversion, resident copies and sums in one pass over the
    host link); other buffers are copied in first.  Both give the same bits,
    and leave the same resident data behind."""
    c = request.getfixturevalue(case)
    ev = c.ev
    D = ev["geom"].shape[0]
    new = ev["noise"] * 0.7 + ev["signal"]
    arrs = [np.stack([new[d].real, new[d].imag], -1) for d in range(D)]
    th = synth.posterior_box(ev["theta_inj"], 300, seed=41)
    outs = {}
    for name, (data, psd) in {
        "mapped": ([_pinned(a, 0) for a in arrs], [_pinned(ev["psd"][d], 0) for d in range(D)]),
        "pinned, 8-byte offset": ([_pinned(a, 1) for a in arrs], [_pinned(ev["psd"][d], 1) for d in range(D)]),
        "pageable": (arrs, [ev["psd"][d] for d in range(D)]),
    }.items():
        L, G = np.zeros(300), np.zeros((300, 13))
        rb.rebuild_loglike_grad_host(c.event, data, psd, th, L, G, mode="mixed")
        # what the step left resident: the batch on the resident copy, the
        # FP64 summary and the full-grid sum (FP32 copy)
        Ld, Gd = rb.rebuild_loglike_grad(c.event, torch.tensor(th, device="cuda"))
        Lf = rb.loglike_full(c.event, torch.tensor(th[:8], device="cuda"))
        outs[name] = (L, G, Ld.cpu().numpy(), Gd.cpu().numpy(), c.event.summary(), Lf.cpu().numpy())
    ref = outs["pageable"]
    np.testing.assert_array_equal(ref[2], ref[0])
    np.testing.assert_array_equal(ref[3], ref[1])
    # pinned outputs are written by the likelihood kernel itself
    data, psd = [_pinned(a, 0) for a in arrs], [_pinned(ev["psd"][d], 0) for d in range(D)]
    Lp = torch.zeros(300, dtype=torch.float64).pin_memory()
    Gp = torch.zeros(300, 13, dtype=torch.float64).pin_memory()
    rb.rebuild_loglike_grad_host(c.event, data, psd, th, Lp, Gp, mode="mixed")
    np.testing.assert_array_equal(Lp.numpy(), ref[0])
    np.testing.assert_array_equal(Gp.numpy(), ref[1])
    Lp.zero_()
    rb.rebuild_loglike_grad_host(c.event, data, psd, th, Lp, None, mode="mixed")
    np.testing.assert_array_equal(Lp.numpy(), ref[0])
    Lp.zero_()
    Gp.zero_()
    rb.loglike_grad_host(c.event, th, Lp, Gp, mode="mixed")
    np.testing.assert_array_equal(Lp.numpy(), ref[0])
    np.testing.assert_array_equal(Gp.numpy(), ref[1])
    # everything pinned, the same buffers call after call: launched directly,
    # then replayed from the graph captured for them -- which reads what the
    # buffers hold at each call
    th_p = torch.tensor(th).pin_memory()
    for _ in range(3):
        Lp.zero_()
        Gp.zero_()
        rb.rebuild_loglike_grad_host(c.event, data, psd, th_p, Lp, Gp, mode="mixed")
        np.testing.assert_array_equal(Lp.numpy(), ref[0])
        np.testing.assert_array_equal(Gp.numpy(), ref[1])
    new2 = ev["noise"] * 0.4 + ev["signal"]
    arrs2 = [np.stack([new2[d].real, new2[d].imag], -1) for d in range(D)]
    for d in range(D):
        data[d].copy_(torch.from_numpy(np.ascontiguousarray(arrs2[d]).ravel()).view_as(data[d]))
    rb.rebuild_loglike_grad_host(c.event, data, psd, th_p, Lp, Gp, mode="mixed")
    L2, G2 = np.zeros(300), np.zeros((300, 13))
    rb.rebuild_loglike_grad_host(c.event, arrs2, [ev["psd"][d] for d in range(D)], th, L2, G2, mode="mixed")
    np.testing.assert_array_equal(Lp.numpy(), L2)
    np.testing.assert_array_equal(Gp.numpy(), G2)
    assert not np.array_equal(L2, ref[0])
    for name, o in outs.items():
        for i in (0, 1, 2, 3, 5):
            np.testing.assert_array_equal(o[i], ref[i], err_msg=name)
        for k in ("A0", "A1", "B0", "B1"):
            np.testing.assert_array_equal(o[4][k], ref[4][k], err_msg=f"{name} {k}")
    orig = [np.ascontiguousarray(np.stack([ev["data"][d].real, ev["data"][d].imag], -1)) for d in range(D)]
    c.event.rebuild(data=orig, psd=[ev["psd"][d] for d in range(D)], mode="fp64")


def test_rebuild_and_batch_graph_survives_workspace_growth(rb, c2):
    """A graph captured with the event's workspace stays valid after a larger
    eager call grows it (outgrown workspaces live as long as the event)."""
    ev = inject(synth.make_event("C2", T=32.0))
    event = rb.Event.from_synth(ev, n_bins=150)
    small = torch.tensor(synth.posterior_box(ev["theta_inj"], 300, seed=5), device="cuda")
    big = torch.tensor(synth.posterior_box(ev["theta_inj"], 2000, seed=6), device="cuda")
    L0, G0 = rb.rebuild_loglike_grad(event, small)  # eager: allocates the event's workspace
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rb.rebuild_loglike_grad(event, small)
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        L, G = rb.rebuild_loglike_grad(event, small)
    Lb, Gb = rb.rebuild_loglike_grad(event, big)  # grows the workspace
    Lb2, Gb2 = rb.loglike_grad(event, big)
    torch.testing.assert_close(Lb, Lb2, rtol=0, atol=0)
    g.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(L, L0, rtol=0, atol=0)
    torch.testing.assert_close(G, G0, rtol=0, atol=0)
    del g
    event.free()


def test_rebuild_and_batch_errors(rb, c2):
    th = torch.tensor(np.array(c2.ev["theta_inj"])[None], device="cuda")
    with pytest.raises(rb.RBError) as e:
        rb.rebuild_loglike_grad(c2.event, th, mode=9)
    assert e.value.status == rb.RB_EINVAL
    lib = rb.load()
    D = c2.ev["geom"].shape[0]
    null = (ctypes.c_void_p * D)()
    L = np.zeros(1)
    rc = lib.rb_rebuild_loglike_grad_host(c2.event.handle, null, null, ctypes.c_void_p(th.cpu().numpy().ctypes.data), 1,
                                          ctypes.c_void_p(L.ctypes.data), None, rb.RB_MIXED, None)
    assert rc == rb.RB_EINVAL and b"NULL data/psd" in lib.rb_last_error()
