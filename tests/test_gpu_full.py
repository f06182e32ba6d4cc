"""Full-grid (un-binned) log-likelihood on the GPU (rb_loglike_full_batch)
against the oracle's direct sum of Eq. 2 with the inner product of Eq. 3 over
every grid point (Sec. II.C: the quantity relative binning approximates).

Tolerance.  <h|h> is exact up to FP64 rounding (the Newtonian amplitude
makes it |K_d|^2 times a theta-free sum).  Each term of <d|h> carries FP32
errors: the data copy and the amplitude series (~1e-7 relative), the phase
(the fractional turn is rounded to FP32, ~4e-7 rad) and the per-lane FP32
sum of <= 32 terms before the float-pair accumulation (<= 31 u ~ 1.9e-6 of
the absolute sum).  So |error| <= 3e-6 * S_abs + 1e-3, where
S_abs = 4 df sum_d |K_d| sum_k |d_k| f_k^-7/6 / S_k bounds the sum of
|terms| (|h_d(f)| = |K_d| f^-7/6 does not depend on the phase)."""
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


class Case:
    def __init__(self, rb, cfg, n_bins=None, **kw):
        self.ev = inject(synth.make_event(cfg, **kw))
        self.n_bins = n_bins or self.ev["n_bins"]
        self.event = rb.Event.from_synth(self.ev, n_bins=self.n_bins)
        f = self.ev["f"]
        # G_d = sum_k |d_k| f_k^-7/6 / S_k per detector
        self.G = np.array([np.sum(np.abs(self.ev["data"][d]) * f ** (-7.0 / 6.0) / self.ev["psd"][d])
                           for d in range(self.ev["geom"].shape[0])])

    def abs_sum(self, theta):
        """S_abs per walker: 4 df sum_d |K_d(theta)| G_d, |K_d| = |h_d(f)| f^7/6 at one grid point."""
        ev = self.ev
        f1 = ev["f"][:1]
        out = np.zeros(theta.shape[0])
        for w, th in enumerate(theta):
            if not np.all(np.isfinite(th)):
                continue
            for d in range(ev["geom"].shape[0]):
                K = abs(oracle.strain(th, ev["geom"][d], ev["gmst"], f1)[0]) * f1[0] ** (7.0 / 6.0)
                out[w] += 4.0 / ev["T"] * K * self.G[d]
        return out

    def check(self, rb, theta, L=None):
        if L is None:
            L = rb.loglike_full(self.event, torch.tensor(theta, device="cuda")).cpu().numpy()
        ref = oracle.loglike_full(self.ev, theta)
        tol = 1e-3 + 3e-6 * self.abs_sum(theta)
        err = np.abs(L - ref)
        assert np.all(err <= tol), (err.max(), np.argmax(err / tol), (err / tol).max())
        return L, ref


@pytest.fixture(scope="module")
def c1(rb):
    c = Case(rb, "C1")
    yield c
    c.event.free()


@pytest.fixture(scope="module")
def c2(rb):
    # three detectors, T = 64 s: ~130k grid points (127 segments of 1024 + a ragged tail)
    c = Case(rb, "C2", n_bins=300, T=64.0)
    yield c
    c.event.free()


def test_full_at_reference_matches_binned_and_oracle(rb, c1, c2):
    """At theta_ref relative binning is exact: full, binned and oracle agree."""
    for c in (c1, c2):
        th = np.array(c.ev["theta_inj"])[None]
        L, ref = c.check(rb, th)
        base = c.event.info()["base_logl"]
        assert abs(L[0] - base) <= 1e-3 + 3e-6 * c.abs_sum(th)[0]


def test_full_posterior_walkers(rb, c1, c2):
    for c, W in ((c1, 257), (c2, 200)):
        th = synth.posterior_box(c.ev["theta_inj"], W, seed=43)
        c.check(rb, th)


def test_full_prior_draws(rb, c2):
    """Prior draws: phases far from the reference (the binned likelihood's hard case)."""
    th = synth.walkers("C2", 300)
    c2.check(rb, th)


def test_full_box_walkers_single_detector(rb, c1):
    th = synth.walkers("C1", 333)
    c1.check(rb, th)


def test_full_size_event_sampled(rb):
    """C2 at its full size (T = 128 s, 3 detectors, ~260k points); 64 walkers of one launch of 1024."""
    c = Case(rb, "C2")
    th = synth.walkers("C2", 1024)
    L = rb.loglike_full(c.event, torch.tensor(th, device="cuda")).cpu().numpy()
    idx = np.linspace(0, th.shape[0] - 1, 64).astype(int)
    c.check(rb, th[idx], L[idx])
    c.event.free()


def test_full_unphysical_and_shapes(rb, c2):
    th = np.tile(c2.ev["theta_inj"], (6, 1))
    th[0, 1] = 1.5
    th[1, 1] = -0.1
    th[2, 6] = 0.0
    th[3, 0] = np.nan
    th[4, 11] = np.inf
    L = rb.loglike_full(c2.event, torch.tensor(th, device="cuda")).cpu().numpy()
    assert np.all(np.isneginf(L[:5])) and np.isfinite(L[5])
    # W = 0 is a no-op; one walker and a ragged slice give the same values (warp per walker)
    empty = rb.loglike_full(c2.event, torch.zeros(0, 13, dtype=torch.float64, device="cuda"))
    assert empty.numel() == 0
    pw = synth.posterior_box(c2.ev["theta_inj"], 37, seed=47)
    full = rb.loglike_full(c2.event, torch.tensor(pw, device="cuda")).cpu().numpy()
    one = rb.loglike_full(c2.event, torch.tensor(pw[9:10], device="cuda")).cpu().numpy()
    assert one[0] == full[9]
    part = rb.loglike_full(c2.event, torch.tensor(pw[3:30], device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(part, full[3:30])


def test_full_follows_rebuilds(rb):
    """The data used are the ones the last rebuild summed over; an FP64 rebuild
    from data read in place leaves no FP32 copy and is refused."""
    c = Case(rb, "C1", n_bins=80)
    th = synth.posterior_box(c.ev["theta_inj"], 64, seed=53)
    # fresh event (built by the FP64 sums): the resident data are converted on
    # demand; <h|h> takes sum_b B0 from whichever summary was built last (FP64
    # here, the FP32 chunk sums after a mixed rebuild), so the two agree to
    # the summary's rounding
    L0 = rb.loglike_full(c.event, torch.tensor(th, device="cuda")).cpu().numpy()
    c.event.rebuild(mode="mixed")
    L1 = rb.loglike_full(c.event, torch.tensor(th, device="cuda")).cpu().numpy()
    assert np.all(np.abs(L0 - L1) <= 1e-3 + 3e-6 * c.abs_sum(th))
    # new data copied in from the host
    ev2 = inject(dict(c.ev), scale=0.5)
    host = [np.ascontiguousarray(np.stack([ev2["data"][0].real, ev2["data"][0].imag], -1))]
    c.event.rebuild(data=host, psd=[ev2["psd"][0]], mode="fp64")
    L2 = rb.loglike_full(c.event, torch.tensor(th, device="cuda")).cpu().numpy()
    ref = oracle.loglike_full(ev2, th)
    assert np.all(np.abs(L2 - ref) <= 1e-3 + 3e-6 * c.abs_sum(th) * 2)
    # data read in place: fine after a mixed rebuild, refused after an FP64 one
    d = torch.tensor(np.stack([c.ev["data"][0].real, c.ev["data"][0].imag], -1), device="cuda")
    p = torch.tensor(c.ev["psd"][0], device="cuda")
    c.event.rebuild(data=[d], psd=[p], mode="mixed")
    L3 = rb.loglike_full(c.event, torch.tensor(th, device="cuda")).cpu().numpy()
    np.testing.assert_array_equal(L3, L1)
    c.event.rebuild(data=[d], psd=[p], mode="fp64")
    with pytest.raises(rb.RBError) as e:
        rb.loglike_full(c.event, torch.tensor(th, device="cuda"))
    assert e.value.status == rb.RB_EINVAL
    c.event.free()


def test_full_errors(rb, c1):
    th = torch.tensor(np.array(c1.ev["theta_inj"])[None], device="cuda")
    for mode in ("fp64", "mixed_f64phase"):
        with pytest.raises(rb.RBError) as e:
            rb.loglike_full(c1.event, th, mode=mode)
        assert e.value.status == rb.RB_EINVAL
    # T f_low < 1024: outside the chunk expansion's range
    ev = inject(synth.make_event("C2", T=8.0, f_low=20.0, f_high=512.0))
    event = rb.Event.from_synth(ev, n_bins=45)
    with pytest.raises(rb.RBError) as e:
        rb.loglike_full(event, th)
    assert e.value.status == rb.RB_EINVAL
    event.free()
