"""What the Python binding hands the C ABI for host inputs, checked on the CPU.

A stand-in for the loaded library records the pointers each call receives and
reads the float64 values behind them; the test compares those bytes with the
strain, PSD and walkers it passed in, for every accepted input form (complex
or (re, im) float pairs, numpy or CPU tensors).  No library call is made."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2404_11397_gb300 import api

T, F_LOW, F_HIGH = 4.0, 20.0, 30.0
N = int(F_HIGH * T) - int(F_LOW * T) + 1  # the grid 80/T .. 120/T, both ends included


def _read(ptr: int, n: int) -> np.ndarray:
    return np.ctypeslib.as_array((ctypes.c_double * n).from_address(ptr)).copy()


class _FakeLib:
    """Records the host buffers of rb_build_summary, rb_event_rebuild,
    rb_rebuild_loglike_grad_host and rb_loglike_grad_host; every call succeeds."""

    def __init__(self):
        self.seen = {}

    def rb_build_summary(self, desc_ref, handle_ref):
        desc = desc_ref._obj
        self.seen["on_device"] = desc.data_on_device
        self.seen["data"] = [_read(desc.det[d].data, 2 * N) for d in range(desc.n_det)]
        self.seen["psd"] = [_read(desc.det[d].psd, N) for d in range(desc.n_det)]
        handle_ref._obj.value = 1
        return 0

    def rb_event_get_info(self, handle, info_ref):
        info_ref._obj.n_freq = N
        return 0

    def rb_event_rebuild(self, handle, th_p, dp, pp, on_dev, mode, stream):
        self.seen["on_device"] = on_dev
        self.seen["data"] = [_read(dp[d], 2 * N) for d in range(len(dp))]
        self.seen["psd"] = [_read(pp[d], N) for d in range(len(pp))]
        return 0

    def rb_rebuild_loglike_grad_host(self, handle, dp, pp, th, W, lo, gr, mode, stream):
        self.seen["data"] = [_read(dp[d], 2 * N) for d in range(len(dp))]
        self.seen["psd"] = [_read(pp[d], N) for d in range(len(pp))]
        self.seen["theta"] = _read(th.value, W * 13).reshape(W, 13)
        self.seen["ptrs"] = (lo.value, gr.value if gr is not None else None)
        return 0

    def rb_loglike_grad_host(self, handle, th, W, lo, gr, mode, stream):
        self.seen["theta"] = _read(th.value, W * 13).reshape(W, 13)
        self.seen["ptrs"] = (lo.value, gr.value if gr is not None else None)
        return 0


class _Stream:
    cuda_stream = 0


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(api, "load", lambda: lib)
    return lib


def _forms(c):
    ri = np.stack([c.real, c.imag], axis=-1)
    return {"complex": c, "re-im pairs": ri, "complex tensor": torch.from_numpy(c.copy()),
            "re-im tensor": torch.from_numpy(ri.copy()), "flat pairs": ri.ravel()}


def test_event_and_rebuild_pass_both_strain_components(fake):
    rng = np.random.default_rng(11)
    geom = np.array([[0.8, -1.5, 100.0, 2.0, 0.4], [0.5, -1.6, 10.0, 4.0, 2.5]])
    c = rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))
    psd = 1.0 + rng.random((2, N))
    expect = [np.stack([c[d].real, c[d].imag], axis=-1).ravel() for d in range(2)]
    for name in _forms(c[0]):
        data = [_forms(c[d])[name] for d in range(2)]
        ev = api.Event(geom, 1.0, T, F_LOW, F_HIGH, data, list(psd), 10, np.zeros(13))
        try:
            assert fake.seen["on_device"] == 0 and ev.n_freq == N
            for d in range(2):
                np.testing.assert_array_equal(fake.seen["data"][d], expect[d], err_msg=name)
                np.testing.assert_array_equal(fake.seen["psd"][d], psd[d], err_msg=name)
            ev.rebuild(data=data, psd=[torch.from_numpy(psd[0]), psd[1]], stream=_Stream())
            assert fake.seen["on_device"] == 0
            for d in range(2):
                np.testing.assert_array_equal(fake.seen["data"][d], expect[d], err_msg=name)
                np.testing.assert_array_equal(fake.seen["psd"][d], psd[d], err_msg=name)
        finally:
            ev._h = None  # a stand-in handle: nothing to free


def test_host_step_passes_strain_walkers_and_outputs(fake):
    rng = np.random.default_rng(12)
    geom = np.array([[0.8, -1.5, 100.0, 2.0, 0.4]])
    c = rng.normal(size=N) + 1j * rng.normal(size=N)
    psd = 1.0 + rng.random(N)
    ev = api.Event(geom, 1.0, T, F_LOW, F_HIGH, [c], [psd], 10, np.zeros(13))
    try:
        th = rng.normal(size=(6, 13))
        expect = np.stack([c.real, c.imag], axis=-1).ravel()
        for name, data in _forms(c).items():
            L, G = np.zeros(6), torch.zeros(6, 13, dtype=torch.float64)
            for theta in (th, torch.from_numpy(th.copy())):
                api.rebuild_loglike_grad_host(ev, [data], [psd], theta, L, G, stream=_Stream())
                np.testing.assert_array_equal(fake.seen["data"][0], expect, err_msg=name)
                np.testing.assert_array_equal(fake.seen["psd"][0], psd)
                np.testing.assert_array_equal(fake.seen["theta"], th)
                assert fake.seen["ptrs"] == (L.ctypes.data, G.data_ptr())  # outputs passed in place
        L, G = torch.zeros(6, dtype=torch.float64), np.zeros((6, 13))
        api.loglike_grad_host(ev, torch.from_numpy(th.copy()), L, None, stream=_Stream())
        np.testing.assert_array_equal(fake.seen["theta"], th)
        assert fake.seen["ptrs"] == (L.data_ptr(), None)
        api.loglike_grad_host(ev, th, L, G, stream=_Stream())
        assert fake.seen["ptrs"] == (L.data_ptr(), G.ctypes.data)
        for bad in ((th[:, :12], L, G), (th, np.zeros(5), G), (th, L, np.zeros((6, 12))), (th, L.float(), G)):
            with pytest.raises(ValueError):
                api.loglike_grad_host(ev, *bad, stream=_Stream())
        with pytest.raises(ValueError):
            api.rebuild_loglike_grad_host(ev, [c], [psd], th, np.zeros(5), None, stream=_Stream())
        with pytest.raises(ValueError):
            api.rebuild_loglike_grad_host(ev, [c[:-1]], [psd], th, np.zeros(6), None, stream=_Stream())
    finally:
        ev._h = None
