"""Python binding of librb: events, batched relative-binning likelihood and
gradient, strain generation, the serving loop, and a torch.autograd.Function.

PyTorch is used for device memory and streams only: tensors are passed to the
C ABI as raw device pointers together with the current CUDA stream.  Every
step of the likelihood runs in librb's kernels; nothing here computes it.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import numpy as np
import torch

from . import _lib
from ._lib import MODES, NPAR, check, load


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _mode(mode) -> int:
    if isinstance(mode, str):
        return MODES[mode]
    return int(mode)


def _theta_dev(theta: torch.Tensor) -> torch.Tensor:
    if not (isinstance(theta, torch.Tensor) and theta.is_cuda):
        raise TypeError("theta must be a CUDA tensor [W, 13]")
    if theta.dim() != 2 or theta.shape[1] != NPAR:
        raise ValueError("theta must have shape [W, 13]")
    return theta.to(torch.float64).contiguous()


def _check_host_arrays(data, psd, n_det: int, n_freq: int) -> None:
    """Per-detector strain ([n_freq][2], or complex [n_freq]) and PSD ([n_freq])
    host arrays of the right count and size: the library reads exactly that
    many points from each pointer (pinned buffers from a kernel), so a shorter
    buffer must be refused here."""
    if len(data) != n_det or len(psd) != n_det:
        raise ValueError(f"need {n_det} strain and {n_det} PSD arrays, got {len(data)} and {len(psd)}")
    for d in range(n_det):
        a, p = data[d], psd[d]
        na = a.numel() if isinstance(a, torch.Tensor) else np.asarray(a).size
        np_ = p.numel() if isinstance(p, torch.Tensor) else np.asarray(p).size
        cplx = (a.is_complex() if isinstance(a, torch.Tensor) else np.iscomplexobj(a))
        if (na if cplx else na // 2) != n_freq or (not cplx and na % 2) or np_ != n_freq:
            raise ValueError(f"detector {d}: strain must hold {n_freq} complex points and the PSD {n_freq} values")


def _host_strain(a, d: int):
    """One detector's host strain as a contiguous float64 [N][2] buffer (complex
    input viewed as its (re, im) pairs, so a pinned complex tensor stays pinned)."""
    if isinstance(a, torch.Tensor):
        if a.is_cuda:
            raise ValueError(f"detector {d}: host strain expected, got a CUDA tensor")
        t = torch.view_as_real(a.to(torch.complex128).resolve_conj()) if a.is_complex() else a.to(torch.float64)
        return t.contiguous()
    a = np.asarray(a)
    if np.iscomplexobj(a):
        return np.ascontiguousarray(a, dtype=np.complex128).view(np.float64)
    return np.ascontiguousarray(a, dtype=np.float64)


def _host_psd(p, d: int):
    if isinstance(p, torch.Tensor):
        if p.is_cuda:
            raise ValueError(f"detector {d}: host PSD expected, got a CUDA tensor")
        return p.to(torch.float64).contiguous()
    return np.ascontiguousarray(p, dtype=np.float64)


def _host_theta(theta):
    """Walkers for a host-buffer call: a host [W, 13] float64 array or CPU tensor."""
    if isinstance(theta, torch.Tensor):
        if theta.is_cuda:
            raise ValueError("theta must be a host array for the host-buffer calls")
        th = theta.to(torch.float64).contiguous()
    else:
        th = np.ascontiguousarray(theta, dtype=np.float64)
    if th.ndim != 2 or th.shape[1] != NPAR:
        raise ValueError("theta must have shape [W, 13]")
    return th


def _check_host_out(a, n: int, what: str) -> None:
    """A host output the library writes n float64 values into (a kernel writes
    pinned buffers directly): it must be that large, float64, contiguous, on
    the host and writable."""
    if isinstance(a, torch.Tensor):
        ok = (not a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() and a.numel() >= n)
    else:
        ok = (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.flags.writeable
              and a.size >= n)
    if not ok:
        raise ValueError(f"{what} must be a contiguous, writable float64 host buffer of at least {n} values")


def _check_mala_shapes(z, logp, gz, xi, u) -> int:
    """z, gz, xi [W, 13] and logp, u [W] (xi and u may be None for the initial
    evaluation): the library reads and writes exactly these extents."""
    if z.dim() != 2 or z.shape[1] != NPAR:
        raise ValueError("z must have shape [W, 13]")
    W = z.shape[0]
    for name, t, shape in (("logp", logp, (W,)), ("gz", gz, (W, NPAR)), ("xi", xi, (W, NPAR)), ("u", u, (W,))):
        if t is not None and tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {list(shape)}, got {list(t.shape)}")
    return W


class Event:
    """A device-resident event: grid, bin edges, summary data and tables.

    geom: [D][5] site rows (lat, lon [rad], elevation [m], x/y arm azimuth [rad]);
    data: [D][N] complex strain (or float64 [D][N][2] as (re, im) pairs) and
    psd: [D][N] one-sided PSD, either all host arrays (numpy or CPU tensors) or
    all CUDA tensors.
    """

    def __init__(self, geom, gmst: float, T: float, f_low: float, f_high: float, data, psd, n_bins: int,
                 theta_ref, stream: Optional[torch.cuda.Stream] = None, bins: str = "pn"):
        lib = load()
        geom = np.asarray(geom, dtype=np.float64).reshape(-1, 5)
        D = geom.shape[0]
        # the grid the library builds: k = ceil(f_low T) .. floor(f_high T), both ends included
        n_freq = math.floor(float(f_high) * float(T) + 1e-9) - math.ceil(float(f_low) * float(T) - 1e-9) + 1
        if n_freq >= 2:
            _check_host_arrays(data, psd, D, n_freq)
        if bins not in _lib.BIN_SCHEMES:
            raise ValueError(f"bins must be one of {sorted(_lib.BIN_SCHEMES)}")
        desc = _lib.EventDesc()
        desc.n_det = D
        desc.n_bins = int(n_bins)
        desc.bin_scheme = _lib.BIN_SCHEMES[bins]
        desc.T, desc.f_low, desc.f_high, desc.gmst = float(T), float(f_low), float(f_high), float(gmst)
        cuda = [isinstance(data[d], torch.Tensor) and data[d].is_cuda for d in range(D)]
        cuda += [isinstance(psd[d], torch.Tensor) and psd[d].is_cuda for d in range(D)]
        if any(cuda) and not all(cuda):
            raise ValueError("strain and PSD must all be CUDA tensors or all host arrays")
        on_device = D > 0 and all(cuda)
        desc.data_on_device = 1 if on_device else 0
        keep = []
        for d in range(D):
            row = desc.det[d]
            row.lat, row.lon, row.elev_m, row.xarm_az, row.yarm_az = map(float, geom[d])
            if on_device:
                a = data[d]
                dd = (torch.view_as_real(a.to(torch.complex128).resolve_conj()) if a.is_complex()
                      else a.to(torch.float64)).contiguous()
                pp = psd[d].to(torch.float64).contiguous()
            else:
                dd, pp = _host_strain(data[d], d), _host_psd(psd[d], d)
            keep += [dd, pp]
            row.data, row.psd = _host_ptr(dd), _host_ptr(pp)
        th = np.asarray(theta_ref, dtype=np.float64).reshape(NPAR)
        for j in range(NPAR):
            desc.theta_ref[j] = float(th[j])
        desc.cuda_stream = _stream_handle(stream).value if torch.cuda.is_available() else None
        handle = ctypes.c_void_p()
        check(lib.rb_build_summary(ctypes.byref(desc), ctypes.byref(handle)), "rb_build_summary")
        del keep
        self._h = handle
        self.n_det = D
        self.n_bins = int(n_bins)
        self.theta_ref = th.copy()
        inf = _lib.EventInfo()
        check(lib.rb_event_get_info(handle, ctypes.byref(inf)), "rb_event_get_info")
        self.n_freq = int(inf.n_freq)

    @classmethod
    def from_synth(cls, ev: dict, n_bins: Optional[int] = None, theta_ref=None, stream=None,
                   bins: str = "pn") -> "Event":
        """Build from a ``synth.make_event`` dict that carries ``data``."""
        return cls(ev["geom"], ev["gmst"], ev["T"], ev["f_low"], ev["f_high"], ev["data"], ev["psd"],
                   n_bins if n_bins is not None else ev["n_bins"],
                   ev["theta_inj"] if theta_ref is None else theta_ref, stream=stream, bins=bins)

    @property
    def handle(self) -> ctypes.c_void_p:
        if self._h is None:
            raise RuntimeError("event has been freed")
        return self._h

    def rebuild(self, theta_ref=None, data=None, psd=None, mode="mixed", stream=None) -> None:
        """Recompute the summary data in place (asynchronous, allocation-free).

        data/psd: per-detector CUDA tensors (read in place), host numpy arrays
        (copied in), or None to reuse the event's resident copy."""
        lib = load()
        th_p = None
        if theta_ref is not None:
            th = np.ascontiguousarray(theta_ref, dtype=np.float64).reshape(NPAR)
            th_p = th.ctypes.data_as(_lib.c_double_p)
            self.theta_ref = th.copy()
        dp = pp = None
        on_dev = 0
        keep = []
        if data is not None:
            D = self.n_det
            _check_host_arrays(data, psd, D, self.n_freq)
            dp = (ctypes.c_void_p * D)()
            pp = (ctypes.c_void_p * D)()
            cuda = [isinstance(a, torch.Tensor) and a.is_cuda for a in list(data) + list(psd)]
            if any(cuda) and not all(cuda):
                raise ValueError("strain and PSD must all be CUDA tensors or all host arrays")
            on_dev = 1 if all(cuda) else 0
            for d in range(D):
                if on_dev:
                    dd, ps = data[d], psd[d]
                    if dd.dtype == torch.complex128 and dd.is_contiguous():
                        dd = torch.view_as_real(dd.resolve_conj())
                    if not (dd.is_contiguous() and ps.is_contiguous() and dd.dtype == torch.float64
                            and ps.dtype == torch.float64):
                        raise ValueError("device data must be contiguous float64 [N][2] (or complex128 [N]) / [N]")
                    dp[d], pp[d] = dd.data_ptr(), ps.data_ptr()
                else:
                    dd, ps = _host_strain(data[d], d), _host_psd(psd[d], d)
                    dp[d], pp[d] = _host_ptr(dd), _host_ptr(ps)
                keep += [dd, ps]
        check(lib.rb_event_rebuild(self.handle, th_p, dp, pp, on_dev, _mode(mode), _stream_handle(stream)),
              "rb_event_rebuild")

    def info(self) -> dict:
        lib = load()
        inf = _lib.EventInfo()
        check(lib.rb_event_get_info(self.handle, ctypes.byref(inf)), "rb_event_get_info")
        out = {f: getattr(inf, f) for f, _ in _lib.EventInfo._fields_}
        out["theta_ref"] = np.array(out["theta_ref"][:], dtype=np.float64)
        return out

    def save(self, path) -> None:
        """Write the event (descriptor, theta_ref, resident strain and PSD) to a file."""
        check(load().rb_event_save(self.handle, str(path).encode()), "rb_event_save")

    @classmethod
    def load(cls, path, stream: Optional[torch.cuda.Stream] = None) -> "Event":
        """Build an event from a file written by save (bit-identical results)."""
        lib = load()
        h = ctypes.c_void_p()
        sh = _stream_handle(stream) if torch.cuda.is_available() else None
        check(lib.rb_event_load(str(path).encode(), sh, ctypes.byref(h)), "rb_event_load")
        ev = cls.__new__(cls)
        ev._h = h
        inf = ev.info()
        ev.n_det, ev.n_bins, ev.theta_ref = int(inf["n_det"]), int(inf["n_bins"]), inf["theta_ref"]
        ev.n_freq = int(inf["n_freq"])
        return ev

    def summary(self) -> dict:
        """FP64 summary data and bin edges copied to the host."""
        lib = load()
        inf = self.info()  # the library's own extents: it copies D x B values per table
        D, B = int(inf["n_det"]), int(inf["n_bins"])
        A0 = np.zeros((D, B, 2))
        A1 = np.zeros((D, B, 2))
        B0 = np.zeros((D, B))
        B1 = np.zeros((D, B))
        edges = np.zeros(B + 1, dtype=np.int64)
        p = lambda a: a.ctypes.data_as(_lib.c_double_p)
        check(lib.rb_event_get_summary(self.handle, p(A0), p(A1), p(B0), p(B1),
                                       edges.ctypes.data_as(_lib.c_int64_p)), "rb_event_get_summary")
        return {"A0": A0[..., 0] + 1j * A0[..., 1], "A1": A1[..., 0] + 1j * A1[..., 1], "B0": B0, "B1": B1,
                "edges": edges}

    def free(self) -> None:
        if getattr(self, "_h", None) is not None:
            load().rb_event_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def loglike(event: Event, theta: torch.Tensor, mode="mixed", stream=None) -> torch.Tensor:
    """Batched RB log-likelihood [W] (float64, on theta's device)."""
    th = _theta_dev(theta)
    out = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
    check(load().rb_loglike_batch(event.handle, ctypes.c_void_p(th.data_ptr()), th.shape[0],
                                  ctypes.c_void_p(out.data_ptr()), _mode(mode), _stream_handle(stream)),
          "rb_loglike_batch")
    return out


def rebuild_loglike_grad(event: Event, theta: torch.Tensor, mode="mixed", stream=None, grad: bool = True):
    """Rebuild the summary data from the event's resident data, then log L [W]
    (and the gradient [W, 13] unless grad=False) in one call, with the walkers'
    set-up overlapped with the summary sums."""
    th = _theta_dev(theta)
    W = th.shape[0]
    out = torch.empty(W, dtype=torch.float64, device=th.device)
    g = torch.empty(W, NPAR, dtype=torch.float64, device=th.device) if grad else None
    check(load().rb_rebuild_loglike_grad(event.handle, ctypes.c_void_p(th.data_ptr()), W,
                                         ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(g.data_ptr()) if g is not None else None, _mode(mode),
                                         _stream_handle(stream)), "rb_rebuild_loglike_grad")
    return (out, g) if grad else out


def rebuild_loglike_grad_host(event: Event, data, psd, theta: np.ndarray, logl_out: np.ndarray,
                              grad_out: Optional[np.ndarray], mode="mixed", stream=None) -> None:
    """End-to-end step on host buffers: new strain/PSD (per detector, [N][2]
    and [N] float64, ideally pinned) and walkers in, summary rebuilt, log L
    (and gradient) out; synchronises the stream."""
    D = event.n_det
    _check_host_arrays(data, psd, D, event.n_freq)
    keep = [_host_strain(data[d], d) for d in range(D)] + [_host_psd(psd[d], d) for d in range(D)]
    ptrs = [_host_ptr(a) for a in keep]
    dp = (ctypes.c_void_p * D)(*ptrs[:D])
    pp = (ctypes.c_void_p * D)(*ptrs[D:])
    th = _host_theta(theta)
    W = th.shape[0]
    _check_host_out(logl_out, W, "logl_out")
    if grad_out is not None:
        _check_host_out(grad_out, W * NPAR, "grad_out")
    th_ptr, lo_ptr = _host_ptr(th), _host_ptr(logl_out)
    gr_ptr = _host_ptr(grad_out) if grad_out is not None else None
    check(load().rb_rebuild_loglike_grad_host(event.handle, dp, pp, ctypes.c_void_p(th_ptr), W, ctypes.c_void_p(lo_ptr),
                                              ctypes.c_void_p(gr_ptr) if gr_ptr else None, _mode(mode),
                                              _stream_handle(stream)), "rb_rebuild_loglike_grad_host")


def loglike_full(event: Event, theta: torch.Tensor, mode="mixed", stream=None) -> torch.Tensor:
    """Full-grid (un-binned) log-likelihood [W] (float64, on theta's device)."""
    th = _theta_dev(theta)
    out = torch.empty(th.shape[0], dtype=torch.float64, device=th.device)
    check(load().rb_loglike_full_batch(event.handle, ctypes.c_void_p(th.data_ptr()), th.shape[0],
                                       ctypes.c_void_p(out.data_ptr()), _mode(mode), _stream_handle(stream)),
          "rb_loglike_full_batch")
    return out


def loglike_grad(event: Event, theta: torch.Tensor, mode="mixed", stream=None):
    """Batched RB log-likelihood [W] and gradient [W, 13]."""
    th = _theta_dev(theta)
    W = th.shape[0]
    out = torch.empty(W, dtype=torch.float64, device=th.device)
    grad = torch.empty(W, NPAR, dtype=torch.float64, device=th.device)
    check(load().rb_loglike_grad_batch(event.handle, ctypes.c_void_p(th.data_ptr()), W,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                       _mode(mode), _stream_handle(stream)), "rb_loglike_grad_batch")
    return out, grad


def _host_ptr(a) -> int:
    return a.data_ptr() if isinstance(a, torch.Tensor) else a.ctypes.data


def loglike_grad_host(event: Event, theta: np.ndarray, logl_out, grad_out=None, mode="mixed", stream=None) -> None:
    """End-to-end call on host buffers (numpy arrays or CPU tensors, ideally
    pinned): copies in, evaluates, copies out (pinned outputs are written by
    the kernel directly), synchronises."""
    th = _host_theta(theta)
    W = th.shape[0]
    _check_host_out(logl_out, W, "logl_out")
    if grad_out is not None:
        _check_host_out(grad_out, W * NPAR, "grad_out")
    check(load().rb_loglike_grad_host(event.handle, ctypes.c_void_p(_host_ptr(th)), W,
                                      ctypes.c_void_p(_host_ptr(logl_out)),
                                      ctypes.c_void_p(_host_ptr(grad_out)) if grad_out is not None else None,
                                      _mode(mode), _stream_handle(stream)), "rb_loglike_grad_host")


def strain(geom, gmst: float, theta, T: float, kmin: int, n_freq: int, device="cuda", stream=None) -> torch.Tensor:
    """Detector strain h_d(f) [n_freq] complex128 on the device (librb kernel)."""
    g = np.ascontiguousarray(geom, dtype=np.float64).reshape(5)
    th = np.ascontiguousarray(theta, dtype=np.float64).reshape(NPAR)
    out = torch.empty(n_freq, 2, dtype=torch.float64, device=device)
    check(load().rb_strain(g.ctypes.data_as(_lib.c_double_p), float(gmst), th.ctypes.data_as(_lib.c_double_p),
                           float(T), int(kmin), int(n_freq), ctypes.c_void_p(out.data_ptr()),
                           _stream_handle(stream)), "rb_strain")
    return torch.view_as_complex(out)


def _host13(v) -> np.ndarray:
    a = np.ascontiguousarray(v, dtype=np.float64).reshape(NPAR)
    return a


def mala_init(event: Event, z: torch.Tensor, lo, hi, mode="mixed", stream=None):
    """log pi(z) [W] and d log pi / dz [W, 13] for chains in the sampling
    coordinates (cos iota, sin dec) with the uniform prior on lo < z < hi."""
    zz = _theta_dev(z)
    W = _check_mala_shapes(zz, None, None, None, None)
    logp = torch.empty(W, dtype=torch.float64, device=zz.device)
    gz = torch.empty(W, NPAR, dtype=torch.float64, device=zz.device)
    lo_, hi_ = _host13(lo), _host13(hi)
    check(load().rb_mala_init(event.handle, ctypes.c_void_p(zz.data_ptr()), W, ctypes.c_void_p(lo_.ctypes.data),
                              ctypes.c_void_p(hi_.ctypes.data), ctypes.c_void_p(logp.data_ptr()),
                              ctypes.c_void_p(gz.data_ptr()), _mode(mode), _stream_handle(stream)), "rb_mala_init")
    return logp, gz


def mala_step(event: Event, z: torch.Tensor, logp: torch.Tensor, gz: torch.Tensor, eps, lo, hi, xi: torch.Tensor,
              u: torch.Tensor, mode="mixed", stream=None) -> torch.Tensor:
    """One MALA step of every chain; z, logp, gz are updated in place (they
    must be contiguous float64 device tensors).  Returns accepted [W] (int32)."""
    for t in (z, logp, gz, xi, u):
        if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
            raise ValueError("mala_step: z, logp, gz, xi, u must be contiguous float64 CUDA tensors")
    W = _check_mala_shapes(z, logp, gz, xi, u)
    acc = torch.empty(W, dtype=torch.int32, device=z.device)
    eps_, lo_, hi_ = _host13(eps), _host13(lo), _host13(hi)
    check(load().rb_mala_step(event.handle, ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(logp.data_ptr()),
                              ctypes.c_void_p(gz.data_ptr()), W, ctypes.c_void_p(eps_.ctypes.data),
                              ctypes.c_void_p(lo_.ctypes.data), ctypes.c_void_p(hi_.ctypes.data),
                              ctypes.c_void_p(xi.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                              ctypes.c_void_p(acc.data_ptr()), _mode(mode), _stream_handle(stream)), "rb_mala_step")
    return acc


def kernel_launch_count() -> int:
    return int(load().rb_kernel_launch_count())


def set_trace_events(before: Optional[torch.cuda.Event], after: Optional[torch.cuda.Event]) -> None:
    """Record `before`/`after` around the main likelihood kernel of every batch call."""
    b = ctypes.c_void_p(before.cuda_event) if before is not None else None
    a = ctypes.c_void_p(after.cuda_event) if after is not None else None
    load().rb_set_trace_events(b, a)


class RBLogLikelihood(torch.autograd.Function):
    """log L(theta) with the hand-written adjoint as its backward.

    forward evaluates log L and d log L / d theta in one pass of the fused
    kernel; backward returns grad_output[:, None] * (d log L / d theta).
    """

    @staticmethod
    def forward(ctx, theta: torch.Tensor, event: Event, mode="mixed"):
        logl, grad = loglike_grad(event, theta.detach(), mode)
        ctx.save_for_backward(grad)
        return logl

    @staticmethod
    def backward(ctx, grad_output):
        (grad,) = ctx.saved_tensors
        return grad_output.to(grad.dtype)[:, None] * grad, None, None


def rb_loglike(theta: torch.Tensor, event: Event, mode="mixed") -> torch.Tensor:
    return RBLogLikelihood.apply(theta, event, mode)


class Server:
    """Continuous-batching request loop (rb_server_* in the C ABI)."""

    def __init__(self, hbm_budget_bytes: int = 0, max_slots: int = 8, max_queue: int = 0, use_graphs: bool = True,
                 mode="mixed", max_walkers: int = 0):
        lib = load()
        o = _lib.ServerOpts(hbm_budget_bytes, max_slots, max_queue, 1 if use_graphs else 0, _mode(mode), max_walkers)
        h = ctypes.c_void_p()
        check(lib.rb_server_create(ctypes.byref(o), ctypes.byref(h)), "rb_server_create")
        self._h = h
        self._req = {}  # ticket -> (W, want_grad) of the requests submitted through this object

    def submit(self, event: Event, theta: np.ndarray, want_grad: bool = True) -> int:
        th = np.ascontiguousarray(theta, dtype=np.float64)
        if th.ndim == 1 and th.size == NPAR:
            th = th.reshape(1, NPAR)
        if th.ndim != 2 or th.shape[1] != NPAR:
            raise ValueError("theta must have shape [W, 13]")
        t = ctypes.c_uint64()
        check(load().rb_submit(self._h, event.handle, th.ctypes.data_as(_lib.c_double_p), th.shape[0],
                               1 if want_grad else 0, ctypes.byref(t)), "rb_submit")
        self._req[t.value] = (th.shape[0], bool(want_grad))
        return t.value

    def _poll_shape(self, ticket: int, W: Optional[int], want_grad: Optional[bool]):
        """The output extents of a poll: the library copies the request's own
        W values (and 13 W gradient values if it asked for them), so buffers
        are sized from the request as the library holds it; a W that disagrees
        is refused, and an unknown ticket raises RB_ENOTFOUND."""
        known = self._req.get(ticket)
        if known is None:  # not submitted through this object: ask the library for its shape
            w, g = ctypes.c_int64(0), ctypes.c_int32(0)
            check(load().rb_ticket_info(self._h, ticket, ctypes.byref(w), ctypes.byref(g)), "rb_ticket_info")
            known = (int(w.value), bool(g.value))
        if W is not None and int(W) != known[0]:
            raise ValueError(f"ticket {ticket} was submitted with W = {known[0]}, not {W}")
        return known[0], known[1] if want_grad is None else (bool(want_grad) and known[1])

    def poll(self, ticket: int, W: Optional[int] = None, timeout_us: int = -1, want_grad: Optional[bool] = None):
        """Returns (status, logl, grad); status RB_OK, RB_PENDING or RB_ETIMEDOUT (others raise).
        W and want_grad default to the request's own; grad is None for a request without it."""
        W, want_grad = self._poll_shape(ticket, W, want_grad)
        logl = np.zeros(W)
        grad = np.zeros((W, NPAR)) if want_grad else None
        st = load().rb_poll(self._h, ticket, int(timeout_us), logl.ctypes.data_as(_lib.c_double_p),
                            grad.ctypes.data_as(_lib.c_double_p) if grad is not None else None)
        if st in (_lib.RB_PENDING, _lib.RB_ETIMEDOUT):
            return st, None, None
        self._req.pop(ticket, None)  # collected, or failed: the library has forgotten it either way
        check(st, "rb_poll")
        return st, logl, grad

    LATENCY_PARTS = ("total", "queue", "issue", "device")

    def latency(self, reset: bool = False) -> dict:
        """Server-side latency of the requests completed since the last reset:
        total (rb_submit to results in host memory) and its parts -- waiting for a
        slot, issuing the launch, device work and completion -- each as
        {count, p50_ms, p99_ms, max_ms}."""
        out = {}
        for part, name in enumerate(self.LATENCY_PARTS):
            n = ctypes.c_int64(0)
            q = [ctypes.c_double(0.0) for _ in range(3)]
            last = part == len(self.LATENCY_PARTS) - 1
            check(load().rb_server_latency(self._h, part, 1 if (reset and last) else 0, ctypes.byref(n),
                                           *(ctypes.byref(x) for x in q)), "rb_server_latency")
            out[name] = {"count": int(n.value), "p50_ms": q[0].value, "p99_ms": q[1].value, "max_ms": q[2].value}
        return out

    def stats(self) -> dict:
        s = _lib.ServerStats()
        check(load().rb_server_get_stats(self._h, ctypes.byref(s)), "rb_server_get_stats")
        return {f: getattr(s, f) for f, _ in _lib.ServerStats._fields_}

    def close(self) -> None:
        if getattr(self, "_h", None) is not None:
            load().rb_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
