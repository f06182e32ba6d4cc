"""rb_loglike_grad_batch_static: the allocation-free batch entry point.

It is for callers that cannot allocate device memory when they need a
likelihood (a host framework whose allocator owns all device memory, or a
sampler loop that must not pay for or synchronise on an allocation): its
per-walker workspace is a fixed device array in the library.  Called through
the C ABI twice in a row (different batches, so the second call runs on the
first call's leftovers), in every mode and with and without the gradient, it
must match the allocating entry point rb_loglike_grad_batch within the parity
tolerance used elsewhere (here it is in fact bit-identical: same kernels, same
inputs).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from tests._events import inject

pytestmark = pytest.mark.gpu


def _call(lib, fn, event, th, mode, grad=True):
    W = th.shape[0]
    L = torch.empty(W, dtype=torch.float64, device="cuda")
    G = torch.empty(W, 13, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = fn(event.handle, ctypes.c_void_p(th.data_ptr()), W, ctypes.c_void_p(L.data_ptr()),
            ctypes.c_void_p(G.data_ptr()) if grad else None, mode, stream)
    assert rc == 0, lib.rb_last_error()
    torch.cuda.synchronize()
    return L.cpu().numpy(), (G.cpu().numpy() if grad else None)


def test_static_workspace_matches_allocating_entry_point():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2404_11397_gb300 as rb
    lib = rb.load()
    ev = inject(synth.make_event("C2", T=16.0))
    event = rb.Event.from_synth(ev, n_bins=200)
    pool = torch.tensor(synth.walkers("C2", 4000), device="cuda")
    for mode in (rb.RB_MIXED, rb.RB_MIXED_F64PHASE, rb.RB_FP64):
        for grad in (True, False):
            for th in (pool[:3000], pool[1000:1700]):  # two calls in a row, different sizes
                Ls, Gs = _call(lib, lib.rb_loglike_grad_batch_static, event, th, mode, grad)
                La, Ga = _call(lib, lib.rb_loglike_grad_batch, event, th, mode, grad)
                tol = np.maximum(1e-3, 2e-6 * np.abs(La))
                assert np.all(np.abs(Ls - La) <= tol), (mode, grad)
                if grad:
                    gscale = np.maximum(np.abs(Ga), 1e-2 * np.max(np.abs(Ga), axis=1, keepdims=True))
                    assert np.all(np.abs(Gs - Ga) <= 1e-4 * gscale), mode
    # batches beyond the fixed array are refused with a clear error, not run
    big = torch.zeros(rb._lib.RB_STATIC_MAX_WALKERS + 1, 13, dtype=torch.float64, device="cuda")
    out = torch.empty(big.shape[0], dtype=torch.float64, device="cuda")
    rc = lib.rb_loglike_grad_batch_static(event.handle, ctypes.c_void_p(big.data_ptr()), big.shape[0],
                                          ctypes.c_void_p(out.data_ptr()), None, rb.RB_MIXED,
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == rb.RB_EINVAL
    assert b"static workspace" in lib.rb_last_error()
    event.free()
