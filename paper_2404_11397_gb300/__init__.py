"""GB300 (sm_103a) relative-binning log-likelihood and gradient for
binary-neutron-star parameter estimation (arXiv:2404.11397, Sec. II).

The compute lives in ``librb.so`` (hand-written CUDA behind the C ABI of
``include/rb.h``); this package is a thin ctypes/torch binding.  Importing it
does not require a GPU, but every compute call needs the built library and a
CUDA device: there is no CPU fallback.
"""
from ._lib import (MODES, NPAR, RB_BINS_AGNOSTIC, RB_BINS_PN, RB_EBUSY, RB_ECLOSED, RB_ECUDA, RB_EINVAL, RB_ENOMEM,
                   RB_ENOTFOUND, RB_ETIMEDOUT, RB_FP64, RB_MIXED, RB_MIXED_F64PHASE, RB_OK, RB_PENDING, RBError, LIB_PATH,
                   load)
from .api import (Event, RBLogLikelihood, Server, kernel_launch_count, loglike, loglike_full, loglike_grad,
                  loglike_grad_host, rebuild_loglike_grad, rebuild_loglike_grad_host,
                  mala_init, mala_step, rb_loglike, set_trace_events, strain)

__all__ = ["Event", "RBLogLikelihood", "Server", "loglike", "loglike_full", "loglike_grad", "loglike_grad_host", "rebuild_loglike_grad", "rebuild_loglike_grad_host", "rb_loglike",
           "mala_init", "mala_step",
           "strain", "set_trace_events", "kernel_launch_count", "load", "LIB_PATH", "MODES", "NPAR", "RBError", "RB_OK", "RB_PENDING",
           "RB_EINVAL", "RB_ENOMEM", "RB_ECUDA", "RB_ETIMEDOUT", "RB_EBUSY", "RB_ENOTFOUND", "RB_ECLOSED",
           "RB_MIXED", "RB_FP64", "RB_MIXED_F64PHASE", "RB_BINS_PN", "RB_BINS_AGNOSTIC"]
