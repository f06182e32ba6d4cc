"""ctypes declarations of the librb C ABI (include/rb.h).  Argument marshalling
only; every computation happens in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

LIB_PATH = Path(__file__).resolve().parent / "librb.so"
# RB_LIB_VARIANT=checked loads the debug build with device-side bounds checks
# (build.py --checked); anything else loads the normal library
if os.environ.get("RB_LIB_VARIANT") == "checked":
    LIB_PATH = LIB_PATH.with_name("librb_checked.so")

RB_OK, RB_PENDING = 0, 1
RB_EINVAL, RB_ENOMEM, RB_ECUDA, RB_ETIMEDOUT, RB_EBUSY, RB_ENOTFOUND, RB_ECLOSED = -1, -2, -3, -4, -5, -6, -7
RB_MIXED, RB_FP64, RB_MIXED_F64PHASE = 0, 1, 2
RB_BINS_PN, RB_BINS_AGNOSTIC = 0, 1
BIN_SCHEMES = {"pn": RB_BINS_PN, "agnostic": RB_BINS_AGNOSTIC}
MODES = {"mixed": RB_MIXED, "fp64": RB_FP64, "mixed_f64phase": RB_MIXED_F64PHASE}
NPAR = 13
MAX_DET = 3
RB_STATIC_MAX_WALKERS = 8192

c_double_p = ctypes.POINTER(ctypes.c_double)
c_int64_p = ctypes.POINTER(ctypes.c_int64)


class DetectorDesc(ctypes.Structure):
    _fields_ = [("lat", ctypes.c_double), ("lon", ctypes.c_double), ("elev_m", ctypes.c_double),
                ("xarm_az", ctypes.c_double), ("yarm_az", ctypes.c_double),
                ("data", ctypes.c_void_p), ("psd", ctypes.c_void_p)]


class EventDesc(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("det", DetectorDesc * MAX_DET),
                ("T", ctypes.c_double), ("f_low", ctypes.c_double), ("f_high", ctypes.c_double),
                ("gmst", ctypes.c_double), ("data_on_device", ctypes.c_int32), ("bin_scheme", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("theta_ref", ctypes.c_double * NPAR)]


class EventInfo(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int32), ("n_bins", ctypes.c_int32), ("kmin", ctypes.c_int64),
                ("n_freq", ctypes.c_int64), ("T", ctypes.c_double), ("gmst", ctypes.c_double),
                ("base_logl", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("theta_ref", ctypes.c_double * 13), ("bin_scheme", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("epsilon", ctypes.c_double)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32),
                ("max_queue", ctypes.c_int32), ("use_graphs", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("max_walkers", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("graph_launches", ctypes.c_uint64), ("plain_launches", ctypes.c_uint64),
                ("graphs_captured", ctypes.c_uint64), ("in_flight", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("hbm_in_use", ctypes.c_size_t), ("max_in_flight", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("graph_updates", ctypes.c_uint64), ("walkers_requested", ctypes.c_uint64),
                ("walkers_run", ctypes.c_uint64)]


# name -> (restype, argtypes); the order follows include/rb.h
SIGNATURES = {
    "rb_build_summary": (ctypes.c_int, [ctypes.POINTER(EventDesc), ctypes.POINTER(ctypes.c_void_p)]),
    "rb_event_free": (ctypes.c_int, [ctypes.c_void_p]),
    "rb_event_rebuild": (ctypes.c_int, [ctypes.c_void_p, c_double_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_void_p]),
    "rb_event_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(EventInfo)]),
    "rb_event_save": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p]),
    "rb_event_load": (ctypes.c_int, [ctypes.c_char_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "rb_event_get_summary": (ctypes.c_int, [ctypes.c_void_p, c_double_p, c_double_p, c_double_p, c_double_p,
                                            c_int64_p]),
    "rb_loglike_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]),
    "rb_loglike_grad_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_mala_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_mala_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_rebuild_loglike_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_rebuild_loglike_grad_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                    ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                                    ctypes.c_void_p]),
    "rb_loglike_full_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                             ctypes.c_int, ctypes.c_void_p]),
    "rb_loglike_grad_batch_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_loglike_grad_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "rb_strain": (ctypes.c_int, [c_double_p, ctypes.c_double, c_double_p, ctypes.c_double, ctypes.c_int64,
                                 ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),
    "rb_server_create": (ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(ctypes.c_void_p)]),
    "rb_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "rb_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, c_double_p, ctypes.c_int64, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "rb_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, c_double_p, c_double_p]),
    "rb_ticket_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, c_int64_p, ctypes.POINTER(ctypes.c_int32)]),
    "rb_server_get_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ServerStats)]),
    "rb_server_latency": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, c_int64_p, c_double_p, c_double_p,
                                         c_double_p]),
    "rb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "rb_last_error": (ctypes.c_char_p, []),
    "rb_set_trace_events": (None, [ctypes.c_void_p, ctypes.c_void_p]),
    "rb_kernel_launch_count": (ctypes.c_uint64, []),
    "rb_abi_version": (ctypes.c_int, []),
    "rb_debug_bounds": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong)]),
}

_lib = None


class RBError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


def load() -> ctypes.CDLL:
    """Load the in-tree librb.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is not None:
        return _lib
    if not LIB_PATH.exists():
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(str(LIB_PATH))
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(status: int, where: str) -> int:
    if status < 0:
        lib = load()
        raise RBError(status, where, lib.rb_last_error().decode(errors="replace"))
    return status
