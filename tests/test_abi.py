"""The C ABI library loads without a GPU, exports exactly what include/rb.h
declares, and rejects malformed arguments on the host before touching CUDA."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2404_11397_gb300 import _lib
    if not _lib.LIB_PATH.exists():
        from paper_2404_11397_gb300 import build
        build.build()
    return _lib.load()


def _declared():
    src = (ROOT / "include" / "rb.h").read_text()
    return sorted(set(re.findall(r"RB_API\s+[\w\s\*]+?\b(rb_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("rb_build_summary", "rb_event_free", "rb_loglike_batch", "rb_loglike_grad_batch", "rb_submit",
                     "rb_poll", "rb_server_create", "rb_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2404_11397_gb300 import _lib
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"{name} missing from the Python binding"


def test_status_strings_and_version(lib):
    assert lib.rb_abi_version() == 2
    assert lib.rb_strerror(0) == b"ok"
    assert lib.rb_strerror(-5).startswith(b"busy")
    assert lib.rb_strerror(12345) == b"unknown status"


def test_host_side_validation(lib):
    from paper_2404_11397_gb300 import _lib
    h = ctypes.c_void_p()
    assert lib.rb_build_summary(None, ctypes.byref(h)) == _lib.RB_EINVAL
    desc = _lib.EventDesc()
    desc.n_det = 0
    assert lib.rb_build_summary(ctypes.byref(desc), ctypes.byref(h)) == _lib.RB_EINVAL
    assert b"n_det" in lib.rb_last_error()
    desc.n_det, desc.n_bins, desc.T, desc.f_low, desc.f_high = 1, 10, 4.0, 20.0, 10.0
    assert lib.rb_build_summary(ctypes.byref(desc), ctypes.byref(h)) == _lib.RB_EINVAL  # f_high < f_low
    desc.f_high, desc.n_bins = 30.0, 100  # 41 grid points < 101 edges
    assert lib.rb_build_summary(ctypes.byref(desc), ctypes.byref(h)) == _lib.RB_EINVAL
    assert b"n_bins" in lib.rb_last_error()
    assert lib.rb_loglike_batch(None, None, 4, None, 0, None) == _lib.RB_EINVAL
    assert lib.rb_loglike_grad_batch(None, None, 4, None, None, 0, None) == _lib.RB_EINVAL
    assert lib.rb_event_rebuild(None, None, None, None, 0, 0, None) == _lib.RB_EINVAL
    assert lib.rb_event_free(None) == _lib.RB_OK
    t = ctypes.c_uint64()
    th = np.zeros(13)
    assert lib.rb_submit(None, None, th.ctypes.data_as(_lib.c_double_p), 1, 1, ctypes.byref(t)) == _lib.RB_EINVAL
    assert lib.rb_poll(None, 1, 0, None, None) == _lib.RB_EINVAL
    assert lib.rb_server_get_stats(None, None) == _lib.RB_EINVAL


def test_package_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2404_11397_gb300 import _lib
    monkeypatch.setattr(_lib, "_lib", None)
    monkeypatch.setattr(_lib, "LIB_PATH", tmp_path / "librb.so")
    with pytest.raises(RuntimeError, match="missing"):
        _lib.load()


def test_bounds_record_absent_from_the_normal_build(lib):
    # the normal library compiles no device-side bounds checks; the debug
    # variant (build.py --checked) is exercised by the GPU tests
    site, index, limit = ctypes.c_int(7), ctypes.c_longlong(7), ctypes.c_longlong(7)
    assert lib.rb_debug_bounds(ctypes.byref(site), ctypes.byref(index), ctypes.byref(limit)) == -1
    assert (site.value, index.value, limit.value) == (7, 7, 7)


def test_event_files_are_validated_before_any_device_work(lib, tmp_path):
    out = ctypes.c_void_p(123)
    missing = str(tmp_path / "missing.rbev").encode()
    assert lib.rb_event_load(missing, None, ctypes.byref(out)) == -1 and out.value is None
    assert b"cannot open" in lib.rb_last_error()
    bad = tmp_path / "bad.rbev"
    bad.write_bytes(b"NOTANEVENTFILE" + bytes(400))
    assert lib.rb_event_load(str(bad).encode(), None, ctypes.byref(out)) == -1
    assert b"not a complete event file" in lib.rb_last_error()
    assert lib.rb_event_load(None, None, ctypes.byref(out)) == -1
    assert lib.rb_event_save(None, str(bad).encode()) == -1


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct of include/rb.h has the size and field offsets the ctypes
    binding uses (a C program compiled against the header prints them)."""
    import shutil
    import subprocess
    from paper_2404_11397_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"rb_detector_desc": _lib.DetectorDesc, "rb_event_desc": _lib.EventDesc,
               "rb_event_info": _lib.EventInfo, "rb_server_opts": _lib.ServerOpts,
               "rb_server_stats": _lib.ServerStats}
    lines = ['#include <stdio.h>', '#include "rb.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", f"-I{ROOT / 'include'}", str(src), "-o", str(exe)], check=True)
    got = {}
    for ln in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        cname, key, val = ln.split()
        got[(cname, key)] = int(val)
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_host_arrays_are_checked_against_the_grid():
    from paper_2404_11397_gb300.api import _check_host_arrays
    N = 17
    good_ri, good_c, psd = np.zeros((N, 2)), np.zeros(N, dtype=complex), np.ones(N)
    _check_host_arrays([good_ri, good_c], [psd, psd], 2, N)
    _check_host_arrays([good_ri.ravel()], [psd], 1, N)  # flat [2N] views are accepted
    for data, p in (([np.zeros((N - 1, 2))], [psd]), ([good_ri], [np.ones(N + 1)]), ([np.zeros(2 * N + 1)], [psd]),
                    ([np.zeros(N - 1, dtype=complex)], [psd])):
        with pytest.raises(ValueError):
            _check_host_arrays(data, p, 1, N)
    with pytest.raises(ValueError):
        _check_host_arrays([good_ri], [psd, psd], 1, N)


def test_host_strain_marshalling_keeps_both_components():
    """Complex strain goes to the library as its (re, im) pairs and [N][2] float
    strain as it is: the library reads 2 N float64 values per detector."""
    import torch
    from paper_2404_11397_gb300.api import _host_psd, _host_strain
    rng = np.random.default_rng(5)
    c = rng.normal(size=9) + 1j * rng.normal(size=9)
    ri = np.stack([c.real, c.imag], axis=-1)
    c64 = c.astype(np.complex64)
    ri64 = np.stack([c64.real, c64.imag], axis=-1).astype(np.float64)
    for a, expect in ((c, ri), (ri, ri), (c64, ri64), (torch.from_numpy(c), ri), (torch.from_numpy(ri), ri),
                      (torch.from_numpy(c64), ri64)):
        out = _host_strain(a, 0)
        flat = out.numpy().ravel() if isinstance(out, torch.Tensor) else out.ravel()
        assert flat.dtype == np.float64 and flat.size == 18
        np.testing.assert_array_equal(flat, expect.ravel())
    t = torch.from_numpy(c)
    assert _host_strain(t, 0).data_ptr() == t.data_ptr()  # a contiguous complex128 tensor is viewed, not copied
    assert _host_strain(t.conj(), 0).numpy()[:, 1].tolist() == (-c.imag).tolist()
    assert _host_psd([1, 2, 3], 0).dtype == np.float64


def test_host_outputs_and_theta_are_checked():
    import torch
    from paper_2404_11397_gb300.api import _check_host_out, _host_theta
    assert _host_theta(np.zeros((4, 13))).shape == (4, 13)
    assert _host_theta(torch.zeros(4, 13, dtype=torch.float32)).dtype == torch.float64
    for bad in (np.zeros(13), np.zeros((4, 12)), np.zeros((2, 4, 13))):
        with pytest.raises(ValueError):
            _host_theta(bad)
    _check_host_out(np.zeros(5), 5, "x")
    _check_host_out(np.zeros(8), 5, "x")  # a larger preallocated buffer is fine
    _check_host_out(torch.zeros(5, dtype=torch.float64), 5, "x")
    ro = np.zeros(5)
    ro.flags.writeable = False
    for bad in (np.zeros(4), np.zeros(5, dtype=np.float32), np.zeros(10)[::2], ro, [0.0] * 5,
                torch.zeros(5, dtype=torch.float32), torch.zeros(10, dtype=torch.float64)[::2]):
        with pytest.raises(ValueError):
            _check_host_out(bad, 5, "x")


def test_mala_shapes_are_checked():
    import torch
    from paper_2404_11397_gb300.api import _check_mala_shapes
    W = 6
    z, g, xi = (torch.zeros(W, 13) for _ in range(3))
    lp, u = torch.zeros(W), torch.zeros(W)
    assert _check_mala_shapes(z, lp, g, xi, u) == W
    assert _check_mala_shapes(z, None, None, None, None) == W
    for args in ((torch.zeros(W * 13), lp, g, xi, u), (z, torch.zeros(W + 1), g, xi, u), (z, lp, torch.zeros(W, 12), xi, u),
                 (z, lp, g, torch.zeros(W - 1, 13), u), (z, lp, g, xi, torch.zeros(W, 1))):
        with pytest.raises(ValueError):
            _check_mala_shapes(*args)


def test_server_poll_buffers_follow_the_submitted_request():
    """rb_poll copies the request's own W values (13 W more with the gradient),
    so the binding sizes its buffers from the submitted request and refuses a
    W that disagrees; a ticket it did not record is sized by the library
    (rb_ticket_info), never from a caller's W; submit refuses walkers that are
    not [W, 13]."""
    from paper_2404_11397_gb300 import RBError
    from paper_2404_11397_gb300.api import Server
    srv = Server.__new__(Server)  # the bookkeeping only: no library server behind it
    srv._h, srv._req = None, {7: (300, True), 8: (5, False)}
    assert srv._poll_shape(7, None, None) == (300, True)
    assert srv._poll_shape(7, 300, False) == (300, False)
    assert srv._poll_shape(8, None, True) == (5, False)  # no gradient to copy for a request without it
    with pytest.raises(ValueError):
        srv._poll_shape(7, 299, None)
    for W in (64, None):  # unknown here: the library is asked (no server behind this object: refused)
        with pytest.raises(RBError):
            srv._poll_shape(9, W, None)
    for bad in (np.zeros(12), np.zeros((4, 12)), np.zeros((2, 2, 13))):
        with pytest.raises(ValueError):
            srv.submit(None, bad)
