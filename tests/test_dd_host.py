"""Float-float arithmetic of the mixed-path set-up (csrc/rb_dd.cuh), built for
the host and checked against long double arithmetic: the set-up needs the
phase coefficients to ~1e-12 relative and the delays to ~1e-12 s, so every
routine must stay well below 1e-12 (relative; absolute for sin and cos)."""
import shutil
import subprocess
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent
SRC = ROOT / "tests" / "dd_host" / "dd_check.cpp"
CSRC = ROOT / "paper_2404_11397_gb300" / "csrc"

LIMITS = {"add": 1e-14, "mul": 5e-14, "div": 5e-14, "sqrt": 5e-14, "cbrt": 1e-13, "rroot5": 1e-13,
          "log": 5e-13, "sin": 1e-12, "cos": 1e-12}


def test_dd_routines_accuracy(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = tmp_path / "dd_check"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", f"-I{CSRC}", str(SRC), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    errs = {k: float(v) for k, v in (ln.split() for ln in out.strip().splitlines())}
    assert set(errs) == set(LIMITS)
    for k, lim in LIMITS.items():
        assert errs[k] <= lim, (k, errs[k], lim)
