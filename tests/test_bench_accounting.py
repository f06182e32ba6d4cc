"""bench.py's roofline accounting on the CPU: the algorithmic work per walker
follows the hot path's cost model (E = B + 1 edges, K = 10 phase-basis
functions, D detectors), and a reported fraction can be recomputed by hand
from the work, the walker count, the kernel time and the derived peak."""
import importlib.util
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parent.parent


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", ROOT / "bench.py")
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _by_hand(D, B, grad, K=10):
    E = B + 1
    fp64 = E * 2 * K + 8 * D * E + 300 + (E * K if grad else 0)  # basis dot product, delay + reduction, set-up
    fp32 = (22 * D * B + 6 * D * E) * (3 if grad else 1)         # r0, r1, contraction; ratio scaling
    sfu = D * E                                                  # one sin/cos per (edge, detector)
    return fp64, fp32, sfu


@pytest.mark.parametrize("D,B,grad", [(1, 100, False), (3, 500, True), (1, 100, True), (3, 1000, True)])
def test_algorithmic_work_matches_the_cost_model(bench, D, B, grad):
    w = bench.algorithmic_work(D, B, grad)
    fp64, fp32, sfu = _by_hand(D, B, grad)
    assert (w["fp64"], w["fp32"], w["sfu_sincos"]) == (fp64, fp32, sfu)
    assert w["total"] == fp64 + fp32 + sfu


def test_headline_work_and_fraction_by_hand(bench):
    # 3 detectors, 500 bins, with the gradient: 27,354 + 126,054 + 1,503
    w = bench.algorithmic_work(3, 500, True)
    assert (w["fp64"], w["fp32"], w["sfu_sincos"], w["total"]) == (27354, 126054, 1503, 154911)
    peak = 152 * 128 * 2 * 2070e6 / 1e12
    assert bench.fp32_peak_tflops() == pytest.approx(peak, rel=1e-12)
    r = bench.roofline_main(4096, 3, 500, True, 30.0e-6)
    assert r["achieved"] == pytest.approx(4096 * 154911 / 30.0e-6 / 1e12, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, rel=1e-12)
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # the implementation's own count is larger (float-pair emulation of the FP64-class work)
    assert r["impl_flops_per_walker"] > w["total"]
