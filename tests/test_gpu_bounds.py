"""The debug library (device-side bounds checks, -DRB_BOUNDS_CHECK) runs the
likelihood, summary, host-link and MALA paths with no index outside its
buffer, and gives the same bits as the normal library."""
import os
import subprocess
import sys
from pathlib import Path

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parents[1]


def test_checked_build_sees_no_out_of_bounds_index(tmp_path):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2404_11397_gb300 import build
    build.build(checked=True)
    res = tmp_path / "checked.npz"
    env = dict(os.environ, RB_LIB_VARIANT="checked")
    r = subprocess.run([sys.executable, str(ROOT / "tests" / "_bounds_run.py"), str(res)], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    chk = np.load(res)
    assert int(chk["count"]) == 0, (int(chk["count"]), int(chk["site"]), int(chk["index"]), int(chk["limit"]))
    # the same paths through the normal library
    import paper_2404_11397_gb300 as rb
    from tests._bounds_paths import run_paths
    assert rb.LIB_PATH.name == "librb.so"
    normal = run_paths(rb)
    for key, v in normal.items():
        np.testing.assert_array_equal(chk[key], v, err_msg=key)
