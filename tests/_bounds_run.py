"""Runs the GPU paths through the bounds-checked debug library and writes
their outputs and the bounds record to the .npz named on the command line.
Started by test_gpu_bounds.py in a child process with RB_LIB_VARIANT=checked."""
import ctypes
import sys
from pathlib import Path

import numpy as np
import torch

sys.path.insert(0, str(Path(__file__).resolve().parents[1]))
from tests._bounds_paths import run_paths  # noqa: E402
import paper_2404_11397_gb300 as rb  # noqa: E402

assert rb.LIB_PATH.name == "librb_checked.so", rb.LIB_PATH
out = run_paths(rb)
torch.cuda.synchronize()
site, index, limit = ctypes.c_int(-1), ctypes.c_longlong(-1), ctypes.c_longlong(-1)
count = rb.load().rb_debug_bounds(ctypes.byref(site), ctypes.byref(index), ctypes.byref(limit))
np.savez(sys.argv[1], count=count, site=site.value, index=index.value, limit=limit.value, **out)
