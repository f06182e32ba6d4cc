"""Multi-process (N > 1) path of bench.py on CPU: world size 2 over gloo.

The path is replicas only (every rank evaluates its own walkers; no
collective on the data path).  The timing aggregation takes the slowest
rank's timed total and counts the units of all ranks; under torchrun the
reference arm runs on rank 0 only and the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys
from pathlib import Path

import pytest
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parent.parent


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, str(ROOT))
    import bench
    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    # rank r timed (r + 1) seconds for 100 units: the job time is the slowest rank's
    t, v = bench.whole_job_rate(d, float(rank + 1), 100.0)
    ref = bench.run_reference(type("A", (), {"steps": 1, "warmup": 0})(), d) if rank != 0 else "skipped"
    out[rank] = (t, v, ref)
    d.close()


def test_whole_job_rate_two_ranks():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        t, v, ref = out[r]
        assert t == pytest.approx(2.0)
        assert v == pytest.approx(100.0 * world / 2.0)
    assert out[1][2] is None  # the reference arm does no work off rank 0


@pytest.mark.slow
def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), str(ROOT / "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    res = json.loads(lines[0])
    assert res["impl"] == "reference" and res["n_gpus"] == 2 and res["value"] > 0
    assert res["cpu_baseline"]["kind"] == "oracle"
    assert res["warmup"] >= 3 and res["steps"] == 1 and res["higher_is_better"] is True
    assert 0 < res["cpu_baseline"]["value_1_core"] <= res["value"] * 1.5
    assert res["e2e"]["value"] == res["value"] and res["e2e"]["h2d_bytes_per_step"] == 0
