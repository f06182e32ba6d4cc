"""Build librb.so in-tree: nvcc for sm_103a, one translation unit per source,
compiled in parallel, linked as a shared library with the C ABI of include/rb.h."""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
INCLUDE = ROOT / "include"
BUILD = PKG / "_build"
LIB = PKG / "librb.so"
SOURCES = ["rb_setup.cu", "rb_loglike.cu", "rb_summary.cu", "rb_api.cu", "rb_server.cu", "rb_static.cu", "rb_mala.cu",
           "rb_full.cu", "rb_bins.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         f"-I{INCLUDE}", f"-I{CSRC}"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out: Path, deps) -> bool:
    if not out.exists():
        return True
    t = out.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build(verbose: bool = False, force: bool = False, checked: bool = False) -> Path:
    """Compile librb.so; with checked=True the debug variant librb_checked.so
    (device-side bounds checks, -DRB_BOUNDS_CHECK) in its own build folder."""
    build_dir = BUILD.with_name("_build_checked") if checked else BUILD
    lib_path = LIB.with_name("librb_checked.so") if checked else LIB
    flags = FLAGS + (["-DRB_BOUNDS_CHECK"] if checked else [])
    build_dir.mkdir(exist_ok=True)
    headers = list(CSRC.glob("*.cuh")) + list(CSRC.glob("*.h")) + list(INCLUDE.glob("*.h"))
    cc = nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        s = CSRC / src
        o = build_dir / (Path(src).stem + ".o")
        objs.append(o)
        if force or _stale(o, [s, *headers]):
            jobs.append([cc, *ARCH, *flags, "-c", str(s), "-o", str(o)])

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r

    with ThreadPoolExecutor(max_workers=min(len(SOURCES), os.cpu_count() or 1)) as ex:
        list(ex.map(run, jobs))
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path.with_suffix(f".{os.getpid()}.tmp")
        run([cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-lpthread", "-ldl"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, checked="--checked" in sys.argv))
