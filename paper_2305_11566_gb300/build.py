"""Build libstereovae.so (the CUDA library behind include/stereovae.h) in-tree.

nvcc compiles every translation unit for sm_103a only, in parallel; the coarse
matcher is compiled once per window radius (1..7) so its template instances build
side by side.  Objects go to _build/, the library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libstereovae.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "--expt-relaxed-constexpr", "-diag-suppress", "177"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libstereovae.so")


def units():
    """(source, extra defines, object name)"""
    out = []
    for f in sorted(os.listdir(CSRC)):
        if not f.endswith(".cu"):
            continue
        src = os.path.join(CSRC, f)
        if f == "zncc_wta.cu":
            for r in range(1, 8):
                out.append((src, [f"-DSV_ZNCC_R={r}"], f"zncc_wta_r{r}.o"))
        else:
            out.append((src, [], f[:-3] + ".o"))
    return out


def _deps_mtime() -> float:
    m = 0.0
    for d in (CSRC, os.path.join(os.path.dirname(HERE), "include")):
        for f in os.listdir(d):
            m = max(m, os.path.getmtime(os.path.join(d, f)))
    return m


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile and link; skipped when the library is newer than every source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    for src, defs, obj in units():
        jobs.append([nvcc, *ARCH, *FLAGS, *defs, "-c", src, "-o", os.path.join(BUILD, obj)])

    def run(cmd):
        p = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, p.returncode, p.stdout + p.stderr

    workers = max(1, min(len(jobs), os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(run, jobs))
    failed = [(c, o) for c, rc, o in results if rc != 0]
    if verbose:
        for c, rc, o in results:
            if o.strip():
                print(o, file=sys.stderr)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(" ".join(c) + "\n" + o for c, o in failed))
    objs = [os.path.join(BUILD, obj) for _, _, obj in units()]
    tmp = LIB + f".{os.getpid()}.tmp"
    p = subprocess.run([nvcc, *ARCH, "-shared", "-Xlinker", "-z", "-Xlinker", "defs", "-o", tmp, *objs], capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("link failed:\n" + p.stdout + p.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv), f"{time.time() - t:.1f}s")
