"""In-tree build of the CUDA library ``libqoco_gpu.so`` for sm_103a.

CUDA sources go through nvcc (``-gencode arch=compute_103a,code=sm_103a``), host
C++ through g++; translation units compile in parallel and link into one shared
library next to this file, with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqoco_gpu.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def sources():
    cu = sorted(f for f in os.listdir(SRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(SRC) if f.endswith(".cpp"))
    return cu, cpp


def build(verbose: bool = False, force: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    cu, cpp = sources()
    inc = ["-I", os.path.join(ROOT, "include"), "-I", SRC]
    nvcc = _nvcc()
    jobs = []
    objs = []
    newest_src = max(os.path.getmtime(os.path.join(d, f))
                     for d, fs in ((SRC, os.listdir(SRC)), (os.path.join(ROOT, "include"),
                                                               os.listdir(os.path.join(ROOT, "include"))))
                     for f in fs)
    for f in cu:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(SRC, f), "-o", o]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((o, cmd))
    for f in cpp:
        o = os.path.join(OUT_DIR, f + ".o")
        objs.append(o)
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", *inc,
               "-I", os.path.join(os.path.dirname(nvcc), "..", "include"),
               "-c", os.path.join(SRC, f), "-o", o]
        jobs.append((o, cmd))
    todo = [(o, c) for o, c in jobs
            if force or ptxas_info or not os.path.exists(o) or os.path.getmtime(o) < newest_src]
    logs = []
    if todo:
        with cf.ThreadPoolExecutor(max_workers=min(len(todo), os.cpu_count() or 4)) as ex:
            for out in ex.map(lambda oc: _run(oc[1]), todo):
                logs.append(out)
    if todo or not os.path.exists(LIB):
        tmp = LIB + ".tmp"
        _run([nvcc, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs, "-lpthread"])
        os.replace(tmp, LIB)
    if verbose:
        print("\n".join(l for l in logs if l.strip()))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, force="--force" in sys.argv, ptxas_info="--ptxas" in sys.argv))
