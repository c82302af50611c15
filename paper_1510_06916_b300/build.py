"""Builds the in-tree shared libraries for sm_103a.

* ``csrc/libnxgraph.so`` — the C-ABI library (every ``csrc/*.cu``).
* ``inputs/librmat.so`` — the seeded workload generator.

Run as ``python -m paper_1510_06916_b300.build``; ``__graft_entry__.build()``
calls :func:`build_all`.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _newer(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd: list[str]) -> None:
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("build failed: " + " ".join(cmd))


def build_nxgraph(verbose_ptxas: bool = False, force: bool = False) -> str:
    out = os.path.join(CSRC, "libnxgraph.so")
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    hdrs = sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(HERE, "..", "include", "nxgraph.h")]
    objdir = os.path.join(CSRC, "_build")
    os.makedirs(objdir, exist_ok=True)
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(objdir, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _newer(o, [s] + hdrs):
            cmd = [NVCC, *ARCH, *FLAGS, "-c", s, "-o", o]
            if verbose_ptxas:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        list(ex.map(_run, jobs))
    if force or jobs or _newer(out, objs):
        _run([NVCC, *ARCH, "-shared", "-o", out, *objs, "-lcudart"])
    return out


def build_rmat(force: bool = False) -> str:
    d = os.path.join(HERE, "inputs")
    src = os.path.join(d, "rmat.cu")
    out = os.path.join(d, "librmat.so")
    if force or _newer(out, [src]):
        _run([NVCC, *ARCH, "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-fopenmp", "-shared", "-o",
              out, src, "-lgomp"])
    return out


def build_all(force: bool = False) -> list[str]:
    return [build_rmat(force), build_nxgraph(force=force)]


if __name__ == "__main__":
    for p in build_all(force="--force" in sys.argv):
        print(p)
