"""FP64 CPU oracle for the NXgraph DSSS update sweep (arXiv 1510.06916).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package. It shares no
code with the CUDA path (``paper_1510_06916_b300``) and never imports it.

Functions and the passage each follows:

* ``pagerank`` — PageRank / personalized / weighted PageRank in double
  precision (the paper's main task, Section IV; the formula it leaves out is
  the standard damped form with dangling mass, written out in nx_oracle.c).
* ``bfs`` — Algorithms 2-4 (root depth 0, others infinity, min depth+1).
* ``wcc`` — weakly connected components, min vertex id per component
  (Section IV-D names WCC; undirected = both directions, Section II-A).
* ``scc`` — strongly connected components, min vertex id per component
  (Section IV-D names SCC), by Tarjan's depth-first search.
* ``bfs_max_depth`` — Algorithm 4's Output: the largest finite depth.
* ``PreparedPageRank`` — the ``pagerank`` arithmetic with its CSR built once,
  so that the iteration loop can be timed on its own.
* ``wpr_adjoint`` — adjoint of weighted PageRank (an extension; the paper has
  no counterpart), the Neumann-series fixed-point formula in nx_oracle.c.
* ``dsss_order`` — the Destination-Sorted Sub-Shard layout of Section II-A and
  III-A: P equal intervals of ceil(n/P) vertices, sub-shard SS_ij holds the
  edges with source in I_i and destination in I_j, sorted by destination then
  by source. Written with numpy's lexsort as the sort step.

Parity is pinned by tests/test_oracle_pins.py (closed forms, brute force,
dense linear algebra, invariants, the Fig. 1 example); every function here has
at least one pin there.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None
INF = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile nx_oracle.c with gcc (-O2, OpenMP) into liboracle.so."""
    import subprocess

    srcf = os.path.join(_HERE, "nx_oracle.c")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(srcf):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, srcf])
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp, u32, u64, dbl, i32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_double, ctypes.c_int)
        lib.orc_pagerank.argtypes = [u32, u64, vp, vp, vp, dbl, u32, vp, i32, vp, vp]
        lib.orc_bfs.argtypes = [u32, u64, vp, vp, u32, vp]
        lib.orc_wcc.argtypes = [u32, u64, vp, vp, vp]
        lib.orc_scc.argtypes = [u32, u64, vp, vp, vp]
        lib.orc_pr_prepare.argtypes = [u32, u64, vp, vp, vp, ctypes.POINTER(vp)]
        lib.orc_pr_iterate.argtypes = [vp, dbl, u32, vp, i32, vp, vp]
        lib.orc_pr_release.argtypes = [vp]
        lib.orc_pr_release.restype = None
        lib.orc_set_threads.argtypes = [i32]
        lib.orc_set_threads.restype = None
        lib.orc_wpr_adjoint.argtypes = [u32, u64, vp, vp, vp, dbl, u32, u32, vp, vp, vp, vp,
                                        vp, vp]
        for f in (lib.orc_pagerank, lib.orc_bfs, lib.orc_wcc, lib.orc_scc, lib.orc_wpr_adjoint,
                  lib.orc_pr_prepare, lib.orc_pr_iterate):
            f.restype = i32
        _lib = lib
    return _lib


def set_threads(k: int | None) -> None:
    """Bound the OpenMP threads the oracle uses from now on (None: no change)."""
    if k is not None:
        os.environ["OMP_NUM_THREADS"] = str(k)
        _load().orc_set_threads(int(k))


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def pagerank(n, src, dst, alpha=0.85, iters=20, w=None, tele=None, dangling_by_tele=False,
             r0=None) -> np.ndarray:
    src, dst = _u32(src), _u32(dst)
    w, tele, r0 = _f64(w), _f64(tele), _f64(r0)
    out = np.empty(n, dtype=np.float64)
    rc = _load().orc_pagerank(n, len(src), _ptr(src), _ptr(dst), _ptr(w), alpha, iters,
                              _ptr(tele), int(dangling_by_tele), _ptr(r0), _ptr(out))
    if rc:
        raise ValueError("orc_pagerank: bad arguments")
    return out


def personalized_pagerank(n, src, dst, tele, alpha=0.85, iters=30) -> np.ndarray:
    """PPR: r0 = t, teleport t, dangling mass spread by t."""
    tele = _f64(tele)
    return pagerank(n, src, dst, alpha, iters, tele=tele, dangling_by_tele=True, r0=tele)


def bfs(n, src, dst, root=0) -> np.ndarray:
    src, dst = _u32(src), _u32(dst)
    out = np.empty(n, dtype=np.uint32)
    if _load().orc_bfs(n, len(src), _ptr(src), _ptr(dst), root, _ptr(out)):
        raise ValueError("orc_bfs: bad arguments")
    return out


def wcc(n, src, dst) -> np.ndarray:
    src, dst = _u32(src), _u32(dst)
    out = np.empty(n, dtype=np.uint32)
    if _load().orc_wcc(n, len(src), _ptr(src), _ptr(dst), _ptr(out)):
        raise ValueError("orc_wcc: bad arguments")
    return out


def scc(n, src, dst) -> np.ndarray:
    src, dst = _u32(src), _u32(dst)
    out = np.empty(n, dtype=np.uint32)
    if _load().orc_scc(n, len(src), _ptr(src), _ptr(dst), _ptr(out)):
        raise ValueError("orc_scc: bad arguments")
    return out


def bfs_max_depth(depth) -> int:
    """Algorithm 4 (Output): the largest finite depth (-1 if none is finite)."""
    depth = np.asarray(depth, dtype=np.uint32)
    fin = depth[depth != INF]
    return int(fin.max()) if len(fin) else -1


class PreparedPageRank:
    """PageRank-family problem with the oracle's CSR built once (same
    arithmetic as :func:`pagerank`); ``iterate`` runs only the iteration loop."""

    def __init__(self, n, src, dst, w=None):
        src, dst = _u32(src), _u32(dst)
        w = _f64(w)
        self.n = n
        self._h = ctypes.c_void_p()
        if _load().orc_pr_prepare(n, len(src), _ptr(src), _ptr(dst), _ptr(w),
                                  ctypes.byref(self._h)):
            raise ValueError("orc_pr_prepare: bad arguments or out of memory")

    def iterate(self, alpha=0.85, iters=20, tele=None, dangling_by_tele=False, r0=None):
        tele, r0 = _f64(tele), _f64(r0)
        out = np.empty(self.n, dtype=np.float64)
        if _load().orc_pr_iterate(self._h, alpha, iters, _ptr(tele), int(dangling_by_tele),
                                  _ptr(r0), _ptr(out)):
            raise ValueError("orc_pr_iterate: bad arguments")
        return out

    def close(self):
        if self._h:
            _load().orc_pr_release(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wpr_adjoint(n, src, dst, w, g, alpha=0.85, fwd_iters=50, adj_terms=50, tele=None):
    """Returns dict(r, lam, dw, dt) in float64."""
    src, dst = _u32(src), _u32(dst)
    w, g, tele = _f64(w), _f64(g), _f64(tele)
    m = len(src)
    r = np.empty(n)
    lam = np.empty(n)
    dw = np.empty(m)
    dt = np.empty(n)
    rc = _load().orc_wpr_adjoint(n, m, _ptr(src), _ptr(dst), _ptr(w), alpha, fwd_iters,
                                 adj_terms, _ptr(tele), _ptr(g), _ptr(r), _ptr(lam), _ptr(dw),
                                 _ptr(dt))
    if rc:
        raise ValueError("orc_wpr_adjoint: bad arguments")
    return {"r": r, "lam": lam, "dw": dw, "dt": dt}


def dsss_order(n, P, src, dst):
    """DSSS layout of Section II-A / III-A.

    Returns (order, sub_off): ``order`` lists input edge indices shard by shard
    (destination interval j), sub-shard by sub-shard within it (source interval
    i), each sub-shard sorted by destination then source; ``sub_off[j*P + i]``
    is where SS_ij starts in that order (length P*P + 1).
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    L = -(-n // P)
    i = src // L
    j = dst // L
    order = np.lexsort((src, dst, i, j))
    sub = (j * P + i)[order]
    counts = np.bincount(sub, minlength=P * P)
    sub_off = np.concatenate([[0], np.cumsum(counts)])
    return order, sub_off
