"""Seeded synthetic inputs: R-MAT graphs, edge weights, PPR seed sets, targets.

Inputs only: nothing here computes any part of the graph method. The FP64
oracle tests and the CUDA path both take their graphs from this module, so the
two sides see bit-identical edge lists. The stream definition is in
``rmat.cu`` (SplitMix64 output function over a counter; R-MAT quadrant choice
per bit level with a/b/c/d = 0.57/0.19/0.19/0.05 unless given).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "librmat.so")
_lib = None

A, B, C = 0.57, 0.19, 0.19


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(
                f"{_LIB_PATH} is missing; run __graft_entry__.build() "
                "(or python -m paper_1510_06916_b300.build) first")
        lib = ctypes.CDLL(_LIB_PATH)
        u64, i32 = ctypes.c_uint64, ctypes.c_int
        vp = ctypes.c_void_p
        lib.rmat_generate_host.argtypes = [u64, i32, u64, u64, u64, u64, u64, vp, vp, vp]
        lib.rmat_generate_host.restype = i32
        lib.rmat_generate_device.argtypes = [u64, i32, u64, u64, u64, u64, u64, vp, vp, vp, vp]
        lib.rmat_generate_device.restype = i32
        lib.rmat_draws_host.argtypes = [u64, u64, u64, vp]
        lib.rmat_draws_host.restype = i32
        _lib = lib
    return _lib


def thresholds(a=A, b=B, c=C):
    """Cumulative quadrant probabilities scaled to 2^64 (truncated)."""
    two64 = float(2 ** 64)
    ta = int(a * two64)
    tab = int((a + b) * two64)
    tabc = int((a + b + c) * two64)
    cap = 2 ** 64 - 1
    return min(ta, cap), min(tab, cap), min(tabc, cap)


def rmat_edges(scale: int, m: int, seed: int, a=A, b=B, c=C, weights=False, e0: int = 0):
    """Host R-MAT edge list: (src uint32[m], dst uint32[m], w float32[m] or None)."""
    lib = _load()
    ta, tab, tabc = thresholds(a, b, c)
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    w = np.empty(m, dtype=np.float32) if weights else None
    lib.rmat_generate_host(seed, scale, e0, m, ta, tab, tabc, src.ctypes.data, dst.ctypes.data,
                           w.ctypes.data if weights else None)
    return src, dst, w


def rmat_edges_device(scale: int, m: int, seed: int, a=A, b=B, c=C, weights=False, device="cuda"):
    """Same stream generated straight into device memory (torch tensors)."""
    import torch

    lib = _load()
    ta, tab, tabc = thresholds(a, b, c)
    src = torch.empty(m, dtype=torch.int32, device=device)
    dst = torch.empty(m, dtype=torch.int32, device=device)
    w = torch.empty(m, dtype=torch.float32, device=device) if weights else None
    stream = torch.cuda.current_stream(src.device).cuda_stream
    rc = lib.rmat_generate_device(seed, scale, 0, m, ta, tab, tabc, src.data_ptr(),
                                  dst.data_ptr(), w.data_ptr() if weights else None, stream)
    if rc != 0:
        raise RuntimeError(f"rmat_generate_device failed with cudaError {rc}")
    return src, dst, w


def draws(seed: int, k0: int, count: int) -> np.ndarray:
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.rmat_draws_host(seed, k0, count, out.ctypes.data)
    return out


def _distinct(seed: int, k0: int, k: int, n: int) -> np.ndarray:
    """k distinct vertices in [0, n): draws k0+1, k0+2, ... taken mod n, repeats skipped."""
    k = min(k, n)
    chosen: list[int] = []
    seen: set[int] = set()
    t = 1
    while len(chosen) < k:
        batch = draws(seed, k0 + t, max(64, 2 * (k - len(chosen))))
        t += len(batch)
        for u in batch:
            v = int(u % np.uint64(n))
            if v not in seen:
                seen.add(v)
                chosen.append(v)
                if len(chosen) == k:
                    break
    return np.array(chosen, dtype=np.int64)


def ppr_teleports(n: int, batch: int, seed: int, max_seeds: int = 1000) -> np.ndarray:
    """[n, batch] float32 teleport matrix; column b is uniform over k_b seeds.

    k_b = 1 + (u(seed, b*2^32) mod max_seeds); the seeds are distinct draws
    u(seed, b*2^32 + t) mod n, t = 1, 2, ...
    """
    T = np.zeros((n, batch), dtype=np.float32)
    for bi in range(batch):
        k0 = bi << 32
        kb = 1 + int(draws(seed, k0, 1)[0] % np.uint64(max_seeds))
        seeds = _distinct(seed, k0, kb, n)
        T[seeds, bi] = np.float32(1.0 / len(seeds))
    return T


def ppr_seed_lists(n: int, batch: int, seed: int, max_seeds: int = 1000):
    """Sparse form of ppr_teleports: (vertex, column, value) arrays of the nonzeros."""
    vs, bs, ts = [], [], []
    for bi in range(batch):
        k0 = bi << 32
        kb = 1 + int(draws(seed, k0, 1)[0] % np.uint64(max_seeds))
        seeds = _distinct(seed, k0, kb, n)
        vs.append(seeds)
        bs.append(np.full(len(seeds), bi, dtype=np.int64))
        ts.append(np.full(len(seeds), 1.0 / len(seeds), dtype=np.float32))
    return np.concatenate(vs), np.concatenate(bs), np.concatenate(ts)


def targets(n: int, count: int, seed: int) -> np.ndarray:
    """`count` distinct target vertices (stream seed, draws 1, 2, ...)."""
    return _distinct(seed, 0, count, n)


def multigraph_scales(count: int, lo: int = 10, hi: int = 18, seed: int = 3) -> list[int]:
    """Scale of graph g = lo + u(seed, 2^48 + g) mod (hi - lo + 1)."""
    u = draws(seed, 1 << 48, count)
    return [lo + int(x % np.uint64(hi - lo + 1)) for x in u]


def multigraph_seed(g: int, base: int = 3) -> int:
    return (base << 16) + g
