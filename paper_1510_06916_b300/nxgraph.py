"""Thin ctypes binding of the C ABI in ``include/nxgraph.h``.

Argument marshalling only: every step of the sweep runs in ``libnxgraph.so``.
Arrays may be numpy arrays (host) or torch CUDA tensors (device); the binding
passes their pointers and the matching ``*_is_device`` flag. Importing this
module without the built library raises immediately — there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "csrc", "libnxgraph.so")

NX_OK, NX_ERR_INVALID_ARG, NX_ERR_OOM, NX_ERR_BUDGET_TOO_SMALL, NX_ERR_CUDA, NX_ERR_TIMEOUT = range(6)
PR, PPR, WPR, BFS, WCC, SCC = range(6)
SPU, DPU, MPU, AUTO, SRC_COARSE, SRC_FINE, DPU_ONCHIP = range(7)
HOST_PTRS, DEV_PTRS, WITH_TRANSPOSE, WITH_WEIGHTS, RELABEL, ONCHIP_HUBS = 0, 1, 2, 4, 8, 16
INF = 0xFFFFFFFF

PROGRAMS = {"pr": PR, "ppr": PPR, "wpr": WPR, "bfs": BFS, "wcc": WCC, "scc": SCC}
STRATEGIES = {"spu": SPU, "dpu": DPU, "mpu": MPU, "auto": AUTO,
              "src_coarse": SRC_COARSE, "src_fine": SRC_FINE, "dpu_onchip": DPU_ONCHIP}

EXPORTS = [
    "nx_set_stream", "nx_trim_memory", "nx_debug_fail_alloc", "nx_last_error", "nx_build_dsss", "nx_graph_get_info", "nx_run",
    "nx_get_values", "nx_set_values", "nx_run_ppr_batch", "nx_adjoint_wpr", "nx_run_multi",
    "nx_graph_free", "nx_io_model", "nx_dsss_export", "nx_pagerank_step_noalloc",
    "nx_autotune", "nx_get_relabel", "nx_bfs_max_depth", "nx_set_barrier_limit",
    "nx_gather_probe", "nx_autotune_shape", "nx_set_batch_shape", "nx_autotune_ppr_batch",
]


class NxParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_float), ("root", ctypes.c_uint32),
                ("teleport", ctypes.c_void_p), ("teleport_is_device", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("band_intervals", ctypes.c_uint32)]


class NxRunStats(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_uint32), ("Q", ctypes.c_uint32),
                ("strategy", ctypes.c_uint32), ("streamed_cols", ctypes.c_uint32),
                ("ms", ctypes.c_float), ("edges_swept", ctypes.c_uint64),
                ("bytes_model", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64), ("launches", ctypes.c_uint32),
                ("intervals_skipped", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class NxShape(ctypes.Structure):
    _fields_ = [("P", ctypes.c_uint32), ("tile_cap_log2", ctypes.c_uint32),
                ("tile_edges_log2", ctypes.c_uint32), ("pad_", ctypes.c_uint32)]


class NxBatchShape(ctypes.Structure):
    _fields_ = [("rows", ctypes.c_uint32), ("sub", ctypes.c_uint32)]


class NxGraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("P", ctypes.c_uint32), ("L", ctypes.c_uint32),
                ("ntiles", ctypes.c_uint32), ("tile_max", ctypes.c_uint32),
                ("lb", ctypes.c_uint32), ("m", ctypes.c_uint64), ("D", ctypes.c_uint64),
                ("D_t", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("build_ms", ctypes.c_float), ("has_transpose", ctypes.c_int32),
                ("has_weights", ctypes.c_int32), ("host_bytes", ctypes.c_uint64),
                ("H_onchip", ctypes.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Loads libnxgraph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1510_06916_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, u32, u64, i32, f32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64,
                                  ctypes.c_int32, ctypes.c_float)
        d = ctypes.c_double
        L.nx_set_stream.argtypes = [vp]
        L.nx_trim_memory.argtypes = []
        L.nx_debug_fail_alloc.argtypes = [ctypes.c_int64]
        L.nx_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        L.nx_last_error.restype = None
        L.nx_build_dsss.argtypes = [vp, vp, u64, u32, u32, u32, vp, ctypes.POINTER(vp)]
        L.nx_graph_get_info.argtypes = [vp, ctypes.POINTER(NxGraphInfo)]
        L.nx_run.argtypes = [vp, i32, ctypes.POINTER(NxParams), u32, i32, u64,
                             ctypes.POINTER(NxRunStats)]
        L.nx_get_values.argtypes = [vp, vp, u64, i32]
        L.nx_set_values.argtypes = [vp, i32, vp, u64, i32]
        L.nx_run_ppr_batch.argtypes = [vp, vp, u32, u32, f32, vp, i32, ctypes.POINTER(NxRunStats)]
        L.nx_adjoint_wpr.argtypes = [vp, vp, u32, vp, vp, i32, ctypes.POINTER(NxRunStats)]
        L.nx_run_multi.argtypes = [ctypes.POINTER(vp), u32, i32, f32, u32,
                                   ctypes.POINTER(NxRunStats)]
        L.nx_dsss_export.argtypes = [vp, i32, vp, vp, vp]
        L.nx_get_relabel.argtypes = [vp, vp, u64, i32]
        L.nx_pagerank_step_noalloc.argtypes = [vp, f32, vp, vp]
        L.nx_autotune.argtypes = [vp, vp, u64, u32, u32, vp, i32, vp, u32, u32,
                                  ctypes.POINTER(u32), vp, ctypes.c_char_p]
        L.nx_bfs_max_depth.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
        L.nx_set_barrier_limit.argtypes = [u64]
        L.nx_gather_probe.argtypes = [vp, u32, ctypes.POINTER(f32)]
        L.nx_autotune_shape.argtypes = [vp, vp, u64, u32, u32, vp, i32, ctypes.POINTER(NxShape),
                                        u32, u32, ctypes.POINTER(u32), vp, ctypes.c_char_p]
        L.nx_set_batch_shape.argtypes = [vp, u32, u32]
        L.nx_autotune_ppr_batch.argtypes = [vp, vp, u32, u32, f32, i32,
                                            ctypes.POINTER(NxBatchShape), u32, ctypes.POINTER(u32),
                                            vp, ctypes.c_char_p]
        L.nx_graph_free.argtypes = [vp]
        L.nx_graph_free.restype = None
        L.nx_io_model.argtypes = [i32, d, d, d, d, d, d, d, d, ctypes.POINTER(d),
                                  ctypes.POINTER(d), ctypes.POINTER(d)]
        for name in EXPORTS:
            f = getattr(L, name)
            if name not in ("nx_last_error", "nx_graph_free"):
                f.restype = i32
        _lib = L
    return _lib


class NxError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"nxgraph error {code}: {msg}")
        self.code = code


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().nx_last_error(buf, 512)
    return buf.value.decode(errors="replace")


def check(rc: int) -> None:
    if rc != NX_OK:
        raise NxError(rc, last_error())


def _ptr(a):
    """(pointer, is_device) of a numpy array or torch tensor (None -> (None, 0))."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be contiguous")
        return a.ctypes.data, 0
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(a, torch.Tensor):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    raise TypeError(f"unsupported array type {type(a)}")


def set_stream(stream) -> None:
    """Stream for later calls: a torch.cuda.Stream, a raw handle, or None."""
    h = getattr(stream, "cuda_stream", stream)
    check(lib().nx_set_stream(ctypes.c_void_p(h or 0)))


def trim_memory() -> None:
    """Returns the library's cached, unused device memory to the driver."""
    check(lib().nx_trim_memory())


def debug_fail_alloc(after: int) -> None:
    """Test hook: the library's device allocation `after` allocations from now
    fails as out of memory (NX_ERR_OOM); a negative value disarms it."""
    check(lib().nx_debug_fail_alloc(int(after)))


def set_barrier_limit(cycles: int) -> None:
    """Grid-barrier wait limit of run_multi in GPU clock cycles (0: default)."""
    check(lib().nx_set_barrier_limit(cycles))


def io_model(strategy, n, m, P, B_M, B_a=4.0, B_v=4.0, B_e=4.0, d=15.0):
    """Section III-B / Table II byte model -> (Q, bytes_read, bytes_write)."""
    q, r, w = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    check(lib().nx_io_model(STRATEGIES.get(strategy, strategy), n, m, P, B_M, B_a, B_v, B_e, d,
                            ctypes.byref(q), ctypes.byref(r), ctypes.byref(w)))
    return q.value, r.value, w.value


class Graph:
    """A DSSS built on the current device (owns it; free() or context exit)."""

    def __init__(self, src, dst, n: int, P: int, transpose: bool = False, weights=None,
                 relabel: bool = False, tile_cap_log2: int = 0, tile_edges_log2: int = 0,
                 onchip: bool = False):
        if isinstance(src, np.ndarray):
            src = np.ascontiguousarray(src, dtype=np.uint32)
        if isinstance(dst, np.ndarray):
            dst = np.ascontiguousarray(dst, dtype=np.uint32)
        if isinstance(weights, np.ndarray):
            weights = np.ascontiguousarray(weights, dtype=np.float32)
        for a in (src, dst, weights):
            if a is not None and not isinstance(a, np.ndarray) and a.element_size() != 4:
                raise ValueError("edge arrays must hold 4-byte elements (int32/uint32/float32)")
        self._keep = (src, dst, weights)  # alive for the duration of the build
        sp, sd = _ptr(src)
        dp, dd = _ptr(dst)
        if sd != dd:
            raise ValueError("src and dst must both be host or both be device arrays")
        m = len(src)
        if len(dst) != m:
            raise ValueError("src and dst differ in length")
        flags = DEV_PTRS if sd else HOST_PTRS
        if transpose:
            flags |= WITH_TRANSPOSE
        if relabel:
            flags |= RELABEL
        if onchip:
            flags |= ONCHIP_HUBS
        flags |= (tile_cap_log2 << 8) | (tile_edges_log2 << 12)
        wp = None
        if weights is not None:
            wp, wd = _ptr(weights)
            if wd != sd:
                raise ValueError("weights must live where src/dst live")
            flags |= WITH_WEIGHTS
        h = ctypes.c_void_p()
        check(lib().nx_build_dsss(sp, dp, m, n, P, flags, wp, ctypes.byref(h)))
        self._h = h
        self.n, self.m, self.P = n, m, P

    @property
    def handle(self):
        return self._h

    def relabel_map(self) -> np.ndarray:
        """old_of_new[k] = caller id of internal vertex k (graphs built with relabel=True)."""
        out = np.empty(self.n, dtype=np.uint32)
        check(lib().nx_get_relabel(self._h, out.ctypes.data, self.n, 0))
        return out

    def free(self):
        if self._h:
            lib().nx_graph_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def info(self) -> dict:
        inf = NxGraphInfo()
        check(lib().nx_graph_get_info(self._h, ctypes.byref(inf)))
        return inf.as_dict()

    def export(self, transpose=False):
        """Stored DSSS order: (src, dst, sub_off) as numpy arrays."""
        s = np.empty(self.m, dtype=np.uint32)
        d = np.empty(self.m, dtype=np.uint32)
        off = np.empty(self.P * self.P + 1, dtype=np.uint64)
        check(lib().nx_dsss_export(self._h, 1 if transpose else 0, s.ctypes.data, d.ctypes.data,
                                   off.ctypes.data))
        return s, d, off

    def run(self, program="pr", iters=20, strategy="spu", budget=0, alpha=0.85, root=0,
            teleport=None, use_graph=False, band=0) -> dict:
        prm = NxParams()
        prm.band_intervals = band
        prm.alpha = alpha
        prm.root = root
        tp, td = _ptr(teleport)
        prm.teleport = tp
        prm.teleport_is_device = td
        prm.use_graph = 1 if use_graph else 0
        st = NxRunStats()
        check(lib().nx_run(self._h, PROGRAMS.get(program, program), ctypes.byref(prm), iters,
                           STRATEGIES.get(strategy, strategy), budget, ctypes.byref(st)))
        return st.as_dict()

    def gather_probe(self, sweeps=10) -> float:
        """ms per pass of the sweep's loads and gathers alone (no reduction)."""
        v = ctypes.c_float()
        check(lib().nx_gather_probe(self._h, sweeps, ctypes.byref(v)))
        return v.value

    def bfs_max_depth(self) -> int:
        """Algorithm 4's Output for the last BFS run: largest finite depth (-1: none)."""
        v = ctypes.c_int64()
        check(lib().nx_bfs_max_depth(self._h, ctypes.byref(v)))
        return v.value

    def values(self, out=None, dtype=None):
        """Current values: float32 ranks (PageRank family) or uint32 depth/labels."""
        if out is None:
            out = np.empty(self.n, dtype=dtype or np.float32)
        p, dev = _ptr(out)
        check(lib().nx_get_values(self._h, p, self.n, dev))
        return out

    def set_values(self, program, values):
        p, dev = _ptr(values)
        check(lib().nx_set_values(self._h, PROGRAMS.get(program, program), p, self.n, dev))

    def ppr_batch(self, teleport, iters=30, alpha=0.85, out=None) -> tuple:
        B = teleport.shape[1]
        if out is None:
            out = np.empty_like(teleport) if isinstance(teleport, np.ndarray) else teleport.new_empty(teleport.shape)
        tp, td = _ptr(teleport)
        op, od = _ptr(out)
        if td != od:
            raise ValueError("teleport and output must both be host or both device")
        st = NxRunStats()
        check(lib().nx_run_ppr_batch(self._h, tp, B, iters, alpha, op, td, ctypes.byref(st)))
        return out, st.as_dict()

    def set_batch_shape(self, rows=4, sub=128):
        """Batched-PPR shape: source rows in flight per lane group, destinations per sub-tile."""
        check(lib().nx_set_batch_shape(self._h, rows, sub))

    def autotune_ppr_batch(self, teleport, iters=5, shapes=((2, 128), (4, 128), (8, 128)),
                           alpha=0.85, cache=None):
        """Fastest batched-PPR shape [(rows, sub), ...], kept on the graph.
        Returns (index, ms_per_iter list)."""
        cand = (NxBatchShape * len(shapes))(*[NxBatchShape(int(r), int(q)) for r, q in shapes])
        ms = np.empty(len(shapes), dtype=np.float32)
        best = ctypes.c_uint32()
        tp, td = _ptr(teleport)
        check(lib().nx_autotune_ppr_batch(self._h, tp, teleport.shape[1], iters, alpha, td, cand,
                                          len(shapes), ctypes.byref(best), ms.ctypes.data,
                                          cache.encode() if cache else None))
        return int(best.value), ms.tolist()

    def adjoint_wpr(self, grad_r, adj_terms, grad_w, grad_t=None) -> dict:
        gp, gd = _ptr(grad_r)
        wp, wd = _ptr(grad_w)
        tp, td = _ptr(grad_t)
        if gd != wd or (grad_t is not None and td != gd):
            raise ValueError("gradient buffers must all be host or all device")
        st = NxRunStats()
        check(lib().nx_adjoint_wpr(self._h, gp, adj_terms, wp, tp, gd, ctypes.byref(st)))
        return st.as_dict()


def autotune(src, dst, n, candidates=(8, 16, 32, 64), program="pr", iters=10, cache=None,
             transpose=False):
    """Fastest P among `candidates` (builds and times each). Returns (P, ms_per_iter list)."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
    sp, sd = _ptr(src)
    dp, _ = _ptr(dst)
    cand = np.ascontiguousarray(candidates, dtype=np.uint32)
    ms = np.empty(len(cand), dtype=np.float32)
    best = ctypes.c_uint32()
    flags = (DEV_PTRS if sd else HOST_PTRS) | (WITH_TRANSPOSE if transpose else 0)
    check(lib().nx_autotune(sp, dp, len(src), n, flags, None, PROGRAMS.get(program, program),
                            cand.ctypes.data, len(cand), iters, ctypes.byref(best), ms.ctypes.data,
                            cache.encode() if cache else None))
    return int(best.value), ms.tolist()


def autotune_shape(src, dst, n, shapes, program="pr", iters=10, cache=None, transpose=False,
                   relabel=False):
    """Fastest of `shapes` [(P, tile_cap_log2, tile_edges_log2), ...] (0 = default).
    Returns (index, ms_per_iter list); ms are -1 when served from the cache."""
    if isinstance(src, np.ndarray):
        src = np.ascontiguousarray(src, dtype=np.uint32)
        dst = np.ascontiguousarray(dst, dtype=np.uint32)
    sp, sd = _ptr(src)
    dp, _ = _ptr(dst)
    cand = (NxShape * len(shapes))(*[NxShape(int(p), int(c), int(e), 0) for p, c, e in shapes])
    ms = np.empty(len(shapes), dtype=np.float32)
    best = ctypes.c_uint32()
    flags = (DEV_PTRS if sd else HOST_PTRS) | (WITH_TRANSPOSE if transpose else 0) | (RELABEL if relabel else 0)
    check(lib().nx_autotune_shape(sp, dp, len(src), n, flags, None,
                                  PROGRAMS.get(program, program), cand, len(shapes), iters,
                                  ctypes.byref(best), ms.ctypes.data,
                                  cache.encode() if cache else None))
    return int(best.value), ms.tolist()


def run_multi(graphs, program="pr", iters=20, alpha=0.85) -> dict:
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    st = NxRunStats()
    check(lib().nx_run_multi(arr, len(graphs), PROGRAMS.get(program, program), alpha, iters,
                             ctypes.byref(st)))
    return st.as_dict()
