"""The allocation-free PageRank step against the FP64 oracle.

nx_pagerank_step_noalloc exists for callers that cannot call cudaMalloc when
they step the iteration (an application that has given the whole device to its
own memory pool, or a latency-critical loop that must not pay for allocation
or for cudaFree's synchronisation). Its scratch is a file-scope device array
shared by every call, so two calls in a row also check that each call clears
what it must. Each step must match one step of the oracle's PageRank started
from the same ranks (oracle.pagerank with iters=1 and r0), within the
tolerances used for PageRank everywhere else (L1 <= 1e-6, max relative error
<= 1e-4), and the two steps must agree with one NX_PR iteration of nx_run.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from nxtol import assert_pr_close
from paper_1510_06916_b300 import inputs
from paper_1510_06916_b300 import nxgraph as nx

pytestmark = pytest.mark.gpu


def _step(g, r_in, r_out):
    fn = nx.lib().nx_pagerank_step_noalloc
    nx.check(fn(g.handle, ctypes.c_float(0.85), ctypes.c_void_p(r_in.data_ptr()),
                ctypes.c_void_p(r_out.data_ptr())))


def _two_steps_vs_oracle(n, s, d, P, what):
    import torch

    torch.cuda.set_device(0)
    nx.set_stream(torch.cuda.current_stream())
    g = nx.Graph(s, d, n, P)
    g.run("pr", 3)
    r0 = g.values().copy()  # a realistic rank vector
    r_in = torch.from_numpy(r0).cuda()
    r_mid = torch.empty_like(r_in)
    r_out = torch.empty_like(r_in)
    _step(g, r_in, r_mid)
    _step(g, r_mid, r_out)
    torch.cuda.synchronize()
    mid = r_mid.cpu().numpy()
    out = r_out.cpu().numpy()
    del r_in, r_mid, r_out
    ref_mid = oracle.pagerank(n, s, d, 0.85, 1, r0=r0.astype(np.float64))
    assert_pr_close(mid, ref_mid, f"{what} step 1")
    ref_out = oracle.pagerank(n, s, d, 0.85, 1, r0=mid.astype(np.float64))
    assert_pr_close(out, ref_out, f"{what} step 2")
    # and the same step as nx_run's PageRank iteration
    g.set_values("pr", r0)
    g.run("pr", 1, "spu")
    assert_pr_close(mid, g.values().astype(np.float64), f"{what} vs nx_run")
    return g


def test_noalloc_step_matches_oracle_twice():
    n = 1 << 15
    s, d, _ = inputs.rmat_edges(15, 16 << 15, 21)
    assert (np.bincount(s, minlength=n) == 0).sum() > 1000  # dangling vertices
    g = _two_steps_vs_oracle(n, s, d, 8, "scale 15")
    # bad arguments are rejected without touching the device
    import torch

    r = torch.zeros(n, dtype=torch.float32, device="cuda")
    with pytest.raises(nx.NxError) as e:
        _step(g, r, r)
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    g.free()


def test_noalloc_step_many_tiles_and_dangling_vertices():
    # 2^29 vertices, 2^22 R-MAT edges, P = 1024: at least 262,144 destination
    # tiles (half the scratch array's limit) and mostly dangling vertices
    scale, m, P = 29, 1 << 22, 1024
    n = 1 << scale
    s, d, _ = inputs.rmat_edges(scale, m, 31)
    g = _two_steps_vs_oracle(n, s, d, P, "2^29 vertices")
    assert g.info()["ntiles"] >= 262144
    g.free()


def test_noalloc_step_rejects_too_many_tiles():
    # 2^30 vertices at P = 1024: 524,288 tiles, above the scratch array's 523,232
    import torch

    n = 1 << 30
    s = np.arange(1024, dtype=np.uint32) * 1024
    g = nx.Graph(s, s[::-1].copy(), n, 1024)
    assert g.info()["ntiles"] == 524288
    r = torch.empty(2, dtype=torch.float32, device="cuda")  # never read: rejected first
    with pytest.raises(nx.NxError) as e:
        _step(g, r[:1], r[1:])
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    g.free()
