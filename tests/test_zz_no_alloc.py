"""The allocation-free PageRank step against the regular entry point.

nx_pagerank_step_noalloc exists for callers that cannot call cudaMalloc when
they step the iteration (an application that has given the whole device to its
own memory pool, or a latency-critical loop that must not pay for allocation
or for cudaFree's synchronisation). Its scratch is a file-scope device array
shared by every call, so two calls in a row also check that each call clears
what it must. The result must match one NX_PR iteration of nx_run started from
the same ranks, within the tolerances used for PageRank everywhere else
(L1 <= 1e-6, max relative error <= 1e-4).

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1510_06916_b300 import inputs
from paper_1510_06916_b300 import nxgraph as nx

pytestmark = pytest.mark.gpu


def _one_step_reference(g, r):
    g.set_values("pr", r)
    g.run("pr", 1, "spu")
    return g.values()


def _close(a, b):
    a = a.astype(np.float64)
    b = b.astype(np.float64)
    l1 = np.abs(a - b).sum()
    rel = (np.abs(a - b)[b != 0] / np.abs(b[b != 0])).max()
    return l1, rel


def test_noalloc_step_matches_nx_run_twice():
    import torch

    torch.cuda.set_device(0)
    nx.set_stream(torch.cuda.current_stream())
    n = 1 << 15
    s, d, _ = inputs.rmat_edges(15, 16 << 15, 21)
    g = nx.Graph(s, d, n, 8)
    g.run("pr", 3)
    r0 = g.values().copy()  # a realistic rank vector
    r_in = torch.from_numpy(r0).cuda()
    r_mid = torch.empty_like(r_in)
    r_out = torch.empty_like(r_in)
    fn = nx.lib().nx_pagerank_step_noalloc
    nx.check(fn(g.handle, ctypes.c_float(0.85), ctypes.c_void_p(r_in.data_ptr()),
                ctypes.c_void_p(r_mid.data_ptr())))
    nx.check(fn(g.handle, ctypes.c_float(0.85), ctypes.c_void_p(r_mid.data_ptr()),
                ctypes.c_void_p(r_out.data_ptr())))
    torch.cuda.synchronize()
    mid = r_mid.cpu().numpy()
    out = r_out.cpu().numpy()
    ref_mid = _one_step_reference(g, r0)
    ref_out = _one_step_reference(g, mid)
    for got, want in ((mid, ref_mid), (out, ref_out)):
        l1, rel = _close(got, want)
        assert l1 <= 1e-6 and rel <= 1e-4, (l1, rel)
    # bad arguments are rejected without touching the device
    with pytest.raises(nx.NxError) as e:
        nx.check(fn(g.handle, ctypes.c_float(0.85), ctypes.c_void_p(r_in.data_ptr()),
                    ctypes.c_void_p(r_in.data_ptr())))
    assert e.value.code == nx.NX_ERR_INVALID_ARG
