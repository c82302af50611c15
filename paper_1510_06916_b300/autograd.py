"""Weighted PageRank as a differentiable torch op (an extension of the paper).

``weighted_pagerank(w, t, src, dst, n, P, iters, adj_terms)`` builds the DSSS
with weights ``w`` (normalised per source inside the library), runs ``iters``
weighted-PageRank sweeps and returns the ranks. ``backward`` calls the
library's hand-written adjoint (a fixed-point solve of the transpose system as
a source-sorted DSSS sweep, ``nx_adjoint_wpr``) for dL/dw and dL/dt. Only
argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import nxgraph as nx


class WeightedPageRank(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, t, src, dst, n, P, iters, adj_terms, alpha):
        if not (w.is_cuda and w.dtype == torch.float32):
            raise ValueError("w must be a float32 CUDA tensor")
        g = nx.Graph(src, dst, n, P, transpose=True, weights=w.detach().contiguous())
        tele = None if t is None else t.detach().contiguous()
        g.run("wpr", iters, "spu", alpha=alpha, teleport=tele)
        r = torch.empty(n, dtype=torch.float32, device=w.device)
        g.values(r)
        ctx.graph = g
        ctx.adj_terms = adj_terms
        ctx.has_t = t is not None
        ctx.shape_w = w.shape
        return r

    @staticmethod
    def backward(ctx, grad_r):
        g = ctx.graph
        dw = torch.empty(ctx.shape_w, dtype=torch.float32, device=grad_r.device)
        dt = torch.empty(g.n, dtype=torch.float32, device=grad_r.device)
        g.adjoint_wpr(grad_r.contiguous().float(), ctx.adj_terms, dw, dt)
        return dw, (dt if ctx.has_t else None), None, None, None, None, None, None, None


def weighted_pagerank(w, t, src, dst, n, P, iters=50, adj_terms=50, alpha=0.85):
    """Ranks r(w, t); src/dst are int32 CUDA tensors (edge endpoints), w > 0."""
    return WeightedPageRank.apply(w, t, src, dst, n, P, iters, adj_terms, alpha)
