"""Full-size parity: the workloads the benchmark measures, against the FP64 oracle.

These build the full graphs (up to R-MAT scale 26, 1,476,395,008 edges) and run
the oracle on the host cores, so they take minutes. Tolerances as everywhere
(tests/nxtol.py): BFS/WCC bit-exact; PageRank and gradients L1 <= 1e-6 (for
gradients relative to the reference's L1 norm) and per-entry relative error
<= 1e-4, with an operand-scale floor only for cancelling dL/dw entries.
"""
import numpy as np
import pytest

import oracle
from nxtol import assert_grad_t_close, assert_grad_w_close, assert_pr_close
from test_gpu_parity import _budget_slack
from paper_1510_06916_b300 import inputs
from paper_1510_06916_b300 import nxgraph as nx

pytestmark = pytest.mark.gpu


def _pr_close(gpu, ref, what):
    return assert_pr_close(gpu, ref, what)


def test_rmat26_p64_spu_and_mpu_6gb():
    # R-MAT scale 26, edge factor 22, seed 5, P = 64: PageRank 10 iterations, BFS, WCC
    # under SPU in HBM, and PageRank / BFS under MPU with a 6 GB device budget.
    scale, ef, seed, P = 26, 22, 5, 64
    n, m = 1 << scale, ef << scale
    s, d, _ = inputs.rmat_edges(scale, m, seed)
    import torch

    src = torch.from_numpy(s.view(np.int32)).cuda()
    dst = torch.from_numpy(d.view(np.int32)).cuda()
    g = nx.Graph(src, dst, n, P, transpose=True, onchip=True)
    del src, dst
    torch.cuda.empty_cache()
    ref = oracle.pagerank(n, s, d, 0.85, 10)
    g.run("pr", 10, "spu")
    _pr_close(g.values(), ref, "rmat26 PR SPU")
    g.run("pr", 10, "dpu_onchip")  # Algorithm 6 with shared-memory intervals
    _pr_close(g.values(), ref, "rmat26 PR DPU on chip")
    st = g.run("pr", 10, "mpu", budget=6 * 10**9)
    assert st["streamed_cols"] > 0 and st["Q"] == P
    _pr_close(g.values(), ref, "rmat26 PR MPU 6GB")
    info = g.info()  # the device holds the budget plus the stated slack only
    print(f"rmat26 PR MPU 6GB: device {info['device_bytes'] / 1e9:.2f} GB, "
          f"pinned host {info['host_bytes'] / 1e9:.2f} GB")
    assert info["device_bytes"] <= 6 * 10**9 + _budget_slack(info, 1), info
    del ref
    bfs = oracle.bfs(n, s, d, 0)
    g.run("bfs", 1000, "spu", root=0)
    assert (g.values(dtype=np.uint32) == bfs).all()
    g.run("bfs", 1000, "mpu", budget=6 * 10**9, root=0)
    assert (g.values(dtype=np.uint32) == bfs).all()
    del bfs
    wcc = oracle.wcc(n, s, d)
    g.run("wcc", 1000, "spu")
    assert (g.values(dtype=np.uint32) == wcc).all()
    st = g.run("wcc", 1000, "mpu", budget=6 * 10**9)
    assert st["streamed_cols"] > 0 and st["Q"] == P
    assert (g.values(dtype=np.uint32) == wcc).all()
    info = g.info()
    print(f"rmat26 WCC MPU 6GB: device {info['device_bytes'] / 1e9:.2f} GB")
    assert info["device_bytes"] <= 6 * 10**9 + _budget_slack(info, 2), info
    g.free()


def test_rmat24_ppr_batch_64_vectors():
    # R-MAT scale 24, seed 3: 64 PPR teleports (1..1000 seeds), 30 iterations in one sweep
    import torch

    scale, seed, B = 24, 3, 64
    n, m = 1 << scale, 16 << scale
    s, d, _ = inputs.rmat_edges(scale, m, seed)
    g = nx.Graph(s, d, n, 16)
    v, b, t = inputs.ppr_seed_lists(n, B, seed)
    T = torch.zeros((n, B), dtype=torch.float32, device="cuda")
    T[torch.from_numpy(v).cuda(), torch.from_numpy(b).cuda()] = torch.from_numpy(t).cuda()
    R, _ = g.ppr_batch(T, iters=30)
    R = R.cpu().numpy()
    sums = R.astype(np.float64).sum(axis=0)
    assert np.abs(sums - 1.0).max() < 1e-5  # every column keeps unit mass
    # eight columns against the oracle: the ones with the most and the fewest
    # seeds and six more spread over the batch
    seeds = np.bincount(b, minlength=B)
    cols = [int(np.argmax(seeds)), int(np.argmin(seeds))]
    cols += [c for c in (0, 9, 21, 37, 50, 63) if c not in cols][:6]
    pp = oracle.PreparedPageRank(n, s, d)
    for col in cols:
        tv = np.zeros(n)
        sel = b == col
        tv[v[sel]] = t[sel]
        ref = pp.iterate(0.85, 30, tele=tv, dangling_by_tele=True, r0=tv)
        _pr_close(R[:, col], ref, f"batch col {col} ({seeds[col]} seeds)")
    pp.close()
    g.free()


def test_rmat24_adjoint_50_50():
    # weighted PageRank on R-MAT scale 24 (seed 4), w ~ U(0.5, 1.5), loss = sum over
    # 1,024 targets; 50 forward and 50 adjoint iterations vs the FP64 adjoint.
    scale, seed = 24, 4
    n, m = 1 << scale, 16 << scale
    s, d, w = inputs.rmat_edges(scale, m, seed, weights=True)
    T = inputs.targets(n, 1024, seed)
    gv = np.zeros(n, np.float32)
    gv[T] = 1.0
    g = nx.Graph(s, d, n, 16, transpose=True, weights=w)
    g.run("wpr", 50)
    dw = np.empty(m, np.float32)
    dt = np.empty(n, np.float32)
    g.adjoint_wpr(gv, 50, dw, dt)
    ref = oracle.wpr_adjoint(n, s, d, w.astype(np.float64), gv.astype(np.float64), 0.85, 50, 50)
    _pr_close(g.values(), ref["r"], "rmat24 WPR forward")
    assert_grad_t_close(dt, ref["dt"], "rmat24 dL/dt")
    assert_grad_w_close(dw, ref, s, d, w, 0.85, "rmat24 dL/dw")
    g.free()


def test_256_graphs_one_launch():
    # 256 R-MAT graphs, scales U{10..18}, edge factor 16: PR x20 / BFS / WCC per graph
    scales = inputs.multigraph_scales(256)
    graphs, data = [], []
    for gi, sc in enumerate(scales):
        n = 1 << sc
        s, d, _ = inputs.rmat_edges(sc, 16 << sc, inputs.multigraph_seed(gi))
        # the tile shape the benchmark's persistent launch uses (E_tile = 2^16)
        graphs.append(nx.Graph(s, d, n, max(1, min(16, n >> 12)), transpose=True, tile_edges_log2=16))
        data.append((n, s, d))
    nx.run_multi(graphs, "pr", 20)
    worst_l1 = worst_rel = 0.0
    for g, (n, s, d) in zip(graphs, data):
        l1, rel = assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "")
        worst_l1, worst_rel = max(worst_l1, l1), max(worst_rel, rel)
    print(f"256 graphs PR: worst L1={worst_l1:.3e} worst max_rel={worst_rel:.3e}")
    nx.run_multi(graphs, "bfs", 60)
    for g, (n, s, d) in zip(graphs, data):
        assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    nx.run_multi(graphs, "wcc", 60)
    for g, (n, s, d) in zip(graphs, data):
        assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    for g in graphs:
        g.free()
