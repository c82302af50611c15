"""CUDA path vs the FP64 oracle, through the C ABI (needs a B300).

Tolerances (PageRank family, FP32 on the GPU vs FP64 oracle): L1 over the
vector <= 1e-6 and max per-vertex relative error <= 1e-4 over vertices with a
non-zero reference. BFS depths and WCC labels: bit-exact.
"""
import numpy as np
import pytest

import oracle
from paper_1510_06916_b300 import inputs
from paper_1510_06916_b300 import nxgraph as nx

pytestmark = pytest.mark.gpu

from nxtol import L1_TOL, REL_TOL, assert_grad_t_close, assert_grad_w_close, assert_pr_close, pr_err  # noqa: E402,F401


def rmat(scale, ef, seed, weights=False):
    return inputs.rmat_edges(scale, ef << scale, seed, weights=weights)


# ------------------------------------------------------------------ builder

@pytest.mark.parametrize("P", [1, 2, 4, 7, 16])
def test_dsss_layout_matches_oracle(P):
    n = 1 << 12
    s, d, _ = rmat(12, 16, 9)
    g = nx.Graph(s, d, n, P, transpose=True)
    order, off = oracle.dsss_order(n, P, s, d)
    gs, gd, goff = g.export()
    assert (goff == off).all()
    assert (gs == s[order]).all() and (gd == d[order]).all()
    # transpose DSSS = the DSSS of the reversed graph
    order_t, off_t = oracle.dsss_order(n, P, d, s)
    ts, td, toff = g.export(transpose=True)
    assert (toff == off_t).all()
    assert (ts == s[order_t]).all() and (td == d[order_t]).all()
    info = g.info()
    heads = np.ones(len(s), bool)
    ks = (d[order].astype(np.int64) // info["L"]) * P + s[order] // info["L"]
    heads[1:] = (ks[1:] != ks[:-1]) | (d[order][1:] != d[order][:-1])
    assert info["D"] == heads.sum()  # distinct (sub-shard, destination) pairs


def test_fig1_example_on_device():
    # Section II-A, Fig. 1: SS_3.2 = e5.2, e4.3, e5.3 with intervals of 2 vertices
    s = np.array([5, 1, 4, 6, 5, 3, 2, 7], np.uint32)
    d = np.array([3, 2, 3, 0, 2, 5, 2, 4], np.uint32)
    g = nx.Graph(s, d, 8, 4)
    gs, gd, off = g.export()
    sel = slice(int(off[1 * 4 + 2]), int(off[1 * 4 + 3]))
    assert list(zip(gs[sel].tolist(), gd[sel].tolist())) == [(5, 2), (4, 3), (5, 3)]


def test_ragged_and_empty_intervals():
    # n = 9, P = 4: L = 3, the last interval is empty
    rng = np.random.default_rng(1)
    s = rng.integers(0, 9, 40).astype(np.uint32)
    d = rng.integers(0, 9, 40).astype(np.uint32)
    g = nx.Graph(s, d, 9, 4, transpose=True)
    order, off = oracle.dsss_order(9, 4, s, d)
    gs, gd, goff = g.export()
    assert (goff == off).all() and (gs == s[order]).all() and (gd == d[order]).all()
    g.run("pr", 20)
    assert_pr_close(g.values(), oracle.pagerank(9, s, d, 0.85, 20), "ragged PR")
    g.run("bfs", 100, root=3)
    assert (g.values(dtype=np.uint32) == oracle.bfs(9, s, d, 3)).all()
    g.run("wcc", 100)
    assert (g.values(dtype=np.uint32) == oracle.wcc(9, s, d)).all()


def test_bfs_max_depth_is_algorithm4_output():
    n = 1 << 14
    s, d, _ = rmat(14, 8, 12)
    g = nx.Graph(s, d, n, 4, transpose=True)
    for root in (0, 77):
        g.run("bfs", 1000, root=root)
        ref = oracle.bfs(n, s, d, root)
        assert g.bfs_max_depth() == oracle.bfs_max_depth(ref) > 0
    g.run("bfs", 1000, root=n - 1)  # a vertex without out-edges: depth 0 only
    assert g.bfs_max_depth() == oracle.bfs_max_depth(oracle.bfs(n, s, d, n - 1))
    g.run("pr", 2)
    with pytest.raises(nx.NxError) as e:
        g.bfs_max_depth()
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    g.free()


@pytest.mark.parametrize("strategy", ["spu", "dpu", "mpu"])
def test_inactive_intervals_are_skipped_and_counted(strategy):
    # Edges only inside interval 0 of P = 4: a BFS from vertex 0 never
    # activates intervals 1-3, so every sweep skips them (Algorithm 1) and
    # reads interval 0's edges alone.
    n, P = 4096, 4
    L = n // P
    rng = np.random.default_rng(5)
    s = rng.integers(0, L, 20000).astype(np.uint32)
    d = rng.integers(0, L, 20000).astype(np.uint32)
    g = nx.Graph(s, d, n, P, transpose=True)
    budget = 2 * n * 4 * 2 // P + 1 if strategy == "mpu" else 0  # Q = 2
    st = g.run("bfs", 1000, strategy, budget=budget, root=0)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    assert st["intervals_skipped"] == 3 * st["iters_done"]
    assert st["edges_swept"] == len(s) * st["iters_done"]
    st = g.run("pr", 5, strategy, budget=budget)
    assert st["intervals_skipped"] == 0 and st["edges_swept"] == 5 * len(s)
    g.free()


# ------------------------------------------------- on-chip double-phase update

def _onchip_hub_count(s, d):
    """Hub entries of the NX_ONCHIP_HUBS layout from its definition: edges in
    (source interval of 2^15, destination interval of 2^14, destination,
    source) order; an entry starts at a new (source interval, destination) or
    at every multiple of 2048 edges."""
    s = np.asarray(s, np.int64)
    d = np.asarray(d, np.int64)
    order = np.lexsort((s & 0x7FFF, d & 0x3FFF, d >> 14, s >> 15))
    k = ((s >> 15) << 40 | d)[order]
    head = np.ones(len(k), bool)
    head[1:] = k[1:] != k[:-1]
    head[::2048] = True
    return int(head.sum())


@pytest.mark.parametrize("scale,ef,seed,P", [(12, 16, 3, 4), (17, 16, 5, 8), (18, 8, 6, 16)])
def test_dpu_onchip_matches_oracle(scale, ef, seed, P):
    # Algorithm 6 with the source interval (2^15) and the destination interval
    # (2^14) held in shared memory: PageRank and PPR vs the FP64 oracle
    n = 1 << scale
    s, d, _ = rmat(scale, ef, seed)
    g = nx.Graph(s, d, n, P, onchip=True)
    assert g.info()["H_onchip"] == _onchip_hub_count(s, d)
    st = g.run("pr", 20, "dpu_onchip")
    assert st["iters_done"] == 20 and st["strategy"] == nx.DPU_ONCHIP
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"onchip PR scale {scale}")
    t = inputs.ppr_teleports(n, 1, seed + 1, max_seeds=50)[:, 0].copy()
    g.run("ppr", 15, "dpu_onchip", teleport=t)
    ref = oracle.personalized_pagerank(n, s, d, t, 0.85, 15)
    assert_pr_close(g.values(), ref, f"onchip PPR scale {scale}")
    # AUTO takes the on-chip update for PageRank on this graph, and SPU on the
    # same graph under a budget or for BFS
    st = g.run("pr", 20, "auto")
    assert st["strategy"] == nx.DPU_ONCHIP
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"onchip AUTO PR scale {scale}")
    st = g.run("pr", 20, "auto", budget=1 << 40)
    assert st["strategy"] == nx.SPU
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"AUTO with a budget, scale {scale}")
    st = g.run("bfs", 1000, "auto")
    assert st["strategy"] == nx.SPU
    g.free()


def test_dpu_onchip_ragged_hub_relabel_and_empty():
    # ragged n (partial last intervals), a 300k-edge in-star (runs cut every
    # 2048 edges), degree-ordered ids, an empty graph, and rejections
    n = 100_003
    rng = np.random.default_rng(4)
    k = 300_000
    s = np.concatenate([rng.integers(0, n, k), rng.integers(0, n, 200_000)]).astype(np.uint32)
    d = np.concatenate([np.full(k, n - 2), rng.integers(0, n, 200_000)]).astype(np.uint32)
    ref = oracle.pagerank(n, s, d, 0.85, 20)
    for relabel in (False, True):
        g = nx.Graph(s, d, n, 7, relabel=relabel, onchip=True)
        g.run("pr", 20, "dpu_onchip")
        assert_pr_close(g.values(), ref, f"onchip ragged relabel={relabel}")
        g.free()
    g = nx.Graph(s, d, n, 7, onchip=True)
    assert g.info()["H_onchip"] == _onchip_hub_count(s, d)
    # the DSSS sweeps on the same graph continue to work, and agree
    g.run("pr", 20, "spu")
    assert_pr_close(g.values(), ref, "spu on an onchip graph")
    for bad in (dict(program="bfs"), dict(budget=1 << 30)):
        with pytest.raises(nx.NxError):
            g.run(bad.get("program", "pr"), 5, "dpu_onchip", budget=bad.get("budget", 0))
    g.free()
    e = np.zeros(0, np.uint32)
    g = nx.Graph(e, e, 50, 2, onchip=True)
    g.run("pr", 5, "dpu_onchip")
    assert_pr_close(g.values(), oracle.pagerank(50, e, e, 0.85, 5), "onchip empty")
    g.free()
    g = nx.Graph(s, d, n, 7)
    with pytest.raises(nx.NxError):
        g.run("pr", 5, "dpu_onchip")  # not built with the on-chip structure
    g.free()


def test_dpu_onchip_under_a_budget_elsewhere():
    # a budgeted SPU run moves the on-chip structure to host memory; the next
    # on-chip run brings it back
    n = 1 << 16
    s, d, _ = rmat(16, 16, 9)
    g = nx.Graph(s, d, n, 8, onchip=True)
    ref = oracle.pagerank(n, s, d, 0.85, 10)
    g.run("pr", 10, "spu", budget=2 * n * 4 + 4 * len(s) // 3)
    assert_pr_close(g.values(), ref, "budget before onchip")
    assert g.info()["host_bytes"] >= 4 * len(s)
    g.run("pr", 10, "dpu_onchip")
    assert_pr_close(g.values(), ref, "onchip after budget")
    g.free()


# ------------------------------------------------------------------ SCC

@pytest.mark.parametrize("P", [1, 3, 8])
def test_scc_bitexact_rmat(P):
    # strongly connected components (Section IV-D) by coloring rounds over the
    # DSSS and its transpose: labels = smallest id per component, bit-exact
    for scale, ef, seed in ((12, 4, 3), (14, 8, 17)):
        n = 1 << scale
        s, d, _ = rmat(scale, ef, seed)
        g = nx.Graph(s, d, n, P, transpose=True)
        st = g.run("scc", 100000)
        ref = oracle.scc(n, s, d)
        assert (g.values(dtype=np.uint32) == ref).all(), (scale, P)
        assert st["Q"] >= 1 and st["iters_done"] >= 2
        print(f"SCC scale {scale} P={P}: {len(np.unique(ref))} components, "
              f"{st['Q']} rounds, {st['iters_done']} sweeps")
        g.free()


def test_scc_special_graphs():
    # a cycle (one component), a path (all singletons), two cycles joined one
    # way, self-loops, an empty graph, a ragged n
    n = 37
    cyc = np.arange(n, dtype=np.uint32)
    for s, d in ((cyc, (cyc + 1) % n), (cyc[:-1], cyc[1:]),
                 (np.array([0, 1, 2, 2, 5, 6, 9, 9], np.uint32),
                  np.array([1, 2, 0, 5, 6, 5, 9, 30], np.uint32)),
                 (np.zeros(0, np.uint32), np.zeros(0, np.uint32))):
        for P in (1, 4, 9):
            g = nx.Graph(s, d, n, P, transpose=True)
            g.run("scc", 10000)
            assert (g.values(dtype=np.uint32) == oracle.scc(n, s, d)).all(), (len(s), P)
            g.free()


def test_scc_relabel_and_limits():
    n = 1 << 13
    s, d, _ = rmat(13, 6, 29)
    ref = oracle.scc(n, s, d)
    g = nx.Graph(s, d, n, 4, transpose=True, relabel=True)
    g.run("scc", 100000)
    assert (g.values(dtype=np.uint32) == ref).all()  # smallest caller id, caller order
    g.free()
    g = nx.Graph(s, d, n, 4, transpose=True)
    st = g.run("scc", 3)  # out of sweeps: unassigned vertices keep 0xFFFFFFFF
    assert st["iters_done"] == 3
    lab = g.values(dtype=np.uint32)
    done = lab != nx.INF
    assert (lab[done] == ref[done]).all()
    with pytest.raises(nx.NxError):
        g.run("scc", 10, "dpu")
    with pytest.raises(nx.NxError):
        g.run("scc", 10, "spu", budget=1 << 30)
    g.free()
    g = nx.Graph(s, d, n, 4)
    with pytest.raises(nx.NxError):
        g.run("scc", 10)  # no transpose
    g.free()


def test_scc_rmat22_bitexact():
    n = 1 << 22
    s, d, _ = rmat(22, 16, 2)
    g = nx.Graph(s, d, n, 16, transpose=True)
    st = g.run("scc", 1000000)
    ref = oracle.scc(n, s, d)
    assert (g.values(dtype=np.uint32) == ref).all()
    print(f"SCC scale 22: {st['Q']} rounds, {st['iters_done']} sweeps, {st['ms']:.1f} ms, "
          f"largest component {np.bincount(ref).max()} vertices")
    g.free()


def test_invalid_inputs():
    s = np.array([0, 5], np.uint32)
    d = np.array([1, 2], np.uint32)
    with pytest.raises(nx.NxError) as e:
        nx.Graph(s, d, 5, 2)  # id 5 >= n
    assert e.value.code == nx.NX_ERR_INVALID_ARG
    g = nx.Graph(np.array([0, 1], np.uint32), np.array([1, 2], np.uint32), 3, 1)
    with pytest.raises(nx.NxError):
        g.run("wcc", 5)  # no transpose
    with pytest.raises(nx.NxError):
        g.run("wpr", 5)  # no weights
    with pytest.raises(nx.NxError):
        g.run("bfs", 5, root=3)
    with pytest.raises(nx.NxError) as e:
        g.run("pr", 5, strategy="spu", budget=8)  # below 2 n B_a
    assert e.value.code == nx.NX_ERR_BUDGET_TOO_SMALL


# ------------------------------------------------------------------ programs

def test_pagerank_rmat16_p4():
    # R-MAT scale 16, edge factor 16, seed 1, P = 4, 20 iterations, SPU
    n = 1 << 16
    s, d, _ = rmat(16, 16, 1)
    g = nx.Graph(s, d, n, 4, transpose=True)
    st = g.run("pr", 20, "spu")
    assert st["iters_done"] == 20
    r = g.values()
    assert abs(r.astype(np.float64).sum() - 1.0) < 1e-5
    assert_pr_close(r, oracle.pagerank(n, s, d, 0.85, 20), "rmat16 PR")


def test_bfs_wcc_rmat16_bitexact():
    n = 1 << 16
    s, d, _ = rmat(16, 16, 1)
    g = nx.Graph(s, d, n, 4, transpose=True)
    g.run("bfs", 1000, root=0)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    g.run("wcc", 1000)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


@pytest.mark.parametrize("P", [1, 3, 16, 64])
def test_programs_across_P(P):
    n = 5000  # not a power of two: ragged last interval and tiles
    s, d, _ = inputs.rmat_edges(13, 60000, 17)
    keep = (s < n) & (d < n)
    s, d = s[keep], d[keep]
    g = nx.Graph(s, d, n, P, transpose=True)
    g.run("pr", 20)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"P={P} PR")
    g.run("bfs", 1000, root=1)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 1)).all()
    g.run("wcc", 1000)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


def test_heavy_hub_split_tiles():
    # in-star with 300k leaves: one destination far heavier than a block's share
    k = 300_000
    n = k + 1
    s = np.arange(1, n, dtype=np.uint32)
    d = np.zeros(k, dtype=np.uint32)
    s = np.concatenate([s, np.array([0, 5], np.uint32)])  # a little extra structure
    d = np.concatenate([d, np.array([7, 0], np.uint32)])
    g = nx.Graph(s, d, n, 4, transpose=True)
    g.run("pr", 20)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "hub PR")
    g.run("bfs", 100, root=5)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 5)).all()
    g.run("wcc", 100)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


def test_tiny_and_empty_graphs():
    g = nx.Graph(np.zeros(0, np.uint32), np.zeros(0, np.uint32), 5, 2, transpose=True)
    g.run("pr", 3)
    assert np.allclose(g.values(), 0.2, rtol=1e-6)
    g.run("bfs", 10, root=2)
    assert (g.values(dtype=np.uint32) == np.array([nx.INF, nx.INF, 0, nx.INF, nx.INF])).all()
    g.run("wcc", 10)
    assert (g.values(dtype=np.uint32) == np.arange(5)).all()
    g1 = nx.Graph(np.zeros(3, np.uint32), np.zeros(3, np.uint32), 1, 1, transpose=True)
    g1.run("pr", 5)
    assert g1.values()[0] == pytest.approx(1.0, rel=1e-6)


def test_cycle_uniform_on_device():
    n = 100_003
    s = np.arange(n, dtype=np.uint32)
    d = ((np.arange(n) + 1) % n).astype(np.uint32)
    g = nx.Graph(s, d, n, 8)
    g.run("pr", 20)
    assert np.allclose(g.values(), 1.0 / n, rtol=1e-5)


def test_ppr_single_vector():
    n = 1 << 14
    s, d, _ = rmat(14, 16, 3)
    t = inputs.ppr_teleports(n, 1, 33)[:, 0].copy()
    g = nx.Graph(s, d, n, 8)
    g.run("ppr", 30, teleport=t)
    assert_pr_close(g.values(), oracle.personalized_pagerank(n, s, d, t, 0.85, 30), "PPR")


def test_weighted_pagerank_forward():
    n = 1 << 13
    s, d, w = rmat(13, 16, 4, weights=True)
    g = nx.Graph(s, d, n, 8, transpose=True, weights=w)
    g.run("wpr", 50)
    ref = oracle.pagerank(n, s, d, 0.85, 50, w=w.astype(np.float64))
    assert_pr_close(g.values(), ref, "WPR")


# ------------------------------------------------------------------ strategies

@pytest.mark.parametrize("P", [1, 4, 9])
def test_dpu_equals_spu(P):
    n = 1 << 14
    s, d, _ = rmat(14, 16, 5)
    g = nx.Graph(s, d, n, P, transpose=True)
    g.run("bfs", 1000, "spu", root=0)
    b_spu = g.values(dtype=np.uint32)
    st = g.run("bfs", 1000, "dpu", root=0)
    assert st["strategy"] == nx.DPU
    assert (g.values(dtype=np.uint32) == b_spu).all()
    assert (b_spu == oracle.bfs(n, s, d, 0)).all()
    g.run("pr", 20, "dpu")
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"DPU P={P}")
    g.run("wcc", 1000, "dpu")  # hubs of the forward and the transpose DSSS
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


def test_resume_from_values():
    n = 1 << 14
    s, d, _ = rmat(14, 16, 6)
    g = nx.Graph(s, d, n, 4, transpose=True)
    g.run("pr", 10)
    mid = g.values()
    g.set_values("pr", mid)
    g.run("pr", 10)
    ref = oracle.pagerank(n, s, d, 0.85, 20)
    assert_pr_close(g.values(), ref, "PR 10+10")
    g.run("bfs", 2, root=0)
    part = g.values(dtype=np.uint32)
    g.set_values("bfs", part)
    g.run("bfs", 1000)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()


# ------------------------------------------------------------------ full size

def test_full_size_rmat22_p16():
    # R-MAT scale 22, edge factor 16 (67,108,864 edges), seed 2, P = 16: the
    # benchmark's launch configuration, checked on the whole vector.
    n = 1 << 22
    s, d, _ = rmat(22, 16, 2)
    g = nx.Graph(s, d, n, 16, transpose=True)
    st = g.run("pr", 20, "spu")
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "rmat22 PR")
    g.run("bfs", 1000, root=0)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    g.run("wcc", 1000)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    st = g.run("pr", 20, "dpu")
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "rmat22 PR DPU")


# ------------------------------------------------------------------ budgets

@pytest.mark.parametrize("P", [4, 7])
def test_mpu_every_q(P):
    # Section III-B3: Q = floor(B_M P / (2 n B_a)); Q = P is SPU, Q = 0 is DPU.
    n = 1 << 13
    s, d, _ = rmat(13, 16, 8)
    g = nx.Graph(s, d, n, P, transpose=True)
    ref_pr = oracle.pagerank(n, s, d, 0.85, 20)
    ref_bfs = oracle.bfs(n, s, d, 0)
    ref_wcc = oracle.wcc(n, s, d)
    L = -(-n // P)
    for Q in range(0, P + 1):
        budget = max(2 * n * 4 * Q // P + 1, 2 * L * 4)
        want_q = min(P, (budget * P) // (2 * n * 4))
        st = g.run("pr", 20, "mpu", budget=budget)
        assert st["Q"] == want_q and st["strategy"] == (nx.SPU if want_q == P else nx.MPU)
        assert_pr_close(g.values(), ref_pr, f"MPU P={P} Q={want_q}")
        st = g.run("bfs", 1000, "mpu", budget=budget, root=0)
        assert (g.values(dtype=np.uint32) == ref_bfs).all(), (P, Q)
        if want_q < P:
            assert st["h2d_bytes"] > 0 and st["d2h_bytes"] > 0
        g.run("wcc", 1000, "mpu", budget=budget)
        assert (g.values(dtype=np.uint32) == ref_wcc).all(), (P, Q)


def test_dpu_with_small_budget_stages_intervals():
    n = 1 << 13
    s, d, _ = rmat(13, 16, 10)
    g = nx.Graph(s, d, n, 8)
    L = n // 8
    st = g.run("pr", 20, "dpu", budget=3 * L * 4)
    assert st["Q"] == 0 and st["h2d_bytes"] > 0
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "staged DPU")
    with pytest.raises(nx.NxError) as e:
        g.run("pr", 5, "mpu", budget=L * 4)  # below one interval pair
    assert e.value.code == nx.NX_ERR_BUDGET_TOO_SMALL


@pytest.mark.parametrize("frac", [0.0, 0.3, 0.8])
def test_spu_streams_shards_from_host(frac):
    n = 1 << 14
    s, d, _ = rmat(14, 16, 12)
    g = nx.Graph(s, d, n, 8, transpose=True)
    m = len(s)
    budget = 2 * n * 4 + int(frac * 4 * m)
    st = g.run("pr", 20, "spu", budget=budget)
    assert st["streamed_cols"] > 0 and st["h2d_bytes"] > 0
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"streamed PR {frac}")
    # byte-granular caching: each iteration moves m B_e + 2 n B_a - B_M (Section III-B1),
    # up to the 16-word alignment of each streamed shard
    want = 4 * m + 2 * n * 4 - budget
    assert abs(st["h2d_bytes"] / 20 - want) <= 8 * 3 * 16 * 4 + 64, (st["h2d_bytes"] / 20, want)
    g.run("bfs", 1000, "spu", budget=budget, root=0)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    st = g.run("wcc", 1000, "spu", budget=budget + int(frac * 4 * m))
    assert st["streamed_cols"] > 0
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


def test_streamed_sub_shard_above_a_chunk_is_cut_by_tiles():
    # Degree-ordered ids put most edges in SS_00: at scale 21, P = 2, it holds
    # far more than one 64 MB staging chunk (16 M words), so the streamed band
    # is cut into ranges of its tiles. Results are unchanged and the staging
    # buffers stay within the stated slack.
    scale = 21
    n = 1 << scale
    s, d, _ = rmat(scale, 16, 14)
    m = len(s)
    g = nx.Graph(s, d, n, 2, transpose=True, relabel=True)
    budget = 2 * n * 4 + (1 << 20)
    st = g.run("pr", 10, "spu", budget=budget)
    assert st["streamed_cols"] == 2
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 10), "PR, split sub-shard")
    info = g.info()
    assert info["device_bytes"] <= budget + _budget_slack(info, 1, True), info
    # every word crosses the link once per iteration, plus the alignment of each band
    assert 4 * m - (1 << 20) <= st["h2d_bytes"] / 10 <= 4 * m + 4096 * 128, (st["h2d_bytes"] / 10, m)
    g.run("bfs", 1000, "spu", budget=budget, root=0)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    st = g.run("wcc", 1000, "spu", budget=budget)
    assert st["streamed_cols"] == 2
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    info = g.info()
    assert info["device_bytes"] <= budget + _budget_slack(info, 2, True), info
    g.free()


def _budget_slack(info, nds, relabeled=False):
    """Device bytes outside a budget's accounting (intervals 2 n B_a + resident
    edge words): out-degrees and PageRank contributions (12 n), the id maps of
    degree-ordered ids (8 n), piece and hub
    offsets of the DSSS the run reads (16 B per piece each), tile tables, the
    accumulators of one streamed column (4 L), two staging buffers (a band
    holds at most 64 MB of words, down to single tiles), and 256 MB for
    plans, split-tile slots and scalars."""
    n, P, nt, L = info["n"], info["P"], info["ntiles"], info["L"]
    return (12 * n + (8 * n if relabeled else 0) + 16 * (P * nt + 1) * nds + 8 * (nt + P + 2) + 4 * L
            + 2 * nds * (64 << 20) + (256 << 20))


def test_budget_bounds_device_memory_and_is_undone():
    # Under a budget, streamed shards, the unread transpose and the hub index
    # live in pinned host memory only; a later run without a budget brings
    # them back; results are unchanged throughout.
    n = 1 << 16
    s, d, _ = rmat(16, 16, 13)
    g = nx.Graph(s, d, n, 8, transpose=True)
    ref = oracle.pagerank(n, s, d, 0.85, 10)
    wcc = oracle.wcc(n, s, d)
    m = len(s)
    for frac in (0.1, 0.5):
        budget = 2 * n * 4 + int(frac * 4 * m)
        st = g.run("pr", 10, "mpu", budget=budget)
        assert st["streamed_cols"] > 0 and st["h2d_bytes"] > 0
        assert_pr_close(g.values(), ref, f"budget {frac} PR")
        info = g.info()
        assert info["device_bytes"] <= budget + _budget_slack(info, 1), (frac, info)
        assert info["host_bytes"] >= 4 * m  # the unread transpose lives in pinned host memory
        st = g.run("wcc", 1000, "mpu", budget=budget + int(frac * 4 * m))
        assert (g.values(dtype=np.uint32) == wcc).all()
        info = g.info()
        assert info["device_bytes"] <= budget + int(frac * 4 * m) + _budget_slack(info, 2)
    # no budget: everything back on the device, same results
    g.run("pr", 10)
    assert_pr_close(g.values(), ref, "PR after budgets")
    back = g.info()
    assert back["host_bytes"] < 64 << 20
    gs, gd, _ = g.export()  # reads the whole (restored) DSSS
    order, _ = oracle.dsss_order(n, 8, s, d)
    assert (gs == s[order]).all() and (gd == d[order]).all()
    g.run("wcc", 1000, "dpu")  # hubs restored
    assert (g.values(dtype=np.uint32) == wcc).all()
    g.free()


# ------------------------------------------------------------------ batched PPR

@pytest.mark.parametrize("B", [1, 8, 33, 64])
def test_ppr_batch_matches_per_vector_oracle(B):
    n = 1 << 13
    s, d, _ = rmat(13, 16, 14)
    T = inputs.ppr_teleports(n, B, 3, max_seeds=50)
    T[:, 0] = 1.0 / n  # one uniform column: equals global PageRank
    g = nx.Graph(s, d, n, 4)
    R, st = g.ppr_batch(T, iters=30)
    assert st["iters_done"] == 30
    for b in range(B):
        ref = oracle.personalized_pagerank(n, s, d, T[:, b], 0.85, 30)
        assert_pr_close(R[:, b], ref, f"batch B={B} col {b}")
    assert_pr_close(R[:, 0], oracle.pagerank(n, s, d, 0.85, 30), "uniform column")


def test_ppr_batch_device_pointers_and_hub():
    import torch
    k = 100_000
    n = k + 1
    s = np.concatenate([np.arange(1, n, dtype=np.uint32), np.array([0], np.uint32)])
    d = np.concatenate([np.zeros(k, np.uint32), np.array([9], np.uint32)])
    T = inputs.ppr_teleports(n, 5, 8, max_seeds=20)
    g = nx.Graph(s, d, n, 2)
    Tt = torch.from_numpy(T).cuda()
    R, _ = g.ppr_batch(Tt, iters=20)
    R = R.cpu().numpy()
    for b in range(5):
        ref = oracle.personalized_pagerank(n, s, d, T[:, b], 0.85, 20)
        assert_pr_close(R[:, b], ref, f"hub batch col {b}")
    R0, _ = g.ppr_batch(T, iters=0)
    assert np.array_equal(R0, T)


# ------------------------------------------------------------------ adjoint

def test_adjoint_matches_fp64_oracle():
    n = 1 << 13
    s, d, w = rmat(13, 16, 4, weights=True)
    T = inputs.targets(n, 64, 4)
    gvec = np.zeros(n, np.float32)
    gvec[T] = 1.0
    g = nx.Graph(s, d, n, 8, transpose=True, weights=w)
    g.run("wpr", 50)
    dw = np.empty(len(s), np.float32)
    dt = np.empty(n, np.float32)
    st = g.adjoint_wpr(gvec, 50, dw, dt)
    ref = oracle.wpr_adjoint(n, s, d, w.astype(np.float64), gvec.astype(np.float64), 0.85, 50, 50)
    assert_grad_t_close(dt, ref["dt"], "scale-13 dL/dt")
    assert_grad_w_close(dw, ref, s, d, w, 0.85, "scale-13 dL/dw")
    assert st["iters_done"] == 50


def test_autograd_function():
    import torch
    from paper_1510_06916_b300.autograd import weighted_pagerank
    n = 1 << 12
    s, d, w = rmat(12, 16, 6, weights=True)
    T = inputs.targets(n, 32, 6)
    src = torch.from_numpy(s.view(np.int32)).cuda()
    dst = torch.from_numpy(d.view(np.int32)).cuda()
    wt = torch.from_numpy(w).cuda().requires_grad_(True)
    t = torch.full((n,), 1.0 / n, device="cuda", requires_grad=True)
    r = weighted_pagerank(wt, t, src, dst, n, 4, iters=50, adj_terms=50)
    loss = r[torch.from_numpy(T).cuda()].sum()
    loss.backward()
    gv = np.zeros(n)
    gv[T] = 1.0
    ref = oracle.wpr_adjoint(n, s, d, w.astype(np.float64), gv, 0.85, 50, 50,
                             tele=np.full(n, 1.0 / n))
    assert_pr_close(r.detach().cpu().numpy(), ref["r"], "autograd forward")
    assert_grad_w_close(wt.grad.cpu().numpy(), ref, s, d, w, 0.85, "autograd dw")
    assert_grad_t_close(t.grad.cpu().numpy(), ref["dt"], "autograd dt")


# ------------------------------------------------------------------ many graphs

@pytest.mark.parametrize("edges_log2", [0, 16])  # the default tile shape and the batching one
def test_run_multi_uneven_graphs(edges_log2):
    scales = inputs.multigraph_scales(12, lo=6, hi=12)
    graphs, edges = [], []
    for gi, sc in enumerate(scales):
        n = 1 << sc
        s, d, _ = inputs.rmat_edges(sc, 16 << sc, inputs.multigraph_seed(gi))
        graphs.append(nx.Graph(s, d, n, 1 + gi % 5, transpose=True, tile_edges_log2=edges_log2))
        edges.append((n, s, d))
    st = nx.run_multi(graphs, "pr", 20)
    assert st["iters_done"] == 20 and st["launches"] == 1
    for g, (n, s, d) in zip(graphs, edges):
        assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"multi PR n={n}")
    nx.run_multi(graphs, "bfs", 40)
    for g, (n, s, d) in zip(graphs, edges):
        assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    nx.run_multi(graphs, "wcc", 40)
    for g, (n, s, d) in zip(graphs, edges):
        assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    # a single graph and repeated calls give the same as nx_run
    g0 = graphs[-1]
    nx.run_multi([g0], "pr", 20)
    a = g0.values().copy()
    g0.run("pr", 20)
    assert_pr_close(a, g0.values().astype(np.float64), "multi vs run")


def test_run_multi_replays_its_cuda_graph():
    # a second call with the same graphs and arguments replays the kept
    # executable graph (stats Q = 1) and gives the same values; freeing a
    # member drops it
    graphs, data = [], []
    for gi, sc in enumerate((9, 11, 10)):
        n = 1 << sc
        s, d, _ = inputs.rmat_edges(sc, 16 << sc, inputs.multigraph_seed(100 + gi))
        graphs.append(nx.Graph(s, d, n, 2, transpose=True))
        data.append((n, s, d))
    st1 = nx.run_multi(graphs, "pr", 15)
    first = [g.values().copy() for g in graphs]
    st2 = nx.run_multi(graphs, "pr", 15)
    assert st1["Q"] == 0 and st2["Q"] == 1
    for g, v, (n, s, d) in zip(graphs, first, data):
        ref = oracle.pagerank(n, s, d, 0.85, 15)
        assert_pr_close(v, ref, f"captured n={n}")
        assert_pr_close(g.values(), ref, f"replayed n={n}")  # (shared-memory atomics
        # fold in a run-dependent order, so two runs agree to rounding, not bit for bit)
    assert nx.run_multi(graphs, "pr", 16)["Q"] == 0  # another iteration count: new capture
    st3 = nx.run_multi(graphs, "bfs", 30)
    assert st3["Q"] == 0 and nx.run_multi(graphs, "bfs", 30)["Q"] == 1
    for g, (n, s, d) in zip(graphs, data):
        assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    graphs[1].free()
    assert nx.run_multi([graphs[0], graphs[2]], "bfs", 30)["Q"] == 0
    for g in graphs:
        g.free()


def test_run_multi_barrier_timeout_then_recovers():
    # The persistent kernel's grid barrier waits a bounded number of cycles.
    # With a limit of 64 cycles the blocks that reach the first barrier early
    # give up: the call returns NX_ERR_TIMEOUT (the kernel ends; nothing traps
    # or hangs). With the default limit restored, the same graphs run again and
    # match the oracle, so the error path left nothing behind.
    graphs, data = [], []
    for gi, sc in enumerate((12, 9, 13, 10, 11, 12)):
        n = 1 << sc
        s, d, _ = inputs.rmat_edges(sc, 16 << sc, inputs.multigraph_seed(200 + gi))
        graphs.append(nx.Graph(s, d, n, 1 + gi % 4, transpose=True))
        data.append((n, s, d))
    try:
        nx.set_barrier_limit(64)
        for prog in ("pr", "wcc"):
            with pytest.raises(nx.NxError) as e:
                nx.run_multi(graphs, prog, 20)
            assert e.value.code == nx.NX_ERR_TIMEOUT
    finally:
        nx.set_barrier_limit(0)
    nx.run_multi(graphs, "pr", 20)
    for g, (n, s, d) in zip(graphs, data):
        assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"after timeout n={n}")
    nx.run_multi(graphs, "wcc", 60)
    for g, (n, s, d) in zip(graphs, data):
        assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    # a single-graph run on the same graph state is also unaffected
    g0, (n, s, d) = graphs[2], data[2]
    g0.run("pr", 20)
    assert_pr_close(g0.values(), oracle.pagerank(n, s, d, 0.85, 20), "nx_run after timeout")
    for g in graphs:
        g.free()


@pytest.mark.parametrize("band", [1, 2, 3])
def test_banded_spu(band):
    # SPU in launches over bands of source intervals, accumulators carried in HBM
    n = 1 << 13
    s, d, _ = rmat(13, 16, 15)
    g = nx.Graph(s, d, n, 7, transpose=True)
    st = g.run("pr", 20, band=band)
    assert st["launches"] == 20 * -(-7 // band)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"band {band} PR")
    g.run("bfs", 1000, root=0, band=band)
    assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, 0)).all()
    g.run("wcc", 1000, band=band)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()


def test_autotune_picks_a_candidate_and_caches(tmp_path):
    n = 1 << 14
    s, d, _ = rmat(14, 16, 16)
    cache = str(tmp_path / "tune.txt")
    P, ms = nx.autotune(s, d, n, candidates=(2, 4, 8), iters=5, cache=cache)
    assert P in (2, 4, 8) and all(x > 0 for x in ms)
    assert P == (2, 4, 8)[int(np.argmin(ms))]
    P2, ms2 = nx.autotune(s, d, n, candidates=(2, 4, 8), iters=5, cache=cache)
    assert P2 == P and all(x == -1 for x in ms2)  # served from the cache file


def test_autotune_shapes_pick_argmin_and_cache(tmp_path):
    # P and tile shape together; every shape gives the oracle's results
    n = 1 << 14
    s, d, _ = rmat(14, 16, 16)
    cache = str(tmp_path / "tune.txt")
    shapes = [(4, 0, 0), (4, 9, 0), (8, 12, 12), (16, 13, 15)]
    best, ms = nx.autotune_shape(s, d, n, shapes, iters=5, cache=cache)
    assert all(x > 0 for x in ms) and best == int(np.argmin(ms))
    best2, ms2 = nx.autotune_shape(s, d, n, shapes, iters=5, cache=cache)
    assert best2 == best and all(x == -1 for x in ms2)
    ref_pr = oracle.pagerank(n, s, d, 0.85, 20)
    ref_wcc = oracle.wcc(n, s, d)
    for P, cap, edges in shapes:
        g = nx.Graph(s, d, n, P, transpose=True, tile_cap_log2=cap, tile_edges_log2=edges)
        info = g.info()
        if cap:
            assert info["tile_max"] <= 1 << cap
        g.run("pr", 20)
        assert_pr_close(g.values(), ref_pr, f"shape {(P, cap, edges)}")
        g.run("wcc", 1000)
        assert (g.values(dtype=np.uint32) == ref_wcc).all()
        g.free()
    with pytest.raises(nx.NxError):
        nx.Graph(s, d, n, 4, tile_cap_log2=14)


def test_autotune_batch_shape_and_every_shape_matches(tmp_path):
    import torch

    n = 1 << 13
    s, d, _ = rmat(13, 16, 14)
    B = 12
    T = inputs.ppr_teleports(n, B, 5, max_seeds=40)
    g = nx.Graph(s, d, n, 4)
    refs = {b: oracle.personalized_pagerank(n, s, d, T[:, b], 0.85, 15) for b in (0, 7, 11)}
    for rows in (2, 4, 8):
        for sub in (32, 64, 128, 256):
            g.set_batch_shape(rows, sub)
            R, _ = g.ppr_batch(T, iters=15)
            for b, ref in refs.items():
                assert_pr_close(R[:, b], ref, f"batch rows={rows} sub={sub} col {b}")
    Tt = torch.from_numpy(T).cuda()
    shapes = [(2, 64), (4, 128), (8, 128), (4, 256)]
    cache = str(tmp_path / "batch.txt")
    best, ms = g.autotune_ppr_batch(Tt, iters=5, shapes=shapes, cache=cache)
    assert all(x > 0 for x in ms) and best == int(np.argmin(ms))
    best2, ms2 = g.autotune_ppr_batch(Tt, iters=5, shapes=shapes, cache=cache)
    assert best2 == best and all(x == -1 for x in ms2)
    R, _ = g.ppr_batch(Tt, iters=15)  # runs with the tuned shape
    assert_pr_close(R[:, 7].cpu().numpy(), refs[7], "tuned batch")
    for bad in ((3, 128), (4, 100)):
        with pytest.raises(nx.NxError):
            g.set_batch_shape(*bad)
    g.free()


# ------------------------------------------------- Table IV ablation (Exp 1)

@pytest.mark.parametrize("strategy", ["src_coarse", "src_fine"])
@pytest.mark.parametrize("P", [1, 3, 16])
def test_source_sorted_push_matches_oracle(strategy, P):
    # the source-sorted, atomic-push sweep computes the same PageRank (ragged n)
    n = 5000
    s, d, _ = inputs.rmat_edges(13, 60000, 17)
    keep = (s < n) & (d < n)
    s, d = s[keep], d[keep]
    g = nx.Graph(s, d, n, P, transpose=True)
    st = g.run("pr", 20, strategy)
    assert st["iters_done"] == 20 and st["launches"] >= 40
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"{strategy} P={P}")


@pytest.mark.parametrize("strategy", ["src_coarse", "src_fine"])
def test_source_sorted_push_hub_and_ppr(strategy):
    k = 300_000  # in-star: 300k atomic adds into one destination
    n = k + 1
    s = np.concatenate([np.arange(1, n, dtype=np.uint32), np.array([0, 5], np.uint32)])
    d = np.concatenate([np.zeros(k, np.uint32), np.array([7, 0], np.uint32)])
    g = nx.Graph(s, d, n, 4, transpose=True)
    g.run("pr", 20, strategy)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"{strategy} hub")
    n2 = 1 << 14
    s2, d2, _ = rmat(14, 16, 3)
    t = inputs.ppr_teleports(n2, 1, 33)[:, 0].copy()
    g2 = nx.Graph(s2, d2, n2, 8, transpose=True)
    g2.run("ppr", 30, strategy, teleport=t)
    ref = oracle.personalized_pagerank(n2, s2, d2, t, 0.85, 30)
    assert_pr_close(g2.values(), ref, f"{strategy} PPR")
    # then the DSSS sweep continues from the pushed values (same state layout)
    g2.set_values("ppr", g2.values())
    g2.run("ppr", 5, "spu", teleport=t)
    ref35 = oracle.personalized_pagerank(n2, s2, d2, t, 0.85, 35)
    assert_pr_close(g2.values(), ref35, f"{strategy} then SPU")


def test_source_sorted_push_rejects():
    n = 64
    s = np.arange(n, dtype=np.uint32)
    d = ((np.arange(n) + 1) % n).astype(np.uint32)
    g = nx.Graph(s, d, n, 2)
    with pytest.raises(nx.NxError):  # no transpose DSSS
        g.run("pr", 2, "src_fine")
    gt = nx.Graph(s, d, n, 2, transpose=True)
    for prog in ("bfs", "wcc"):
        with pytest.raises(nx.NxError):
            gt.run(prog, 2, "src_coarse")
    with pytest.raises(nx.NxError):
        gt.run("pr", 2, "src_coarse", budget=1 << 20)
    gt.run("pr", 2, "src_coarse")
    assert np.allclose(gt.values(), 1.0 / n, rtol=1e-6)


# ------------------------------------------- degree-ordered ids (NX_RELABEL)

def _ragged_graph():
    n = 5000
    s, d, _ = inputs.rmat_edges(13, 60000, 17)
    keep = (s < n) & (d < n)
    return n, s[keep], d[keep]


@pytest.mark.parametrize("transpose", [True, False])  # False: new ids applied while making keys
@pytest.mark.parametrize("P", [1, 4, 7])
def test_relabel_order_and_layout(P, transpose):
    n, s, d = _ragged_graph()
    g = nx.Graph(s, d, n, P, transpose=transpose, relabel=True)
    old_of_new = g.relabel_map()
    assert (np.sort(old_of_new) == np.arange(n)).all()  # a permutation
    od = np.bincount(s, minlength=n)[old_of_new]
    assert (np.diff(od) <= 0).all()  # out-degree non-increasing
    tie = np.diff(od) == 0
    assert (np.diff(old_of_new.astype(np.int64))[tie] > 0).all()  # ties by caller id
    new_of_old = np.empty(n, np.uint32)
    new_of_old[old_of_new] = np.arange(n, dtype=np.uint32)
    ns, nd = new_of_old[s], new_of_old[d]
    order, off = oracle.dsss_order(n, P, ns, nd)  # the DSSS of the renamed graph
    gs, gd, goff = g.export()
    assert (goff == off).all()
    assert (gs == ns[order]).all() and (gd == nd[order]).all()
    if transpose:
        order_t, _ = oracle.dsss_order(n, P, nd, ns)
        ts, td, _ = g.export(transpose=True)
        assert (ts == ns[order_t]).all() and (td == nd[order_t]).all()
    g.run("pr", 20)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"relabel P={P} PR")


def test_gather_probe_times_and_leaves_the_run_alone():
    n = 1 << 15
    s, d, _ = rmat(15, 16, 13)
    g = nx.Graph(s, d, n, 8, relabel=True)
    g.run("pr", 10)
    r = g.values().copy()
    ms = g.gather_probe(sweeps=3)
    assert ms > 0.0
    assert (g.values() == r).all()  # the probe writes nothing the run owns
    g.run("pr", 10)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 10), "PR after the probe")


def test_trim_memory_keeps_graphs_and_later_builds_correct():
    n = 1 << 14
    s, d, _ = rmat(14, 16, 9)
    g = nx.Graph(s, d, n, 8, relabel=True)
    g.run("pr", 10)
    ref = oracle.pagerank(n, s, d, 0.85, 10)
    assert_pr_close(g.values(), ref, "before trim")
    nx.trim_memory()  # cached blocks back to the driver; the live graph keeps its own
    g.run("pr", 10)
    assert_pr_close(g.values(), ref, "after trim")
    g.free()
    nx.trim_memory()
    g2 = nx.Graph(s, d, n, 8, relabel=True)
    g2.run("pr", 10)
    assert_pr_close(g2.values(), ref, "new graph after trim")


@pytest.mark.parametrize("P", [3, 16])
def test_relabel_programs_in_caller_ids(P):
    n, s, d = _ragged_graph()
    g = nx.Graph(s, d, n, P, transpose=True, relabel=True)
    g.run("pr", 20)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"relabel P={P} PR")
    for strat in ("dpu", "src_fine"):
        g.run("pr", 20, strat)
        assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), f"relabel {strat}")
    g.run("pr", 20, "mpu", budget=2 * n * 4 // 2 + 1)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "relabel MPU")
    t = inputs.ppr_teleports(n, 1, 5)[:, 0].copy()
    g.run("ppr", 30, teleport=t)
    assert_pr_close(g.values(), oracle.personalized_pagerank(n, s, d, t, 0.85, 30), "relabel PPR")
    for root in (1, 4999):
        g.run("bfs", 1000, root=root)
        assert (g.values(dtype=np.uint32) == oracle.bfs(n, s, d, root)).all()
    g.run("wcc", 1000)
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    g.run("wcc", 1000, "dpu")
    assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
    # resume: values set in caller order continue in caller order
    g.run("pr", 10)
    mid = g.values().copy()
    g.set_values("pr", mid)
    g.run("pr", 10)
    assert_pr_close(g.values(), oracle.pagerank(n, s, d, 0.85, 20), "relabel resume")


def test_relabel_device_pointers_batch_and_adjoint():
    import torch

    n = 1 << 12
    s, d, w = rmat(12, 16, 4, weights=True)
    g = nx.Graph(torch.from_numpy(s.view(np.int32)).cuda(), torch.from_numpy(d.view(np.int32)).cuda(),
                 n, 4, transpose=True, weights=torch.from_numpy(w).cuda(), relabel=True)
    T = inputs.ppr_teleports(n, 8, 21)
    R, _ = g.ppr_batch(torch.from_numpy(T).cuda(), iters=30)
    R = R.cpu().numpy()
    for b in (0, 5):
        ref = oracle.personalized_pagerank(n, s, d, T[:, b].astype(np.float64), 0.85, 30)
        assert_pr_close(R[:, b], ref, f"relabel batch col {b}")
    tv = torch.from_numpy(T[:, 3].copy()).cuda()
    g.run("ppr", 30, teleport=tv)  # device teleport
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    g.values(out)
    ref = oracle.personalized_pagerank(n, s, d, T[:, 3].astype(np.float64), 0.85, 30)
    assert_pr_close(out.cpu().numpy(), ref, "relabel device PPR")
    gv = np.zeros(n, np.float32)
    gv[inputs.targets(n, 64, 4)] = 1.0
    g.run("wpr", 20)
    dw = np.empty(len(s), np.float32)
    dt = np.empty(n, np.float32)
    g.adjoint_wpr(gv, 20, dw, dt)
    ref = oracle.wpr_adjoint(n, s, d, w.astype(np.float64), gv.astype(np.float64), 0.85, 20, 20)
    assert_pr_close(g.values(), ref["r"], "relabel WPR")
    assert_grad_t_close(dt, ref["dt"], "relabel dL/dt")
    assert_grad_w_close(dw, ref, s, d, w, 0.85, "relabel dL/dw")


def test_relabel_rejected_where_unsupported():
    import torch

    n, s, d = _ragged_graph()
    g = nx.Graph(s, d, n, 4, relabel=True)
    with pytest.raises(nx.NxError):
        nx.run_multi([g], "pr", 2)
    r_in = torch.full((n,), 1.0 / n, dtype=torch.float32, device="cuda")
    r_out = torch.empty_like(r_in)
    rc = nx.lib().nx_pagerank_step_noalloc(g.handle, 0.85, r_in.data_ptr(), r_out.data_ptr())
    assert rc == nx.NX_ERR_INVALID_ARG
    plain = nx.Graph(s, d, n, 4)
    with pytest.raises(nx.NxError):
        plain.relabel_map()


# 3, 7, 5 and 8 sorted chunks to merge: the first two leave runs of unequal
# rank in different buffers at the end (the copy before the merge)
@pytest.mark.parametrize("m", [3000, 7000, 8200, 100_000])
@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_host_upload_sorts_while_edges_arrive(kind, m):
    # Host edges without weights are sorted chunk by chunk as they land and the
    # sorted chunks merged; the DSSS (both directions, degree-ordered ids and
    # the on-chip structure) must equal the oracle's for every input kind.
    import torch

    n = 3001
    rng = np.random.default_rng(m)
    s = (rng.zipf(1.7, m) % n).astype(np.uint32)  # skewed, with duplicate edges
    d = rng.integers(0, n, m).astype(np.uint32)
    if kind == "pageable":
        a, b = s, d
    else:
        a = torch.from_numpy(s.view(np.int32))
        b = torch.from_numpy(d.view(np.int32))
        a, b = (a.pin_memory(), b.pin_memory()) if kind == "pinned" else (a.cuda(), b.cuda())
    for relabel in (False, True):
        g = nx.Graph(a, b, n, 5, transpose=True, relabel=relabel, onchip=True)
        if relabel:
            old_of_new = g.relabel_map()
            new_of_old = np.empty(n, np.uint32)
            new_of_old[old_of_new] = np.arange(n, dtype=np.uint32)
            ns, nd = new_of_old[s], new_of_old[d]
        else:
            ns, nd = s, d
        order, off = oracle.dsss_order(n, 5, ns, nd)
        gs, gd, goff = g.export()
        assert (goff == off).all()
        assert (gs == ns[order]).all() and (gd == nd[order]).all()
        order_t, off_t = oracle.dsss_order(n, 5, nd, ns)
        ts, td, toff = g.export(transpose=True)
        assert (toff == off_t).all()
        assert (ts == ns[order_t]).all() and (td == nd[order_t]).all()
        assert g.info()["H_onchip"] == _onchip_hub_count(ns, nd)
        ref = oracle.pagerank(n, s, d, 0.85, 10)
        g.run("pr", 10)
        assert_pr_close(g.values(), ref, f"{kind} relabel={relabel} PR")
        g.run("pr", 10, "dpu_onchip")
        assert_pr_close(g.values(), ref, f"{kind} relabel={relabel} on-chip PR")
        g.run("wcc", 1000)
        assert (g.values(dtype=np.uint32) == oracle.wcc(n, s, d)).all()
        g.free()
    # an id far beyond n is rejected, whatever the path
    bad = s.copy()
    bad[m // 2] = 0xFFFFFFF0
    if kind == "pageable":
        a = bad
    else:
        a = torch.from_numpy(bad.view(np.int32))
        a = a.pin_memory() if kind == "pinned" else a.cuda()
    with pytest.raises(nx.NxError) as e:
        nx.Graph(a, b, n, 5, transpose=True, relabel=True)
    assert e.value.code == nx.NX_ERR_INVALID_ARG


def test_injected_allocation_failures_leave_the_library_usable():
    # Host-side fault injection: every device allocation of a build and of its
    # runs fails in turn (SPU, SPU with streamed shards, MPU with staged
    # intervals, DPU). The failing call returns NX_ERR_OOM and says so; the
    # graph, when it exists, stays usable (the same runs repeated match the
    # oracle), and so does the library.
    import torch

    n = 1 << 12
    s, d, _ = rmat(12, 16, 21)
    m = len(s)
    ref = oracle.pagerank(n, s, d, 0.85, 5)
    wcc = oracle.wcc(n, s, d)
    hs = torch.from_numpy(s.view(np.int32)).pin_memory()
    hd = torch.from_numpy(d.view(np.int32)).pin_memory()
    runs = [("pr", 5, "spu", 0), ("pr", 5, "spu", 2 * n * 4 + 4 * m // 3),
            ("wcc", 100, "mpu", n * 4 + 1), ("pr", 5, "dpu", 0)]  # MPU: Q = 2 of P = 4
    k, failures, in_runs = 0, 0, 0
    while True:
        nx.debug_fail_alloc(k)
        g = None
        try:
            g = nx.Graph(hs, hd, n, 4, transpose=True, relabel=True)
            for prog, it, strat, budget in runs:
                g.run(prog, it, strat, budget=budget)
            nx.debug_fail_alloc(-1)
            g.free()
            break
        except nx.NxError as e:
            nx.debug_fail_alloc(-1)
            assert e.code == nx.NX_ERR_OOM and "injected" in str(e), (k, e)
            failures += 1
            if g is not None:
                in_runs += 1
                for prog, it, strat, budget in runs:
                    g.run(prog, it, strat, budget=budget)
                    if prog == "pr":
                        assert_pr_close(g.values(), ref, f"{strat} after failure {k}")
                    else:
                        assert (g.values(dtype=np.uint32) == wcc).all(), k
                g.free()
        k += 1
        assert k < 2000
    assert failures >= 20 and in_runs >= 10, (failures, in_runs)
    g = nx.Graph(s, d, n, 4, transpose=True)
    g.run("pr", 5)
    assert_pr_close(g.values(), ref, "a fresh build after the failures")
    g.free()
