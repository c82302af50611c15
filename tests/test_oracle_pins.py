"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms,
brute force from the definition, dense linear algebra, invariants, and the
Fig. 1 worked example (Section II-A).
"""
import os
from collections import deque

import numpy as np
import pytest

import oracle
from paper_1510_06916_b300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ALPHA = 0.85


def _rand_graph(n, m, seed, self_loops=True):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, m).astype(np.uint32)
    d = rng.integers(0, n, m).astype(np.uint32)
    if not self_loops:
        keep = s != d
        s, d = s[keep], d[keep]
    return s, d


def _dense_transition(n, s, d, w=None):
    """Column-stochastic Pt[v, u] = sum over edges u->v of p_uv; d_u = dangling."""
    w = np.ones(len(s)) if w is None else np.asarray(w, dtype=np.float64)
    W = np.zeros(n)
    np.add.at(W, s, w)
    Pt = np.zeros((n, n))
    np.add.at(Pt, (d, s), w / W[s])
    return Pt, (W == 0).astype(np.float64)


# ---------------------------------------------------------------- PageRank

@pytest.mark.parametrize("n", [1, 2, 7, 64, 1000])
@pytest.mark.parametrize("iters", [1, 5, 20])
def test_cycle_is_uniform(n, iters):
    s = np.arange(n, dtype=np.uint32)
    d = ((np.arange(n) + 1) % n).astype(np.uint32)
    r = oracle.pagerank(n, s, d, ALPHA, iters)
    assert np.allclose(r, 1.0 / n, rtol=4e-16 * 8, atol=0)


@pytest.mark.parametrize("k", [1, 3, 10, 63])
@pytest.mark.parametrize("iters", [0, 1, 2, 7, 20, 200])
def test_in_star_closed_form(k, iters):
    # k leaves -> centre c = 0; the centre is dangling, leaves have no in-edges.
    n = k + 1
    s = np.arange(1, n, dtype=np.uint32)
    d = np.zeros(k, dtype=np.uint32)
    r = oracle.pagerank(n, s, d, ALPHA, iters)
    # r_c^{t+1} = (1-a)/n + a - a(1-1/n) r_c^t  => geometric approach to r*.
    a = ALPHA
    rstar = (1 + a * k) / (n + a * k)
    q = -a * (1 - 1 / n)
    rc = rstar + q ** iters * (1 / n - rstar)
    assert r[0] == pytest.approx(rc, rel=1e-13, abs=1e-16)
    # leaves: (1-a)/n + a r_c^{t-1} / n for t >= 1
    if iters > 0:
        rc_prev = rstar + q ** (iters - 1) * (1 / n - rstar)
        leaf = (1 - a) / n + a * rc_prev / n
    else:
        leaf = 1 / n
    assert np.allclose(r[1:], leaf, rtol=1e-13)
    if iters >= 200:
        assert r[0] == pytest.approx(rstar, rel=1e-12)
        assert np.allclose(r[1:], (1 - rstar) / k, rtol=1e-12)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("weighted", [False, True])
def test_dense_power_iteration_and_solve(seed, weighted):
    n = 5 + 13 * seed  # up to 44 vertices
    s, d = _rand_graph(n, 3 * n, seed)
    w = np.random.default_rng(100 + seed).uniform(0.5, 1.5, len(s)) if weighted else None
    Pt, dang = _dense_transition(n, s, d, w)
    G = ALPHA * (Pt + np.outer(np.ones(n), dang) / n) + (1 - ALPHA) / n * np.ones((n, n))
    x = np.full(n, 1.0 / n)
    for _ in range(20):
        x = G @ x
    r = oracle.pagerank(n, s, d, ALPHA, 20, w=w)
    assert np.abs(r - x).max() < 1e-14
    # fixed point by Gaussian elimination (textbook): (I - a(Pt + 1 d^T/n)) r = (1-a)/n
    A = np.eye(n) - ALPHA * (Pt + np.outer(np.ones(n), dang) / n)
    rstar = np.linalg.solve(A, np.full(n, (1 - ALPHA) / n))
    r300 = oracle.pagerank(n, s, d, ALPHA, 300, w=w)
    assert np.abs(r300 - rstar).max() < 1e-13


@pytest.mark.parametrize("iters", [1, 3, 20])
def test_rank_mass_sums_to_one_with_dangling(iters):
    s, d, _ = inputs.rmat_edges(12, 8 << 12, 7)
    n = 1 << 12
    outdeg = np.bincount(s, minlength=n)
    assert (outdeg == 0).sum() > 100  # plenty of dangling vertices
    r = oracle.pagerank(n, s, d, ALPHA, iters)
    assert abs(r.sum() - 1.0) < 1e-12
    assert (r > 0).all()


@pytest.mark.parametrize("weighted", [False, True])
def test_prepared_problem_is_the_same_arithmetic(weighted):
    # the prepared form (CSR built once, iterations timed alone) returns exactly
    # the one-call result, and repeated iterate() calls do not interfere
    s, d, w = inputs.rmat_edges(10, 8 << 10, 8, weights=weighted)
    n = 1 << 10
    w = None if w is None else w.astype(np.float64)
    pp = oracle.PreparedPageRank(n, s, d, w)
    for iters in (1, 7):
        assert (pp.iterate(ALPHA, iters) == oracle.pagerank(n, s, d, ALPHA, iters, w=w)).all()
    t = np.zeros(n)
    t[[3, 9]] = 0.5
    assert (pp.iterate(ALPHA, 4, tele=t, dangling_by_tele=True, r0=t)
            == oracle.pagerank(n, s, d, ALPHA, 4, w=w, tele=t, dangling_by_tele=True, r0=t)).all()
    pp.close()


def test_thread_count_does_not_change_the_oracle():
    # every vertex's sum is taken by one thread in edge order, so one thread
    # and all of them give the same bits (the CPU baseline times both)
    s, d, _ = inputs.rmat_edges(12, 16 << 12, 11)
    n = 1 << 12
    pp = oracle.PreparedPageRank(n, s, d)
    oracle.set_threads(1)
    try:
        one = pp.iterate(ALPHA, 5)
    finally:
        oracle.set_threads(os.cpu_count() or 1)
    assert (pp.iterate(ALPHA, 5) == one).all()
    pp.close()


def test_pagerank_dangling_term_matters():
    # A plausible mistake (dropping the dangling mass) breaks the sum-to-one pin:
    # a 2-vertex path 0 -> 1 with 1 dangling.
    r = oracle.pagerank(2, [0], [1], ALPHA, 1)
    # r'_0 = (1-a)/2 + a*(0 + 0.5/2); r'_1 = (1-a)/2 + a*(0.5 + 0.5/2)
    assert r[0] == pytest.approx((1 - ALPHA) / 2 + ALPHA * 0.25, rel=1e-15)
    assert r[1] == pytest.approx((1 - ALPHA) / 2 + ALPHA * 0.75, rel=1e-15)


# ---------------------------------------------------------------- PPR

def test_ppr_uniform_teleport_equals_pagerank():
    s, d, _ = inputs.rmat_edges(10, 16 << 10, 3)
    n = 1024
    t = np.full(n, 1.0 / n)
    assert np.abs(oracle.personalized_pagerank(n, s, d, t, ALPHA, 30)
                  - oracle.pagerank(n, s, d, ALPHA, 30)).max() < 1e-15


@pytest.mark.parametrize("iters", [1, 7, 30])
def test_ppr_is_linear_in_the_teleport_without_dangling_vertices(iters):
    # With every vertex holding an out-edge there is no dangling mass, so each
    # step r' = (1-a) t + a Pt r (from r0 = t) is linear in t: the result for a
    # mix of two teleports is the same mix of their results. (With dangling
    # vertices the term Dm(r) t is bilinear and this does not hold.)
    n = 500
    s, d = _rand_graph(n, 3000, 11)
    ring_s = np.arange(n, dtype=np.uint32)
    ring_d = ((np.arange(n) + 1) % n).astype(np.uint32)
    s, d = np.concatenate([s, ring_s]), np.concatenate([d, ring_d])
    rng = np.random.default_rng(5)
    t1 = np.zeros(n)
    t1[rng.choice(n, 3, replace=False)] = 1.0 / 3
    t2 = rng.random(n)
    t2 /= t2.sum()
    # weights that do not sum to one, so a constant term (an affine map) fails too
    beta, gamma = 0.3, 1.1
    mix = oracle.personalized_pagerank(n, s, d, beta * t1 + gamma * t2, ALPHA, iters)
    r1 = oracle.personalized_pagerank(n, s, d, t1, ALPHA, iters)
    r2 = oracle.personalized_pagerank(n, s, d, t2, ALPHA, iters)
    assert np.abs(mix - (beta * r1 + gamma * r2)).max() < 1e-15
    assert abs(mix.sum() - (beta + gamma)) < 1e-12  # no dangling vertex: mass is kept


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ppr_fixed_point_dense(seed):
    # With dangling mass spread by t the fixed point is x / sum(x),
    # x = (I - a Pt)^{-1} t (textbook linear solve).
    n = 30
    s, d = _rand_graph(n, 60, seed)
    t = np.zeros(n)
    t[np.random.default_rng(seed).choice(n, 4, replace=False)] = 0.25
    Pt, _ = _dense_transition(n, s, d)
    x = np.linalg.solve(np.eye(n) - ALPHA * Pt, t)
    r = oracle.personalized_pagerank(n, s, d, t, ALPHA, 400)
    assert np.abs(r - x / x.sum()).max() < 1e-13
    # and one step from r0 = t by hand
    dang = np.bincount(s, minlength=n) == 0
    r1 = (1 - ALPHA) * t + ALPHA * (Pt @ t + t * t[dang].sum())
    assert np.abs(oracle.personalized_pagerank(n, s, d, t, ALPHA, 1) - r1).max() < 1e-16


# ---------------------------------------------------------------- BFS

def _bellman_ford(n, s, d, root):
    INF = oracle.INF
    depth = [INF] * n
    depth[root] = 0
    changed = True
    while changed:  # relax every edge until nothing changes (Algorithm 3)
        changed = False
        for u, v in zip(s, d):
            if depth[u] != INF and depth[v] > depth[u] + 1:
                depth[v] = depth[u] + 1
                changed = True
    return np.array(depth, dtype=np.uint32)


def _read_fixture(name):
    out = {"edge": [], "expect": []}
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            k, *v = line.split()
            if k in ("edge", "expect"):
                out[k].append(tuple(int(x) for x in v))
            else:
                out[k] = v
    return out


def test_bfs_golden_fixture():
    fx = _read_fixture("bfs_levels.txt")
    n = int(fx["n"][0])
    s = [e[0] for e in fx["edge"]]
    d = [e[1] for e in fx["edge"]]
    depth = oracle.bfs(n, s, d, int(fx["root"][0]))
    want = [oracle.INF if x == "inf" else int(x) for x in fx["depth"]]
    assert depth.tolist() == want
    finite = depth[depth != oracle.INF]
    assert int(finite.max()) == int(fx["maxdepth"][0])  # Algorithm 4 output
    assert oracle.bfs_max_depth(depth) == int(fx["maxdepth"][0])
    assert oracle.bfs_max_depth(np.full(3, oracle.INF, np.uint32)) == -1


@pytest.mark.parametrize("seed", range(6))
def test_bfs_matches_bellman_ford(seed):
    n = 3 + 7 * seed
    s, d = _rand_graph(n, 2 * n, seed)
    for root in (0, n - 1):
        assert (oracle.bfs(n, s, d, root) == _bellman_ford(n, s, d, root)).all()


# ---------------------------------------------------------------- WCC

def _wcc_dfs(n, s, d):
    adj = [[] for _ in range(n)]
    for u, v in zip(s, d):
        adj[u].append(v)
        adj[v].append(u)
    label = [-1] * n
    for start in range(n):  # increasing ids: each component is first hit at its minimum
        if label[start] >= 0:
            continue
        label[start] = start
        q = deque([start])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if label[v] < 0:
                    label[v] = start
                    q.append(v)
    return np.array(label, dtype=np.uint32)


@pytest.mark.parametrize("seed", range(6))
def test_wcc_matches_dfs(seed):
    n = 4 + 9 * seed
    s, d = _rand_graph(n, n, seed)
    assert (oracle.wcc(n, s, d) == _wcc_dfs(n, s, d)).all()


def test_wcc_matches_scipy_components():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    s, d, _ = inputs.rmat_edges(11, 2 << 11, 5)
    n = 1 << 11
    lab = oracle.wcc(n, s, d)
    A = sp.coo_matrix((np.ones(len(s)), (s, d)), shape=(n, n))
    k, comp = connected_components(A, directed=True, connection="weak")
    assert len(np.unique(lab)) == k
    # same partition, and each label is its component's minimum id
    for c in range(k):
        members = np.flatnonzero(comp == c)
        assert (lab[members] == members.min()).all()


# ---------------------------------------------------------------- SCC

def _scc_brute(n, s, d):
    """u and v share a component iff each reaches the other (reachability by
    a breadth-first search from every vertex); label = smallest member."""
    adj = [[] for _ in range(n)]
    for u, v in zip(s, d):
        adj[int(u)].append(int(v))
    reach = np.zeros((n, n), dtype=bool)
    for r in range(n):
        reach[r, r] = True
        q = deque([r])
        while q:
            u = q.popleft()
            for v in adj[u]:
                if not reach[r, v]:
                    reach[r, v] = True
                    q.append(v)
    mutual = reach & reach.T
    return np.array([int(np.flatnonzero(mutual[v]).min()) for v in range(n)], dtype=np.uint32)


@pytest.mark.parametrize("seed", range(8))
def test_scc_matches_mutual_reachability(seed):
    n = 3 + 6 * seed
    s, d = _rand_graph(n, int(1.3 * n), seed)
    assert (oracle.scc(n, s, d) == _scc_brute(n, s, d)).all()


def test_scc_special_cases():
    # a directed cycle is one component; a path (a DAG) is all singletons;
    # a self-loop does not join anything; isolated vertices are their own
    n = 10
    cyc = np.arange(n, dtype=np.uint32)
    assert (oracle.scc(n, cyc, (cyc + 1) % n) == 0).all()
    assert (oracle.scc(n, cyc[:-1], cyc[1:]) == cyc).all()
    assert (oracle.scc(n, [3, 3], [3, 4]) == cyc).all()
    # two cycles joined one way stay apart: {0,1,2} -> {5,6}
    s = np.array([0, 1, 2, 2, 5, 6], np.uint32)
    d = np.array([1, 2, 0, 5, 6, 5], np.uint32)
    lab = oracle.scc(7, s, d)
    assert lab.tolist() == [0, 0, 0, 3, 4, 5, 5]


def test_scc_matches_scipy_strong_components():
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components

    s, d, _ = inputs.rmat_edges(12, 4 << 12, 6)
    n = 1 << 12
    lab = oracle.scc(n, s, d)
    A = sp.coo_matrix((np.ones(len(s)), (s, d)), shape=(n, n))
    k, comp = connected_components(A, directed=True, connection="strong")
    assert len(np.unique(lab)) == k
    assert k < n - 100  # a non-trivial case: many vertices share components
    for c in range(k):
        members = np.flatnonzero(comp == c)
        assert (lab[members] == members.min()).all()


def test_scc_is_finer_than_wcc():
    s, d, _ = inputs.rmat_edges(11, 8 << 11, 2)
    n = 1 << 11
    scc, wcc = oracle.scc(n, s, d), oracle.wcc(n, s, d)
    # every strong component lies inside one weak component, and the labels are minima
    assert (wcc[scc] == wcc).all()
    assert (scc <= np.arange(n)).all() and (scc[scc] == scc).all()


# ---------------------------------------------------------------- adjoint

def _dense_M(n, s, d, w):
    Pt, dang = _dense_transition(n, s, d, w)
    return ALPHA * (Pt + np.outer(np.ones(n), dang) / n), dang


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_teleport_grad_is_unrolled_exact(seed):
    # L = g . r^K, r^K = M^K r0 + sum_{k<K} M^k (1-a) t  =>  dL/dt = (1-a) sum_{k<K} (M^T)^k g
    n = 20
    s, d = _rand_graph(n, 50, seed)
    w = np.random.default_rng(seed).uniform(0.5, 1.5, len(s))
    g = np.zeros(n)
    g[[1, 4, 7]] = 1.0
    K = 12
    M, _ = _dense_M(n, s, d, w)
    acc = np.zeros(n)
    v = g.copy()
    for _ in range(K):
        acc += v
        v = M.T @ v
    out = oracle.wpr_adjoint(n, s, d, w, g, ALPHA, fwd_iters=K, adj_terms=K)
    assert np.abs(out["dt"] - (1 - ALPHA) * acc).max() < 1e-14


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_adjoint_weight_grad_fixed_point_dense(seed):
    # Exact implicit gradient at the fixed point: lambda = (I - M^T)^{-1} g,
    # dL/dwhat_uv = a lambda_v r_u, chain rule through what = w / W_u.
    n = 16
    s, d = _rand_graph(n, 40, seed)
    w = np.random.default_rng(seed + 9).uniform(0.5, 1.5, len(s))
    g = np.zeros(n)
    g[[0, 3]] = 1.0
    M, dang = _dense_M(n, s, d, w)
    A = np.eye(n) - M
    r = np.linalg.solve(A, np.full(n, (1 - ALPHA) / n))
    lam = np.linalg.solve(A.T, g)
    W = np.zeros(n)
    np.add.at(W, s, w)
    dwhat = ALPHA * lam[d] * r[s]  # per edge
    # dL/dw_e = dwhat_e / W_u - sum_{e' from u} dwhat_e' w_e' / W_u^2
    tmp = np.zeros(n)
    np.add.at(tmp, s, dwhat * w)
    dw = dwhat / W[s] - tmp[s] / W[s] ** 2
    out = oracle.wpr_adjoint(n, s, d, w, g, ALPHA, fwd_iters=400, adj_terms=400)
    assert np.abs(out["dw"] - dw).max() < 1e-13
    assert np.abs(out["dt"] - (1 - ALPHA) * lam).max() < 1e-13


def test_adjoint_central_differences_and_scale_invariance():
    n = 1 << 8
    s, d, w = inputs.rmat_edges(8, 8 << 8, 4, weights=True)
    w = w.astype(np.float64)
    T = inputs.targets(n, 16, 44)
    g = np.zeros(n)
    g[T] = 1.0
    K = 200  # a^200 ~ 8e-15: truncation far below the FD error
    out = oracle.wpr_adjoint(n, s, d, w, g, ALPHA, fwd_iters=K, adj_terms=K)
    rng = np.random.default_rng(0)
    for e in rng.choice(len(s), 12, replace=False):
        h = 1e-6 * w[e]
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        Lp = oracle.pagerank(n, s, d, ALPHA, K, w=wp)[T].sum()
        Lm = oracle.pagerank(n, s, d, ALPHA, K, w=wm)[T].sum()
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - out["dw"][e]) <= 1e-7 * max(abs(fd), 1e-3)
    # scaling all of u's weights leaves L unchanged => sum_v w_uv dL/dw_uv = 0 per u
    per_u = np.zeros(n)
    np.add.at(per_u, s, w * out["dw"])
    assert np.abs(per_u).max() < 1e-14


def test_adjoint_central_differences_on_100_edges():
    # The differentiation workload checks 100 random edges against central
    # differences; here at R-MAT scale 12 (edge factor 16, 64 targets), with
    # 200 forward steps and 200 adjoint terms (a^200 ~ 8e-15 truncation).
    # Central differences err by rounding, about eps |L| / h, and by h^2 times
    # the third derivative / 6.
    n = 1 << 12
    s, d, w = inputs.rmat_edges(12, 16 << 12, 4, weights=True)
    w = w.astype(np.float64)
    T = inputs.targets(n, 64, 4)
    g = np.zeros(n)
    g[T] = 1.0
    K = 200
    out = oracle.wpr_adjoint(n, s, d, w, g, ALPHA, fwd_iters=K, adj_terms=K)
    L0 = oracle.pagerank(n, s, d, ALPHA, K, w=w)[T].sum()
    rng = np.random.default_rng(100)
    worst = 0.0
    for e in rng.choice(len(s), 100, replace=False):
        h = 1e-5 * w[e]
        wp, wm = w.copy(), w.copy()
        wp[e] += h
        wm[e] -= h
        fd = (oracle.pagerank(n, s, d, ALPHA, K, w=wp)[T].sum()
              - oracle.pagerank(n, s, d, ALPHA, K, w=wm)[T].sum()) / (2 * h)
        err = abs(fd - out["dw"][e])
        tol = 1e-6 * abs(fd) + 50 * np.finfo(float).eps * L0 / h
        worst = max(worst, err / tol)
        assert err <= tol, (e, fd, out["dw"][e])
    print(f"100-edge central differences: worst error / tolerance = {worst:.3f}")


# ---------------------------------------------------------------- DSSS layout

def test_fig1_subshard_order():
    fx = _read_fixture("fig1_dsss.txt")
    n, P = int(fx["n"][0]), int(fx["P"][0])
    s = np.array([e[0] for e in fx["edge"]])
    d = np.array([e[1] for e in fx["edge"]])
    order, off = oracle.dsss_order(n, P, s, d)
    i, j = 2, 1  # paper's SS_3.2 (1-based)
    sel = order[off[j * P + i]:off[j * P + i + 1]]
    assert list(zip(s[sel].tolist(), d[sel].tolist())) == fx["expect"]


def test_dsss_order_invariants():
    n, P = 1000, 7
    s, d = _rand_graph(n, 5000, 11)
    order, off = oracle.dsss_order(n, P, s, d)
    assert sorted(order.tolist()) == list(range(len(s)))  # a permutation
    L = -(-n // P)
    for j in range(P):
        for i in range(P):
            sel = order[off[j * P + i]:off[j * P + i + 1]]
            assert (s[sel] // L == i).all() and (d[sel] // L == j).all()
            key = d[sel].astype(np.int64) * n + s[sel]
            assert (np.diff(key) >= 0).all()
