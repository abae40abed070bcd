"""Pins of the oracle against things other than itself.

Each test checks an oracle function against a value the paper prints, a
closed form, a textbook/library routine (SciPy's csgraph) or brute force on a
tiny input, so that a dropped term, a wrong sign or index, or a transposed
operand in oracle.c fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_graph(n, ne, seed, sym=True, weights=None):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, (ne, 2))
    return gg.from_edge_list(n, map(tuple, e), symmetrize=sym, weights=weights)


def _scipy(g, weighted=False):
    data = g.wt.astype(np.float64) if weighted else np.ones(g.m)
    return sp.csr_matrix((data, g.col, g.row_ptr), shape=(g.n, g.n))


# ---------------------------------------------------------------- CSR checks

def test_validate_catches_each_defect():
    g = gg.from_edge_list(5, [(0, 1), (1, 2), (2, 3), (3, 4)])
    assert oracle.validate_csr(g) == 0
    bad = lambda **kw: type("G", (), dict(n=g.n, row_ptr=g.row_ptr.copy(), col=g.col.copy(), wt=None, **kw))
    b = bad(); b.row_ptr[2], b.row_ptr[3] = b.row_ptr[3], b.row_ptr[2]
    assert oracle.validate_csr(b) != 0          # non-monotone offsets
    b = bad(); b.col[0] = 9
    assert oracle.validate_csr(b) == 4          # index out of range
    b = bad(); b.col[0] = 0
    assert oracle.validate_csr(b) == 5          # self-loop
    b = bad(); b.col[1:3] = b.col[1:3][::-1]
    assert oracle.validate_csr(b) == 6          # unsorted row
    d = gg.from_edge_list(3, [(0, 1), (1, 2)], symmetrize=False)
    assert oracle.validate_csr(d, require_symmetric=True) == 7
    assert oracle.validate_csr(d, require_symmetric=False) == 0


# ------------------------------------------------------------ edge selection

def test_worked_example_from_selection():
    ex = json.load(open(os.path.join(GOLDEN, "gis_worked_example.json")))
    g = gg.from_edge_list(ex["n"], map(tuple, ex["edges_directed"]), symmetrize=False)
    mask = np.zeros(ex["n"], np.uint8)
    mask[ex["frontier"]] = 1
    u, v = oracle.edgeset_select(g, from_mask=mask)
    assert sorted(zip(u.tolist(), v.tolist())) == sorted(map(tuple, ex["push_space"]))
    # pull space = the same edges written (dst, src)
    assert sorted(zip(v.tolist(), u.tolist())) == sorted(map(tuple, ex["pull_space"]))


def test_selection_brute_force():
    g = _rand_graph(30, 120, 3, sym=False)
    rng = np.random.default_rng(5)
    for _ in range(5):
        f, t, fs, fd = (rng.integers(0, 2, g.n).astype(np.uint8) for _ in range(4))
        u, v = oracle.edgeset_select(g, f, t, fs, fd)
        want = [(a, int(g.col[e])) for a in range(g.n) for e in range(g.row_ptr[a], g.row_ptr[a + 1])
                if f[a] and fs[a] and t[g.col[e]] and fd[g.col[e]]]
        assert list(zip(u.tolist(), v.tolist())) == want
    u, v = oracle.edgeset_select(g)
    assert len(u) == g.m


# ---------------------------------------------------------------------- BFS

def _bfs_brute(n, adj, src):
    depth = [-1] * n
    depth[src] = 0
    changed = True
    while changed:  # relax until fixpoint: depth = shortest hop count
        changed = False
        for u in range(n):
            if depth[u] < 0:
                continue
            for v in adj[u]:
                if depth[v] == -1 or depth[v] > depth[u] + 1:
                    depth[v] = depth[u] + 1
                    changed = True
    return depth


@pytest.mark.parametrize("seed", range(4))
def test_bfs_brute_force_and_parent_rule(seed):
    g = _rand_graph(48, 70, seed, sym=(seed % 2 == 0))
    adj = [g.col[g.row_ptr[u]:g.row_ptr[u + 1]].tolist() for u in range(g.n)]
    inn = [[u for u in range(g.n) if v in adj[u]] for v in range(g.n)]
    in_edges = gg.transpose(g)[:2]
    for src in range(0, g.n, 7):
        depth, parent, levels = oracle.bfs(g, src, in_edges=in_edges)
        bd = _bfs_brute(g.n, adj, src)
        assert depth.tolist() == bd
        for v in range(g.n):
            if bd[v] <= 0:
                assert parent[v] == (src if v == src else -1)
            else:
                assert parent[v] == min(w for w in inn[v] if bd[w] == bd[v] - 1)
        assert levels.sum() == sum(d >= 0 for d in bd)


def test_bfs_matches_scipy_and_invariant():
    g = gg.rmat_graph(11, seed=2)
    src = 0
    depth, parent, _ = oracle.bfs(g, src)
    ref = csg.shortest_path(_scipy(g), unweighted=True, indices=src)
    ref = np.where(np.isinf(ref), -1, ref).astype(np.int32)
    assert np.array_equal(depth, ref)
    u = np.repeat(np.arange(g.n), g.degrees())
    both = (depth[u] >= 0)
    assert (np.abs(depth[u][both] - depth[g.col][both]) <= 1).all()


def test_bfs_grid_manhattan_closed_form():
    side = 23
    g = gg.grid_graph(side, shortcut_frac=0.0)
    sx, sy = 5, 17
    depth, parent, _ = oracle.bfs(g, sy * side + sx)
    xs, ys = np.meshgrid(np.arange(side), np.arange(side))
    assert np.array_equal(depth.reshape(side, side), np.abs(xs - sx) + np.abs(ys - sy))


def test_bfs_path_star():
    n = 17
    path = gg.from_edge_list(n, [(i, i + 1) for i in range(n - 1)])
    d, p, lv = oracle.bfs(path, 4)
    assert d.tolist() == [abs(i - 4) for i in range(n)]
    assert p[0] == 1 and p[16] == 15 and p[4] == 4 and p[5] == 4 and p[3] == 4
    star = gg.from_edge_list(n, [(0, i) for i in range(1, n)])
    d, p, lv = oracle.bfs(star, 3)
    assert d[3] == 0 and d[0] == 1 and all(d[i] == 2 for i in range(1, n) if i != 3)
    assert lv.tolist() == [1, 1, n - 2]


# --------------------------------------------------------------------- SSSP

@pytest.mark.parametrize("seed", range(3))
def test_sssp_matches_dijkstra(seed):
    g = _rand_graph(200, 700, seed, weights=(seed, 1, 1000))
    for src in (0, 17, 150):
        dist, fs = oracle.sssp(g, src)
        ref = csg.dijkstra(_scipy(g, True), indices=src)
        ref = np.where(np.isinf(ref), np.iinfo(np.int32).max, ref).astype(np.int64)
        assert np.array_equal(dist.astype(np.int64), ref)


def test_sssp_rmat_invariants_and_unit_weights():
    g = gg.rmat_graph(10, weights=(1, 1000))
    dist, _ = oracle.sssp(g, 0)
    u = np.repeat(np.arange(g.n), g.degrees())
    reach = dist[u] < np.iinfo(np.int32).max
    assert (dist[g.col][reach].astype(np.int64) <= dist[u][reach].astype(np.int64) + g.wt[reach]).all()
    tight = np.zeros(g.n, bool)
    ok = reach & (dist[g.col].astype(np.int64) == dist[u].astype(np.int64) + g.wt)
    tight[g.col[ok]] = True
    reached = dist < np.iinfo(np.int32).max
    reached[0] = False
    assert tight[reached].all()
    g.wt = np.ones_like(g.wt)
    dist, _ = oracle.sssp(g, 0)
    depth, _, _ = oracle.bfs(g, 0)
    assert np.array_equal(np.where(depth < 0, np.iinfo(np.int32).max, depth), dist)


def test_sssp_round_structure_on_path():
    n = 12
    g = gg.from_edge_list(n, [(i, i + 1) for i in range(n - 1)], weights=(1, 1, 2))
    dist, fs = oracle.sssp(g, 0)
    assert dist.tolist() == list(range(n))
    assert fs.tolist() == [1] * n   # frontier {0}, {1}, ..., {n-1}


# ----------------------------------------------------------------------- CC

@pytest.mark.parametrize("seed", range(3))
def test_cc_partition_and_min_label(seed):
    g = _rand_graph(300, 260, seed)
    label, _ = oracle.cc(g)
    ncomp, comp = csg.connected_components(_scipy(g), directed=False)
    want = np.zeros(g.n, np.int32)
    for c in range(ncomp):
        members = np.flatnonzero(comp == c)
        want[members] = members.min()
    assert np.array_equal(label, want)


def test_cc_rmat_labels_constant_on_arcs():
    g = gg.rmat_graph(12)
    label, fs = oracle.cc(g)
    u = np.repeat(np.arange(g.n), g.degrees())
    assert (label[u] == label[g.col]).all()
    assert (label <= np.arange(g.n)).all()
    assert fs[0] == g.n


# ----------------------------------------------------------------- PageRank

def test_pagerank_dense_power_iteration():
    g = _rand_graph(40, 90, 9, sym=False)
    A = np.zeros((g.n, g.n))
    for u in range(g.n):
        for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            A[v, u] = 1.0 / (g.row_ptr[u + 1] - g.row_ptr[u])
    x = np.full(g.n, 1.0 / g.n)
    for _ in range(20):
        x = (1 - 0.85) / g.n + 0.85 * A @ x
    in_edges = gg.transpose(g)[:2]
    r = oracle.pagerank(g, 0.85, 20, normalize=False, in_edges=in_edges)
    assert np.allclose(r, x, rtol=1e-12, atol=0)
    rn = oracle.pagerank(g, 0.85, 20, normalize=True, in_edges=in_edges)
    assert np.allclose(rn, x / x.sum(), rtol=1e-12) and abs(rn.sum() - 1) < 1e-12


@pytest.mark.parametrize("kind", ["cycle", "complete", "torus"])
def test_pagerank_regular_graph_uniform(kind):
    if kind == "cycle":
        n = 31
        g = gg.from_edge_list(n, [(i, (i + 1) % n) for i in range(n)])
    elif kind == "complete":
        n = 9
        g = gg.from_edge_list(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    else:
        s = 8
        n = s * s
        g = gg.from_edge_list(n, [(y * s + x, y * s + (x + 1) % s) for y in range(s) for x in range(s)] +
                              [(y * s + x, ((y + 1) % s) * s + x) for y in range(s) for x in range(s)])
    r = oracle.pagerank(g, 0.85, 20, normalize=False)
    assert np.allclose(r, 1.0 / n, rtol=1e-13)


def test_pagerank_mass_recurrence_with_dangling():
    g = gg.rmat_graph(10)   # has isolated vertices
    d = 0.85
    deg = g.degrees()
    prev = oracle.pagerank(g, d, 0, normalize=False)
    S = prev.sum()
    for k in range(1, 6):
        cur = oracle.pagerank(g, d, k, normalize=False)
        S_next = (1 - d) + d * (S - prev[deg == 0].sum())
        assert abs(cur.sum() - S_next) < 1e-12
        S, prev = cur.sum(), cur
    assert abs(oracle.pagerank(g, d, 20).sum() - 1.0) < 1e-12


# ------------------------------------------------------------ PageRankDelta

def test_prdelta_eps0_equals_pagerank_iterates():
    g = gg.rmat_graph(10)
    for k in (1, 2, 5, 10):
        rank, fs = oracle.prdelta(g, 0.85, 0.0, k)
        pr = oracle.pagerank(g, 0.85, k, normalize=False)
        assert np.allclose(rank, pr, rtol=1e-11, atol=1e-15), k
    assert fs[0] == g.n


def test_prdelta_history_matches_pagerank_iterates_and_frontiers():
    """The per-round history: with eps = 0, Rank after round k is PR_k and
    Delta after round k is PR_k - PR_{k-1} (PR_0 = 1/V, Fig. 1's Delta), both
    from the independently pinned power iteration; with eps > 0 the frontier
    entering round k+1 is {v : |Delta_k(v)| > eps * Rank_k(v)}."""
    g = gg.rmat_graph(10)
    k = 6
    rank, fs, dh, rh = oracle.prdelta(g, 0.85, 0.0, k, history=True)
    prev = np.full(g.n, 1.0 / g.n)
    for r in range(k):
        pr = oracle.pagerank(g, 0.85, r + 1, normalize=False)
        assert np.allclose(rh[r], pr, rtol=1e-11, atol=1e-15), r
        assert np.allclose(dh[r], pr - prev, rtol=1e-9, atol=1e-15), r
        prev = pr
    assert np.array_equal(rh[-1], rank)
    rank, fs, dh, rh = oracle.prdelta(g, 0.85, 1e-2, 8, history=True)
    for r in range(1, 8):
        assert fs[r] == int(np.sum(np.abs(dh[r - 1]) > 1e-2 * rh[r - 1])), r


def test_prdelta_huge_eps_freezes_after_round1():
    g = gg.rmat_graph(9)
    r1, _ = oracle.prdelta(g, 0.85, 0.0, 1)
    r, fs = oracle.prdelta(g, 0.85, 1e9, 6)
    assert np.array_equal(r, r1)
    assert fs[0] == g.n and (fs[1:] == 0).all()


def test_prdelta_round1_by_hand():
    # path 0-1-2: out-degrees 1,2,1; round 1 DeltaSum = sum over in-nbrs of (1/3)/deg
    g = gg.from_edge_list(3, [(0, 1), (1, 2)])
    a, n = 0.85, 3
    ds = np.array([(1 / 3) / 2, (1 / 3) / 1 + (1 / 3) / 1, (1 / 3) / 2])
    rank, _ = oracle.prdelta(g, a, 0.0, 1)
    assert np.allclose(rank, a * ds + (1 - a) / n, rtol=1e-14)


# ------------------------------------------------ frontier stats and rules

def test_frontier_stats_brute():
    g = gg.rmat_graph(9)
    rng = np.random.default_rng(1)
    f = rng.integers(0, 2, g.n).astype(np.uint8)
    vis = rng.integers(0, 2, g.n).astype(np.uint8)
    deg = g.degrees().astype(np.int64)
    assert oracle.frontier_stats(g, f, vis) == (int(f.sum()), int(deg[f == 1].sum()),
                                                  int((vis == 0).sum()), int(deg[vis == 0].sum()))


def test_beamer_and_ligra_rules():
    # push -> pull when m_f > m_u/alpha
    assert oracle.beamer(1000, 10, 11, 14 * 10, 0) == 1
    assert oracle.beamer(1000, 10, 10, 14 * 10, 0) == 0
    # pull -> push when |F| < V/beta
    assert oracle.beamer(2400, 99, 0, 0, 1) == 0
    assert oracle.beamer(2400, 100, 0, 0, 1) == 1
    assert oracle.ligra_dense(2000, 50, 51) == 1 and oracle.ligra_dense(2000, 50, 50) == 0


def test_features_closed_form():
    x = oracle.features(n=1023, m=4095, maxdeg=255, nf=7, mf=63, nu=511, mu=2047, level=3, was_pull=1,
                        nf_prev=15)
    want = [3, 6, 9, 11, 10, 12, 7 / 1023, 63 / 4095, 511 / 1023, 2047 / 4095, np.log2(10), 8,
            np.log2(1 + 4095 / 1023), 2, 1, 4]
    assert np.allclose(x, want, rtol=1e-14)


# ---------------------------------------------------------------------- MLP

def _mlp_init(seed):
    rng = np.random.default_rng(seed)
    return rng.normal(0, 0.3, oracle.mlp_num_params())


def test_mlp_param_count():
    assert oracle.mlp_num_params() == 64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3


def test_mlp_forward_matches_matrix_form():
    p = _mlp_init(1)
    X = np.random.default_rng(2).normal(size=(5, 16))
    o = 0
    W1 = p[o:o + 1024].reshape(64, 16); o += 1024
    b1 = p[o:o + 64]; o += 64
    W2 = p[o:o + 4096].reshape(64, 64); o += 4096
    b2 = p[o:o + 64]; o += 64
    W3 = p[o:o + 192].reshape(3, 64); o += 192
    b3 = p[o:o + 3]
    h = np.maximum(X @ W1.T + b1, 0)
    h = np.maximum(h @ W2.T + b2, 0)
    assert np.allclose(oracle.mlp_forward(p, X), h @ W3.T + b3, rtol=1e-12)


def test_mlp_gradient_finite_differences():
    p = _mlp_init(3)
    rng = np.random.default_rng(4)
    X = rng.normal(size=(6, 16))
    T = rng.normal(size=(6, 3))
    M = rng.integers(0, 2, (6, 3)).astype(np.float64)
    M[0] = 1
    loss, g = oracle.mlp_loss_grad(p, X, T, M)
    Y = oracle.mlp_forward(p, X)
    assert abs(loss - (M * (Y - T) ** 2).sum() / M.sum()) < 1e-12
    h = 1e-6
    idx = np.r_[0:20, 1024:1030, 1088:1100, 5184:5190, 5376:5380, 5440:5443,
                rng.integers(0, p.size, 40)]
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, X, T, M)[0] - oracle.mlp_loss_grad(pm, X, T, M)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), i


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m = np.zeros(3)
    v = np.zeros(3)
    oracle.adam_step(p, g, m, v, 1, lr=0.01, eps=1e-8)
    # bias-corrected first step moves each parameter by lr * g/(|g| + eps)
    assert np.allclose(p, [1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4 / (4 + 1e-8), 0.5], rtol=1e-14)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


# ------------------------------------------- synchronous (Jacobi) rounds, by hand

def test_sssp_rounds_are_synchronous_hand_example():
    # 0-1 (1), 1-2 (1), 2-3 (1), 0-2 (10), 0-3 (10).  Round 2 must relax 2's arcs
    # with its start-of-round distance 10, so 3 only improves in round 3:
    # frontiers {0}, {1,2,3}, {2}, {3}.  An in-place (Gauss-Seidel) sweep gives {0},{1,2,3},{2,3}.
    edges = [(0, 1, 1), (1, 2, 1), (2, 3, 1), (0, 2, 10), (0, 3, 10)]
    g = gg.from_edge_list(4, [(a, b) for a, b, _ in edges])
    w = {(a, b): c for a, b, c in edges}
    w.update({(b, a): c for (a, b), c in list(w.items())})
    u = np.repeat(np.arange(g.n), g.degrees())
    g.wt = np.array([w[(int(a), int(b))] for a, b in zip(u, g.col)], np.int32)
    dist, fs = oracle.sssp(g, 0)
    assert dist.tolist() == [0, 1, 2, 3]
    assert fs.tolist() == [1, 3, 1, 1]


def test_cc_rounds_are_synchronous_hand_example():
    # path 0-1-2: round 1 (all active) gives labels 0,0,1; round 2 (active {1,2}) gives 0,0,0;
    # round 3 (active {2}) changes nothing.  An in-place sweep would finish in 2 rounds.
    g = gg.from_edge_list(3, [(0, 1), (1, 2)])
    label, fs = oracle.cc(g)
    assert label.tolist() == [0, 0, 0]
    assert fs.tolist() == [3, 2, 1]
