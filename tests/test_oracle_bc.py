"""Pins of the oracle's single-source betweenness dependencies (Brandes).

Independent of the oracle's accumulation: closed forms on paths, stars,
cycles and complete graphs; grid path counts (binomial coefficients); the
pair-dependency definition delta_s(v) = sum_t sigma_sv sigma_vt / sigma_st
over t with d(s,v) + d(v,t) = d(s,t), evaluated from all-pairs BFS on tiny
random graphs; the identity sum_v delta_s(v) = sum_t (d(s,t) - 1); and
NetworkX's betweenness_centrality where NetworkX is installed.
"""
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle


def _und(n, pairs):
    return gg.from_edge_list(n, pairs)


def test_path_closed_form():
    n = 9
    g = _und(n, [(i, i + 1) for i in range(n - 1)])
    d, s, nl = oracle.bc(g, 0)
    assert nl == n
    assert np.array_equal(s, np.ones(n))
    assert np.array_equal(d, np.array([0] + [n - 1 - v for v in range(1, n)], float))
    d, s, _ = oracle.bc(g, 4)  # middle: each side counts the vertices beyond it
    assert np.array_equal(d, np.array([0, 1, 2, 3, 0, 3, 2, 1, 0], float))


def test_star_and_complete_graph():
    k = 12
    star = _und(k + 1, [(0, i) for i in range(1, k + 1)])
    d, s, _ = oracle.bc(star, 3)
    want = np.zeros(k + 1)
    want[0] = k - 1
    assert np.array_equal(d, want) and np.array_equal(s, np.ones(k + 1))
    n = 8
    kn = _und(n, [(i, j) for i in range(n) for j in range(i + 1, n)])
    d, s, nl = oracle.bc(kn, 5)
    assert nl == 2 and not d.any() and np.array_equal(s, np.ones(n))


def test_even_cycle_closed_form():
    n = 6
    g = _und(n, [(i, (i + 1) % n) for i in range(n)])
    d, s, _ = oracle.bc(g, 0)
    assert np.array_equal(s, np.array([1, 1, 1, 2, 1, 1], float))
    # 1 and 5 carry their successor fully and half of the antipode; 2 and 4 half of it
    assert np.allclose(d, [0, 1.5, 0.5, 0, 0.5, 1.5], rtol=0, atol=1e-15)


def test_grid_path_counts_are_binomials():
    side = 7
    g = gg.grid_graph(side, shortcut_frac=0.0, seed=1)
    d, s, nl = oracle.bc(g, 0)
    ij = np.arange(side * side)
    r, c = ij // side, ij % side
    assert np.array_equal(s, np.array([comb(int(a + b), int(a)) for a, b in zip(r, c)], float))
    assert nl == 2 * side - 1
    # the far corner lies on no shortest path to any other vertex
    assert d[side * side - 1] == 0


def _all_pairs(n, rp, ci):
    dist = np.full((n, n), -1, np.int64)
    sig = np.zeros((n, n))
    for x in range(n):
        dist[x, x], sig[x, x] = 0, 1.0
        q = [x]
        for v in q:
            for e in range(rp[v], rp[v + 1]):
                w = ci[e]
                if dist[x, w] < 0:
                    dist[x, w] = dist[x, v] + 1
                    q.append(w)
                if dist[x, w] == dist[x, v] + 1:
                    sig[x, w] += sig[x, v]
    return dist, sig


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_pair_dependency_definition_tiny_random(seed):
    rng = np.random.default_rng(seed)
    n = 24
    pairs = [tuple(x) for x in rng.integers(0, n, (40, 2))]
    g = _und(n, pairs)
    dist, sig = _all_pairs(n, g.row_ptr, g.col)
    for s in range(0, n, 5):
        want = np.zeros(n)
        for v in range(n):
            if v == s or dist[s, v] < 0:
                continue
            for t in range(n):
                if t in (s, v) or dist[s, t] < 0 or dist[v, t] < 0:
                    continue
                if dist[s, v] + dist[v, t] == dist[s, t]:
                    want[v] += sig[s, v] * sig[v, t] / sig[s, t]
        d, sg, _ = oracle.bc(g, s)
        assert np.allclose(d, want, rtol=1e-12, atol=1e-12)
        assert np.array_equal(sg, np.where(dist[s] >= 0, sig[s], 0.0))


def test_dependency_sum_identity_rmat():
    g = gg.rmat_graph(10, seed=3)
    for s in gg.pick_sources(g, 3, seed=1):
        d, sg, _ = oracle.bc(g, int(s))
        depth, _, _ = oracle.bfs(g, int(s))
        reached = depth > 0
        assert np.isclose(d.sum(), float((depth[reached] - 1).sum()), rtol=1e-12)
        assert (sg[depth >= 0] >= 1).all() and not sg[depth < 0].any()


def test_directed_graph_uses_in_arcs():
    # 0->1->3, 0->2->3, 3->4: two shortest paths to 3 and 4; 1 and 2 carry half of each
    g = gg.from_edge_list(5, [(0, 1), (0, 2), (1, 3), (2, 3), (3, 4)], symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(g)
    d, s, nl = oracle.bc(g, 0, in_edges=(in_ptr, in_col))
    assert np.array_equal(s, [1, 1, 1, 2, 2]) and nl == 4
    assert np.allclose(d, [0, 1.0, 1.0, 1.0, 0], rtol=0, atol=1e-15)


def test_networkx_betweenness():
    nx = pytest.importorskip("networkx")
    g = gg.rmat_graph(8, edge_factor=4, seed=5)
    total = np.zeros(g.n)
    for s in range(g.n):
        total += oracle.bc(g, s)[0]
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    u = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    G.add_edges_from(zip(u.tolist(), g.col.tolist()))
    ref = nx.betweenness_centrality(G, normalized=False)
    # NetworkX counts each unordered pair once on undirected graphs
    assert np.allclose(total / 2, [ref[v] for v in range(g.n)], rtol=1e-9, atol=1e-9)
