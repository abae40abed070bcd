"""Seeded input generators: determinism, CSR structure, grid shape, weights."""
import numpy as np
import pytest

import graphgen as gg
import oracle


def _brute_csr(n, src, dst, symmetrize):
    pairs = set()
    for s, t in zip(src.tolist(), dst.tolist()):
        if s == t:
            continue
        pairs.add((s, t))
        if symmetrize:
            pairs.add((t, s))
    pairs = sorted(pairs)
    rp = np.zeros(n + 1, np.int64)
    for s, _ in pairs:
        rp[s + 1] += 1
    return np.cumsum(rp).astype(np.int32), np.array([t for _, t in pairs], np.int32)


@pytest.mark.parametrize("sym", [True, False])
def test_csr_matches_brute_force(sym):
    rng = np.random.default_rng(7)
    n = 40
    src = rng.integers(0, n, 300).astype(np.int32)
    dst = rng.integers(0, n, 300).astype(np.int32)
    rp, col = gg.csr_from_edges(n, src, dst, sym)
    brp, bcol = _brute_csr(n, src, dst, sym)
    assert np.array_equal(rp, brp) and np.array_equal(col, bcol)


def test_csr_rejects_bad_ids():
    with pytest.raises(RuntimeError):
        gg.csr_from_edges(4, np.array([0, 5], np.int32), np.array([1, 2], np.int32))


def test_rmat_deterministic_and_valid():
    g1 = gg.rmat_graph(12, seed=3)
    g2 = gg.rmat_graph(12, seed=3)
    g3 = gg.rmat_graph(12, seed=4)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col, g2.col)
    assert not (g1.m == g3.m and np.array_equal(g1.col, g3.col))
    assert oracle.validate_csr(g1, require_symmetric=True) == 0
    assert int(g1.degrees().sum()) == g1.m
    # vertex 0 is the hub when there is no relabelling
    assert int(np.argmax(g1.degrees())) == 0


def test_rmat_quadrant_probabilities():
    scale, ne = 8, 200000
    src, dst = gg.rmat_edges(scale, ne, 0.57, 0.19, 0.19, seed=11)
    top = 1 << (scale - 1)
    s1, t1 = (src & top) != 0, (dst & top) != 0
    frac = {"a": np.mean(~s1 & ~t1), "b": np.mean(~s1 & t1), "c": np.mean(s1 & ~t1), "d": np.mean(s1 & t1)}
    for k, p in {"a": 0.57, "b": 0.19, "c": 0.19, "d": 0.05}.items():
        assert abs(frac[k] - p) < 0.01, (k, frac[k])


def test_grid_structure_without_shortcuts():
    side = 9
    g = gg.grid_graph(side, shortcut_frac=0.0)
    assert g.m == 2 * 2 * side * (side - 1)
    deg = g.degrees().reshape(side, side)
    assert deg[0, 0] == 2 and deg[0, side - 1] == 2 and deg[side - 1, 0] == 2
    assert deg[0, 4] == 3 and deg[4, 0] == 3
    assert (deg[1:-1, 1:-1] == 4).all()
    assert oracle.validate_csr(g) == 0


def test_grid_shortcuts_are_local():
    side = 64
    g = gg.grid_graph(side, shortcut_frac=0.05, max_l1=8, seed=5)
    u = np.repeat(np.arange(g.n), g.degrees())
    v = g.col
    l1 = np.abs(u % side - v % side) + np.abs(u // side - v // side)
    assert l1.min() >= 1 and l1.max() <= 8
    n_short_arcs = int((l1 >= 2).sum())
    assert 0 < n_short_arcs <= 2 * int(0.05 * 2 * side * (side - 1))
    assert oracle.validate_csr(g) == 0


def test_weights_symmetric_and_in_range():
    g = gg.rmat_graph(10, weights=(1, 1000))
    assert g.wt.min() >= 1 and g.wt.max() < 1000
    u = np.repeat(np.arange(g.n), g.degrees())
    w = {(int(a), int(b)): int(c) for a, b, c in zip(u, g.col, g.wt)}
    assert all(w[(b, a)] == c for (a, b), c in w.items())


def test_sources_have_degree():
    g = gg.rmat_graph(10)
    s = gg.pick_sources(g, 64, seed=1)
    assert (g.degrees()[s] >= 1).all()
    assert np.array_equal(s, gg.pick_sources(g, 64, seed=1))
