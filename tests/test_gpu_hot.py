"""Hot-source DensePull (gi_schedule.hot_cache = 1: shared memory + L1, 2: L1 array).

The shared-memory source cache changes only where an arc's value is read, not
the tiles or the order of any reduction, so PageRank and PageRankDelta must
equal the plain tiled pull bit for bit, and the oracle within the fp32
tolerance.  Cases: every source hot (n <= 24,576), only the high-degree head
hot (R-MAT 18, 2-D grid with ties at the threshold degree), a hub row split
over tiles, a graph without arcs (no hot set), a directed graph with separate
in-edges, and every block tile size (mode 1 covers 512..2048 arcs and falls
back to the plain pull above; mode 2 covers 512..8192).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from _graphs import adversarial, grid, rmat

pytestmark = pytest.mark.gpu
PR_TOL = 1e-4
HOT_MAX = 24576


def _np(t):
    return t.cpu().numpy()


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30))) if a.size else 0.0


def _hot_info(gi, g):
    return g.hot_info()


CASES = {
    "rmat14_all_hot": lambda: rmat(14),
    "rmat18_head_hot": lambda: rmat(18),
    "grid300_ties": lambda: grid(300),
    "hub_tail_split_row": lambda: adversarial("hub_tail"),
    "star": lambda: adversarial("star"),
    "path": lambda: adversarial("path"),
    "isolated_no_arcs": lambda: adversarial("isolated"),
}


@pytest.mark.parametrize("name", list(CASES))
def test_hot_set_is_the_degree_head(gi, name):
    """k sources of out-degree >= min_deg, min_deg the smallest threshold with <= 24,576 sources."""
    hg = CASES[name]()
    g = gi.Graph.from_host(hg)
    k, d = _hot_info(gi, g)
    deg = np.diff(hg.row_ptr)
    if hg.m == 0:
        assert (k, d) == (0, 0)
        return
    assert 1 <= d and k == int(np.sum(deg >= d)) and k <= HOT_MAX
    if d > 1:
        assert int(np.sum(deg >= d - 1)) > HOT_MAX


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("te", [512, 1024, 2048, 4096])
@pytest.mark.parametrize("name", list(CASES))
def test_hot_pagerank_bit_identical(gi, name, te, mode):
    hg = CASES[name]()
    g = gi.Graph.from_host(hg)
    s0, s1 = gi.schedule("dense_pull", tile_edges=te), gi.schedule("dense_pull", tile_edges=te, hot_cache=mode)
    gi.pagerank(g, 0.85, 1, sched=s0)  # builds the tiles and the hot set, so the counts below are per run
    gi.pagerank(g, 0.85, 1, sched=s1)
    gi.stats_reset()
    plain = _np(gi.pagerank(g, 0.85, 20, sched=s0))
    n_plain = gi.stats_read()[0]
    gi.stats_reset()
    hot = _np(gi.pagerank(g, 0.85, 20, sched=s1))
    n_hot = gi.stats_read()[0]
    assert np.array_equal(plain.view(np.uint32), hot.view(np.uint32))
    assert _max_rel(hot, oracle.pagerank(hg, 0.85, 20)) < PR_TOL
    # the hot path adds one gather launch per iteration where it applies
    k, _ = g.hot_info()
    assert n_hot - n_plain == (20 if (k > 0 and (te <= 2048 or mode == 2)) else 0)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("te", [512, 2048])
@pytest.mark.parametrize("name", ["rmat14_all_hot", "rmat18_head_hot", "hub_tail_split_row", "grid300_ties"])
def test_hot_prdelta_bit_identical(gi, name, te, mode):
    hg = CASES[name]()
    g = gi.Graph.from_host(hg)
    tr0, tr1 = gi.Trace(16), gi.Trace(16)
    plain = _np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=gi.schedule("hybrid_pull", tile_edges=te), trace=tr0))
    hot = _np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=gi.schedule("hybrid_pull", tile_edges=te, hot_cache=mode),
                                trace=tr1))
    assert np.array_equal(plain.view(np.uint32), hot.view(np.uint32))
    assert np.array_equal(tr0.as_dict()["frontier"], tr1.as_dict()["frontier"])
    want, _ = oracle.prdelta(hg, 0.85, 1e-7, 10)
    assert _max_rel(hot, want) < PR_TOL


def test_hot_directed_graph_with_separate_in_edges(gi):
    rng = np.random.default_rng(12)
    n = 60_000
    src = np.concatenate([rng.integers(0, 50, 200_000), rng.integers(0, n, 300_000)])
    dst = rng.integers(0, n, src.size)
    hg = gg.from_edge_list(n, zip(src.tolist(), dst.tolist()), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None), validate=True)
    k, d = _hot_info(gi, g)
    assert 0 < k <= HOT_MAX
    plain = _np(gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull")))
    for mode in (1, 2):
        hot = _np(gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull", hot_cache=mode)))
        assert np.array_equal(plain.view(np.uint32), hot.view(np.uint32))
    assert _max_rel(hot, oracle.pagerank(hg, 0.85, 20, in_edges=(in_ptr, in_col))) < PR_TOL


def test_hot_set_rebuilt_after_new_in_edges(gi):
    """gi_load_csc replaces the in-edges: the hot set (derived from them) follows."""
    rng = np.random.default_rng(4)
    n = 5000
    e = rng.integers(0, n, (40_000, 2))
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None))
    first = _np(gi.pagerank(g, 0.85, 10, sched=gi.schedule("dense_pull", hot_cache=1)))
    g.load_in_edges(in_ptr, in_col)
    again = _np(gi.pagerank(g, 0.85, 10, sched=gi.schedule("dense_pull", hot_cache=1)))
    assert np.array_equal(first.view(np.uint32), again.view(np.uint32))
    assert _max_rel(again, oracle.pagerank(hg, 0.85, 10, in_edges=(in_ptr, in_col))) < PR_TOL


WEIGHTED = {
    "rmat14_all_hot": lambda: rmat(14, weights=True),
    "rmat18_head_hot": lambda: rmat(18, weights=True),
    "grid300_ties": lambda: grid(300, weights=True),
    "hub_tail_split_row": lambda: adversarial("hub_tail", weights=True),
}


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("name", list(WEIGHTED))
def test_hot_cc_sssp_exact(gi, name, mode):
    """Min-label pulls (CC, SSSP) read snap[u] of hot sources from the hot
    set (shared memory and L1 in mode 1, L1 in mode 2): labels, distances and
    per-round frontiers equal the oracle's."""
    hg = WEIGHTED[name]()
    g = gi.Graph.from_host(hg)
    for direction in ("dense_pull", "hybrid_pull"):
        sc = gi.schedule(direction, hot_cache=mode)
        want, fs = oracle.cc(hg)
        tr = gi.Trace(1 << 12)
        assert np.array_equal(_np(gi.cc(g, sched=sc, trace=tr)), want)
        assert np.array_equal(tr.as_dict()["frontier"], fs)
        src = int(gg.pick_sources(hg, 1, seed=3)[0])
        want, fs = oracle.sssp(hg, src)
        tr = gi.Trace(1 << 14)
        assert np.array_equal(_np(gi.sssp(g, src, sched=sc, trace=tr)), want)
        assert np.array_equal(tr.as_dict()["frontier"], fs)


LOAD_CASES = {
    "rmat14_all_hot": lambda: rmat(14),
    "rmat19_three_pieces": lambda: rmat(19),
    "grid300_ties_weighted": lambda: grid(300, weights=True),
    "hub_tail_split_row": lambda: adversarial("hub_tail"),
    "isolated_no_arcs": lambda: adversarial("isolated"),
}


@pytest.mark.parametrize("source", ["host", "pinned", "device"])
@pytest.mark.parametrize("validate", [False, True])
@pytest.mark.parametrize("name", list(LOAD_CASES))
def test_hot_set_built_during_load(gi, name, validate, source):
    """GI_HOT_SOURCES: the hot set remapped piece by piece while the indices
    arrive equals the one built on first use (same threshold and count, and
    the hot pulls give the plain pull's ranks bit for bit)."""
    import torch
    hg = LOAD_CASES[name]()
    wt = getattr(hg, "wt", None)
    arrs = [hg.row_ptr, hg.col] + ([wt] if wt is not None else [])
    if source == "pinned":
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy() for a in arrs]
    elif source == "device":
        arrs = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in arrs]
    g_load = gi.Graph(arrs[0], arrs[1], arrs[2] if wt is not None else None, symmetric=True, validate=validate,
                      hot_sources=True)
    g_lazy = gi.Graph.from_host(hg)
    assert g_load.hot_info() == g_lazy.hot_info()
    plain = _np(gi.pagerank(g_lazy, 0.85, 10, sched=gi.schedule("dense_pull")))
    for mode in (1, 2):
        for g in (g_load, g_lazy):
            hot = _np(gi.pagerank(g, 0.85, 10, sched=gi.schedule("dense_pull", hot_cache=mode)))
            assert np.array_equal(plain.view(np.uint32), hot.view(np.uint32))
    if wt is not None and hg.m:
        src = int(gg.pick_sources(hg, 1, seed=5)[0])
        want, _ = oracle.sssp(hg, src)
        assert np.array_equal(_np(gi.sssp(g_load, src, sched=gi.schedule("hybrid_pull", hot_cache=2))), want)
    g_load.free()
    g_lazy.free()


def test_hot_set_built_with_separate_in_edges(gi):
    """On a directed graph the flag acts on the call that loads the in-edges."""
    rng = np.random.default_rng(21)
    n = 70_000
    src = np.concatenate([rng.integers(0, 40, 300_000), rng.integers(0, n, 9_000_000)]).astype(np.int32)
    dst = rng.integers(0, n, src.size).astype(np.int32)
    row_ptr, col = gg.csr_from_edges(n, src, dst, False)
    hg = gg.HostGraph(n, row_ptr, col, None, False, "directed_two_pieces", {})
    in_ptr, in_col, _ = gg.transpose(hg)
    g_load = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None), hot_sources=True)
    g_lazy = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None))
    assert g_load.hot_info() == g_lazy.hot_info() and g_load.hot_info()[0] > 0
    plain = _np(gi.pagerank(g_lazy, 0.85, 20, sched=gi.schedule("dense_pull")))
    hot = _np(gi.pagerank(g_load, 0.85, 20, sched=gi.schedule("dense_pull", hot_cache=2)))
    assert np.array_equal(plain.view(np.uint32), hot.view(np.uint32))
    assert _max_rel(hot, oracle.pagerank(hg, 0.85, 20, in_edges=(in_ptr, in_col))) < PR_TOL
