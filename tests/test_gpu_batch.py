"""Batched persistent engine: every query's result equals the oracle's
(bit-exact BFS depths and SSSP distances) for all cluster sizes and
direction selectors; the level cap ends a run cleanly with GI_ERR_TIMEOUT."""
import ctypes
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from _graphs import adversarial, grid, rmat

pytestmark = pytest.mark.gpu
INT_MAX = np.iinfo(np.int32).max


def _graphs():
    return [rmat(12, weights=True), rmat(14, weights=True), grid(64, weights=True), adversarial("path", True),
            adversarial("components", True), adversarial("hub_tail", True)]


def _queries(hgs, n_q, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_q):
        gi_ = int(rng.integers(0, len(hgs)))
        src = int(rng.integers(0, hgs[gi_].n))
        out.append((gi_, src, "bfs" if i % 2 == 0 else "sssp"))
    return out


def _check(hgs, queries, results):
    for (gidx, src, algo), got in zip(queries, results):
        hg = hgs[gidx]
        got = got.cpu().numpy()
        if algo == "bfs":
            want, _, _ = oracle.bfs(hg, src)
        else:
            want, _ = oracle.sssp(hg, src)
        assert np.array_equal(got, want), (gidx, src, algo)


@pytest.mark.parametrize("cluster", [1, 2, 4, 8])
@pytest.mark.parametrize("selector", ["sparse_push", "hybrid_pull"])
def test_batch_matches_oracle(gi, cluster, selector):
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 48, seed=cluster)
    res, ns = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=cluster, selector=selector))
    _check(hgs, qs, res)
    assert (ns > 0).all()


@pytest.mark.parametrize("cluster", [0, 1, 4])
@pytest.mark.parametrize("selector", ["sparse_push", "hybrid_pull"])
def test_batch_bfs_parents(gi, cluster, selector):
    """BFS queries with a parent array get the canonical (smallest-id) parent
    of gi_bfs and the oracle, bit-exact; SSSP queries beside them are unchanged."""
    import torch
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 24, seed=20 + cluster)
    pars = [torch.empty(max(hgs[g_].n, 1), dtype=torch.int32, device="cuda") if a == "bfs" else None
            for g_, _, a in qs]
    res, _ = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=cluster, selector=selector), parents=pars)
    _check(hgs, qs, res)
    for (gidx, src, algo), par in zip(qs, pars):
        if algo == "bfs":
            assert np.array_equal(par[:hgs[gidx].n].cpu().numpy(), oracle.bfs(hgs[gidx], src)[1]), (gidx, src)


@pytest.mark.parametrize("tw,tc", [(1, 1), (8, 64), (32, 32), (16, 4096)])
def test_batch_bin_thresholds(gi, tw, tc):
    """Every expansion bin setting (thread / warp / CTA by degree) gives the oracle's results."""
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 32, seed=tw + tc)
    res, _ = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=2, t_warp=tw, t_cta=tc))
    _check(hgs, qs, res)


def test_batch_bin_thresholds_rejected(gi):
    hgs = _graphs()[:1]
    gs = [gi.Graph.from_host(h) for h in hgs]
    for tw, tc in ((33, 1024), (16, 8)):
        with pytest.raises(gi.GIError) as e:
            gi.batch_run(gs, [(0, 0, "bfs")], opts=gi.batch_opts(t_warp=tw, t_cta=tc))
        assert e.value.code == -1


def test_batch_autotune_returns_valid_faster_options(gi):
    """gi_batch_autotune: the best options found time no slower than the start
    and still give the oracle's results for every query."""
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 32, seed=77)
    best, best_ms, start_ms = gi.batch_autotune(gs, qs, start=gi.batch_opts(cluster_size=4), budget=8, seed=5)
    assert best_ms <= start_ms
    assert best.cluster_size in (1, 2, 4, 8) and 1 <= best.t_warp <= 32 and best.t_cta >= best.t_warp
    res, _ = gi.batch_run(gs, qs, opts=best)
    _check(hgs, qs, res)


def test_batch_fewer_clusters_than_queries(gi):
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 40, seed=11)
    res, _ = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=2, clusters=3))
    _check(hgs, qs, res)


WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_00923_gb300",
                       "selector_weights.npz")


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained selector weights committed")
def test_batch_learned_selector(gi):
    from paper_1805_00923_gb300 import selector as sel
    sel.install(WEIGHTS)
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 32, seed=5)
    res, _ = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=4, selector="learned"))
    _check(hgs, qs, res)


def test_batch_level_cap_returns_timeout(gi):
    hg = adversarial("path", True)
    g = gi.Graph.from_host(hg)
    with pytest.raises(gi.GIError) as e:
        gi.batch_run([g], [(0, 0, "bfs")], opts=gi.batch_opts(level_cap=10))
    assert e.value.code == -5
    # the context is still usable
    res, _ = gi.batch_run([g], [(0, 0, "bfs"), (0, 5, "sssp")])
    _check([hg], [(0, 0, "bfs"), (0, 5, "sssp")], res)


def test_batch_plan_graph_capture_replay(gi):
    """The plan's launch is captured in a CUDA graph and replayed; each replay
    recomputes every query (outputs are cleared in between)."""
    import torch
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 24, seed=21)
    plan = gi.BatchPlan(gs, qs, opts=gi.batch_opts(cluster_size=2))
    plan.launch()
    res, ns, lev = plan.results()
    _check(hgs, qs, res)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.launch()
    for _ in range(2):
        for o in plan.outs:
            o.fill_(12345)
        graph.replay()
        torch.cuda.synchronize()
        res, ns2, lev2 = plan.results()
        _check(hgs, qs, res)
        assert np.array_equal(lev, lev2)
    plan.free()


@pytest.mark.parametrize("delta", [-1.0, 0.5, 2.0, 20.0])
def test_batch_sssp_threshold_orders(gi, delta):
    """Any distance-threshold step (or none) gives the oracle's distances."""
    hgs = [grid(48, weights=True), rmat(12, weights=True), adversarial("hub_tail", True)]
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = [(k, s, "sssp") for k in range(3) for s in (0, 7, hgs[k].n - 1)]
    res, _ = gi.batch_run(gs, qs, opts=gi.batch_opts(cluster_size=2, sssp_delta=delta))
    _check(hgs, qs, res)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("selector", ["sparse_push", "hybrid_pull", "learned"])
def test_persistent_single_queries(gi, selector, mode):
    """BFS (depth + canonical parent) and SSSP in the whole-GPU persistent mode
    (1) and with the level loop as a CUDA graph (2; SSSP then runs host-driven)."""
    if selector == "learned":
        if not os.path.exists(WEIGHTS):
            pytest.skip("no trained selector weights committed")
        from paper_1805_00923_gb300 import selector as sel
        sel.install(WEIGHTS)
    for hg in [rmat(14, weights=True), grid(64, weights=True), adversarial("path", True),
               adversarial("components", True), adversarial("single", True)]:
        g = gi.Graph.from_host(hg)
        sc = gi.schedule(selector, persistent=mode)
        for src in sorted({0, hg.n // 3, hg.n - 1}):
            wd, wp, levels = oracle.bfs(hg, src)
            tr = gi.Trace(16)
            d, p = gi.bfs(g, src, sched=sc, trace=tr)
            assert np.array_equal(d.cpu().numpy(), wd) and np.array_equal(p.cpu().numpy(), wp)
            assert tr.iterations == len(levels)
            assert np.array_equal(gi.sssp(g, src, sched=sc).cpu().numpy(), oracle.sssp(hg, src)[0])


def test_grid_barrier_wait_runs_out(gi):
    """A barrier waiting for arrivals that never come gives up (~2 s) with
    GI_ERR_TIMEOUT; the context stays usable."""
    hg = rmat(10)
    g = gi.Graph.from_host(hg)
    lib = gi.lib()
    assert lib.gi_debug_barrier_phantoms(1) == 0
    try:
        with pytest.raises(gi.GIError) as e:
            gi.batch_run([g], [(0, 0, "bfs")], opts=gi.batch_opts(cluster_size=0))
        assert e.value.code == -5 and b"grid barrier" in lib.gi_last_error()
    finally:
        lib.gi_debug_barrier_phantoms(0)
    res, _ = gi.batch_run([g], [(0, 0, "bfs"), (0, 3, "bfs")], opts=gi.batch_opts(cluster_size=0))
    _check([hg], [(0, 0, "bfs"), (0, 3, "bfs")], res)


def test_graph_driven_bfs_cache_and_reuse(gi):
    """The cached graph is rebuilt when the schedule changes and reused across
    sources and output buffers; results stay the oracle's."""
    import torch
    hg = rmat(13)
    g = gi.Graph.from_host(hg)
    for k, sc in enumerate([gi.schedule("hybrid_pull", persistent=2), gi.schedule("hybrid_pull", persistent=2),
                            gi.schedule("sparse_push", persistent=2), gi.schedule("hybrid_pull", persistent=2,
                                                                                   alpha=4.0)]):
        for src in (0, 100 + k, hg.n - 1):
            out = (torch.full((hg.n,), 77, dtype=torch.int32, device="cuda"),
                   torch.full((hg.n,), 77, dtype=torch.int32, device="cuda"))
            tr = gi.Trace(8)
            d, p = gi.bfs(g, src, sched=sc, trace=tr, out=out)
            wd, wp, levels = oracle.bfs(hg, src)
            assert np.array_equal(d.cpu().numpy(), wd) and np.array_equal(p.cpu().numpy(), wp)
            assert tr.iterations == len(levels)


def test_graph_driven_bfs_directed_without_in_edges(gi):
    """Without in-edges the graph-driven loop pushes every level."""
    rng = np.random.default_rng(2)
    n = 2000
    e = rng.integers(0, n, (10_000, 2))
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False)
    d, _ = gi.bfs(g, 5, want_parent=False, sched=gi.schedule("hybrid_pull", persistent=2))
    want = oracle.bfs(hg, 5, in_edges=gg.transpose(hg)[:2])[0]
    assert np.array_equal(d.cpu().numpy(), want)


def test_graph_driven_bfs_follows_new_in_edges(gi):
    """gi_load_csc drops the cached graph (its kernels hold the in-edge arrays)."""
    rng = np.random.default_rng(6)
    n = 3000
    e = rng.integers(0, n, (12_000, 2))
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    ip, ic, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(ip, ic, None))
    sc = gi.schedule("dense_pull", persistent=2)
    want = oracle.bfs(hg, 1, in_edges=(ip, ic))[0]
    assert np.array_equal(gi.bfs(g, 1, want_parent=False, sched=sc)[0].cpu().numpy(), want)
    g.load_in_edges(ip.copy(), ic.copy())
    assert np.array_equal(gi.bfs(g, 1, want_parent=False, sched=sc)[0].cpu().numpy(), want)


def test_batch_claim_order_does_not_change_results(gi):
    """Largest-first and as-given claim orders give the same per-query results,
    the same BFS level counts (SSSP's asynchronous rounds vary with timing) and
    a time for every query."""
    hgs = _graphs()
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs = _queries(hgs, 40, seed=17)
    levels = {}
    for order in (0, 1):
        lv = np.zeros(len(qs), np.int32)
        opts = gi.batch_opts(cluster_size=2, order=order,
                             levels=lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        res, ns = gi.batch_run(gs, qs, opts=opts)
        _check(hgs, qs, res)
        assert (ns > 0).all()
        levels[order] = lv
    bfs = np.array([q[2] == "bfs" for q in qs])
    assert np.array_equal(levels[0][bfs], levels[1][bfs]) and (levels[1] > 0).all()
