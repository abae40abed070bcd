"""Parity at the full workload sizes, in the schedules bench.py times.

R-MAT scale 22 (4.19M vertices, 128M arcs): PageRank (20 iterations, DensePull),
PageRankDelta (eps 1e-7, 10 rounds, hybrid) and CC (hybrid) against the
oracle on every vertex.  R-MAT scale 24 (16.8M vertices, ~510M arcs, weights in
[1,1000)): BFS and SSSP from one sampled source, bit-exact against the oracle,
plus the per-arc invariants (|depth(u)-depth(v)| <= 1, dist(v) <= dist(u)+w).
R-MAT scale 22: Betweenness Centrality from one sampled source (path counts
exact, dependencies within 1e-9 relative).
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu
PR_TOL = 1e-4


@pytest.fixture(scope="module")
def rmat22():
    return gg.rmat_graph(22, seed=1)


@pytest.fixture(scope="module")
def rmat24():
    return gg.rmat_graph(24, seed=1, weights=(1, 1000))


def test_scale22_pagerank_prdelta_cc(gi, rmat22):
    hg = rmat22
    g = gi.Graph.from_host(hg)
    got = gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull")).cpu().numpy().astype(np.float64)
    want = oracle.pagerank(hg, 0.85, 20)
    assert np.max(np.abs(got - want) / want) < PR_TOL
    got = gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=gi.schedule("hybrid_pull")).cpu().numpy().astype(np.float64)
    want, _ = oracle.prdelta(hg, 0.85, 1e-7, 10)
    assert np.max(np.abs(got - want) / want) < PR_TOL
    tr = gi.Trace(64)
    lab = gi.cc(g, sched=gi.schedule("hybrid_pull"), trace=tr).cpu().numpy()
    want, fs = oracle.cc(hg)
    assert np.array_equal(lab, want)
    assert np.array_equal(tr.as_dict()["frontier"], fs)


def test_scale24_bfs_sssp_sampled_source(gi, rmat24):
    hg = rmat24
    g = gi.Graph.from_host(hg)
    src = int(gg.pick_sources(hg, 1, seed=24)[0])
    depth, parent = gi.bfs(g, src, sched=gi.schedule("hybrid_pull"))
    depth = depth.cpu().numpy()
    parent = parent.cpu().numpy()
    want_d, want_p, _ = oracle.bfs(hg, src)
    assert np.array_equal(depth, want_d) and np.array_equal(parent, want_p)
    u = np.repeat(np.arange(hg.n, dtype=np.int64), np.diff(hg.row_ptr))
    both = (depth[u] >= 0)
    assert (np.abs(depth[u][both] - depth[hg.col][both]) <= 1).all()
    dist = gi.sssp(g, src, sched=gi.schedule("hybrid_pull")).cpu().numpy()
    want, _ = oracle.sssp(hg, src)
    assert np.array_equal(dist, want)
    reach = dist[u] < np.iinfo(np.int32).max
    assert (dist[hg.col][reach].astype(np.int64) <= dist[u][reach].astype(np.int64) + hg.wt[reach]).all()


def test_scale22_bc_sampled_source(gi, rmat22):
    hg = rmat22
    g = gi.Graph.from_host(hg)
    src = int(gg.pick_sources(hg, 1, seed=22)[0])
    dep, sig = gi.bc(g, src, sched=gi.schedule("hybrid_pull"), want_sigma=True)
    want_d, want_s, _ = oracle.bc(hg, src)
    assert np.array_equal(sig.cpu().numpy(), want_s)
    dep = dep.cpu().numpy()
    assert np.array_equal(dep == 0, want_d == 0)
    assert np.allclose(dep, want_d, rtol=1e-9, atol=0)
    # sum of dependencies = sum over reached t of (d(s,t) - 1)
    depth = oracle.bfs(hg, src)[0]
    assert np.isclose(dep.sum(), float((depth[depth > 0] - 1).sum()), rtol=1e-9)
