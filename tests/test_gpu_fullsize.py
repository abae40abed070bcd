"""Parity at the full workload sizes, in the schedules bench.py times.

R-MAT scale 22 (4.19M vertices, 128M arcs): PageRank (20 iterations, DensePull),
PageRankDelta (eps 1e-7, 10 rounds, hybrid) and CC (hybrid) against the
oracle on every vertex.  R-MAT scale 24 (16.8M vertices, ~521M arcs, weights in
[1,1000)), the BFS/SSSP configuration with 64 seeded sources: BFS depth and
parent and SSSP distance from every one of the 64 sources, bit-exact against
the oracle under each schedule the benchmark times (one test id per
schedule), plus the per-arc invariants (|depth(u)-depth(v)| <= 1,
dist(v) <= dist(u)+w) for one source.  The oracle runs on every host core
(one thread per source and algorithm: its C calls release the interpreter
lock) while the GPU works; its results are kept on the GPU for comparison.
R-MAT scale 22: Betweenness Centrality from one sampled source (path counts
exact, dependencies within 1e-9 relative).
"""
import concurrent.futures as cf
import os

import numpy as np
import pytest
import torch

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


L_SOURCES = 64   # the scale-24 BFS/SSSP configuration: 64 seeded sources (bench.py --workload rmat24_bfs_sssp)
BFS_SCHEDULES = {"hybrid_pull": dict(direction="hybrid_pull"), "learned": dict(direction="learned"),
                 "graph_driven": dict(direction="hybrid_pull", persistent=2),
                 "graph_driven_learned": dict(direction="learned", persistent=2)}
SSSP_SCHEDULES = {"hybrid_pull": dict(direction="hybrid_pull"), "learned": dict(direction="learned"),
                  "delta_hybrid": dict(direction="hybrid_pull", delta=64),
                  "delta_learned": dict(direction="learned", delta=64),
                  "graph_driven_delta_learned": dict(direction="learned", delta=64, persistent=2),
                  "graph_driven_bellman_ford": dict(direction="hybrid_pull", persistent=2)}


@pytest.fixture(scope="module")
def rmat24_expected(rmat24):
    """Oracle BFS (depth, parent) and SSSP distance for the 64 sources, on the GPU."""
    hg = rmat24
    srcs = [int(x) for x in gg.pick_sources(hg, L_SOURCES, seed=1)]
    oracle.build()
    out = {"sources": srcs, "bfs": {}, "sssp": {}}
    with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
        futs = {ex.submit(oracle.sssp, hg, s): ("sssp", s) for s in srcs}
        futs.update({ex.submit(oracle.bfs, hg, s): ("bfs", s) for s in srcs})
        for f in cf.as_completed(futs):
            kind, s = futs[f]
            r = f.result()
            if kind == "bfs":
                out["bfs"][s] = (torch.from_numpy(r[0]).cuda(), torch.from_numpy(r[1]).cuda())
            else:
                out["sssp"][s] = torch.from_numpy(r[0]).cuda()
    return out


@pytest.fixture(scope="module")
def g24(gi, rmat24):
    from paper_1805_00923_gb300 import selector as sel
    sel.install()
    g = gi.Graph.from_host(rmat24)
    yield g
    g.free()


@pytest.mark.parametrize("name", list(BFS_SCHEDULES))
def test_scale24_bfs_64_sources(gi, g24, rmat24_expected, name):
    sc = gi.schedule(**BFS_SCHEDULES[name])
    n = g24.n
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    bad = []
    for s in rmat24_expected["sources"]:
        gi.bfs(g24, s, sched=sc, out=(depth, parent))
        wd, wp = rmat24_expected["bfs"][s]
        if not (torch.equal(depth, wd) and torch.equal(parent, wp)):
            bad.append(s)
    assert bad == [], f"{len(bad)} of {L_SOURCES} sources differ, first {bad[:4]}"


@pytest.mark.parametrize("name", list(SSSP_SCHEDULES))
def test_scale24_sssp_64_sources(gi, g24, rmat24_expected, name):
    sc = gi.schedule(**SSSP_SCHEDULES[name])
    dist = torch.empty(g24.n, dtype=torch.int32, device="cuda")
    bad = []
    for s in rmat24_expected["sources"]:
        gi.sssp(g24, s, sched=sc, out=dist)
        if not torch.equal(dist, rmat24_expected["sssp"][s]):
            bad.append(s)
    assert bad == [], f"{len(bad)} of {L_SOURCES} sources differ, first {bad[:4]}"


def test_scale24_invariants_one_source(gi, g24, rmat24, rmat24_expected):
    hg = rmat24
    s = rmat24_expected["sources"][0]
    depth = rmat24_expected["bfs"][s][0].cpu().numpy()
    dist = rmat24_expected["sssp"][s].cpu().numpy()
    u = np.repeat(np.arange(hg.n, dtype=np.int64), np.diff(hg.row_ptr))
    both = (depth[u] >= 0)
    assert (np.abs(depth[u][both] - depth[hg.col][both]) <= 1).all()
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
