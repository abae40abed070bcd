"""CUDA path vs the oracle, element by element, through the C ABI.

Integer outputs (BFS depth and parent, SSSP distance, CC label, per-round
frontier sizes, selected-edge probes) must be bit-exact; PageRank within 1e-4
max relative error of the FP64 oracle.  Each schedule is forced in turn, then
the hybrid rules.
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _graphs import ADVERSARIAL, adversarial, grid, rmat
from _prd_bound import FlipBound

pytestmark = pytest.mark.gpu

INT_MAX = np.iinfo(np.int32).max
DIRS = ["sparse_push", "dense_push", "dense_pull", "hybrid_pull", "hybrid_dpush"]
PR_TOL = 1e-4


def _load(gi, hg):
    return gi.Graph.from_host(hg, validate=True)


def _np(t):
    return t.cpu().numpy()


def _max_rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-30))) if a.size else 0.0


# ----------------------------------------------------------------------- BFS

@pytest.mark.parametrize("direction", DIRS)
@pytest.mark.parametrize("balance", ["edge_aware", "vertex", "edge_parallel"])
def test_bfs_rmat16_all_schedules(gi, direction, balance):
    hg = rmat(16)
    g = _load(gi, hg)
    for src in [0, *gg.pick_sources(hg, 3, seed=2)]:
        want_d, want_p, levels = oracle.bfs(hg, int(src))
        tr = gi.Trace(64)
        d, p = gi.bfs(g, int(src), sched=gi.schedule(direction, balance=balance), trace=tr)
        assert np.array_equal(_np(d), want_d)
        assert np.array_equal(_np(p), want_p)
        t = tr.as_dict()
        assert t["iterations"] == len(levels)
        assert np.array_equal(t["frontier"], levels)


@pytest.mark.parametrize("expand", ["block", "all_blocks"])
@pytest.mark.parametrize("name", ADVERSARIAL)
@pytest.mark.parametrize("direction", DIRS)
def test_bfs_adversarial(gi, name, direction, expand):
    """Sources of degree >= 256 are expanded by one block (t_heavy off) or
    split over all blocks (the default t_heavy)."""
    hg = adversarial(name)
    g = _load(gi, hg)
    kw = dict(t_cta=256, t_heavy=INT_MAX) if expand == "block" else {}
    for src in sorted({0, hg.n // 2, hg.n - 1}):
        want_d, want_p, _ = oracle.bfs(hg, src)
        d, p = gi.bfs(g, src, sched=gi.schedule(direction, **kw))
        assert np.array_equal(_np(d), want_d), (name, src)
        assert np.array_equal(_np(p), want_p), (name, src)


def test_bfs_grid_high_diameter(gi):
    hg = grid(96)
    g = _load(gi, hg)
    want_d, want_p, levels = oracle.bfs(hg, 5)
    for direction in ["sparse_push", "hybrid_pull"]:
        d, p = gi.bfs(g, 5, sched=gi.schedule(direction))
        assert np.array_equal(_np(d), want_d) and np.array_equal(_np(p), want_p)


def test_bfs_beamer_decisions_replayed_on_cpu(gi):
    """The hybrid's per-level choice equals Beamer's rule evaluated by the oracle."""
    hg = rmat(16)
    g = _load(gi, hg)
    src = 0
    depth, _, levels = oracle.bfs(hg, src)
    deg = hg.degrees().astype(np.int64)
    tr = gi.Trace(64)
    gi.bfs(g, src, sched=gi.schedule("hybrid_pull"), trace=tr)
    t = tr.as_dict()
    visited_deg = 0
    nu, mu = hg.n, int(deg.sum())
    was_pull = 0
    for lvl in range(len(levels)):
        front = depth == lvl
        nf, mf = int(front.sum()), int(deg[front].sum())
        nu, mu = nu - nf, mu - mf
        assert t["frontier"][lvl] == nf and t["edges"][lvl] == mf
        want = oracle.beamer(hg.n, nf, mf, mu, was_pull)
        got = 1 if t["direction"][lvl] == gi.GI_DIR_DENSE_PULL else 0
        assert got == want, lvl
        x = oracle.features(hg.n, hg.m, int(deg.max()), nf, mf, nu, mu, lvl, was_pull,
                            0 if lvl == 0 else int(levels[lvl - 1]))
        assert np.allclose(t["features"][lvl], x, rtol=2e-6, atol=1e-6), lvl
        was_pull = want
        visited_deg += mf


# ---------------------------------------------------------------------- SSSP

@pytest.mark.parametrize("balance", ["edge_aware", "edge_parallel"])
@pytest.mark.parametrize("direction", DIRS)
def test_sssp_rmat_all_schedules(gi, direction, balance):
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    for src in [0, *gg.pick_sources(hg, 2, seed=4)]:
        want, fs = oracle.sssp(hg, int(src))
        tr = gi.Trace(256)
        d = gi.sssp(g, int(src), sched=gi.schedule(direction, balance=balance), trace=tr)
        assert np.array_equal(_np(d), want)
        t = tr.as_dict()
        assert np.array_equal(t["frontier"], fs)   # synchronous rounds: same frontiers


@pytest.mark.parametrize("name", ["path", "components", "hub_tail", "single"])
@pytest.mark.parametrize("direction", ["sparse_push", "dense_pull", "dense_push"])
def test_sssp_adversarial(gi, name, direction):
    hg = adversarial(name, weights=True)
    g = _load(gi, hg)
    want, _ = oracle.sssp(hg, 0)
    assert np.array_equal(_np(gi.sssp(g, 0, sched=gi.schedule(direction))), want)
    # block-cooperative expansion instead of the all-block split
    assert np.array_equal(_np(gi.sssp(g, 0, sched=gi.schedule(direction, t_cta=256, t_heavy=INT_MAX))), want)
    # one thread per arc
    assert np.array_equal(_np(gi.sssp(g, 0, sched=gi.schedule(direction, balance="edge_parallel"))), want)


def test_sssp_grid(gi):
    hg = grid(64, weights=True)
    g = _load(gi, hg)
    want, fs = oracle.sssp(hg, 100)
    tr = gi.Trace(4096)
    d = gi.sssp(g, 100, sched=gi.schedule("hybrid_pull"), trace=tr)
    assert np.array_equal(_np(d), want)
    assert np.array_equal(tr.as_dict()["frontier"], fs)


# ------------------------------------------------------ SSSP, delta-stepping

DS_DIRS = ["sparse_push", "dense_pull", "dense_push", "hybrid_pull", "learned"]


@pytest.mark.parametrize("delta", [1, 7, 64, 333, 1 << 20])
@pytest.mark.parametrize("direction", DS_DIRS)
def test_sssp_delta_stepping_rmat(gi, direction, delta):
    """Delta-stepping (gi_schedule.delta) gives the oracle's distances for bucket
    widths from one weight unit (every arc heavy) to beyond the largest
    distance (every arc light, one bucket)."""
    from paper_1805_00923_gb300 import selector as sel
    sel.install()
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    for src in [0, *gg.pick_sources(hg, 2, seed=4)]:
        want, _ = oracle.sssp(hg, int(src))
        d = gi.sssp(g, int(src), sched=gi.schedule(direction, delta=delta))
        assert np.array_equal(_np(d), want), (src, delta)


@pytest.mark.parametrize("te", [256, 512, 2048, 8192])
@pytest.mark.parametrize("persistent", [0, 2])
def test_sssp_delta_stepping_pull_tile_sizes(gi, te, persistent):
    """The delta-stepping pulls over the row-compacted light / heavy views
    (block tiles: only the rows with arcs of the class) and over the full
    rows (warp tiles, 256 arcs), host- and graph-driven, forced DensePull and
    the hybrid rule, against the oracle; the R-MAT graph has isolated
    vertices and hubs whose rows are split over several tiles."""
    hg = rmat(16, weights=True)
    g = _load(gi, hg)
    for src in [0, *gg.pick_sources(hg, 2, seed=5)]:
        want, _ = oracle.sssp(hg, int(src))
        for direction in ("dense_pull", "hybrid_pull"):
            for delta in (64, 1 << 20):
                d = gi.sssp(g, int(src), sched=gi.schedule(direction, delta=delta, tile_edges=te,
                                                           persistent=persistent))
                assert np.array_equal(_np(d), want), (src, direction, delta)
    g.free()


@pytest.mark.parametrize("balance", ["edge_aware", "vertex", "edge_parallel"])
def test_sssp_delta_stepping_rounds_do_not_depend_on_direction(gi, balance):
    """Push and pull relax the same arcs of the same sources in every round
    (the light / heavy split is its own in-edge view on symmetric graphs), so
    the per-round source counts and arc counts agree across directions."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    src = int(gg.pick_sources(hg, 1, seed=9)[0])
    want, _ = oracle.sssp(hg, src)
    traces = []
    for direction in ["sparse_push", "dense_pull", "hybrid_pull"]:
        tr = gi.Trace(4096)
        d = gi.sssp(g, src, sched=gi.schedule(direction, delta=48, balance=balance), trace=tr)
        assert np.array_equal(_np(d), want)
        t = tr.as_dict()
        traces.append((t["frontier"], t["edges"]))
    for f, e in traces[1:]:
        assert np.array_equal(f, traces[0][0]) and np.array_equal(e, traces[0][1])
    # every arc of every reached vertex is relaxed at least once (light arcs in
    # its bucket's light rounds, heavy arcs once in the bucket's heavy round)
    deg = np.diff(hg.row_ptr)
    assert traces[0][1].sum() >= deg[want < INT_MAX].sum()


@pytest.mark.parametrize("name", ["path", "components", "hub_tail", "single", "isolated", "star"])
@pytest.mark.parametrize("direction", ["sparse_push", "dense_pull", "hybrid_pull"])
def test_sssp_delta_stepping_adversarial(gi, name, direction):
    hg = adversarial(name, weights=True)
    g = _load(gi, hg)
    want, _ = oracle.sssp(hg, 0)
    for delta in (1, 10, 100):
        assert np.array_equal(_np(gi.sssp(g, 0, sched=gi.schedule(direction, delta=delta))), want), delta
        assert np.array_equal(_np(gi.sssp(g, 0, sched=gi.schedule(direction, delta=delta,
                                                                    balance="edge_parallel"))), want), delta


def test_sssp_delta_stepping_grid_and_directed(gi):
    hg = grid(64, weights=True)
    g = _load(gi, hg)
    for delta in (3, 20, 250):
        assert np.array_equal(_np(gi.sssp(g, 100, sched=gi.schedule("hybrid_pull", delta=delta))),
                              oracle.sssp(hg, 100)[0])
    # a directed graph: delta-stepping pushes along the out-edges (pull needs a symmetric graph)
    hd = _directed(3000, 12000, 4, weights=True)
    in_ptr, in_col, in_wt = gg.transpose(hd)
    gd = gi.Graph(hd.row_ptr, hd.col, hd.wt, symmetric=False, in_edges=(in_ptr, in_col, in_wt), validate=True)
    for direction in ("sparse_push", "dense_pull", "hybrid_pull"):
        for src in (0, 1234):
            assert np.array_equal(_np(gi.sssp(gd, src, sched=gi.schedule(direction, delta=40))),
                                  oracle.sssp(hd, src)[0])


@pytest.mark.parametrize("delta", [0, 1, 48, 1 << 20])
@pytest.mark.parametrize("direction", ["sparse_push", "dense_pull", "hybrid_pull", "learned"])
def test_sssp_graph_driven(gi, direction, delta):
    """The graph-driven loop (persistent = 2) gives the oracle's distances, and
    runs the same rounds as the host-driven loop: Bellman-Ford's synchronous
    rounds for delta = 0, delta-stepping's otherwise."""
    from paper_1805_00923_gb300 import selector as sel
    sel.install()
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    for src in [0, *gg.pick_sources(hg, 2, seed=6)]:
        want, fs = oracle.sssp(hg, int(src))
        tg, th = gi.Trace(8), gi.Trace(8192)
        d = gi.sssp(g, int(src), sched=gi.schedule(direction, delta=delta, persistent=2), trace=tg)
        assert np.array_equal(_np(d), want), (src, delta)
        gi.sssp(g, int(src), sched=gi.schedule(direction, delta=delta), trace=th)
        assert tg.iterations == th.iterations
        if delta == 0:
            assert tg.iterations == len(fs)


@pytest.mark.parametrize("name", ["path", "components", "hub_tail", "single", "isolated", "star"])
def test_sssp_graph_driven_adversarial(gi, name):
    hg = adversarial(name, weights=True)
    g = _load(gi, hg)
    want, _ = oracle.sssp(hg, 0)
    for delta in (0, 1, 10):
        for direction in ("hybrid_pull", "sparse_push", "dense_pull"):
            d = gi.sssp(g, 0, sched=gi.schedule(direction, delta=delta, persistent=2))
            assert np.array_equal(_np(d), want), (delta, direction)


def test_sssp_graph_driven_grid_directed_and_reuse(gi):
    hg = grid(64, weights=True)
    g = _load(gi, hg)
    want = oracle.sssp(hg, 100)[0]
    for delta in (3, 0, 3, 250):  # the cached loop is rebuilt when the schedule changes
        assert np.array_equal(_np(gi.sssp(g, 100, sched=gi.schedule("hybrid_pull", delta=delta, persistent=2))), want)
    hd = _directed(3000, 12000, 4, weights=True)
    in_ptr, in_col, in_wt = gg.transpose(hd)
    gd = gi.Graph(hd.row_ptr, hd.col, hd.wt, symmetric=False, in_edges=(in_ptr, in_col, in_wt), validate=True)
    for delta in (0, 40):
        for src in (0, 1234):
            assert np.array_equal(_np(gi.sssp(gd, src, sched=gi.schedule("hybrid_pull", delta=delta, persistent=2))),
                                  oracle.sssp(hd, src)[0])


def test_sssp_delta_stepping_split_reused_and_rebuilt(gi):
    """The light/heavy split is cached per graph and delta: alternating deltas
    rebuilds it each time and keeps every result exact."""
    hg = rmat(12, weights=True)
    g = _load(gi, hg)
    want, _ = oracle.sssp(hg, 5)
    for delta in (16, 16, 200, 16, 0, 200):
        assert np.array_equal(_np(gi.sssp(g, 5, sched=gi.schedule("hybrid_pull", delta=delta))), want), delta


# ------------------------------------------------------------------------ CC

@pytest.mark.parametrize("balance", ["edge_aware", "edge_parallel"])
@pytest.mark.parametrize("direction", DIRS)
def test_cc_all_schedules(gi, direction, balance):
    for hg in [rmat(14), adversarial("components"), adversarial("path"), grid(40, shortcut_frac=0.0)]:
        g = _load(gi, hg)
        want, fs = oracle.cc(hg)
        tr = gi.Trace(4096)
        lab = gi.cc(g, sched=gi.schedule(direction, balance=balance), trace=tr)
        assert np.array_equal(_np(lab), want)
        assert np.array_equal(tr.as_dict()["frontier"], fs)


# ------------------------------------------------------------------ PageRank

@pytest.mark.parametrize("variant", ["pull", "pull_vertex", "push", "seg4", "tile256", "tile512", "tile8192"])
def test_pagerank_rmat16(gi, variant):
    hg = rmat(16)
    g = _load(gi, hg)
    sched = {"pull": gi.schedule("dense_pull"),
             "pull_vertex": gi.schedule("dense_pull", balance="vertex"),
             "push": gi.schedule("dense_push"),
             "seg4": gi.schedule("dense_pull", num_segments=4),
             "tile256": gi.schedule("dense_pull", tile_edges=256),
             "tile512": gi.schedule("dense_pull", tile_edges=512),
             "tile8192": gi.schedule("dense_pull", tile_edges=8192)}[variant]
    want = oracle.pagerank(hg, 0.85, 20)
    got = _np(gi.pagerank(g, 0.85, 20, sched=sched))
    assert _max_rel(got, want) < PR_TOL
    assert abs(float(np.sum(got.astype(np.float64))) - 1.0) < 1e-5


@pytest.mark.parametrize("name", ["single", "isolated", "star", "path", "hub_tail"])
def test_pagerank_adversarial(gi, name):
    hg = adversarial(name)
    g = _load(gi, hg)
    want = oracle.pagerank(hg, 0.85, 20)
    for d in ["dense_pull", "dense_push"]:
        assert _max_rel(_np(gi.pagerank(g, 0.85, 20, sched=gi.schedule(d))), want) < PR_TOL


def test_pagerank_zero_iterations_and_grid(gi):
    hg = grid(50)
    g = _load(gi, hg)
    assert _max_rel(_np(gi.pagerank(g, 0.85, 0)), oracle.pagerank(hg, 0.85, 0)) < 1e-6
    assert _max_rel(_np(gi.pagerank(g, 0.85, 20)), oracle.pagerank(hg, 0.85, 20)) < PR_TOL


# ------------------------------------------------------------- PageRankDelta

def _prd_explained(fb, got, tr):
    """Every vertex within 1e-4 of the oracle, or off by no more than the
    threshold flips of _prd_bound allow; every round's frontier size equal to
    the oracle's up to the flip-possible count of the round before."""
    t = tr.as_dict()
    # the driver stops once no vertex is active: the remaining rounds have |F| = 0
    front = np.zeros(len(fb.fs), np.int64)
    front[:len(t["frontier"])] = t["frontier"][:len(fb.fs)]
    bad_v, bad_r = fb.violations(got, front, PR_TOL)
    assert bad_v == [] and bad_r == [], (bad_v[:10], bad_r, fb.near_counts)


@pytest.mark.parametrize("direction", ["dense_pull", "sparse_push", "dense_push", "hybrid_pull"])
def test_prdelta_rmat16(gi, direction):
    hg = rmat(16)
    g = _load(gi, hg)
    fb = FlipBound(hg, 1e-7, 10)
    tr = gi.Trace(16)
    got = _np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=gi.schedule(direction), trace=tr))
    assert _max_rel(got, fb.rank) < PR_TOL
    _prd_explained(fb, got, tr)


@pytest.mark.parametrize("balance", ["edge_aware", "edge_parallel"])
@pytest.mark.parametrize("direction", ["dense_pull", "sparse_push", "hybrid_pull"])
def test_prdelta_sparse_rounds(gi, direction, balance):
    """eps = 1e-2 makes the active set shrink, exercising sparse rounds.  A
    vertex may differ from the oracle by more than 1e-4 only where a decision
    |Delta| > eps*Rank within rounding of its threshold can reach it (the
    per-round margins come from the oracle's history, _prd_bound)."""
    hg = rmat(14)
    g = _load(gi, hg)
    fb = FlipBound(hg, 1e-2, 10)
    tr = gi.Trace(16)
    got = _np(gi.pagerank_delta(g, 0.85, 1e-2, 10, sched=gi.schedule(direction, balance=balance), trace=tr))
    _prd_explained(fb, got, tr)
    assert fb.fs[-1] < fb.fs[0]


def test_prdelta_eps0_is_pagerank(gi):
    hg = rmat(12)
    g = _load(gi, hg)
    want = oracle.pagerank(hg, 0.85, 5, normalize=False)
    assert _max_rel(_np(gi.pagerank_delta(g, 0.85, 0.0, 5, sched=gi.schedule("dense_pull"))), want) < PR_TOL


# -------------------------------------------------------------- edgeset apply

def _mask_set(gi, g, mask):
    vs = gi.VertexSet(g)
    vs.import_ids(torch.from_numpy(np.flatnonzero(mask).astype(np.int32)).cuda())
    return vs


@pytest.mark.parametrize("balance", ["edge_aware", "edge_parallel"])
@pytest.mark.parametrize("direction", ["sparse_push", "dense_push", "dense_pull", "hybrid_pull", "sparse_pull"])
@pytest.mark.parametrize("dedup", [True, False])
def test_edgeset_apply_selection_probe(gi, direction, dedup, balance):
    """from/to selection and applyModified output equal the oracle's edge set
    (edge_parallel with a forced direction reads the frontier size back)."""
    hg = rmat(12)
    g = _load(gi, hg)
    rng = np.random.default_rng(11)
    for p_from, p_to in [(0.05, 1.0), (0.5, 0.3), (1.0, 1.0)]:
        fm = (rng.random(hg.n) < p_from).astype(np.uint8)
        tm = (rng.random(hg.n) < p_to).astype(np.uint8)
        u, v = oracle.edgeset_select(hg, fm, tm)
        cnt = np.bincount(v, minlength=hg.n)
        ssum = np.bincount(v, weights=u.astype(np.float64) + 1, minlength=hg.n).astype(np.uint64)
        F, T, OUT = _mask_set(gi, g, fm), _mask_set(gi, g, tm), gi.VertexSet(g)
        count = torch.zeros(hg.n, dtype=torch.int32, device="cuda")
        srcsum = torch.zeros(hg.n, dtype=torch.int64, device="cuda")
        args = gi.gi_probe_args(count.data_ptr(), srcsum.data_ptr())
        gi.edgeset_apply(g, F, T if p_to < 1 else None, gi.schedule(direction, balance=balance), gi.GI_K_PROBE,
                         args, OUT, flags=0 if dedup else gi.GI_NO_DEDUP)
        assert np.array_equal(_np(count), cnt)
        assert np.array_equal(_np(srcsum).astype(np.uint64), ssum)
        mod = _np(OUT.export())
        assert np.array_equal(mod, np.flatnonzero(cnt > 0))


def test_edgeset_apply_worked_example(gi):
    import json
    import os
    ex = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "gis_worked_example.json")))
    n = ex["n"]
    hg = gg.from_edge_list(n, map(tuple, ex["edges_directed"]), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col), validate=True)
    fm = np.zeros(n, np.uint8)
    fm[ex["frontier"]] = 1
    for direction in ["sparse_push", "dense_push", "dense_pull"]:
        count = torch.zeros(n, dtype=torch.int32, device="cuda")
        srcsum = torch.zeros(n, dtype=torch.int64, device="cuda")
        gi.edgeset_apply(g, _mask_set(gi, g, fm), None, gi.schedule(direction), gi.GI_K_PROBE,
                         gi.gi_probe_args(count.data_ptr(), srcsum.data_ptr()))
        got = sorted((int(s) - 1, v) for v in range(n) for s in ([_np(srcsum)[v]] if _np(count)[v] else []))
        assert got == sorted(map(tuple, ex["push_space"])), direction


# ----------------------------------------------------------------- vertexsets

def test_vertexset_roundtrip(gi):
    hg = rmat(12)
    g = _load(gi, hg)
    rng = np.random.default_rng(2)
    ids = np.unique(rng.integers(0, hg.n, 700)).astype(np.int32)
    vs = gi.VertexSet(g)
    vs.import_ids(torch.from_numpy(rng.permutation(np.r_[ids, ids[:50]]).astype(np.int32)).cuda())
    assert vs.size() == ids.size
    assert np.array_equal(_np(vs.export()), ids)
    vs.to_dense(gi.GI_REP_BOOL)
    vs.to_sparse()
    assert vs.reps() & gi.GI_REP_SPARSE
    assert np.array_equal(_np(vs.export()), ids)
    assert gi.VertexSet(g, gi.GI_VSET_ALL).size() == hg.n
    assert gi.VertexSet(g, gi.GI_VSET_EMPTY).size() == 0
    one = gi.VertexSet(g, gi.GI_VSET_SINGLE, 77)
    assert _np(one.export()).tolist() == [77]


def test_bad_graph_rejected(gi):
    hg = rmat(8)
    col = hg.col.copy()
    col[5] = hg.n + 3
    with pytest.raises(gi.GIError) as e:
        gi.Graph(hg.row_ptr, col, validate=True)
    assert e.value.code == -2


@pytest.mark.parametrize("te", [256, 512, 8192, "vertex"])
def test_pull_tile_sizes(gi, te):
    """Every tile shape (and the vertex-parallel pull) gives the oracle's results
    for min, sum and probe pulls."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    sc = gi.schedule("dense_pull", balance="vertex") if te == "vertex" else gi.schedule("dense_pull", tile_edges=te)
    te = 2048 if te == "vertex" else te
    want, fs = oracle.cc(hg)
    tr = gi.Trace(64)
    assert np.array_equal(_np(gi.cc(g, sched=sc, trace=tr)), want)
    assert np.array_equal(tr.as_dict()["frontier"], fs)
    want, _ = oracle.sssp(hg, 3)
    assert np.array_equal(_np(gi.sssp(g, 3, sched=sc)), want)
    want, _ = oracle.prdelta(hg, 0.85, 1e-7, 10)
    assert _max_rel(_np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=sc)), want) < PR_TOL
    hub = adversarial("hub_tail")
    gh = _load(gi, hub)
    assert _max_rel(_np(gi.pagerank(gh, 0.85, 20, sched=sc)), oracle.pagerank(hub, 0.85, 20)) < PR_TOL
    fm = (np.random.default_rng(te).random(hg.n) < 0.3).astype(np.uint8)
    u, v = oracle.edgeset_select(hg, fm)
    count = torch.zeros(hg.n, dtype=torch.int32, device="cuda")
    srcsum = torch.zeros(hg.n, dtype=torch.int64, device="cuda")
    OUT = gi.VertexSet(g)
    gi.edgeset_apply(g, _mask_set(gi, g, fm), None, sc, gi.GI_K_PROBE,
                     gi.gi_probe_args(count.data_ptr(), srcsum.data_ptr()), OUT)
    assert np.array_equal(_np(count), np.bincount(v, minlength=hg.n))
    assert np.array_equal(_np(OUT.export()), np.flatnonzero(np.bincount(v, minlength=hg.n) > 0))


# ----------------------------------------------------------------- autotuner

@pytest.mark.parametrize("block", [128, 512])
@pytest.mark.parametrize("direction", ["sparse_push", "hybrid_pull"])
def test_push_block_sizes(gi, direction, block):
    """SparsePush in 128- and 512-thread blocks (gi_schedule.block) keeps every result exact."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    for src in (0, 77):
        wd, wp, _ = oracle.bfs(hg, src)
        d, p = gi.bfs(g, src, sched=gi.schedule(direction, block=block))
        assert np.array_equal(_np(d), wd) and np.array_equal(_np(p), wp)
        assert np.array_equal(_np(gi.sssp(g, src, sched=gi.schedule(direction, block=block))), oracle.sssp(hg, src)[0])
        assert np.array_equal(_np(gi.sssp(g, src, sched=gi.schedule(direction, block=block, delta=40))),
                              oracle.sssp(hg, src)[0])
    assert np.array_equal(_np(gi.cc(g, sched=gi.schedule(direction, block=block))), oracle.cc(hg)[0])


def test_schedule_block_must_be_a_supported_size(gi):
    g = _load(gi, rmat(10))
    with pytest.raises(gi.GIError) as e:
        gi.bfs(g, 0, sched=gi.schedule("sparse_push", block=192))
    assert e.value.code == -1


@pytest.mark.parametrize("algo", ["bfs", "sssp", "cc", "pagerank", "pagerank_delta"])
def test_autotune_returns_valid_faster_schedule(gi, algo):
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    start = gi.schedule("dense_pull" if algo == "pagerank" else "hybrid_pull")
    best, best_ms, start_ms = gi.autotune(g, algo, src=0, start=start, budget=8, seed=3)
    assert best_ms <= start_ms
    assert best.direction == start.direction and best.balance == start.balance
    if algo == "bfs":
        d, p = gi.bfs(g, 0, sched=best)
        wd, wp, _ = oracle.bfs(hg, 0)
        assert np.array_equal(_np(d), wd) and np.array_equal(_np(p), wp)
    elif algo == "sssp":
        assert np.array_equal(_np(gi.sssp(g, 0, sched=best)), oracle.sssp(hg, 0)[0])
    elif algo == "cc":
        assert np.array_equal(_np(gi.cc(g, sched=best)), oracle.cc(hg)[0])
    elif algo == "pagerank":
        assert _max_rel(_np(gi.pagerank(g, 0.85, 20, sched=best)), oracle.pagerank(hg, 0.85, 20)) < PR_TOL
    else:
        assert _max_rel(_np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=best)),
                        oracle.prdelta(hg, 0.85, 1e-7, 10)[0]) < PR_TOL


# ------------------------------------------------------------ directed graphs

def _directed(n, ne, seed, weights=False):
    rng = np.random.default_rng(seed)
    e = rng.integers(0, n, (ne, 2))
    return gg.from_edge_list(n, map(tuple, e), symmetrize=False, weights=(seed, 1, 500) if weights else None)


@pytest.mark.parametrize("direction", ["sparse_push", "dense_push", "dense_pull", "hybrid_pull"])
def test_directed_graph_with_separate_in_edges(gi, direction):
    """Pull directions read the in-edges loaded by gi_load_csc; results still match."""
    hg = _directed(3000, 12000, 4, weights=True)
    in_ptr, in_col, in_wt = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, hg.wt, symmetric=False, in_edges=(in_ptr, in_col, in_wt), validate=True)
    sc = gi.schedule(direction)
    for src in (0, 1234):
        wd, wp, _ = oracle.bfs(hg, src, in_edges=(in_ptr, in_col))
        d, p = gi.bfs(g, src, sched=sc)
        assert np.array_equal(_np(d), wd) and np.array_equal(_np(p), wp)
        assert np.array_equal(_np(gi.sssp(g, src, sched=sc)), oracle.sssp(hg, src)[0])
    want = oracle.pagerank(hg, 0.85, 20, in_edges=(in_ptr, in_col))
    pr_dir = "dense_push" if direction in ("sparse_push", "dense_push") else "dense_pull"
    assert _max_rel(_np(gi.pagerank(g, 0.85, 20, sched=gi.schedule(pr_dir))), want) < PR_TOL


def test_directed_graph_without_in_edges_rejects_pull(gi):
    hg = _directed(100, 300, 5)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False)
    with pytest.raises(gi.GIError) as e:
        gi.bfs(g, 0, sched=gi.schedule("dense_pull"))
    assert e.value.code == -6
    d, _ = gi.bfs(g, 0, sched=gi.schedule("hybrid_pull"))   # hybrid falls back to push
    assert np.array_equal(_np(d), oracle.bfs(hg, 0, in_edges=gg.transpose(hg)[:2])[0])


@pytest.mark.parametrize("strategy", ["fvc", "evc"])
@pytest.mark.parametrize("segs", [2, 5])
def test_segmented_pull_all_algorithms(gi, segs, strategy):
    """Cache-partitioned (segmented) pull for PR, PRD, CC and SSSP matches the oracle."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    sc = gi.schedule("dense_pull", num_segments=segs, seg_strategy=strategy)
    assert _max_rel(_np(gi.pagerank(g, 0.85, 20, sched=sc)), oracle.pagerank(hg, 0.85, 20)) < PR_TOL
    want, _ = oracle.prdelta(hg, 0.85, 1e-7, 10)
    assert _max_rel(_np(gi.pagerank_delta(g, 0.85, 1e-7, 10, sched=sc)), want) < PR_TOL
    want, fs = oracle.cc(hg)
    tr = gi.Trace(64)
    assert np.array_equal(_np(gi.cc(g, sched=sc, trace=tr)), want)
    assert np.array_equal(tr.as_dict()["frontier"], fs)
    want, fs = oracle.sssp(hg, 9)
    tr = gi.Trace(256)
    assert np.array_equal(_np(gi.sssp(g, 9, sched=sc, trace=tr)), want)
    assert np.array_equal(tr.as_dict()["frontier"], fs)


@pytest.mark.parametrize("direction", ["dense_push", "dense_pull", "hybrid_pull"])
def test_boolean_map_frontier(gi, direction):
    """configApplyDenseVertexSet: dense traversals reading a boolean map instead of a bitvector."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    sc = gi.schedule(direction, dense_rep=gi.GI_REP_BOOL)
    wd, wp, _ = oracle.bfs(hg, 0)
    d, p = gi.bfs(g, 0, sched=sc)
    assert np.array_equal(_np(d), wd) and np.array_equal(_np(p), wp)
    assert np.array_equal(_np(gi.sssp(g, 4, sched=sc)), oracle.sssp(hg, 4)[0])
    assert np.array_equal(_np(gi.cc(g, sched=sc)), oracle.cc(hg)[0])
    fm = (np.random.default_rng(3).random(hg.n) < 0.2).astype(np.uint8)
    u, v = oracle.edgeset_select(hg, fm)
    count = torch.zeros(hg.n, dtype=torch.int32, device="cuda")
    srcsum = torch.zeros(hg.n, dtype=torch.int64, device="cuda")
    gi.edgeset_apply(g, _mask_set(gi, g, fm), None, sc, gi.GI_K_PROBE,
                     gi.gi_probe_args(count.data_ptr(), srcsum.data_ptr()))
    assert np.array_equal(_np(count), np.bincount(v, minlength=hg.n))


@pytest.mark.parametrize("strategy", ["fvc", "evc"])
def test_segment_bounds_and_arc_counts(gi, strategy):
    """Segments partition the sources; EVC cuts the out-degree prefix at s*m/S."""
    hg = rmat(16)
    g = _load(gi, hg)
    S = 8
    g.build_segments(S, strategy)
    st, b, arcs = g.segment_info()
    assert st == (0 if strategy == "fvc" else 1)
    assert b[0] == 0 and b[-1] == hg.n and (np.diff(b) >= 0).all()
    deg = np.diff(hg.row_ptr).astype(np.int64)
    want = np.array([deg[b[k]:b[k + 1]].sum() for k in range(S)])   # symmetric: in-arcs per source = out-degree
    assert np.array_equal(arcs, want) and arcs.sum() == hg.m
    if strategy == "fvc":
        size = -(-hg.n // S)
        assert np.array_equal(b[:-1], np.arange(S) * size)
    else:
        for k in range(1, S):
            assert hg.row_ptr[b[k]] >= hg.m * k // S and (b[k] == 0 or hg.row_ptr[b[k] - 1] < hg.m * k // S)
        assert arcs.max() <= hg.m // S + deg.max() + 1
    g.build_segments(1)
    assert g.segment_info()[1].tolist() == [0, hg.n]


@pytest.mark.parametrize("bal", ["edge_aware", "vertex"])
def test_sparse_pull_matches_dense_pull_with_to_set(gi, bal):
    """SparsePull (only the `to` destinations pull) computes what DensePull
    with the same `to` filter computes, for every edge function."""
    hg = rmat(13, weights=True)
    g = _load(gi, hg)
    rng = np.random.default_rng(21)
    fm = (rng.random(hg.n) < 0.2).astype(np.uint8)
    fm[7] = 1  # a hub of R-MAT
    tm = (rng.random(hg.n) < 0.05).astype(np.uint8)
    tm[np.argsort(np.diff(hg.row_ptr))[-3:]] = 1  # the highest in-degree rows: block-cooperative path
    F, T = _mask_set(gi, g, fm), _mask_set(gi, g, tm)
    u, v = oracle.edgeset_select(hg, fm, tm)
    snap_h = rng.integers(0, 1000, hg.n)
    results = {}
    for d in ("dense_pull", "sparse_pull"):
        sc = gi.schedule(d, balance=bal)
        # BFS step: unvisited = everything but a few; canonical parent = min frontier in-neighbour
        depth = torch.full((hg.n,), -1, dtype=torch.int32, device="cuda")
        depth[:50] = 0
        parent = torch.full((hg.n,), 2**31 - 1, dtype=torch.int32, device="cuda")
        OUT = gi.VertexSet(g)
        gi.edgeset_apply(g, F, T, sc, gi.GI_K_BFS, gi.gi_bfs_args(depth.data_ptr(), parent.data_ptr(), 1), OUT)
        # CC / SSSP min relaxations from snap
        snap = torch.tensor(snap_h, dtype=torch.int32, device="cuda")
        lab = torch.full((hg.n,), 500, dtype=torch.int32, device="cuda")
        gi.edgeset_apply(g, F, T, sc, gi.GI_K_CC, gi.gi_cc_args(lab.data_ptr(), snap.data_ptr()))
        dist = torch.full((hg.n,), 900, dtype=torch.int32, device="cuda")
        gi.edgeset_apply(g, F, T, sc, gi.GI_K_SSSP, gi.gi_sssp_args(dist.data_ptr(), snap.data_ptr()))
        contrib = torch.linspace(0.1, 1.0, hg.n, dtype=torch.float32, device="cuda")
        acc = torch.zeros(hg.n, dtype=torch.float32, device="cuda")
        gi.edgeset_apply(g, F, T, sc, gi.GI_K_SUM, gi.gi_sum_args(contrib.data_ptr(), acc.data_ptr()))
        results[d] = (_np(depth), _np(parent), _np(OUT.export()), _np(lab), _np(dist), _np(acc))
    a, b = results["dense_pull"], results["sparse_pull"]
    for k in range(5):
        assert np.array_equal(a[k], b[k]), k
    assert np.allclose(a[5], b[5], rtol=1e-5, atol=0)
    # and the sums are the oracle's selected edges
    want = np.bincount(v, weights=np.linspace(0.1, 1.0, hg.n, dtype=np.float32)[u].astype(np.float64),
                       minlength=hg.n)
    assert np.allclose(b[5], want, rtol=1e-5, atol=1e-6)
    # CC relaxation: the oracle's selected edges give the minimum snap per destination
    lab_want = np.full(hg.n, 500)
    np.minimum.at(lab_want, v, snap_h[u])
    assert np.array_equal(b[3], lab_want)


@pytest.mark.parametrize("direction", ["dense_pull", "hybrid_pull"])
def test_bfs_pull_deferred_long_rows(gi, direction):
    """Rows whose first 1,028 in-arcs hold no frontier source and that have
    more than 2,048 arcs left are finished by every block in 2,048-arc
    chunks.  A hub of 20,000 leaves is pulled with its only frontier source
    deep in the row, with frontier sources in two different chunks (the
    parent must be the lower id), and with none at all."""
    N = 20_000
    S = N + 1
    edges = [(0, i) for i in range(1, N + 1)] + [(S, 9_000), (S, 17_000)]
    hg = gg.from_edge_list(N + 2, edges)
    g = _load(gi, hg)
    # S: hits at positions 8,999 and 16,999 (two chunks); 15,000 and 1,500:
    # one deferred hit; 500: a hit inside the warp's own scan; 0: the hub
    for src in (S, 15_000, 1_500, 500, 0):
        want_d, want_p, _ = oracle.bfs(hg, src)
        d, p = gi.bfs(g, src, sched=gi.schedule(direction))
        assert np.array_equal(_np(d), want_d), src
        assert np.array_equal(_np(p), want_p), src


def test_bfs_pull_deferred_rows_directed_graph(gi):
    """Deferred long rows on a directed graph whose in-edges are loaded
    separately: hub H has in-arcs from 20,000 sources, and the BFS reaches two
    of them (9,000 and 17,000) one level before H."""
    N = 20_000
    H, S = N + 1, N + 2
    src = list(range(1, N + 1)) + [S, S]
    dst = [H] * N + [9_000, 17_000]
    row_ptr, col = gg.csr_from_edges(N + 3, np.array(src, np.int32), np.array(dst, np.int32), False)
    hg = gg.HostGraph(N + 3, row_ptr, col, None, False, "directed_hub", {})
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None))
    for direction in ("dense_pull", "hybrid_pull"):
        for s in (S, 12_345):
            want_d, want_p, _ = oracle.bfs(hg, s, in_edges=(in_ptr, in_col))
            d, p = gi.bfs(g, s, sched=gi.schedule(direction))
            assert np.array_equal(_np(d), want_d), (direction, s)
            assert np.array_equal(_np(p), want_p), (direction, s)


def _two_rmat_blobs_on_a_path():
    """Two R-MAT 12 components (each with its isolated vertices) joined by a
    30-vertex path, so that a BFS from the first pulls, pushes along the path
    and pulls again in the second: the compacted unvisited list is walked,
    goes stale over push levels and is walked again."""
    a = rmat(12)
    src = np.repeat(np.arange(a.n, dtype=np.int64), np.diff(a.row_ptr))
    e = np.stack([src, a.col.astype(np.int64)], 1)
    e = e[e[:, 0] < e[:, 1]]
    off = a.n + 30
    path = [(int(a.col[0]) if a.m else 0, a.n)] + [(a.n + i, a.n + i + 1) for i in range(29)]
    hub_b = off + int(np.argmax(np.diff(a.row_ptr)))
    path.append((a.n + 29, hub_b))
    pairs = np.concatenate([e, e + off, np.array(path, np.int64)])
    return gg.from_edge_list(off + a.n, map(tuple, pairs.tolist()))


@pytest.mark.parametrize("persistent", [0, 2])
@pytest.mark.parametrize("direction", ["dense_pull", "hybrid_pull", "learned"])
def test_bfs_unvisited_list(gi, direction, persistent):
    """DensePull levels over the compacted list of unvisited vertices with
    in-arcs (dst_list 1) and over every vertex (dst_list 0): identical depths
    and parents, equal to the oracle's, on R-MAT (isolated vertices), on two
    components joined by a path (pull, push, pull again) and on a grid."""
    graphs = [rmat(16), _two_rmat_blobs_on_a_path(), grid(64)]
    for hg in graphs:
        g = _load(gi, hg)
        for src in [0, *gg.pick_sources(hg, 2, seed=4)]:
            want_d, want_p, _ = oracle.bfs(hg, int(src))
            for dl in (1, 0):
                d, p = gi.bfs(g, int(src), sched=gi.schedule(direction, persistent=persistent, dst_list=dl))
                assert np.array_equal(_np(d), want_d), (hg.name, src, dl)
                assert np.array_equal(_np(p), want_p), (hg.name, src, dl)
        g.free()


def test_bfs_unvisited_list_survives_push_levels(gi):
    """The path graph's hybrid run really pulls, pushes, then pulls again."""
    hg = _two_rmat_blobs_on_a_path()
    g = _load(gi, hg)
    src = int(gg.pick_sources(hg, 1, seed=4)[0])
    tr = gi.Trace(256)
    gi.bfs(g, src, sched=gi.schedule("hybrid_pull"), trace=tr)
    dirs = tr.as_dict()["direction"].tolist()
    pulls = [i for i, x in enumerate(dirs) if x == gi.GI_DIR_DENSE_PULL]
    assert pulls and any(dirs[i] != gi.GI_DIR_DENSE_PULL for i in range(pulls[0], pulls[-1])), dirs


@pytest.mark.parametrize("name", ADVERSARIAL)
def test_bfs_unvisited_list_adversarial(gi, name):
    """No arcs at all (an empty live list), one vertex, a star, a path."""
    hg = adversarial(name)
    g = _load(gi, hg)
    for src in sorted({0, hg.n // 2, hg.n - 1}):
        want_d, want_p, _ = oracle.bfs(hg, src)
        for direction in ("dense_pull", "hybrid_pull"):
            for persistent in (0, 2):
                d, p = gi.bfs(g, src, sched=gi.schedule(direction, persistent=persistent))
                assert np.array_equal(_np(d), want_d), (name, src, direction, persistent)
                assert np.array_equal(_np(p), want_p), (name, src, direction, persistent)


def test_bfs_unvisited_list_directed_and_profile(gi):
    """A directed graph: the list holds the vertices with in-arcs (some have
    none, some have no out-arcs); and gi_selector_profile walks it too, with
    the same per-level features either way."""
    rng = np.random.default_rng(21)
    n = 6000
    e = rng.integers(0, n // 2, (30_000, 2))
    e[:, 1] += rng.integers(0, 2, e.shape[0]) * (n // 2)  # half the ids have no out-arcs, some no in-arcs
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None))
    for s_ in (0, 7, 2999):
        want_d, want_p, _ = oracle.bfs(hg, s_, in_edges=(in_ptr, in_col))
        for direction in ("dense_pull", "hybrid_pull"):
            for dl in (0, 1):
                d, p = gi.bfs(g, s_, sched=gi.schedule(direction, dst_list=dl))
                assert np.array_equal(_np(d), want_d), (s_, direction, dl)
                assert np.array_equal(_np(p), want_p), (s_, direction, dl)
    from paper_1805_00923_gb300 import selector as sel
    hs = rmat(14)
    gs = _load(gi, hs)
    f1, t1 = sel.profile(gs, gi.GI_K_BFS, 3, sched=gi.schedule("hybrid_pull", dst_list=1))
    f0, t0 = sel.profile(gs, gi.GI_K_BFS, 3, sched=gi.schedule("hybrid_pull", dst_list=0))
    assert f1.shape == f0.shape and np.array_equal(f1, f0)
    assert (t1[:, 2] > 0).all() and (t0[:, 2] > 0).all()
    # the run after the profile starts from a fresh list
    want_d, want_p, _ = oracle.bfs(hs, 3)
    d, p = gi.bfs(gs, 3, sched=gi.schedule("dense_pull"))
    assert np.array_equal(_np(d), want_d) and np.array_equal(_np(p), want_p)


def test_schedule_rejects_unknown_fields_and_bad_dst_list(gi):
    with pytest.raises(TypeError):
        gi.schedule("hybrid_pull", no_such_field=1)
    g = _load(gi, rmat(10))
    with pytest.raises(gi.GIError):
        gi.bfs(g, 0, sched=gi.schedule("hybrid_pull", dst_list=2))


@pytest.mark.parametrize("hub_in_to", [True, False])
def test_edgeset_apply_bfs_deferred_row_with_to_set(gi, hub_in_to):
    """The operator form of the early-exit pull: a hub whose frontier sources
    sit deep in its row is finished by the deferred scan only if the `to` set
    holds it; the parent is the smallest frontier source."""
    N = 20_000
    hg = gg.from_edge_list(N + 1, [(0, i) for i in range(1, N + 1)])
    g = _load(gi, hg)
    fm = np.zeros(hg.n, np.uint8)
    fm[[15_000, 17_500, 19_999]] = 1
    tm = np.zeros(hg.n, np.uint8)
    tm[[0, 3, 4]] = 1 if hub_in_to else 0
    tm[[3, 4]] = 1
    depth = torch.full((hg.n,), -1, dtype=torch.int32, device="cuda")
    depth[torch.from_numpy(np.flatnonzero(fm)).cuda()] = 0
    parent = torch.full((hg.n,), -1, dtype=torch.int32, device="cuda")
    OUT = gi.VertexSet(g)
    gi.edgeset_apply(g, _mask_set(gi, g, fm), _mask_set(gi, g, tm), gi.schedule("dense_pull"), gi.GI_K_BFS,
                     gi.gi_bfs_args(depth.data_ptr(), parent.data_ptr(), 1), OUT)
    d, p, out = _np(depth), _np(parent), np.sort(_np(OUT.export()))
    if hub_in_to:
        assert d[0] == 1 and p[0] == 15_000 and out.tolist() == [0]
    else:
        assert d[0] == -1 and out.size == 0
    assert d[3] == -1 and d[4] == -1  # leaves 3 and 4: their only in-neighbour (the hub) is not in F


def test_pull_arc_counter(gi):
    """gi_stats_pull_arcs: with timing on, a block-tiled PageRank pull gathers
    every arc once per iteration; a delta-stepping pull skips the long rows
    its bound filter rejects, so it gathers at most the class's arcs per
    round; with timing off nothing is counted."""
    hg = rmat(14, weights=True)
    g = _load(gi, hg)
    gi.stats_pull_arcs(g, reset=True)
    gi.pagerank(g, 0.85, 3, sched=gi.schedule("dense_pull", tile_edges=2048))
    assert gi.stats_pull_arcs(g) == 0  # timing off
    gi.stats_enable(True)
    try:
        gi.stats_pull_arcs(g, reset=True)
        gi.pagerank(g, 0.85, 3, sched=gi.schedule("dense_pull", tile_edges=2048))
        assert gi.stats_pull_arcs(g, reset=True) == 3 * hg.m
        tr = gi.Trace(1 << 12)
        d = gi.sssp(g, 0, sched=gi.schedule("dense_pull", delta=64), trace=tr)
        arcs = gi.stats_pull_arcs(g, reset=True)
        rounds = tr.as_dict()["iterations"]
        assert 0 < arcs <= rounds * hg.m
    finally:
        gi.stats_enable(False)
        gi.stats_reset()
    want, _ = oracle.sssp(hg, 0)
    assert np.array_equal(_np(d), want)


def test_prepare_then_queries(gi):
    """gi_prepare builds a schedule's per-graph set-up ahead of the queries
    (also from a second host thread while queries run on another graph); the
    queries then give the oracle's results."""
    import threading
    hg = rmat(15, weights=True)
    srcs = [int(s) for s in gg.pick_sources(hg, 3, seed=8)]
    want = {s: oracle.sssp(hg, s)[0] for s in srcs}
    want_b = {s: oracle.bfs(hg, s)[:2] for s in srcs}
    for sched in (gi.schedule("hybrid_pull", delta=64, persistent=2), gi.schedule("hybrid_pull", delta=64),
                  gi.schedule("learned", persistent=2)):
        g = _load(gi, hg)
        gi.prepare(g, "sssp", sched)
        gi.prepare(g, "bfs", sched)
        for s in srcs:
            assert np.array_equal(_np(gi.sssp(g, s, sched=sched)), want[s])
            d, p = gi.bfs(g, s, sched=sched)
            assert np.array_equal(_np(d), want_b[s][0]) and np.array_equal(_np(p), want_b[s][1])
        g.free()
    # a second graph loaded and prepared in another thread while the first one serves queries
    sched = gi.schedule("learned", delta=64, persistent=2)
    g1 = _load(gi, hg)
    box = {}

    def other():
        torch.cuda.set_device(0)
        st = torch.cuda.Stream()
        g2 = gi.Graph.from_host(hg, stream=st)
        gi.prepare(g2, "sssp", sched, stream=st)
        gi.prepare(g2, "bfs", sched, stream=st)
        box["g"] = g2

    th = threading.Thread(target=other)
    th.start()
    for s in srcs:
        assert np.array_equal(_np(gi.sssp(g1, s, sched=sched)), want[s])
    th.join()
    for s in srcs:
        assert np.array_equal(_np(gi.sssp(box["g"], s, sched=sched)), want[s])
    g1.free()
    box["g"].free()
    with pytest.raises(gi.GIError):
        gi.prepare(_load(gi, rmat(10)), "sssp", gi.schedule("hybrid_pull", delta=64))  # no weights
