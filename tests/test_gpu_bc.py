"""Betweenness Centrality (gi_bc) against the oracle's Brandes dependencies.

Path counts sigma are sums of integers in FP64, exact below 2^53, so they must
equal the oracle's bit for bit.  Dependencies are FP64 sums whose order
differs from the oracle's (the GPU factors sigma[u] out of each level's sum):
each delta is a sum of at most max-degree positive terms per level, so over
L levels its relative error stays below about L * max_deg * 2^-53 (< 1e-9 at
the sizes tested); zeros (sources, leaves, unreached vertices) are exact.
"""
import os

import numpy as np
import pytest

import graphgen as gg
import oracle
from _graphs import ADVERSARIAL, adversarial, grid, rmat

pytestmark = pytest.mark.gpu
REL = 1e-9
IMAX = 2**31 - 1
WEIGHTS = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1805_00923_gb300",
                       "selector_weights.npz")


def _check(gi, g, hg, src, sched, in_edges=None):
    want_d, want_s, levels = oracle.bc(hg, src, in_edges=in_edges)
    tr = gi.Trace(1 << 12)
    dep, sig = gi.bc(g, src, sched=sched, trace=tr, want_sigma=True)
    dep, sig = dep.cpu().numpy(), sig.cpu().numpy()
    assert np.array_equal(sig, want_s), src
    assert np.array_equal(dep == 0, want_d == 0), src
    assert np.allclose(dep, want_d, rtol=REL, atol=0), (src, float(np.max(np.abs(dep - want_d) / np.maximum(want_d, 1e-300))))
    assert tr.iterations == levels
    return dep


def _sources(hg):
    return sorted({0, hg.n // 2, hg.n - 1, int(gg.pick_sources(hg, 1, seed=7)[0]) if hg.m else 0})


DIRS = ["sparse_push", "dense_push", "dense_pull", "hybrid_pull", "hybrid_dpush", "sparse_pull"]


@pytest.mark.parametrize("direction", DIRS)
@pytest.mark.parametrize("graph", ["rmat12", "rmat16", "grid64"])
def test_bc_matches_oracle(gi, graph, direction):
    hg = {"rmat12": lambda: rmat(12), "rmat16": lambda: rmat(16), "grid64": lambda: grid(64)}[graph]()
    g = gi.Graph.from_host(hg)
    for src in _sources(hg):
        _check(gi, g, hg, src, gi.schedule(direction))


@pytest.mark.parametrize("name", ADVERSARIAL)
def test_bc_adversarial(gi, name):
    hg = adversarial(name)
    g = gi.Graph.from_host(hg)
    for direction in ("sparse_push", "dense_pull", "hybrid_pull"):
        for src in _sources(hg):
            _check(gi, g, hg, src, gi.schedule(direction))


@pytest.mark.parametrize("balance", ["vertex", "block", "all_blocks", "edge_parallel"])
def test_bc_load_balance_modes(gi, balance):
    """Thread-per-vertex gathers, block-cooperative rows, all-block push split,
    one thread per arc."""
    hg = adversarial("hub_tail")
    g = gi.Graph.from_host(hg)
    kw = {"vertex": dict(balance="vertex"), "block": dict(t_cta=256, t_heavy=IMAX), "all_blocks": {},
          "edge_parallel": dict(balance="edge_parallel")}[balance]
    for direction in ("sparse_push", "hybrid_pull"):
        for src in (7, 0, 41_000):
            _check(gi, g, hg, src, gi.schedule(direction, **kw))


def test_bc_directed_graph(gi):
    rng = np.random.default_rng(8)
    n = 3000
    e = rng.integers(0, n, (15_000, 2))
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col, None))
    for direction in ("sparse_push", "dense_pull", "hybrid_pull"):
        for src in (0, 1500):
            _check(gi, g, hg, src, gi.schedule(direction), in_edges=(in_ptr, in_col))


def test_bc_accumulate_over_sources(gi):
    hg = rmat(11)
    g = gi.Graph.from_host(hg)
    srcs = [int(s) for s in gg.pick_sources(hg, 6, seed=3)]
    acc = None
    for s in srcs:
        acc = gi.bc(g, s, out=acc, accumulate=acc is not None)
    want = sum(oracle.bc(hg, s)[0] for s in srcs)
    assert np.allclose(acc.cpu().numpy(), want, rtol=REL, atol=0)


@pytest.mark.skipif(not os.path.exists(WEIGHTS), reason="no trained selector weights committed")
def test_bc_learned_selector(gi):
    from paper_1805_00923_gb300 import selector as sel
    sel.install(WEIGHTS)
    hg = rmat(14)
    g = gi.Graph.from_host(hg)
    for src in _sources(hg):
        _check(gi, g, hg, src, gi.schedule("learned"))


def test_bc_tile_sizes(gi):
    hg = rmat(14)
    g = gi.Graph.from_host(hg)
    for te in (256, 512, 8192):
        _check(gi, g, hg, 3, gi.schedule("dense_pull", tile_edges=te))
