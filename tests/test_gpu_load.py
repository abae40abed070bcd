"""Graph loading: the index copy on the side stream in pieces, the pooled
pinned control blocks and loads from several host threads.

Each load copies its indices (and weights) on one non-blocking stream per
device and records an event per piece; control blocks come from 64 KB
pinned slabs of 128 blocks kept for the process.  These tests load and free
more graphs than one slab holds, load graphs from two threads at once on
their own streams while a third thread runs traversals, and check every
graph against the oracle.
"""
import threading

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _graphs import grid, rmat

pytestmark = pytest.mark.gpu


def _np(t):
    return t.cpu().numpy()


def test_many_loads_reuse_pooled_control_blocks(gi):
    """300 live graphs (more than two slabs of control blocks), then freed and
    loaded again: every one answers BFS like the oracle."""
    hgs = [gg.rmat_graph(8, 8, seed=100 + i) for i in range(6)]
    want = [oracle.bfs(hg, 0)[0] for hg in hgs]
    for _ in range(2):
        gs = [gi.Graph.from_host(hgs[i % len(hgs)]) for i in range(300)]
        for i in range(0, 300, 37):
            d, _ = gi.bfs(gs[i], 0, want_parent=False)
            assert np.array_equal(_np(d), want[i % len(hgs)])
        for g in gs:
            g.free()


@pytest.mark.parametrize("hot", [False, True])
def test_loads_on_two_threads_beside_a_traversal(gi, hot):
    """Two threads load graphs on their own streams while the main thread runs
    PageRank on another graph; each thread's graphs equal the oracle's."""
    base = rmat(16)
    g0 = gi.Graph.from_host(base)
    pr_want = oracle.pagerank(base, 0.85, 20)
    cases = [rmat(14, weights=True), grid(200, weights=True)]
    want = [oracle.sssp(hg, 0)[0] for hg in cases]
    pinned = [(torch.from_numpy(hg.row_ptr).pin_memory(), torch.from_numpy(hg.col).pin_memory(),
               torch.from_numpy(hg.wt).pin_memory()) for hg in cases]
    errors, results = [], {}
    dev = torch.cuda.current_device()

    def worker(k):
        try:
            torch.cuda.set_device(dev)
            s = torch.cuda.Stream()
            rp, col, wt = pinned[k]
            out = []
            for _ in range(4):
                g = gi.Graph(rp.numpy(), col.numpy(), wt.numpy(), symmetric=True, stream=s, hot_sources=hot)
                with torch.cuda.stream(s):
                    dist = gi.sssp(g, 0, stream=s)
                s.synchronize()
                out.append(_np(dist))
                g.free()
            results[k] = out
        except Exception as e:  # reported in the main thread
            errors.append(e)

    ths = [threading.Thread(target=worker, args=(k,)) for k in range(2)]
    for t in ths:
        t.start()
    for _ in range(3):
        r = _np(gi.pagerank(g0, 0.85, 20))
        assert np.max(np.abs(r - pr_want) / np.maximum(np.abs(pr_want), 1e-30)) < 1e-4
    for t in ths:
        t.join()
    assert not errors, errors
    for k in range(2):
        assert len(results[k]) == 4
        for dist in results[k]:
            assert np.array_equal(dist, want[k])
    g0.free()
