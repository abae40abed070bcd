"""Failure paths, injected on the host: allocation failures at every step of a
graph load and of each driver return GI_ERR_OOM, leak no device memory, and
leave the library usable; malformed graphs are rejected."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from _graphs import rmat

pytestmark = pytest.mark.gpu


def _used(lib):
    b = ctypes.c_int64()
    assert lib.gi_debug_pool_used(ctypes.byref(b)) == 0
    return b.value


def test_allocation_failures_do_not_leak(gi):
    lib = gi.lib()
    hg = rmat(12, weights=True)
    torch.cuda.synchronize()
    base = _used(lib)
    seen_ok = False
    for k in range(0, 40):
        lib.gi_debug_fail_allocs_after(k)
        try:
            g = gi.Graph.from_host(hg)
        except gi.GIError as e:
            assert e.code == -3
            continue
        finally:
            lib.gi_debug_fail_allocs_after(-1)
        # the graph loaded; now make each driver fail part-way
        for run in (lambda: gi.bfs(g, 0), lambda: gi.sssp(g, 0), lambda: gi.cc(g),
                    lambda: gi.pagerank(g, 0.85, 3), lambda: gi.pagerank_delta(g, 0.85, 1e-7, 3)):
            for j in range(0, 6):
                lib.gi_debug_fail_allocs_after(j)
                try:
                    run()
                except gi.GIError as e:
                    assert e.code == -3
                finally:
                    lib.gi_debug_fail_allocs_after(-1)
        d, p = gi.bfs(g, 0)
        assert np.array_equal(d.cpu().numpy(), oracle.bfs(hg, 0)[0])
        g.free()
        seen_ok = True
        break
    assert seen_ok
    torch.cuda.synchronize()
    assert _used(lib) == base


def test_malformed_offsets_rejected(gi):
    hg = rmat(8)
    rp = hg.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3] + 1
    with pytest.raises(gi.GIError) as e:
        gi.Graph(rp, hg.col, validate=True)
    assert e.value.code in (-2,)
