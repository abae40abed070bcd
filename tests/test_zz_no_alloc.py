"""gi_pagerank_static: PageRank for callers that may not allocate GPU memory.

Some callers must not allocate device memory while they run (a fixed memory
budget reserved up front, or a host application whose allocator owns the
device heap), so they cannot use gi_load_csr/gi_pagerank.  This entry point
works on CSR arrays the caller already holds and keeps its working vectors in
a fixed device array inside the library.  Each case calls it twice in a row
through the C ABI and compares it with the FP64 oracle and with gi_pagerank
(1e-4 max relative error, the PageRank tolerance of the other tests), with the
library's allocation hook set to fail every allocation and the device pool
and torch's allocator checked to be unchanged.  This file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
from _graphs import rmat

pytestmark = pytest.mark.gpu

PR_TOL = 1e-4


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b) / np.abs(b)))


def _static_twice(gi, in_ptr, in_col, out_ptr, n, m, iters):
    """Two calls in a row with every library allocation set to fail; returns both results."""
    lib = gi.lib()
    in_ptr = torch.from_numpy(np.ascontiguousarray(in_ptr, np.int32)).cuda()
    in_col = torch.from_numpy(np.ascontiguousarray(in_col, np.int32)).cuda()
    out_ptr = None if out_ptr is None else torch.from_numpy(np.ascontiguousarray(out_ptr, np.int32)).cuda()
    outs = [torch.full((n,), -1.0, dtype=torch.float32, device="cuda") for _ in range(2)]
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # the first call on a device looks up the scratch array (set-up, before the checks)
    assert lib.gi_pagerank_static(ctypes.c_void_p(in_ptr.data_ptr()), ctypes.c_void_p(in_col.data_ptr()),
                                  None if out_ptr is None else ctypes.c_void_p(out_ptr.data_ptr()), n, m, 0.85,
                                  1, ctypes.c_void_p(outs[0].data_ptr()), stream) == 0, lib.gi_last_error()
    torch.cuda.synchronize()
    pool0, torch0 = ctypes.c_int64(), torch.cuda.memory_allocated()
    assert lib.gi_debug_pool_used(ctypes.byref(pool0)) == 0
    lib.gi_debug_fail_allocs_after(0)
    try:
        for out in outs:
            out.fill_(-1.0)
            rc = lib.gi_pagerank_static(ctypes.c_void_p(in_ptr.data_ptr()), ctypes.c_void_p(in_col.data_ptr()),
                                        None if out_ptr is None else ctypes.c_void_p(out_ptr.data_ptr()), n, m,
                                        0.85, iters, ctypes.c_void_p(out.data_ptr()), stream)
            assert rc == 0, lib.gi_last_error()
        torch.cuda.synchronize()
    finally:
        lib.gi_debug_fail_allocs_after(-1)
    pool1 = ctypes.c_int64()
    assert lib.gi_debug_pool_used(ctypes.byref(pool1)) == 0
    assert pool1.value == pool0.value and torch.cuda.memory_allocated() == torch0
    return [o.cpu().numpy() for o in outs]


def test_static_pagerank_symmetric_matches_oracle_and_library(gi):
    hg = rmat(16)
    want = oracle.pagerank(hg, 0.85, 20)
    g = gi.Graph.from_host(hg)
    lib_rank = gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull")).cpu().numpy()
    g.free()
    for got in _static_twice(gi, hg.row_ptr, hg.col, None, hg.n, hg.m, 20):
        assert _rel(got, want) < PR_TOL
        assert _rel(got, lib_rank) < PR_TOL


def test_static_pagerank_directed_with_out_offsets(gi):
    """A directed graph: in-edges from the transpose, out-degrees from the real out_offsets."""
    rng = np.random.default_rng(11)
    n = 5000
    e = rng.integers(0, n, (40_000, 2))
    hg = gg.from_edge_list(n, map(tuple, e), symmetrize=False)
    in_ptr, in_col, _ = gg.transpose(hg)
    want = oracle.pagerank(hg, 0.85, 20, in_edges=(in_ptr, in_col))
    g = gi.Graph(hg.row_ptr, hg.col, symmetric=False, in_edges=(in_ptr, in_col))
    lib_rank = gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull")).cpu().numpy()
    g.free()
    for got in _static_twice(gi, in_ptr, in_col, hg.row_ptr, hg.n, hg.m, 20):
        assert _rel(got, want) < PR_TOL
        assert _rel(got, lib_rank) < PR_TOL


def test_static_pagerank_at_the_vertex_limit(gi):
    """n = GI_STATIC_PR_MAX_N exactly (R-MAT scale 20 has 2^20 vertices)."""
    from paper_1805_00923_gb300 import _lib as L
    hg = rmat(20)
    assert hg.n == L.GI_STATIC_PR_MAX_N
    want = oracle.pagerank(hg, 0.85, 20)
    for got in _static_twice(gi, hg.row_ptr, hg.col, None, hg.n, hg.m, 20):
        assert _rel(got, want) < PR_TOL


def test_static_pagerank_zero_iterations(gi):
    hg = rmat(12)
    for got in _static_twice(gi, hg.row_ptr, hg.col, None, hg.n, hg.m, 0):
        assert _rel(got, np.full(hg.n, 1.0 / hg.n)) < 1e-6
        assert _rel(got, oracle.pagerank(hg, 0.85, 0)) < 1e-6


def test_static_pagerank_rejects_too_many_vertices(gi):
    lib = gi.lib()
    from paper_1805_00923_gb300 import _lib as L
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = lib.gi_pagerank_static(ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None,
                                L.GI_STATIC_PR_MAX_N + 1, 0, 0.85, 20, ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == L.GI_ERR_INVALID_ARG
    assert b"at most" in lib.gi_last_error()
