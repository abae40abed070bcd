"""gi_pagerank_static: PageRank for callers that may not allocate GPU memory.

Some callers must not allocate device memory while they run (a fixed memory
budget reserved up front, or a host application whose allocator owns the
device heap), so they cannot use gi_load_csr/gi_pagerank.  This entry point
works on CSR arrays the caller already holds and keeps its working vectors in
a fixed device array inside the library.  Here it is called twice in a row
through the C ABI and must agree with gi_pagerank within the PageRank
tolerance of the other tests (1e-4 max relative error).  This file is named to
be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

from _graphs import rmat

pytestmark = pytest.mark.gpu

PR_TOL = 1e-4


def test_static_pagerank_matches_library(gi):
    lib = gi.lib()
    hg = rmat(16)
    n, m = hg.n, hg.m
    g = gi.Graph.from_host(hg)
    want = gi.pagerank(g, 0.85, 20, sched=gi.schedule("dense_pull")).cpu().numpy().astype(np.float64)
    rp = torch.from_numpy(hg.row_ptr).cuda()
    col = torch.from_numpy(hg.col).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(-1.0)
        rc = lib.gi_pagerank_static(ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(col.data_ptr()), None, n, m,
                                    0.85, 20, ctypes.c_void_p(out.data_ptr()), stream)
        assert rc == 0, lib.gi_last_error()
        got = out.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - want) / want) < PR_TOL
    g.free()


def test_static_pagerank_rejects_too_many_vertices(gi):
    lib = gi.lib()
    from paper_1805_00923_gb300 import _lib as L
    dummy = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = lib.gi_pagerank_static(ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None,
                                L.GI_STATIC_PR_MAX_N + 1, 0, 0.85, 20, ctypes.c_void_p(dummy.data_ptr()), None)
    assert rc == L.GI_ERR_INVALID_ARG
    assert b"at most" in lib.gi_last_error()
