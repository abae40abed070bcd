"""GB300 edgeset-apply library (GraphIt's operators and schedules on sm_103a).

Thin Python binding of the C ABI in include/graphit_gb.h: every function here
marshals arguments (torch tensors for device memory, torch streams) and calls
the CUDA library; all graph work runs in its kernels.  Importing the package
loads (and if needed builds) libgraphit_gb.so and raises if that fails: there
is no CPU path.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib as L
from ._lib import (GI_BAL_EDGE_AWARE, GI_BAL_VERTEX, GI_DIR_DENSE_PULL, GI_DIR_DENSE_PUSH,  # noqa: F401
                   GI_DIR_HYBRID_DPUSH, GI_DIR_HYBRID_PULL, GI_DIR_LEARNED, GI_DIR_SPARSE_PUSH, GI_K_BFS,
                   GI_K_CC, GI_K_PROBE, GI_K_SSSP, GI_K_SUM, GI_NO_DEDUP, GI_REP_BITMAP, GI_REP_BOOL,
                   GI_REP_SPARSE, GI_RULE_BEAMER, GI_RULE_LIGRA, GI_VSET_ALL, GI_VSET_EMPTY, GI_VSET_SINGLE,
                   GIError, gi_batch_opts, gi_bfs_args, gi_cc_args, gi_probe_args, gi_schedule, gi_sssp_args, gi_sum_args,
                   gi_trace)

_C = L.load()
check = L.check


def lib():
    """The loaded ctypes library (functions named as in graphit_gb.h)."""
    return _C


def _vp(x) -> ctypes.c_void_p:
    if x is None:
        return ctypes.c_void_p(None)
    if isinstance(x, torch.Tensor):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def schedule(direction="hybrid_pull", **kw) -> gi_schedule:
    """A gi_schedule with the library defaults, overridden by keyword fields."""
    s = gi_schedule()
    _C.gi_schedule_default(ctypes.byref(s))
    if isinstance(direction, str):
        direction = L.DIRECTIONS[direction]
    s.direction = direction
    fields = {f for f, _ in gi_schedule._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise TypeError(f"gi_schedule has no field {k!r}")
        if k == "balance" and isinstance(v, str):
            v = {"vertex": GI_BAL_VERTEX, "edge_aware": GI_BAL_EDGE_AWARE, "edge_parallel": L.GI_BAL_EDGE_PARALLEL}[v]
        if k == "seg_strategy" and isinstance(v, str):
            v = {"fvc": L.GI_SEG_FVC, "evc": L.GI_SEG_EVC}[v]
        if k == "rule" and isinstance(v, str):
            v = {"beamer": GI_RULE_BEAMER, "ligra": GI_RULE_LIGRA}[v]
        setattr(s, k, v)
    return s


class Graph:
    """A graph loaded into the library (gi_load_csr / gi_load_csc).

    row_ptr/col/wt are host numpy arrays (copied host-to-device) or CUDA
    tensors (copied device-to-device), int32.  hot_sources=True builds the
    hot-source set of the on-chip pull during the load (GI_HOT_SOURCES).
    """

    def __init__(self, row_ptr, col, wt=None, symmetric=True, validate=False, in_edges=None, stream=None,
                 hot_sources=False):
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        if not on_dev:
            row_ptr = np.ascontiguousarray(row_ptr, np.int32)
            col = np.ascontiguousarray(col, np.int32)
            wt = None if wt is None else np.ascontiguousarray(wt, np.int32)
        self._keep = (row_ptr, col, wt)
        n = int(row_ptr.shape[0]) - 1
        m = int(col.shape[0])
        flags = (L.GI_DEV_PTRS if on_dev else L.GI_HOST_PTRS) | (L.GI_SYMMETRIC if symmetric else 0) | \
            (L.GI_VALIDATE if validate else 0) | (L.GI_HOT_SOURCES if hot_sources else 0)
        h = ctypes.c_void_p()
        check(_C.gi_load_csr(_vp(row_ptr), _vp(col), _vp(wt), n, m, flags, _stream(stream), ctypes.byref(h)))
        self.handle = h
        self._keep = None
        if in_edges is not None and not symmetric:
            self.load_in_edges(*(list(in_edges) + [None])[:3], validate=validate, stream=stream,
                               hot_sources=hot_sources)
        n_, m_, md = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        check(_C.gi_graph_info(h, ctypes.byref(n_), ctypes.byref(m_), ctypes.byref(md)))
        self.n, self.m, self.max_deg = n_.value, m_.value, md.value
        self.weighted = wt is not None

    @classmethod
    def from_host(cls, hg, validate=False, stream=None, in_edges=None, hot_sources=False):
        """From a graphgen.HostGraph-like object (n, row_ptr, col, wt, symmetric)."""
        return cls(hg.row_ptr, hg.col, getattr(hg, "wt", None), symmetric=getattr(hg, "symmetric", True),
                   validate=validate, in_edges=in_edges, stream=stream, hot_sources=hot_sources)

    def load_in_edges(self, in_ptr, in_col, in_wt=None, validate=False, stream=None, hot_sources=False):
        """gi_load_csc: attach (or replace) the in-edges of a non-symmetric graph."""
        on_dev = isinstance(in_ptr, torch.Tensor) and in_ptr.is_cuda
        if not on_dev:
            in_ptr, in_col = np.ascontiguousarray(in_ptr, np.int32), np.ascontiguousarray(in_col, np.int32)
            in_wt = None if in_wt is None else np.ascontiguousarray(in_wt, np.int32)
        check(_C.gi_load_csc(self.handle, _vp(in_ptr), _vp(in_col), _vp(in_wt),
                             (L.GI_DEV_PTRS if on_dev else L.GI_HOST_PTRS) | (L.GI_VALIDATE if validate else 0) |
                             (L.GI_HOT_SOURCES if hot_sources else 0),
                             _stream(stream)))

    def hot_info(self, stream=None):
        """gi_graph_hot_info: (k, min_deg) of the hot-source set of the shared-memory pull."""
        k, d = ctypes.c_int32(), ctypes.c_int32()
        check(_C.gi_graph_hot_info(self.handle, ctypes.byref(k), ctypes.byref(d), _stream(stream)))
        return k.value, d.value

    def build_segments(self, num_segments: int, strategy="fvc", stream=None):
        """gi_graph_build_segments; strategy "fvc" (equal source ranges) or "evc" (about m/S arcs each)."""
        st = {"fvc": L.GI_SEG_FVC, "evc": L.GI_SEG_EVC}.get(strategy, strategy)
        check(_C.gi_graph_build_segments(self.handle, int(num_segments), int(st), _stream(stream)))

    def segment_info(self):
        """(strategy, bounds[S+1], arcs[S]) of the current segments."""
        num, strat = ctypes.c_int32(), ctypes.c_int32()
        check(_C.gi_graph_segment_info(self.handle, ctypes.byref(num), ctypes.byref(strat), None, None, 0))
        b = np.zeros(num.value + 1, np.int32)
        a = np.zeros(num.value, np.int64)
        check(_C.gi_graph_segment_info(self.handle, None, None, _vp(b), _vp(a), num.value))
        return strat.value, b, a

    def free(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            check(_C.gi_graph_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class VertexSet:
    """A gi_vset (sparse queue / bool map / bitmap frontier)."""

    def __init__(self, g: Graph, init=GI_VSET_EMPTY, v: int = 0, stream=None):
        h = ctypes.c_void_p()
        check(_C.gi_vset_create(g.handle, int(init), int(v), _stream(stream), ctypes.byref(h)))
        self.handle, self.g = h, g

    def size(self, stream=None) -> int:
        out = ctypes.c_int64()
        check(_C.gi_vset_size(self.handle, ctypes.byref(out), _stream(stream)))
        return out.value

    def reps(self) -> int:
        out = ctypes.c_uint32()
        check(_C.gi_vset_reps(self.handle, ctypes.byref(out)))
        return out.value

    def to_sparse(self, stream=None):
        check(_C.gi_vset_to_sparse(self.handle, _stream(stream)))

    def to_dense(self, rep=GI_REP_BITMAP, stream=None):
        check(_C.gi_vset_to_dense(self.handle, int(rep), _stream(stream)))

    def export(self, stream=None) -> torch.Tensor:
        out = torch.empty(max(self.g.n, 1), dtype=torch.int32, device="cuda")
        cnt = ctypes.c_int64()
        check(_C.gi_vset_export(self.handle, _vp(out), out.numel(), ctypes.byref(cnt), _stream(stream)))
        return out[:cnt.value]

    def import_ids(self, ids: torch.Tensor, stream=None):
        ids = ids.to(device="cuda", dtype=torch.int32).contiguous()
        check(_C.gi_vset_import(self.handle, _vp(ids), ids.numel(), _stream(stream)))

    def free(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            check(_C.gi_vset_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Trace:
    """Host arrays for a gi_trace of up to `cap` iterations."""

    def __init__(self, cap: int = 4096):
        self.direction = np.zeros(cap, np.int32)
        self.frontier = np.zeros(cap, np.int64)
        self.edges = np.zeros(cap, np.int64)
        self.features = np.zeros((cap, 16), np.float32)
        self.phase = np.zeros(cap, np.int32)
        self.c = gi_trace(cap, 0, self.direction.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                          self.frontier.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          self.edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                          self.features.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                          self.phase.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))

    @property
    def iterations(self) -> int:
        return int(self.c.iterations)

    def as_dict(self):
        k = min(self.iterations, self.direction.shape[0])
        return dict(direction=self.direction[:k].copy(), frontier=self.frontier[:k].copy(),
                    edges=self.edges[:k].copy(), features=self.features[:k].copy(), phase=self.phase[:k].copy(),
                    iterations=self.iterations)


def _sched(s):
    return s if s is not None else schedule()


def _tr(trace):
    return ctypes.byref(trace.c) if trace is not None else None


def bfs(g: Graph, src: int, want_parent=True, sched=None, trace: Trace | None = None, stream=None, out=None):
    """gi_bfs: (depth, parent or None) as int32 CUDA tensors."""
    depth = out[0] if out else torch.empty(g.n, dtype=torch.int32, device="cuda")
    parent = (out[1] if out else torch.empty(g.n, dtype=torch.int32, device="cuda")) if want_parent else None
    check(_C.gi_bfs(g.handle, int(src), _vp(depth), _vp(parent), ctypes.byref(_sched(sched)), _tr(trace),
                    _stream(stream)))
    return depth, parent


def sssp(g: Graph, src: int, sched=None, trace: Trace | None = None, stream=None, out=None):
    dist = out if out is not None else torch.empty(g.n, dtype=torch.int32, device="cuda")
    check(_C.gi_sssp(g.handle, int(src), _vp(dist), ctypes.byref(_sched(sched)), _tr(trace), _stream(stream)))
    return dist


def cc(g: Graph, sched=None, trace: Trace | None = None, stream=None, out=None):
    label = out if out is not None else torch.empty(max(g.n, 1), dtype=torch.int32, device="cuda")
    check(_C.gi_cc(g.handle, _vp(label), ctypes.byref(_sched(sched)), _tr(trace), _stream(stream)))
    return label[:g.n]


def pagerank(g: Graph, damping=0.85, iters=20, sched=None, stream=None, out=None):
    rank = out if out is not None else torch.empty(max(g.n, 1), dtype=torch.float32, device="cuda")
    check(_C.gi_pagerank(g.handle, float(damping), int(iters), _vp(rank),
                         ctypes.byref(_sched(sched if sched is not None else schedule("dense_pull"))),
                         _stream(stream)))
    return rank[:g.n]


def pagerank_delta(g: Graph, damping=0.85, eps=1e-7, iters=10, sched=None, trace: Trace | None = None,
                   stream=None, out=None):
    rank = out if out is not None else torch.empty(max(g.n, 1), dtype=torch.float32, device="cuda")
    check(_C.gi_pagerank_delta(g.handle, float(damping), float(eps), int(iters), _vp(rank),
                               ctypes.byref(_sched(sched)), _tr(trace), _stream(stream)))
    return rank[:g.n]


def bc(g: Graph, src: int, sched=None, trace: Trace | None = None, stream=None, out=None, accumulate=False,
       want_sigma=False):
    """gi_bc: single-source betweenness dependencies (FP64 CUDA tensor), and
    the shortest-path counts if want_sigma.  With accumulate, adds into out."""
    dep = out if out is not None else torch.zeros(max(g.n, 1), dtype=torch.float64, device="cuda")
    sig = torch.empty(max(g.n, 1), dtype=torch.float64, device="cuda") if want_sigma else None
    check(_C.gi_bc(g.handle, int(src), _vp(dep), _vp(sig), int(bool(accumulate)), ctypes.byref(_sched(sched)),
                   _tr(trace), _stream(stream)))
    return (dep[:g.n], sig[:g.n]) if want_sigma else dep[:g.n]


def edgeset_apply(g: Graph, frm: VertexSet | None, to: VertexSet | None, sched, kernel_id: int, args,
                  out: VertexSet | None = None, flags: int = 0, stream=None):
    """gi_edgeset_apply: args is one of the gi_*_args ctypes structs."""
    check(_C.gi_edgeset_apply(g.handle, frm.handle if frm else None, to.handle if to else None,
                              ctypes.byref(_sched(sched)), int(kernel_id), ctypes.byref(args),
                              out.handle if out else None, int(flags), _stream(stream)))


def selector_load(params: np.ndarray, mean: np.ndarray, inv_std: np.ndarray):
    p = np.ascontiguousarray(params, np.float32)
    mu = np.ascontiguousarray(mean, np.float32)
    isd = np.ascontiguousarray(inv_std, np.float32)
    check(_C.gi_selector_load(_vp(p), int(p.size), _vp(mu), _vp(isd)))


def selector_num_params() -> int:
    return int(_C.gi_selector_num_params())


def stats_enable(timing: bool = True):
    check(_C.gi_stats_enable(1 if timing else 0))


def stats_reset():
    check(_C.gi_stats_reset())


def stats_read(kclass: int | str = -1):
    """(launches since reset, timed launches of kclass, their device ms)."""
    if isinstance(kclass, str):
        kclass = L.KCLASS[kclass]
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
    check(_C.gi_stats_read(int(kclass), ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def prepare(g: Graph, algo: str, sched=None, stream=None):
    """gi_prepare: build what `algo` ("bfs", "sssp", ...) run with `sched` needs on g, ahead of the queries."""
    check(_C.gi_prepare(g.handle, int(ALGOS[algo] if isinstance(algo, str) else algo), ctypes.byref(_sched(sched)),
                        _stream(stream)))


def stats_pull_arcs(g: Graph, reset: bool = False) -> int:
    """gi_stats_pull_arcs: arcs the block-tiled pulls on g gathered while timing was on."""
    a = ctypes.c_int64()
    check(_C.gi_stats_pull_arcs(g.handle, 1 if reset else 0, ctypes.byref(a)))
    return a.value


def gather_rate(idx: torch.Tensor, table: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """gi_gather_rate: launch the gather-ceiling kernel over idx (int32, CUDA) into table (float32, CUDA)."""
    out = out if out is not None else torch.zeros(1, dtype=torch.float32, device="cuda")
    check(_C.gi_gather_rate(_vp(idx), idx.numel(), _vp(table), table.numel(), _vp(out), _stream(stream)))
    return out


ALGOS = {"bfs": L.GI_ALGO_BFS, "sssp": L.GI_ALGO_SSSP, "cc": L.GI_ALGO_CC, "pagerank": L.GI_ALGO_PAGERANK,
         "pagerank_delta": L.GI_ALGO_PAGERANK_DELTA}


def autotune(g: Graph, algo, src: int = 0, start=None, budget: int = 30, seed: int = 1, stream=None):
    """gi_autotune: (best schedule, best ms, start ms)."""
    algo = ALGOS[algo] if isinstance(algo, str) else int(algo)
    best = gi_schedule()
    bms, sms = ctypes.c_double(), ctypes.c_double()
    st = start if start is not None else schedule()
    check(_C.gi_autotune(g.handle, algo, int(src), ctypes.byref(st), int(budget), int(seed), ctypes.byref(best),
                         ctypes.byref(bms), ctypes.byref(sms), _stream(stream)))
    return best, bms.value, sms.value


def schedule_dict(s: gi_schedule) -> dict:
    return {f: getattr(s, f) for f, _ in gi_schedule._fields_}


def batch_opts(**kw) -> gi_batch_opts:
    o = gi_batch_opts()
    _C.gi_batch_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "selector" and isinstance(v, str):
            v = L.DIRECTIONS[v]
        setattr(o, k, v)
    return o


def _with_parents(opts, parents, n_q):
    """A copy of opts whose parents field points at the device tensors in
    `parents` (one per query, None for no parents); returns (opts, keep-alive)."""
    o = gi_batch_opts()
    ctypes.pointer(o)[0] = opts if opts is not None else batch_opts()
    if parents is None:
        return o, None
    arr = (ctypes.c_void_p * max(n_q, 1))(*[None if p is None else p.data_ptr() for p in parents])
    o.parents = ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p))
    return o, arr


def batch_run(graphs, queries, outs=None, opts=None, stream=None, parents=None):
    """gi_batch_run.  queries: list of (graph index, source, "bfs"|"sssp").
    parents: optional list (one int32 CUDA tensor or None per query) that BFS
    queries fill with canonical parents.
    Returns (list of int32 CUDA result tensors, per-query ns as numpy int64)."""
    n_q = len(queries)
    qg = np.array([q[0] for q in queries], np.int32)
    qs = np.array([q[1] for q in queries], np.int32)
    qa = np.array([ALGOS[q[2]] if isinstance(q[2], str) else q[2] for q in queries], np.int32)
    if outs is None:
        outs = [torch.empty(max(graphs[q[0]].n, 1), dtype=torch.int32, device="cuda") for q in queries]
    handles = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    optr = (ctypes.c_void_p * max(n_q, 1))(*[o.data_ptr() for o in outs])
    ns = np.zeros(max(n_q, 1), np.int64)
    o, keep = _with_parents(opts, parents, n_q)
    check(_C.gi_batch_run(handles, len(graphs), _vp(qg), _vp(qs), _vp(qa), n_q, optr, _vp(ns), ctypes.byref(o),
                          _stream(stream)))
    del keep
    return [o_[:graphs[q[0]].n] for o_, q in zip(outs, queries)], ns[:n_q]


def batch_autotune(graphs, queries, start=None, budget: int = 12, seed: int = 1, stream=None):
    """gi_batch_autotune: (best gi_batch_opts, best ms, start ms) for the launch of these queries."""
    n_q = len(queries)
    qg = np.array([q[0] for q in queries], np.int32)
    qs = np.array([q[1] for q in queries], np.int32)
    qa = np.array([ALGOS[q[2]] if isinstance(q[2], str) else q[2] for q in queries], np.int32)
    handles = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
    best = gi_batch_opts()
    bms, sms = ctypes.c_double(), ctypes.c_double()
    check(_C.gi_batch_autotune(handles, len(graphs), _vp(qg), _vp(qs), _vp(qa), n_q,
                               ctypes.byref(start if start is not None else batch_opts()), int(budget), int(seed),
                               ctypes.byref(best), ctypes.byref(bms), ctypes.byref(sms), _stream(stream)))
    return best, bms.value, sms.value


class BatchPlan:
    """gi_batch_plan: the batched engine split into create / launch (capturable) / results."""

    def __init__(self, graphs, queries, opts=None, outs=None, stream=None, parents=None):
        n_q = len(queries)
        qg = np.array([q[0] for q in queries], np.int32)
        qs = np.array([q[1] for q in queries], np.int32)
        qa = np.array([ALGOS[q[2]] if isinstance(q[2], str) else q[2] for q in queries], np.int32)
        self.outs = outs if outs is not None else [torch.empty(max(graphs[q[0]].n, 1), dtype=torch.int32,
                                                               device="cuda") for q in queries]
        self.queries = queries
        self.graphs = graphs
        handles = (ctypes.c_void_p * len(graphs))(*[g.handle.value for g in graphs])
        optr = (ctypes.c_void_p * n_q)(*[o.data_ptr() for o in self.outs])
        h = ctypes.c_void_p()
        o, keep = _with_parents(opts, parents, n_q)
        check(_C.gi_batch_plan_create(handles, len(graphs), _vp(qg), _vp(qs), _vp(qa), n_q, optr, ctypes.byref(o),
                                      _stream(stream), ctypes.byref(h)))
        del keep
        self.parents = parents
        self.handle = h

    def launch(self, stream=None):
        check(_C.gi_batch_plan_launch(self.handle, _stream(stream)))

    def results(self, stream=None):
        n_q = len(self.queries)
        ns = np.zeros(n_q, np.int64)
        lev = np.zeros(n_q, np.int32)
        check(_C.gi_batch_plan_results(self.handle, _vp(ns), _vp(lev), _stream(stream)))
        return [o[:self.graphs[q[0]].n] for o, q in zip(self.outs, self.queries)], ns, lev

    def free(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            check(_C.gi_batch_plan_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
