"""ORACLE -- test infrastructure only.

ctypes wrapper around oracle.c: plain single-threaded CPU implementations of
the edgeset-apply path (selection, BFS, Bellman-Ford SSSP, label-propagation
CC, PageRank, PageRankDelta, single-source betweenness dependencies, frontier
statistics, the direction rules and the schedule-selector MLP).  Only tests/, the smoke check and the benchmark's CPU
baseline may import this package; the library under paper_1805_00923_gb300/
never does, and the two share no code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

D_IN, H, D_OUT = 16, 64, 3


def build(force: bool = False) -> str:
    """Compile oracle.c (gcc -O2, single-threaded, strict IEEE: no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)
_F64 = ctypes.POINTER(ctypes.c_double)
_i64, _i32, _f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "or_validate_csr": (ctypes.c_int, [_i64, _i64, _I32, _I32, ctypes.c_int]),
            "or_edgeset_select": (_i64, [_i64, _I32, _I32, _U8, _U8, _U8, _U8, _I32, _I32, _i64]),
            "or_bfs": (_i32, [_i64, _I32, _I32, _I32, _I32, _i32, _I32, _I32, _I64, _i32]),
            "or_sssp": (_i32, [_i64, _I32, _I32, _I32, _i32, _I32, _I64, _i32]),
            "or_cc": (_i32, [_i64, _I32, _I32, _I32, _I64, _i32]),
            "or_bc": (_i32, [_i64, _I32, _I32, _I32, _I32, _i32, _F64, _F64]),
            "or_pagerank": (None, [_i64, _I32, _I32, _I32, _f64, _i32, _i32, _F64]),
            "or_prdelta": (None, [_i64, _I32, _I32, _f64, _f64, _i32, _F64, _I64, _F64, _F64]),
            "or_frontier_stats": (None, [_i64, _I32, _U8, _U8, _I64]),
            "or_beamer": (_i32, [_i64, _i64, _i64, _i64, _i32, _f64, _f64]),
            "or_ligra_dense": (_i32, [_i64, _i64, _i64]),
            "or_mlp_num_params": (_i32, []),
            "or_mlp_forward": (None, [_F64, _F64, _i64, _F64]),
            "or_mlp_loss_grad": (_f64, [_F64, _F64, _F64, _F64, _i64, _F64]),
            "or_adam_step": (None, [_i64, _F64, _F64, _F64, _F64, _i32, _f64, _f64, _f64, _f64]),
            "or_features": (None, [_i64, _i64, _i64, _i64, _i64, _i64, _i64, _i32, _i32, _i64, _F64]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctype)


class _G:
    """Normalised CSR (+CSC) view of a graph-like object or tuple."""

    def __init__(self, g, in_edges=None):
        self.n = int(g.n)
        self.rp = _c(g.row_ptr, np.int32)
        self.ci = _c(g.col, np.int32)
        self.wt = _c(g.wt, np.int32) if getattr(g, "wt", None) is not None else None
        if in_edges is None:
            self.in_rp, self.in_ci = self.rp, self.ci
        else:
            self.in_rp, self.in_ci = _c(in_edges[0], np.int32), _c(in_edges[1], np.int32)

    @property
    def m(self):
        return int(self.ci.shape[0])


def validate_csr(g, require_symmetric=True) -> int:
    G = _G(g)
    return int(_load().or_validate_csr(G.n, G.m, _ptr(G.rp, _I32), _ptr(G.ci, _I32), int(require_symmetric)))


def edgeset_select(g, from_mask=None, to_mask=None, src_keep=None, dst_keep=None):
    """List of selected (u, v) in push order (Table 2 semantics)."""
    G = _G(g)
    masks = [None if x is None else _c(x, np.uint8) for x in (from_mask, to_mask, src_keep, dst_keep)]
    lib = _load()
    k = int(lib.or_edgeset_select(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32),
                                  *[_ptr(x, _U8) for x in masks], None, None, 0))
    ou = np.empty(max(k, 1), np.int32)
    ov = np.empty(max(k, 1), np.int32)
    lib.or_edgeset_select(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), *[_ptr(x, _U8) for x in masks],
                          _ptr(ou, _I32), _ptr(ov, _I32), k)
    return ou[:k], ov[:k]


def bfs(g, src: int, in_edges=None, level_cap: int = 1 << 16):
    """(depth, parent, level_sizes) with the canonical min-id parent rule."""
    G = _G(g, in_edges)
    depth = np.empty(G.n, np.int32)
    parent = np.empty(G.n, np.int32)
    ls = np.zeros(level_cap, np.int64)
    nl = int(_load().or_bfs(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), _ptr(G.in_rp, _I32), _ptr(G.in_ci, _I32),
                            int(src), _ptr(depth, _I32), _ptr(parent, _I32), _ptr(ls, _I64), level_cap))
    return depth, parent, ls[:nl].copy()


def sssp(g, src: int, round_cap: int = 1 << 16):
    """(dist, frontier_sizes) of synchronous frontier Bellman-Ford; INT32_MAX = unreachable."""
    G = _G(g)
    assert G.wt is not None, "sssp needs edge weights"
    dist = np.empty(G.n, np.int32)
    fs = np.zeros(round_cap, np.int64)
    r = int(_load().or_sssp(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), _ptr(G.wt, _I32), int(src),
                            _ptr(dist, _I32), _ptr(fs, _I64), round_cap))
    return dist, fs[:min(r, round_cap)].copy()


def cc(g, round_cap: int = 1 << 16):
    """(label, frontier_sizes) of synchronous min-label propagation."""
    G = _G(g)
    label = np.empty(G.n, np.int32)
    fs = np.zeros(round_cap, np.int64)
    r = int(_load().or_cc(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), _ptr(label, _I32), _ptr(fs, _I64), round_cap))
    return label, fs[:min(r, round_cap)].copy()


def bc(g, src: int, in_edges=None):
    """(delta, sigma, levels): Brandes' single-source dependencies and path counts."""
    G = _G(g, in_edges)
    delta = np.empty(G.n, np.float64)
    sigma = np.empty(G.n, np.float64)
    nl = int(_load().or_bc(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), _ptr(G.in_rp, _I32), _ptr(G.in_ci, _I32),
                           int(src), _ptr(delta, _F64), _ptr(sigma, _F64)))
    return delta, sigma, nl


def pagerank(g, damping=0.85, iters=20, normalize=True, in_edges=None):
    G = _G(g, in_edges)
    out_deg = np.diff(G.rp).astype(np.int32)
    rank = np.empty(G.n, np.float64)
    _load().or_pagerank(G.n, _ptr(G.in_rp, _I32), _ptr(G.in_ci, _I32), _ptr(out_deg, _I32), float(damping),
                        int(iters), int(normalize), _ptr(rank, _F64))
    return rank


def prdelta(g, damping=0.85, eps=1e-7, iters=10, history=False):
    """(rank, frontier_sizes) of PageRankDelta (Fig. 1 / Fig. 3).  With
    history=True also (delta_hist, rank_hist), each iters x n: Delta and Rank
    of every vertex at the end of each round."""
    G = _G(g)
    rank = np.empty(G.n, np.float64)
    fs = np.zeros(max(iters, 1), np.int64)
    dh = np.empty((max(iters, 1), G.n), np.float64) if history else None
    rh = np.empty((max(iters, 1), G.n), np.float64) if history else None
    _load().or_prdelta(G.n, _ptr(G.rp, _I32), _ptr(G.ci, _I32), float(damping), float(eps), int(iters),
                       _ptr(rank, _F64), _ptr(fs, _I64), _ptr(dh, _F64), _ptr(rh, _F64))
    if history:
        return rank, fs[:iters].copy(), dh[:iters], rh[:iters]
    return rank, fs[:iters].copy()


def frontier_stats(g, front_mask, visited_mask=None):
    G = _G(g)
    out = np.zeros(4, np.int64)
    f = _c(front_mask, np.uint8)
    vis = None if visited_mask is None else _c(visited_mask, np.uint8)
    _load().or_frontier_stats(G.n, _ptr(G.rp, _I32), _ptr(f, _U8), _ptr(vis, _U8), _ptr(out, _I64))
    return tuple(int(x) for x in out)


def beamer(n, nf, mf, mu, was_pull, alpha=14.0, beta=24.0) -> int:
    return int(_load().or_beamer(int(n), int(nf), int(mf), int(mu), int(was_pull), float(alpha), float(beta)))


def ligra_dense(m, nf, mf) -> int:
    return int(_load().or_ligra_dense(int(m), int(nf), int(mf)))


def mlp_num_params() -> int:
    return int(_load().or_mlp_num_params())


def mlp_forward(params, X):
    p = _c(params, np.float64)
    X = _c(X, np.float64).reshape(-1, D_IN)
    Y = np.empty((X.shape[0], D_OUT), np.float64)
    _load().or_mlp_forward(_ptr(p, _F64), _ptr(X, _F64), X.shape[0], _ptr(Y, _F64))
    return Y


def mlp_loss_grad(params, X, T, M):
    p = _c(params, np.float64)
    X = _c(X, np.float64).reshape(-1, D_IN)
    T = _c(T, np.float64).reshape(-1, D_OUT)
    M = _c(M, np.float64).reshape(-1, D_OUT)
    g = np.empty(p.shape[0], np.float64)
    loss = float(_load().or_mlp_loss_grad(_ptr(p, _F64), _ptr(X, _F64), _ptr(T, _F64), _ptr(M, _F64),
                                          X.shape[0], _ptr(g, _F64)))
    return loss, g


def adam_step(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """In-place Adam update of float64 arrays p, m, v."""
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    g = _c(g, np.float64)
    _load().or_adam_step(p.shape[0], _ptr(p, _F64), _ptr(g, _F64), _ptr(m, _F64), _ptr(v, _F64), int(t),
                         float(lr), float(b1), float(b2), float(eps))


def features(n, m, maxdeg, nf, mf, nu, mu, level, was_pull, nf_prev):
    x = np.empty(D_IN, np.float64)
    _load().or_features(int(n), int(m), int(maxdeg), int(nf), int(mf), int(nu), int(mu), int(level),
                        int(was_pull), int(nf_prev), _ptr(x, _F64))
    return x
