"""Seeded synthetic graph inputs (R-MAT, grids with local shortcuts, CSR assembly).

This module is shared by the oracle tests and the GPU path and holds no part of
the traversal method: it only produces CSR inputs, edge weights and sources.
The C code (graphgen.c) is compiled on first use with gcc (OpenMP); results do
not depend on the thread count.

Workload shapes follow the paper's evaluation graphs (Sec. 7, Table 6): R-MAT
graphs stand in for the social/web graphs (power-law, low diameter) and 2-D
grids with local shortcuts for the road graph (high diameter, degree ~4).
Undirected graphs are stored with both arcs, as the paper counts them (Sec. 7).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into a shared library (gcc, -O2, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i32p = ctypes.POINTER(ctypes.c_int32)
        lib.gg_splitmix64.restype = ctypes.c_uint64
        lib.gg_splitmix64.argtypes = [ctypes.c_uint64]
        lib.gg_rmat_edges.restype = None
        lib.gg_rmat_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, i32p, i32p]
        lib.gg_grid_base_edges.restype = ctypes.c_int64
        lib.gg_grid_base_edges.argtypes = [ctypes.c_int32]
        lib.gg_grid_edges.restype = ctypes.c_int64
        lib.gg_grid_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64,
                                      i32p, i32p]
        lib.gg_csr_from_edges.restype = ctypes.c_int64
        lib.gg_csr_from_edges.argtypes = [ctypes.c_int64, ctypes.c_int64, i32p, i32p, ctypes.c_int32,
                                          i32p, i32p, ctypes.c_int64]
        lib.gg_pair_weights.restype = None
        lib.gg_pair_weights.argtypes = [ctypes.c_int64, i32p, i32p, ctypes.c_uint64, ctypes.c_int32,
                                        ctypes.c_int32, i32p]
        lib.gg_pick_sources.restype = ctypes.c_int32
        lib.gg_pick_sources.argtypes = [ctypes.c_int64, i32p, ctypes.c_uint64, ctypes.c_int32, i32p]
        _lib = lib
        return lib


def _p(a: np.ndarray):
    assert a.dtype == np.int32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def splitmix64(x: int) -> int:
    return int(_load().gg_splitmix64(ctypes.c_uint64(x & (2**64 - 1))))


@dataclass
class HostGraph:
    """CSR arrays on the host.  For the symmetric inputs here CSC == CSR."""
    n: int
    row_ptr: np.ndarray          # int32[n+1]
    col: np.ndarray              # int32[m]
    wt: np.ndarray | None = None  # int32[m] or None
    symmetric: bool = True
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(self.col.shape[0])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int32)


def rmat_edges(scale: int, n_edges: int, a=0.57, b=0.19, c=0.19, seed=1):
    src = np.empty(n_edges, np.int32)
    dst = np.empty(n_edges, np.int32)
    _load().gg_rmat_edges(scale, n_edges, a, b, c, seed, _p(src), _p(dst))
    return src, dst


def grid_edges(side: int, shortcut_frac=0.01, max_l1=8, seed=1):
    lib = _load()
    base = int(lib.gg_grid_base_edges(side))
    n_short = int(shortcut_frac * base)
    src = np.empty(base + n_short, np.int32)
    dst = np.empty(base + n_short, np.int32)
    k = int(lib.gg_grid_edges(side, n_short, max_l1, seed, _p(src), _p(dst)))
    if k < 0:
        raise MemoryError("grid generator out of host memory")
    return src[:k], dst[:k]


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray, symmetrize=True):
    src = np.ascontiguousarray(src, np.int32)
    dst = np.ascontiguousarray(dst, np.int32)
    ne = src.shape[0]
    cap = 2 * ne if symmetrize else ne
    row_ptr = np.empty(n + 1, np.int32)
    col = np.empty(max(cap, 1), np.int32)
    m = int(_load().gg_csr_from_edges(n, ne, _p(src), _p(dst), 1 if symmetrize else 0,
                                      _p(row_ptr), _p(col), cap))
    if m < 0:
        raise RuntimeError({-1: "out of host memory", -2: "capacity", -3: "E >= 2^31",
                            -4: "vertex id out of range"}.get(m, str(m)))
    return row_ptr, col[:m]


def pair_weights(row_ptr: np.ndarray, col: np.ndarray, seed: int, lo: int, hi: int) -> np.ndarray:
    n = row_ptr.shape[0] - 1
    wt = np.empty(col.shape[0], np.int32)
    _load().gg_pair_weights(n, _p(row_ptr), _p(np.ascontiguousarray(col)), seed, lo, hi, _p(wt))
    return wt


def pick_sources(g: HostGraph, k: int, seed: int) -> np.ndarray:
    out = np.empty(k, np.int32)
    got = int(_load().gg_pick_sources(g.n, _p(g.row_ptr), seed, k, _p(out)))
    if got != k:
        raise RuntimeError("graph has no vertex with degree >= 1")
    return out


def rmat_graph(scale: int, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1,
               weights: tuple | None = None) -> HostGraph:
    """Symmetrized R-MAT graph with 2^scale vertices and edge_factor*2^scale generated edges."""
    n = 1 << scale
    src, dst = rmat_edges(scale, edge_factor * n, a, b, c, seed)
    row_ptr, col = csr_from_edges(n, src, dst, True)
    del src, dst
    wt = pair_weights(row_ptr, col, seed, *weights) if weights else None
    return HostGraph(n, row_ptr, col, wt, True, f"rmat{scale}_ef{edge_factor}",
                     dict(kind="rmat", scale=scale, edge_factor=edge_factor, a=a, b=b, c=c, seed=seed,
                          weights=weights))


def grid_graph(side: int, shortcut_frac=0.01, max_l1=8, seed=1, weights: tuple | None = None) -> HostGraph:
    """side x side 4-neighbour grid plus shortcut_frac local shortcuts (2 <= L1 <= max_l1)."""
    n = side * side
    src, dst = grid_edges(side, shortcut_frac, max_l1, seed)
    row_ptr, col = csr_from_edges(n, src, dst, True)
    wt = pair_weights(row_ptr, col, seed, *weights) if weights else None
    return HostGraph(n, row_ptr, col, wt, True, f"grid{side}",
                     dict(kind="grid", side=side, shortcut_frac=shortcut_frac, max_l1=max_l1, seed=seed,
                          weights=weights))


def from_edge_list(n: int, edges, symmetrize=True, weights=None, name="custom") -> HostGraph:
    """Small hand-written graphs for tests: edges is an iterable of (u, v)."""
    e = np.asarray(list(edges), np.int32).reshape(-1, 2)
    row_ptr, col = csr_from_edges(n, e[:, 0].copy(), e[:, 1].copy(), symmetrize)
    wt = pair_weights(row_ptr, col, *weights) if weights else None
    return HostGraph(n, row_ptr, col, wt, symmetrize, name, dict(kind="custom"))


def transpose(g: HostGraph):
    """In-edge (CSC) arrays of a directed HostGraph: (in_ptr, in_col, in_wt)."""
    n = g.n
    deg = g.degrees()
    src = np.repeat(np.arange(n, dtype=np.int32), deg)
    order = np.lexsort((src, g.col))
    in_col = src[order].astype(np.int32)
    in_ptr = np.zeros(n + 1, np.int64)
    np.add.at(in_ptr, g.col.astype(np.int64) + 1, 1)
    in_ptr = np.cumsum(in_ptr).astype(np.int32)
    in_wt = g.wt[order].astype(np.int32) if g.wt is not None else None
    return in_ptr, in_col, in_wt
