"""ctypes declarations of the C ABI in include/graphit_gb.h (names kept as in C)."""
from __future__ import annotations

import ctypes
import os

from . import _build

GI_OK = 0
GI_ERR_INVALID_ARG = -1
GI_ERR_BAD_GRAPH = -2
GI_ERR_OOM = -3
GI_ERR_CUDA = -4
GI_ERR_TIMEOUT = -5
GI_ERR_UNSUPPORTED = -6
ERR_NAMES = {0: "GI_OK", -1: "GI_ERR_INVALID_ARG", -2: "GI_ERR_BAD_GRAPH", -3: "GI_ERR_OOM",
             -4: "GI_ERR_CUDA", -5: "GI_ERR_TIMEOUT", -6: "GI_ERR_UNSUPPORTED"}

GI_HOST_PTRS, GI_DEV_PTRS, GI_SYMMETRIC, GI_VALIDATE, GI_HOT_SOURCES = 0x1, 0x2, 0x4, 0x8, 0x10
GI_VSET_EMPTY, GI_VSET_ALL, GI_VSET_SINGLE = 0, 1, 2
GI_REP_SPARSE, GI_REP_BOOL, GI_REP_BITMAP = 0x1, 0x2, 0x4
GI_DIR_SPARSE_PUSH, GI_DIR_DENSE_PUSH, GI_DIR_DENSE_PULL = 0, 1, 2
GI_DIR_HYBRID_PULL, GI_DIR_HYBRID_DPUSH, GI_DIR_LEARNED, GI_DIR_SPARSE_PULL = 3, 4, 5, 6
GI_BAL_VERTEX, GI_BAL_EDGE_AWARE, GI_BAL_EDGE_PARALLEL = 0, 1, 2
GI_SEG_FVC, GI_SEG_EVC = 0, 1
GI_RULE_BEAMER, GI_RULE_LIGRA = 0, 1
GI_K_BFS, GI_K_SSSP, GI_K_CC, GI_K_SUM, GI_K_PROBE = 1, 2, 3, 4, 5
GI_NO_DEDUP = 0x1
GI_STATIC_PR_MAX_N = 1 << 20
GI_ALGO_BFS, GI_ALGO_SSSP, GI_ALGO_CC, GI_ALGO_PAGERANK, GI_ALGO_PAGERANK_DELTA = 1, 2, 3, 4, 5

DIRECTIONS = {"sparse_push": 0, "dense_push": 1, "dense_pull": 2, "hybrid_pull": 3, "hybrid_dpush": 4,
              "learned": 5, "sparse_pull": 6}

_vp = ctypes.c_void_p
_i32, _i64, _u32, _f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_float
_P = ctypes.POINTER


class gi_schedule(ctypes.Structure):
    _fields_ = [("direction", _i32), ("dense_rep", _u32), ("balance", _i32), ("num_segments", _i32),
                ("block", _i32), ("t_warp", _i32), ("t_cta", _i32), ("rule", _i32), ("alpha", _f32),
                ("beta", _f32), ("tile_edges", _i32), ("t_heavy", _i32), ("persistent", _i32),
                ("hot_cache", _i32), ("seg_strategy", _i32), ("delta", _i32),
                ("dst_list", _i32)]


class gi_trace(ctypes.Structure):
    _fields_ = [("cap", _i32), ("iterations", _i32), ("direction", _P(_i32)), ("frontier", _P(_i64)),
                ("edges", _P(_i64)), ("features", _P(_f32)), ("phase", _P(_i32))]


class gi_batch_opts(ctypes.Structure):
    _fields_ = [("cluster_size", _i32), ("clusters", _i32), ("selector", _i32), ("alpha", _f32), ("beta", _f32),
                ("level_cap", _i64), ("levels", _P(_i32)), ("sssp_delta", _f32), ("order", _i32),
                ("t_warp", _i32), ("t_cta", _i32), ("parents", _P(_vp))]


class gi_bfs_args(ctypes.Structure):
    _fields_ = [("depth", _vp), ("parent", _vp), ("level", _i32)]


class gi_sssp_args(ctypes.Structure):
    _fields_ = [("dist", _vp), ("snap", _vp)]


class gi_cc_args(ctypes.Structure):
    _fields_ = [("label", _vp), ("snap", _vp)]


class gi_sum_args(ctypes.Structure):
    _fields_ = [("contrib", _vp), ("acc", _vp)]


class gi_probe_args(ctypes.Structure):
    _fields_ = [("count", _vp), ("srcsum", _vp)]


SIGNATURES = {
    "gi_last_error": (ctypes.c_char_p, []),
    "gi_version": (ctypes.c_int, []),
    "gi_load_csr": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _u32, _vp, _P(_vp)]),
    "gi_load_csc": (ctypes.c_int, [_vp, _vp, _vp, _vp, _u32, _vp]),
    "gi_graph_free": (ctypes.c_int, [_vp]),
    "gi_graph_info": (ctypes.c_int, [_vp, _P(_i64), _P(_i64), _P(_i32)]),
    "gi_graph_device_csr": (ctypes.c_int, [_vp, _P(_vp), _P(_vp), _P(_vp)]),
    "gi_graph_build_segments": (ctypes.c_int, [_vp, _i32, _i32, _vp]),
    "gi_graph_segment_info": (ctypes.c_int, [_vp, _P(_i32), _P(_i32), _vp, _vp, _i32]),
    "gi_vset_create": (ctypes.c_int, [_vp, _i32, _i32, _vp, _P(_vp)]),
    "gi_vset_free": (ctypes.c_int, [_vp]),
    "gi_vset_size": (ctypes.c_int, [_vp, _P(_i64), _vp]),
    "gi_vset_reps": (ctypes.c_int, [_vp, _P(_u32)]),
    "gi_vset_to_sparse": (ctypes.c_int, [_vp, _vp]),
    "gi_vset_to_dense": (ctypes.c_int, [_vp, _u32, _vp]),
    "gi_vset_export": (ctypes.c_int, [_vp, _vp, _i64, _P(_i64), _vp]),
    "gi_vset_import": (ctypes.c_int, [_vp, _vp, _i64, _vp]),
    "gi_schedule_default": (None, [_P(gi_schedule)]),
    "gi_edgeset_apply": (ctypes.c_int, [_vp, _vp, _vp, _P(gi_schedule), _i32, _vp, _vp, _u32, _vp]),
    "gi_bfs": (ctypes.c_int, [_vp, _i32, _vp, _vp, _P(gi_schedule), _P(gi_trace), _vp]),
    "gi_sssp": (ctypes.c_int, [_vp, _i32, _vp, _P(gi_schedule), _P(gi_trace), _vp]),
    "gi_cc": (ctypes.c_int, [_vp, _vp, _P(gi_schedule), _P(gi_trace), _vp]),
    "gi_pagerank": (ctypes.c_int, [_vp, _f32, _i32, _vp, _P(gi_schedule), _vp]),
    "gi_pagerank_delta": (ctypes.c_int, [_vp, _f32, _f32, _i32, _vp, _P(gi_schedule), _P(gi_trace), _vp]),
    "gi_bc": (ctypes.c_int, [_vp, _i32, _vp, _vp, _i32, _P(gi_schedule), _P(gi_trace), _vp]),
    "gi_pagerank_static": (ctypes.c_int, [_vp, _vp, _vp, _i64, _i64, _f32, _i32, _vp, _vp]),
    "gi_selector_load": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
    "gi_selector_num_params": (ctypes.c_int, []),
    "gi_mlp_loss_grad": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp, _vp]),
    "gi_mlp_forward": (ctypes.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "gi_mlp_adam": (ctypes.c_int, [_vp, _vp, _vp, _vp, _i32, _f32, _f32, _f32, _f32, _vp]),
    "gi_selector_profile": (ctypes.c_int, [_vp, _i32, _i32, _P(gi_schedule), _i32, _vp, _vp, _P(_i32), _vp]),
    "gi_autotune": (ctypes.c_int, [_vp, _i32, _i32, _P(gi_schedule), _i32, ctypes.c_uint64, _P(gi_schedule),
                                   _P(ctypes.c_double), _P(ctypes.c_double), _vp]),
    "gi_batch_opts_default": (None, [_P(gi_batch_opts)]),
    "gi_batch_autotune": (ctypes.c_int, [_P(_vp), _i32, _vp, _vp, _vp, _i32, _P(gi_batch_opts), _i32,
                                         ctypes.c_uint64, _P(gi_batch_opts), _P(ctypes.c_double),
                                         _P(ctypes.c_double), _vp]),
    "gi_batch_run": (ctypes.c_int, [_P(_vp), _i32, _vp, _vp, _vp, _i32, _P(_vp), _vp, _P(gi_batch_opts), _vp]),
    "gi_batch_plan_create": (ctypes.c_int, [_P(_vp), _i32, _vp, _vp, _vp, _i32, _P(_vp), _P(gi_batch_opts), _vp,
                                            _P(_vp)]),
    "gi_batch_plan_launch": (ctypes.c_int, [_vp, _vp]),
    "gi_batch_plan_results": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "gi_batch_plan_free": (ctypes.c_int, [_vp]),
    "gi_debug_fail_allocs_after": (ctypes.c_int, [_i64]),
    "gi_debug_pool_used": (ctypes.c_int, [_P(_i64)]),
    "gi_graph_hot_info": (ctypes.c_int, [_vp, _P(_i32), _P(_i32), _vp]),
    "gi_debug_barrier_phantoms": (ctypes.c_int, [_i32]),
    "gi_gather_rate": (ctypes.c_int, [_vp, _i64, _vp, _i64, _vp, _vp]),
    "gi_stats_enable": (ctypes.c_int, [ctypes.c_int]),
    "gi_stats_reset": (ctypes.c_int, []),
    "gi_stats_read": (ctypes.c_int, [_i32, _P(_i64), _P(_i64), _P(ctypes.c_double)]),
    "gi_stats_pull_arcs": (ctypes.c_int, [_vp, _i32, _P(_i64)]),
    "gi_prepare": (ctypes.c_int, [_vp, _i32, _vp, _vp]),
}
KCLASS = {"pr_pull": 0, "prd_pull": 1, "min_pull": 2, "push": 3, "bfs_pull": 4, "other_pull": 5, "batch": 6}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgraphit_gb.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class GIError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int):
    if code != GI_OK:
        msg = _lib.gi_last_error().decode(errors="replace") if _lib is not None else ""
        raise GIError(code, msg)
