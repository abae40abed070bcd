"""The C ABI library loads and exports every function include/*.h declares.

Only argument checks run here (they return before any CUDA call), so this
needs no GPU.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(?:int|void|const char\s*\*)\s*\*?\s*(gi_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1805_00923_gb300 import _lib
    return _lib.load()


def test_header_declares_functions():
    names = _declared()
    assert "gi_load_csr" in names and "gi_edgeset_apply" in names and "gi_bfs" in names
    assert len(names) >= 25


def test_every_declared_symbol_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header(lib):
    from paper_1805_00923_gb300 import _lib
    assert set(_declared()) <= set(_lib.SIGNATURES), set(_declared()) - set(_lib.SIGNATURES)


def test_argument_errors_without_gpu(lib):
    from paper_1805_00923_gb300 import _lib as L
    out = ctypes.c_void_p()
    a = (ctypes.c_int32 * 2)(0, 0)
    # NULL output handle
    assert lib.gi_load_csr(a, a, None, 1, 0, L.GI_HOST_PTRS, None, None) == L.GI_ERR_INVALID_ARG
    # negative sizes
    assert lib.gi_load_csr(a, a, None, -1, 0, L.GI_HOST_PTRS, None, ctypes.byref(out)) == L.GI_ERR_INVALID_ARG
    # both / neither pointer kinds
    assert lib.gi_load_csr(a, a, None, 1, 0, L.GI_HOST_PTRS | L.GI_DEV_PTRS, None,
                           ctypes.byref(out)) == L.GI_ERR_INVALID_ARG
    assert lib.gi_load_csr(a, a, None, 1, 0, 0, None, ctypes.byref(out)) == L.GI_ERR_INVALID_ARG
    # too large for int32 offsets
    assert lib.gi_load_csr(a, a, None, 1, 2**31, L.GI_HOST_PTRS, None, ctypes.byref(out)) == L.GI_ERR_UNSUPPORTED
    assert b"int32" in lib.gi_last_error()
    # NULL graph handles
    s = L.gi_schedule()
    lib.gi_schedule_default(ctypes.byref(s))
    assert lib.gi_bfs(None, 0, None, None, ctypes.byref(s), None, None) == L.GI_ERR_INVALID_ARG
    assert lib.gi_pagerank(None, 0.85, 20, None, ctypes.byref(s), None) == L.GI_ERR_INVALID_ARG
    assert lib.gi_graph_free(None) == L.GI_OK
    assert lib.gi_selector_load(None, 0, None, None) == L.GI_ERR_INVALID_ARG


def test_schedule_defaults(lib):
    from paper_1805_00923_gb300 import _lib as L
    s = L.gi_schedule()
    lib.gi_schedule_default(ctypes.byref(s))
    assert s.direction == L.GI_DIR_HYBRID_PULL and s.dense_rep == L.GI_REP_BITMAP
    assert s.balance == L.GI_BAL_EDGE_AWARE and s.num_segments == 1 and s.block == 256
    assert (s.t_warp, s.t_cta, s.rule, s.alpha, s.beta, s.tile_edges) == (32, 256, L.GI_RULE_BEAMER, 14.0, 24.0,
                                                                          2048)
    assert (s.t_heavy, s.persistent, s.hot_cache, s.seg_strategy) == (256, 0, 0, 0)
    assert (s.delta, s.dst_list) == (0, 1)


def test_schedule_binding_fields(lib):
    """The binding's schedule(): library defaults, a named direction, string
    enums mapped to the header's values, and no silently ignored field."""
    import pytest
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import _lib as L
    s = gi.schedule("learned", balance="edge_parallel", rule="ligra", seg_strategy="evc", delta=128, tile_edges=4096)
    assert s.direction == L.GI_DIR_LEARNED and s.balance == L.GI_BAL_EDGE_PARALLEL
    assert s.rule == L.GI_RULE_LIGRA and s.seg_strategy == L.GI_SEG_EVC
    assert (s.delta, s.tile_edges, s.t_warp, s.dst_list) == (128, 4096, 32, 1)
    with pytest.raises(TypeError):
        gi.schedule("dense_pull", tile_edge=4096)


def test_selector_param_count_matches_oracle(lib):
    import oracle
    assert lib.gi_selector_num_params() == oracle.mlp_num_params()


def test_struct_layouts_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field
    offsets: a C program built against include/graphit_gb.h prints them."""
    from paper_1805_00923_gb300 import _lib as L
    structs = ["gi_schedule", "gi_trace", "gi_batch_opts", "gi_bfs_args", "gi_sssp_args", "gi_cc_args",
               "gi_sum_args", "gi_probe_args"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "graphit_gb.h"', "int main(void) {"]
    for name in structs:
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f, _ in getattr(L, name)._fields_:
            lines.append(f'  printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, c = ln.split()
            got[(a, b)] = int(c)
    for name in structs:
        cls = getattr(L, name)
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)


def test_constants_match_the_header(tmp_path):
    """Every GI_* constant the header defines has the same value in the
    binding (the timing classes as its KCLASS table): a C program built
    against include/graphit_gb.h prints them."""
    import re
    import subprocess
    from paper_1805_00923_gb300 import _lib as L
    header = open(os.path.join(ROOT, "include", "graphit_gb.h")).read()
    names = re.findall(r"^#define (GI_[A-Z0-9_]+)[ \t]+\S", header, re.M)
    assert len(names) > 40
    lines = ['#include <stdio.h>', '#include "graphit_gb.h"', "int main(void) {"]
    lines += [f'  printf("{n} %lld\\n", (long long)({n}));' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    r = subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(ln.split() for ln in subprocess.run([str(exe)], capture_output=True, text=True,
                                                     check=True).stdout.splitlines())
    for n in names:
        if n.startswith("GI_KCLASS_"):
            mine = L.KCLASS[n[len("GI_KCLASS_"):].lower()]
        else:
            assert hasattr(L, n), n
            mine = getattr(L, n)
        assert int(got[n]) == int(mine), n


def test_null_handles_are_argument_errors(lib):
    """Each entry point that takes a graph, vertexset or plan reports a NULL
    one as GI_ERR_INVALID_ARG with a message, before any device work (so
    this runs without a GPU); the free functions take NULL as a no-op."""
    from paper_1805_00923_gb300 import _lib as L
    s = L.gi_schedule()
    lib.gi_schedule_default(ctypes.byref(s))
    o = L.gi_batch_opts()
    lib.gi_batch_opts_default(ctypes.byref(o))
    p, i64, i32, u32, d = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_uint32(), ctypes.c_double()
    f = ctypes.c_float
    calls = {
        "gi_load_csc": lambda: lib.gi_load_csc(None, None, None, None, 0, None),
        "gi_graph_info": lambda: lib.gi_graph_info(None, ctypes.byref(i64), ctypes.byref(i64), ctypes.byref(i32)),
        "gi_graph_hot_info": lambda: lib.gi_graph_hot_info(None, ctypes.byref(i32), ctypes.byref(i32), None),
        "gi_graph_build_segments": lambda: lib.gi_graph_build_segments(None, 2, 0, None),
        "gi_vset_create": lambda: lib.gi_vset_create(None, 0, 0, None, ctypes.byref(p)),
        "gi_vset_size": lambda: lib.gi_vset_size(None, ctypes.byref(i64), None),
        "gi_vset_reps": lambda: lib.gi_vset_reps(None, ctypes.byref(u32)),
        "gi_vset_to_sparse": lambda: lib.gi_vset_to_sparse(None, None),
        "gi_edgeset_apply": lambda: lib.gi_edgeset_apply(None, None, None, ctypes.byref(s), 0, None, None, 0, None),
        "gi_sssp": lambda: lib.gi_sssp(None, 0, None, ctypes.byref(s), None, None),
        "gi_prepare": lambda: lib.gi_prepare(None, 0, ctypes.byref(s), None),
        "gi_cc": lambda: lib.gi_cc(None, None, ctypes.byref(s), None, None),
        "gi_pagerank_delta": lambda: lib.gi_pagerank_delta(None, f(0.85), f(1e-7), 10, None, ctypes.byref(s), None,
                                                           None),
        "gi_bc": lambda: lib.gi_bc(None, 0, None, None, 0, ctypes.byref(s), None, None),
        "gi_pagerank_static": lambda: lib.gi_pagerank_static(None, None, None, 10, 5, f(0.85), 20, None, None),
        "gi_batch_plan_launch": lambda: lib.gi_batch_plan_launch(None, None),
        "gi_autotune": lambda: lib.gi_autotune(None, 0, 0, ctypes.byref(s), 4, 1, ctypes.byref(s), ctypes.byref(d),
                                               ctypes.byref(d), None),
        "gi_stats_pull_arcs": lambda: lib.gi_stats_pull_arcs(None, 0, ctypes.byref(i64)),
        "gi_mlp_forward": lambda: lib.gi_mlp_forward(None, None, 4, None, None),
        "gi_selector_profile": lambda: lib.gi_selector_profile(None, 0, 0, ctypes.byref(s), 16, None, None, None,
                                                               None),
    }
    for name, call in calls.items():
        assert call() == L.GI_ERR_INVALID_ARG, name
        assert lib.gi_last_error().startswith(b"invalid argument"), name
    assert lib.gi_stats_read(99, ctypes.byref(i64), ctypes.byref(i64), None) == L.GI_ERR_INVALID_ARG
    assert lib.gi_vset_free(None) == L.GI_OK
    assert lib.gi_batch_plan_free(None) == L.GI_OK
