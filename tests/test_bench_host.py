"""Host-side pieces of bench.py that need no GPU: the per-level byte model of
the early-exit BFS pull (checked against a brute-force scan), the JSON line
of the CPU reference arm, and the rule that ties a recorded ncu traffic
figure to the kernel code it was captured on."""
import json
import os
import subprocess
import sys

import numpy as np
import torch

import graphgen as gg
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_bfs_level_bytes_match_brute_force():
    """|F|, m_f, |F_next|, n_u and E_scanned (in-arcs up to and including the
    first frontier source, all of them if none) per level, from the depths."""
    hg = gg.rmat_graph(10, seed=3)
    src = int(gg.pick_sources(hg, 1, seed=1)[0])
    depth, _, _ = oracle.bfs(hg, src)
    deg = np.diff(hg.row_ptr)
    levels = int(depth.max()) + 1
    got = bench._bfs_level_bytes(torch.from_numpy(depth.astype(np.int32)), torch.from_numpy(hg.col),
                                 torch.repeat_interleave(torch.arange(hg.n, dtype=torch.int32),
                                                         torch.from_numpy(deg.astype(np.int64))),
                                 torch.from_numpy(hg.row_ptr), torch.from_numpy(deg.astype(np.int32)), levels)
    for d in range(levels):
        scanned = 0
        for v in range(hg.n):
            if 0 <= depth[v] <= d:
                continue
            a, b = hg.row_ptr[v], hg.row_ptr[v + 1]
            k = b - a
            for j in range(a, b):
                if depth[hg.col[j]] == d:
                    k = j - a + 1
                    break
            scanned += k
        front = depth == d
        assert got[d] == dict(frontier=int(front.sum()), m_f=int(deg[front].sum()),
                              next=int((depth == d + 1).sum()), n_u=int(((depth > d) | (depth < 0)).sum()),
                              e_scanned=scanned)


def test_sssp_pull_bytes_counts_pull_rounds_only():
    """Per pull round 4(V+1) + 8m + 8 m_f + V/4 + 4|F_next|; push rounds add nothing."""
    class T:
        def as_dict(self):
            return {"frontier": np.array([1, 40, 900, 50]), "edges": np.array([3, 200, 5000, 300]),
                    "direction": np.array([0, 2, 2, 0])}
    n, m = 1000, 20000
    want = sum(4 * (n + 1) + 8 * m + 8 * e + n // 4 + 4 * nx for e, nx in ((200, 900), (5000, 50)))
    assert bench._sssp_pull_bytes(n, m, T()) == (want, 2, 2 * m)

    class D:  # delta-stepping: light (phase 0) and heavy (1) rounds; a pull round without arcs launches nothing
        def as_dict(self):
            return {"frontier": np.array([1, 40, 900, 50, 7]), "edges": np.array([3, 200, 5000, 300, 0]),
                    "direction": np.array([0, 2, 2, 0, 2]), "phase": np.array([0, 0, 1, 0, 1])}
    ml = 6000
    want = (4 * (n + 1) + 8 * ml + 8 * 200 + n // 4) + (4 * (n + 1) + 8 * (m - ml) + 8 * 5000 + n // 4)
    assert bench._sssp_pull_bytes(n, m, D(), ml) == (want, 2, m)


def test_reference_arm_json_line():
    """`--impl reference` prints one JSON line with the contract's keys and
    exits 0 (oracle BFS / SSSP queries of the BFS/SSSP workload on a small graph)."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--scale", "12",
                        "--steps", "2", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "dtype", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["config"]["workload"] == "rmat24_bfs_sssp" and d["config"]["sources"] == 64


def test_recorded_traffic_follows_the_kernel_code(tmp_path, monkeypatch):
    """roofline.traffic is read from profiles/traffic.txt only while the code
    it was captured on is unchanged: comment and blank-line edits keep the
    kernel hash, an edit of the tile loop or of the edge function drops it."""
    csrc = tmp_path / "paper_1805_00923_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    real = os.path.join(ROOT, "paper_1805_00923_gb300", "csrc")
    traverse = open(os.path.join(real, "gi_traverse.cuh")).read()
    (csrc / "gi_internal.cuh").write_text(open(os.path.join(real, "gi_internal.cuh")).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    op = "OpMinInt+OpMinIntBounded"

    def hashed(text):
        (csrc / "gi_traverse.cuh").write_text(text)
        return bench.kernel_source_hash(op)

    h = hashed(traverse)
    (tmp_path / "profiles" / "traffic.txt").write_text(f"# hash kernel workload bytes\n{h} kname wl 123 (1 launch)\n")
    assert bench.recorded_traffic("kname", "wl", op=op) == 123.0
    assert bench.recorded_traffic("kname", "other", op=op) is None

    line = "constexpr int kBatch = 8;"
    assert traverse.count(line) == 1
    assert hashed(traverse.replace(line, line + "  // a note\n\n// another\n")) == h
    assert bench.recorded_traffic("kname", "wl", op=op) == 123.0

    staged = "u[j] = k < ne ? G.src(idx + e0 + k) : -1;"  # the tile staging loop
    assert staged in traverse
    assert hashed(traverse.replace(staged, staged.replace("-1", "-2"), 1)) != h
    assert bench.recorded_traffic("kname", "wl", op=op) is None

    combine = "__device__ static V combine(V a, V b) { return a < b ? a : b; }"
    i = traverse.index("struct OpMinInt ")
    edited = traverse[:i] + traverse[i:].replace(combine, combine.replace("a < b", "a <= b"), 1)
    assert hashed(edited) != h
    assert bench.recorded_traffic("kname", "wl", op=op) is None
