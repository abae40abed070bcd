#!/usr/bin/env python
"""Benchmark of the edgeset-apply hot path on one GB300 (or N replicas).

Workload (one "step", the default): on a symmetrized R-MAT graph of scale 24
(edge factor 16, a=.57 b=.19 c=.19, seed 1; 16.8M vertices, ~521M arcs, int32
arc weights uniform in [1,1000) from the pair hash), run from each of 64 seeded
sources (uniform among vertices of degree >= 1)
  BFS    depth + canonical (smallest-id) parent
  SSSP   Bellman-Ford distances
with the direction of every level chosen by the learned selector.  Value =
arcs of the reached components (per query the sum of the reached vertices'
degrees) / step time, in GTEPS (10^9 arcs/s).  Beside it: Beamer's rule
(SSSP: Ligra's |F| + m_f > m/20) on the same queries, three interleaved
repeats of each, the BFS level loop as a CUDA graph, and the exhaustive
best-direction-per-level sum; the PR + PRD + CC step on R-MAT 22 rides along
as an extra.  Inputs (CSR + weights ~4.2 GB) exceed the 126 MB L2.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.  --workload selects the other
configurations, each printing its own line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS per algorithm & graph, learned vs heuristic schedule; % of HBM roofline"
DAMPING, PR_ITERS, PRD_EPS, PRD_ITERS = 0.85, 20, 1e-7, 10
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["gi", "reference"], default="gi")
    p.add_argument("--scale", type=int, default=24, help="R-MAT scale of the BFS/SSSP workload")
    p.add_argument("--m-scale", type=int, default=22, help="R-MAT scale of the PR/PRD/CC workload (and BC)")
    p.add_argument("--m-steps", type=int, default=5, help="timed steps of the PR/PRD/CC extra")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--repeats", type=int, default=3, help="repeats of the learned vs rule comparison")
    p.add_argument("--delta", type=int, default=128, help="SSSP bucket width the autotuner starts from")
    p.add_argument("--exhaustive-sources", type=int, default=8)
    p.add_argument("--cpu-sources", type=int, default=4, help="sources of the CPU oracle sample (BFS + SSSP)")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="PR/PRD/CC workload: CPU time of the oracle sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--tune-budget", type=int, default=12, help="autotuner trials per algorithm (untimed)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the untimed autotuning and direction comparison (profiling runs)")
    p.add_argument("--workload", choices=["rmat24_bfs_sssp", "rmat22", "rmat24_levels", "grid4096", "batch512", "bc"],
                   default="rmat24_bfs_sssp",
                   help="rmat24_bfs_sssp (default): BFS + SSSP from 64 sources on R-MAT 24, learned vs Beamer, "
                        "with the PR+PRD+CC step on R-MAT 22 as an extra; the others measure the remaining "
                        "configurations and print their own JSON line")
    p.add_argument("--sources", type=int, default=64, help="sources per graph for the BFS/SSSP workloads")
    p.add_argument("--only", choices=["pagerank", "pagerank_delta", "cc", "bfs", "sssp", "bc"], default=None,
                   help="profiling case: run just this algorithm --steps times on the workload graph")
    p.add_argument("--hot-cache", type=int, choices=[0, 1, 2], default=0,
                   help="profiling case: PageRank / PageRankDelta pulls with the hot-source cache")
    p.add_argument("--only-delta", type=int, default=0,
                   help="profiling case: SSSP bucket width (0 = Bellman-Ford)")
    p.add_argument("--only-persistent", type=int, choices=[0, 1, 2], default=0,
                   help="profiling case: single-query mode of BFS / SSSP (2 = graph-driven loop)")
    p.add_argument("--only-source", type=int, default=0,
                   help="profiling case: BFS / SSSP source (-1: the first seeded source of the BFS/SSSP workload)")
    p.add_argument("--only-direction", default="hybrid_pull",
                   help="profiling case: direction of BFS / SSSP (hybrid_pull, learned, ...)")
    return p.parse_args()


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_config(hg, scale):
    return {"workload": f"rmat{scale}_pr{PR_ITERS}_prd{PRD_ITERS}_cc", "graph": "R-MAT symmetrized",
            "scale": scale, "edge_factor": 16, "abc": [0.57, 0.19, 0.19], "seed": 1, "n": hg.n, "m": hg.m,
            "pagerank": {"iters": PR_ITERS, "damping": DAMPING,
                         "schedule": "DensePull, autotuned from the hot-source L1 pull"},
            "pagerank_delta": {"iters": PRD_ITERS, "eps": PRD_EPS,
                               "schedule": "DensePull-SparsePush (Ligra rule), autotuned from the hot-source L1 pull"},
            "cc": {"schedule": "DensePull-SparsePush (Ligra rule), autotuned from the hot-source L1 pull"},
            "l2": "inputs larger than L2 (CSR %.0f MB vs 126 MB L2); no flush" % ((4 * (hg.n + 1) + 4 * hg.m) / 1e6)}


def oracle_sample(hg, seconds):
    """Time the oracle's PageRank on the full graph for as many iterations as fit ~`seconds`."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.pagerank(hg, DAMPING, 1)
    t1 = time.perf_counter() - t0
    iters = max(1, min(PR_ITERS, int(seconds / max(t1, 1e-3))))
    t0 = time.perf_counter()
    oracle.pagerank(hg, DAMPING, iters)
    t = time.perf_counter() - t0
    return iters * hg.m / t / 1e9, iters, t


def run_reference(args):
    """The oracle on the BFS/SSSP workload: each step is one oracle query (BFS
    with parents, then SSSP, alternating over the 64 sources), single-threaded
    C; the steps run on the host cores at once, so value = arcs of the timed
    queries / wall time of the timed region on `cores` threads."""
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    import numpy as np
    import graphgen as gg
    hg = gg.rmat_graph(args.scale, seed=1, weights=(1, 1000))
    srcs = [int(x) for x in gg.pick_sources(hg, args.sources, seed=1)]
    qs = [("bfs" if i % 2 == 0 else "sssp", srcs[(i // 2) % len(srcs)]) for i in range(args.warmup + args.steps)]
    cores, model = host_cpu()
    threads = max(1, min(cores, len(qs)))
    if args.warmup:
        oracle_queries(hg, qs[:args.warmup], threads)
    timed = qs[args.warmup:]
    secs, arcs = oracle_queries(hg, timed, min(threads, max(1, len(timed))))
    value = arcs / secs / 1e9
    used = min(threads, max(1, len(timed)))
    sample = (f"{len(timed)} oracle queries (BFS with parents / SSSP alternating over the seeded sources) of "
              f"the scale-{args.scale} workload, one per step, on {used} threads at once")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": l_config(hg, len(srcs)),
            "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": used, "kind": "oracle", "sample": sample,
                             "host": {"nproc": cores, "model": model, "used": f"{used} of {cores} cores"}},
            "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class ClockSampler:
    """nvidia-smi clocks/throttle samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash(op="OpPR"):
    """Hash of the code of the timed kernel (k_pull_tiled with its staging
    helpers, the edge function `op` -- "+"-joined names for an edge function
    and the one it extends -- and the hot-source cap), so a recorded ncu
    traffic figure is used only while that code is unchanged."""
    import re
    with open(os.path.join(ROOT, "paper_1805_00923_gb300", "csrc", "gi_traverse.cuh")) as fh:
        src = fh.read()
    a = src.index("constexpr int kBatch = 8;")
    b = src.index("// Warp tiles (tile_edges = 256)")
    parts = src[a:b]
    for name in op.split("+"):
        c = re.search(rf"struct {name}\b[^{{;]*{{", src).start()
        parts += src[c:src.index("};", c)]
    # code only: comment lines and blank lines do not change the kernel
    code = [ln.split("//")[0].rstrip() for ln in parts.splitlines()]
    # the hot-source cap (a constant of the shared header) changes what the kernel reads
    with open(os.path.join(ROOT, "paper_1805_00923_gb300", "csrc", "gi_internal.cuh")) as fh:
        code += [ln.split("//")[0].rstrip() for ln in fh if ln.startswith("constexpr int kHotMax")]
    return hashlib.sha256("\n".join(ln for ln in code if ln).encode()).hexdigest()[:16]


def recorded_traffic(kernel, workload, op="OpPR"):
    """DRAM bytes per launch from profiles/traffic.txt if recorded for the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(op)
    for ln in open(path):
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == want and parts[1] == kernel \
                and parts[2] == workload:
            return float(parts[3])
    return None


def measured_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def run_rmat22(args, extra=False):
    """The PageRank + PageRankDelta + CC step on R-MAT scale --m-scale.  As the
    workload of `--workload rmat22` it prints its own line; with extra=True it
    runs --m-steps timed steps (no end-to-end, comparison or CPU legs) and
    returns the line for embedding in the BFS/SSSP line."""
    import numpy as np
    import torch
    import torch.distributed as dist

    world, rank, local = dist_setup()
    if not extra:
        torch.cuda.set_device(local)
        if world > 1:
            dist.init_process_group("nccl")
    import graphgen as gg
    import paper_1805_00923_gb300 as gi

    steps = args.m_steps if extra else args.steps
    hg = gg.rmat_graph(args.m_scale, seed=1)
    n, m = hg.n, hg.m
    stream = torch.cuda.current_stream()
    g = gi.Graph.from_host(hg)
    # the autotuner picks tile shape / thresholds / segment count (untimed setup)
    tune_budget = 1 if args.no_extras else args.tune_budget
    # PageRank / PageRankDelta start from the L1-resident hot-source pull
    # (faster on R-MAT at these sizes); the tuner may move every knob
    pr_s, pr_tuned_ms, pr_start_ms = gi.autotune(g, "pagerank", start=gi.schedule("dense_pull", hot_cache=2),
                                                 budget=tune_budget, seed=1)
    prd_s, prd_tuned_ms, prd_start_ms = gi.autotune(g, "pagerank_delta",
                                                    start=gi.schedule("hybrid_pull", hot_cache=2),
                                                    budget=tune_budget, seed=2)
    cc_s, cc_tuned_ms, cc_start_ms = gi.autotune(g, "cc", start=gi.schedule("hybrid_pull", hot_cache=2),
                                                 budget=tune_budget, seed=3)
    tuned = {"pagerank": dict(gi.schedule_dict(pr_s), tuned_ms=pr_tuned_ms, default_ms=pr_start_ms),
             "pagerank_delta": dict(gi.schedule_dict(prd_s), tuned_ms=prd_tuned_ms, default_ms=prd_start_ms),
             "cc": dict(gi.schedule_dict(cc_s), tuned_ms=cc_tuned_ms, default_ms=cc_start_ms)}
    if not args.no_extras:
        # the tuner's own gain: the same search from the library's default
        # DensePull schedule (no hot-source cache), reported beside the timed one
        d_s, d_tuned, d_start = gi.autotune(g, "pagerank", start=gi.schedule("dense_pull"),
                                            budget=2 * args.tune_budget, seed=1)
        tuned["pagerank_from_library_defaults"] = dict(gi.schedule_dict(d_s), tuned_ms=d_tuned, default_ms=d_start)
    # the three PageRank directions of the workload, one timed run each (untimed setup)
    compare = {}
    for name, sc in ([] if (args.no_extras or extra) else
                     [("dense_pull", gi.schedule("dense_pull")),
                      ("dense_pull_hot_cache", gi.schedule("dense_pull", hot_cache=1)),
                      ("segmented_pull_4", gi.schedule("dense_pull", num_segments=4)),
                      ("dense_push", gi.schedule("dense_push"))]):
        gi.pagerank(g, DAMPING, PR_ITERS, sched=sc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gi.pagerank(g, DAMPING, PR_ITERS, sched=sc)
        e1.record()
        torch.cuda.synchronize()
        compare[name] = PR_ITERS * m / (e0.elapsed_time(e1) * 1e-3) / 1e9
    g.build_segments(1)
    hyb = prd_s
    rank_buf = torch.empty(n, dtype=torch.float32, device="cuda")
    prd_buf = torch.empty(n, dtype=torch.float32, device="cuda")
    lab_buf = torch.empty(n, dtype=torch.int32, device="cuda")
    tr_p, tr_c = gi.Trace(64), gi.Trace(256)

    def traversed(tr):
        """PageRankDelta's actual work: m per pull round, m_f per push round."""
        t = tr.as_dict()
        return int(sum(m if d == gi.GI_DIR_DENSE_PULL else e for d, e in zip(t["direction"], t["edges"])))

    def step(graph, ev=None, after=None):
        """One pass of the workload; after(i), if given, runs once algorithm i is enqueued."""
        if ev:
            ev[0].record()
        gi.pagerank(graph, DAMPING, PR_ITERS, sched=pr_s, out=rank_buf)
        if ev:
            ev[1].record()
        if after:
            after(0)
        gi.pagerank_delta(graph, DAMPING, PRD_EPS, PRD_ITERS, sched=hyb, trace=tr_p, out=prd_buf)
        if ev:
            ev[2].record()
        if after:
            after(1)
        gi.cc(graph, sched=cc_s, trace=tr_c, out=lab_buf)
        if ev:
            ev[3].record()
        if after:
            after(2)
        # CC reaches every vertex: sum of degrees = m, counted once
        return PR_ITERS * m, traversed(tr_p), m

    for _ in range(args.warmup):
        step(g)
    torch.cuda.synchronize()
    if world > 1 and not extra:
        dist.barrier()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    gi.stats_reset()
    gi.stats_enable(True)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    edges = np.zeros(3, np.float64)
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record()
    for k in range(steps):
        edges += step(g, evs[k])
    stop.record()
    torch.cuda.synchronize()
    if world > 1 and not extra:
        dist.barrier()
    torch.cuda.synchronize()
    gi.stats_enable(False)
    launches, pr_launches, pr_ms = gi.stats_read("pr_pull")
    clocks = sampler.stop()
    total_ms = start.elapsed_time(stop)
    per_alg_ms = np.zeros(3)
    for ev in evs:
        per_alg_ms += [ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])]
    if world > 1 and not extra:
        from paper_1805_00923_gb300 import replicas
        total_ms = replicas.max_over_ranks(total_ms, device="cuda")
    value = (1 if extra else world) * edges.sum() / (total_ms * 1e-3) / 1e9
    if extra:
        return rmat22_summary(args, hg, g, steps, value, total_ms, per_alg_ms, edges, launches, pr_launches, pr_ms,
                              pr_s, tuned, clocks)

    # end to end through the C ABI from pinned host buffers
    rp_h = torch.from_numpy(hg.row_ptr).pin_memory()
    col_h = torch.from_numpy(hg.col).pin_memory()
    out_h = [torch.empty(n, dtype=torch.float32).pin_memory(), torch.empty(n, dtype=torch.float32).pin_memory(),
             torch.empty(n, dtype=torch.int32).pin_memory()]
    h2d = 4 * (n + 1) + 4 * m
    # the hot-source set is built while the indices arrive when a schedule uses it
    want_hot = any(int(x.hot_cache) > 0 for x in (pr_s, hyb, cc_s))
    d2h = 3 * 4 * n
    # each result vector goes back on a side stream as soon as its algorithm
    # is done, under the next algorithm's kernels
    side = torch.cuda.Stream()
    res_dev = (rank_buf, prd_buf, lab_buf)

    def fetch(i):
        done = torch.cuda.Event()
        done.record()
        side.wait_event(done)
        with torch.cuda.stream(side):
            out_h[i].copy_(res_dev[i], non_blocking=True)

    # serial form: load, step, copy back, free, one after another
    serial_ms = []
    for k in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ge = gi.Graph(rp_h.numpy(), col_h.numpy(), symmetric=True, hot_sources=want_hot)
        step(ge, after=fetch)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.current_stream().synchronize()
        ge.free()
        if k > 0:  # the first one warms the allocator pool
            serial_ms.append((time.perf_counter() - t0) * 1e3)

    # pipelined form (the reported number): like a data loader, a second host
    # thread loads step k+1's graph (host-to-device copy on its own stream,
    # tiles, hot-source set) while step k runs.  Every step's copy in, from the
    # first load on, and every result copy out lie inside the timed region.
    load_stream = torch.cuda.Stream()
    dev = torch.cuda.current_device()

    def load_graph(box):
        torch.cuda.set_device(dev)
        box["g"] = gi.Graph(rp_h.numpy(), col_h.numpy(), symmetric=True, hot_sources=want_hot, stream=load_stream)

    def pipelined(K):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        box = {}
        load_graph(box)
        edges = 0.0
        for k in range(K):
            cur, box = box["g"], {}
            th = threading.Thread(target=load_graph, args=(box,)) if k + 1 < K else None
            if th:
                th.start()
            edges += sum(step(cur, after=fetch))
            torch.cuda.current_stream().wait_stream(side)
            torch.cuda.current_stream().synchronize()
            if th:
                th.join()
                if "g" not in box:
                    raise RuntimeError("graph load in the loader thread failed")
            cur.free()  # after the join: its device-wide sync waits for nothing
        return (time.perf_counter() - t0) * 1e3, edges

    pipelined(2)  # warm-up
    e2e_total, e2e_edges = pipelined(args.e2e_steps)
    if world > 1:
        from paper_1805_00923_gb300 import replicas
        e2e_total = replicas.max_over_ranks(e2e_total, device="cuda")
    e2e_value = world * e2e_edges / (e2e_total * 1e-3) / 1e9

    # learned vs heuristic direction selection on the same graph (BFS from 8 sources; untimed extra)
    selector = None
    if not args.no_extras:
        from paper_1805_00923_gb300 import selector as sel
        sel.install()
        srcs = gg.pick_sources(hg, 8, seed=7)
        selector = {}
        for pol in ("hybrid_pull", "learned"):
            ms, ed = 0.0, 0
            for s_ in srcs:
                tr = gi.Trace(64)
                gi.bfs(g, int(s_), want_parent=False, sched=gi.schedule(pol), trace=tr)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                gi.bfs(g, int(s_), want_parent=False, sched=gi.schedule(pol), trace=tr)
                e1.record()
                torch.cuda.synchronize()
                ms += e0.elapsed_time(e1)
                ed += int(tr.as_dict()["edges"].sum())
            selector["bfs_" + ("beamer" if pol == "hybrid_pull" else "learned") + "_gteps"] = ed / (ms * 1e-3) / 1e9

    peak, peak_kind = measured_hbm()
    # algorithmic bytes of one PageRank DensePull launch: offsets 4(n+1), indices 4m,
    # one gathered 4-byte contribution per arc 4m, 1/outdeg 4n, one output vector 4n
    bytes_per_launch = 8 * m + 12 * n + 4
    avg_ms = pr_ms / max(pr_launches, 1)
    achieved = bytes_per_launch / (avg_ms * 1e-3) / 1e9
    hot = int(pr_s.hot_cache) if pr_s.direction == gi.GI_DIR_DENSE_PULL and pr_s.num_segments == 1 else 0
    kname = {0: "k_pull_tiled_OpPR", 1: "k_pull_hot_OpPR", 2: "k_pull_tiled_hotL1_OpPR"}[hot]
    traffic = recorded_traffic(kname, f"rmat{args.m_scale}")

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(hg, args.m_scale),
            "per_algorithm": {
                "pagerank": {"gteps": edges[0] / (per_alg_ms[0] * 1e-3) / 1e9, "ms": per_alg_ms[0] / steps},
                "pagerank_delta": {"gteps": edges[1] / (per_alg_ms[1] * 1e-3) / 1e9,
                                   "gteps_nominal": PRD_ITERS * m * steps / (per_alg_ms[1] * 1e-3) / 1e9,
                                   "ms": per_alg_ms[1] / steps},
                "cc": {"gteps": edges[2] / (per_alg_ms[2] * 1e-3) / 1e9, "ms": per_alg_ms[2] / steps}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": {0: "k_pull_tiled<OpPR> (PageRank DensePull iteration)",
                                    1: "k_hot_gather + k_pull_hot<OpPR> (PageRank DensePull iteration, hot sources "
                                       "in shared memory)",
                                    2: "k_hot_gather + k_pull_tiled<OpPR, hot L1> (PageRank DensePull iteration, hot "
                                       "sources kept in L1)"}[hot],
                         "bytes_model": "8m + 12n + 4 per launch (offsets, indices, one gathered contribution "
                                        "per arc, 1/outdeg, output vector)", "launches_timed": pr_launches,
                         "avg_launch_ms": avg_ms, "peak_kind": f"{peak_kind} hbm_gbs"},
            "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_total / args.e2e_steps, "steps": args.e2e_steps,
                    "form": "next step's graph loaded by a second host thread on its own stream under the "
                            "current step; first load and every copy in the timed region",
                    "serial_ms_per_step": statistics.median(serial_ms)},
            "gpu_launches": launches, "clocks": clocks,
            "autotuned": tuned, "pagerank_direction_gteps": compare, "selector": selector}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, iters, t = oracle_sample(hg, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                                "sample": f"oracle PageRank, {iters} iterations on the full graph ({t:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.free()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_only(args):
    """A small fixed case for profilers: one algorithm, default schedule, --steps runs."""
    import torch
    import graphgen as gg
    import paper_1805_00923_gb300 as gi
    torch.cuda.set_device(0)
    hg = gg.rmat_graph(args.scale, seed=1, weights=(1, 1000) if args.only == "sssp" else None)
    g = gi.Graph.from_host(hg)
    # BFS / SSSP source: --only-source, or the first of the BFS/SSSP workload's seeded sources when -1
    src = args.only_source if args.only_source >= 0 else int(gg.pick_sources(hg, 1, seed=1)[0])
    if args.only_direction == "learned":
        from paper_1805_00923_gb300 import selector as sel
        sel.install()
    for _ in range(args.steps):
        if args.only == "pagerank":
            gi.pagerank(g, DAMPING, PR_ITERS, sched=gi.schedule("dense_pull", hot_cache=args.hot_cache))
        elif args.only == "pagerank_delta":
            gi.pagerank_delta(g, DAMPING, PRD_EPS, PRD_ITERS, sched=gi.schedule("hybrid_pull", hot_cache=args.hot_cache))
        elif args.only == "cc":
            gi.cc(g)
        elif args.only == "bfs":
            gi.bfs(g, src, sched=gi.schedule(args.only_direction, persistent=args.only_persistent))
        elif args.only == "bc":
            gi.bc(g, int(gg.pick_sources(hg, 10, seed=1)[0]), sched=gi.schedule("hybrid_pull", rule="ligra"))
        else:
            gi.sssp(g, src, sched=gi.schedule(args.only_direction, delta=args.only_delta,
                                               persistent=args.only_persistent))
    torch.cuda.synchronize()
    print(json.dumps({"only": args.only, "scale": args.scale, "n": hg.n, "m": hg.m, "runs": args.steps, "source": src}))
    return 0


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def run_bc(args):
    """R-MAT scale --scale, single-source Betweenness Centrality from 10 sources
    (the paper averages BC over 10 starting points), per forward/backward schedule."""
    import time as _time
    import torch
    import graphgen as gg
    import oracle
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import selector as sel
    torch.cuda.set_device(0)
    sel.install()
    hg = gg.rmat_graph(args.m_scale, seed=1)
    g = gi.Graph.from_host(hg)
    srcs = [int(x) for x in gg.pick_sources(hg, 10, seed=1)]
    out = {}
    dep = torch.zeros(hg.n, dtype=torch.float64, device="cuda")
    for name, sc in [("hybrid_pull", gi.schedule("hybrid_pull")),
                     ("hybrid_pull_ligra", gi.schedule("hybrid_pull", rule="ligra")),
                     ("learned", gi.schedule("learned")),
                     ("sparse_push", gi.schedule("sparse_push")),
                     ("dense_pull", gi.schedule("dense_pull"))]:
        gi.bc(g, srcs[0], sched=sc, out=dep)
        a, b = _events()
        a.record()
        for s_ in srcs:
            gi.bc(g, s_, sched=sc, out=dep)
        b.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / len(srcs)
        out[name] = {"ms_per_source": ms, "gteps_nominal": hg.m / (ms * 1e-3) / 1e9}
    oracle.build()
    t0 = _time.perf_counter()
    oracle.bc(hg, srcs[0])
    cpu_ms = (_time.perf_counter() - t0) * 1e3
    best = min(out.values(), key=lambda r: r["ms_per_source"])
    print(json.dumps({"metric": METRIC, "workload": f"rmat{args.m_scale}_bc10", "value": out["hybrid_pull"]["gteps_nominal"],
                      "unit": "GTEPS", "n": hg.n, "m": hg.m, "sources": len(srcs), "results": out,
                      "best_ms_per_source": best["ms_per_source"],
                      "cpu_baseline": {"kind": "oracle", "cores": 1, "ms_per_source": cpu_ms,
                                       "sample": "oracle Brandes BC from the first source"},
                      "note": "nominal GTEPS = m / time per source; forward and backward applies per level"}))
    return 0


def _sssp_pull_bytes(n, m, tr, m_light=None):
    """Algorithmic bytes of the SSSP DensePull rounds of one traced query, per
    pull round 4(V+1) offsets + 8m' (index and frontier-folded distance per
    arc) + 8 m_f (weight and distance per source arc) + V/4 (bitmaps) +
    4|F_next|, where m' is the arcs the round scans: m for Bellman-Ford, the
    light or heavy arc count for a delta-stepping round (phase 0 / 1; then
    |F_next| is not recorded and the term is left out).  Returns (bytes,
    pull rounds, arcs the pull rounds scanned)."""
    import numpy as np
    t = tr.as_dict()
    fr, ed, dr = t["frontier"], t["edges"], t["direction"]
    ph = t.get("phase", np.zeros(len(dr), np.int32))
    total, rounds, arcs = 0, 0, 0
    for i in range(len(dr)):
        if dr[i] == 2:  # GI_DIR_DENSE_PULL
            if m_light is None:
                scanned = m
                nxt = int(fr[i + 1]) if i + 1 < len(fr) else 0
            else:
                if ed[i] == 0:  # sources without arcs of the class: nothing is launched
                    continue
                scanned = m_light if ph[i] == 0 else m - m_light
                nxt = 0
            total += 4 * (n + 1) + 8 * scanned + 8 * int(ed[i]) + n // 4 + 4 * nxt
            rounds += 1
            arcs += scanned
    return total, rounds, arcs


PULL_TRAFFIC_NOTE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, average over the 6 pull launches of one "
                     "query (source 16536593, width 128, host-driven, Ligra's rule)")


def host_cpu():
    """(nproc, CPU model name) of this host."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model Name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model


def oracle_queries(hg, queries, threads):
    """Run oracle BFS / SSSP queries [(algo, src)] on `threads` host threads
    (each oracle call is single-threaded C that releases the interpreter lock);
    returns (wall seconds, arcs = sum over queries of the reached vertices' degrees)."""
    import concurrent.futures as cf
    import numpy as np
    import oracle
    oracle.build()
    deg = np.diff(hg.row_ptr).astype(np.int64)

    def one(q):
        algo, s = q
        if algo == "bfs":
            d = oracle.bfs(hg, s)[0]
            return int(deg[d >= 0].sum())
        d = oracle.sssp(hg, s)[0]
        return int(deg[d < np.iinfo(np.int32).max].sum())

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=max(1, threads)) as ex:
        arcs = sum(ex.map(one, queries))
    return time.perf_counter() - t0, arcs


def l_config(hg, n_sources, delta=None):
    return {"workload": "rmat24_bfs_sssp", "graph": "R-MAT symmetrized, int32 weights uniform in [1,1000)",
            "scale": max(0, int(hg.n).bit_length() - 1), "edge_factor": 16, "abc": [0.57, 0.19, 0.19],
            "seed": 1, "n": hg.n, "m": hg.m, "sources": n_sources,
            "sources_rule": "uniform among vertices of degree >= 1, seeded (pick_sources seed 1)",
            "step": f"BFS (depth + canonical parent) then SSSP (distance) from each of the {n_sources} sources",
            "gteps_numerator": "per query the sum of degrees of the reached vertices (arcs of the reached "
                               "component, both directions); Graph500 count = half",
            "schedule": "learned selector per level / round (SparsePush / DensePush / DensePull); BFS and SSSP "
                        "level loops as CUDA graphs (gi_schedule.persistent = 2); SSSP by delta-stepping "
                        f"(bucket width {delta}, autotuned), BFS with canonical parents",
            "l2": "inputs larger than L2 (CSR + weights %.2f GB vs 126 MB L2); no flush"
                  % ((4 * (hg.n + 1) + 8 * hg.m) / 1e9)}


def run_config_l(args):
    """R-MAT scale 24 (weights [1,1000)), BFS + SSSP from 64 seeded sources:
    the timed step runs every source under the learned selector (level loops
    as CUDA graphs, SSSP by delta-stepping with the autotuned bucket width);
    the fixed rules (Beamer's for BFS, Ligra's |F| + m_f > m/20 for SSSP) on
    the same loops and the exhaustive per-level optimum are measured beside it."""
    import numpy as np
    import torch
    import torch.distributed as dist
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import graphgen as gg
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import selector as sel
    sel.install()
    hg = gg.rmat_graph(args.scale, seed=1, weights=(1, 1000))
    n, m = hg.n, hg.m
    g = gi.Graph.from_host(hg)
    # replicas: rank r serves its own 64 seeded sources (weak scaling)
    srcs = [int(x) for x in gg.pick_sources(hg, args.sources, seed=1 + rank)]
    depth = torch.empty(n, dtype=torch.int32, device="cuda")
    parent = torch.empty(n, dtype=torch.int32, device="cuda")
    dist_ = torch.empty(n, dtype=torch.int32, device="cuda")
    # SSSP schedule: the autotuner picks the bucket width and the other knobs
    # from the learned graph-driven start (untimed set-up; outputs checked)
    tune_budget = 1 if args.no_extras else args.tune_budget
    ss_learned, ss_tuned_ms, ss_start_ms = gi.autotune(
        g, "sssp", src=srcs[0], start=gi.schedule("learned", delta=args.delta, persistent=2), budget=tune_budget,
        seed=7)
    delta = int(ss_learned.delta)
    # the tuner's own gain: the same search from the library's default SSSP
    # schedule (Bellman-Ford rounds, learned, graph-driven), reported only
    tune_defaults = None
    if not args.no_extras:
        d_s, d_tuned, d_start = gi.autotune(g, "sssp", src=srcs[0], start=gi.schedule("learned", persistent=2),
                                            budget=2 * args.tune_budget, seed=7)
        tune_defaults = {"schedule": gi.schedule_dict(d_s), "tuned_ms": d_tuned, "start_ms": d_start}
    ss_rule = gi.schedule("hybrid_pull")
    for f, _ in ss_learned._fields_:
        setattr(ss_rule, f, getattr(ss_learned, f))
    ss_rule.direction = gi.GI_DIR_HYBRID_PULL
    # learned: the timed schedule; rule: the same loops and bucket width with
    # the fixed direction rules; fixed_heuristic: the paper's own schedule
    # (host-driven levels, Bellman-Ford rounds, Beamer's / Ligra's rule)
    pols = {"learned": (gi.schedule("learned", persistent=2), ss_learned),
            "rule": (gi.schedule("hybrid_pull", persistent=2), ss_rule),
            "fixed_heuristic": (gi.schedule("hybrid_pull"), gi.schedule("hybrid_pull"))}
    deg = torch.from_numpy(np.diff(hg.row_ptr).astype(np.int64)).cuda()
    # per-query GTEPS numerator: arcs of the reached component (BFS and SSSP
    # reach the same vertices: weights are positive), untimed
    reach = {}
    for s_ in srcs:
        gi.bfs(g, s_, want_parent=False, sched=pols["learned"][0], out=(depth, None))
        reach[s_] = int(deg[depth >= 0].sum())
    arcs_per_step = 2 * sum(reach.values())

    def one_pass(pol):
        bs, ss = pols[pol]
        for s_ in srcs:
            gi.bfs(g, s_, sched=bs, out=(depth, parent))
            gi.sssp(g, s_, sched=ss, out=dist_)
        return arcs_per_step

    for _ in range(args.warmup):
        one_pass("learned")
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    gi.stats_reset()
    start, stop = _events()
    start.record()
    for _ in range(args.steps):
        one_pass("learned")
    stop.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches, _, _ = gi.stats_read()
    clocks = sampler.stop()
    total_ms = start.elapsed_time(stop)
    if world > 1:
        from paper_1805_00923_gb300 import replicas
        total_ms = replicas.max_over_ranks(total_ms, device="cuda")
    value = world * args.steps * arcs_per_step / (total_ms * 1e-3) / 1e9

    # roofline of the dominant kernel, the SSSP DensePull rounds
    # (k_pull_tiled<OpMinInt / OpMinIntBounded>): kernels inside a CUDA graph cannot be timed one
    # by one, so the same 64 queries run once more with the same schedule
    # host-driven, every pull launch bracketed by CUDA events on its stream
    m_light = int((hg.wt < delta).sum()) if delta > 0 else None
    ss_host = gi.schedule("learned")
    for f, _ in ss_learned._fields_:
        setattr(ss_host, f, getattr(ss_learned, f))
    ss_host.persistent = 0
    traces = {s_: gi.Trace(4096) for s_ in srcs}
    for s_ in srcs[:2]:
        gi.sssp(g, s_, sched=ss_host, trace=traces[s_], out=dist_)
    torch.cuda.synchronize()
    gi.stats_reset()
    gi.stats_pull_arcs(g, reset=True)
    gi.stats_enable(True)
    a0, a1 = _events()
    a0.record()
    for s_ in srcs:
        gi.sssp(g, s_, sched=ss_host, trace=traces[s_], out=dist_)
    a1.record()
    torch.cuda.synchronize()
    gi.stats_enable(False)
    host_ms = a0.elapsed_time(a1) / len(srcs)
    _, pull_launches, pull_ms = gi.stats_read("min_pull")
    # the arcs the pulls gathered, counted by the library (a delta-stepping
    # pull skips the long rows at or below the round's least candidate), in
    # place of every arc of the class in the 8m' term
    gathered = gi.stats_pull_arcs(g, reset=True)
    pull_bytes, pull_rounds, class_arcs = 0, 0, 0
    for s_ in srcs:
        b_, r_, a_ = _sssp_pull_bytes(n, m, traces[s_], m_light)
        pull_bytes += b_
        pull_rounds += r_
        class_arcs += a_
    pull_bytes += 8 * (gathered - class_arcs)
    pull_arcs = gathered
    peak, peak_kind = measured_hbm()
    achieved = pull_bytes / (pull_ms * 1e-3) / 1e9 if pull_ms > 0 else 0.0
    # the second ceiling of a pull: one gathered 4-byte value per arc
    # (gi_gather_rate over this graph's source ids into an n-entry table)
    ceil = gather_ceiling(hg.col, n)
    pull_rate = pull_arcs / (pull_ms * 1e-3) if pull_ms > 0 else 0.0
    # DRAM traffic per launch from one ncu capture of this workload's pulls
    # (recorded with the kernel's source hash; null once the code changes)
    traffic = recorded_traffic("k_pull_tiled_OpMinInt_and_Bounded", f"rmat{args.scale}_delta{delta}",
                               op="OpMinInt+OpMinIntBounded")

    # learned vs rule per algorithm, 3 interleaved repeats each (outside the timed region)
    def per_alg(pol):
        bs, ss = pols[pol]
        a0, a1 = _events()
        b_ms = s_ms = 0.0
        for s_ in srcs:
            a0.record()
            gi.bfs(g, s_, sched=bs, out=(depth, parent))
            a1.record()
            torch.cuda.synchronize()
            b_ms += a0.elapsed_time(a1)
            a0.record()
            gi.sssp(g, s_, sched=ss, out=dist_)
            a1.record()
            torch.cuda.synchronize()
            s_ms += a0.elapsed_time(a1)
        half = arcs_per_step / 2
        return {"bfs_gteps": half / (b_ms * 1e-3) / 1e9, "sssp_gteps": half / (s_ms * 1e-3) / 1e9,
                "gteps": arcs_per_step / ((b_ms + s_ms) * 1e-3) / 1e9,
                "bfs_ms_per_query": b_ms / len(srcs), "sssp_ms_per_query": s_ms / len(srcs)}

    reps = {"learned": [], "rule": [], "fixed_heuristic": []}
    for _ in range(args.repeats):
        for pol in reps:
            reps[pol].append(per_alg(pol))
    compare = {}
    for pol, rs in reps.items():
        d = {}
        for k in rs[0]:
            vals = [r[k] for r in rs]
            d[k] = {"mean": float(np.mean(vals)), "min": float(np.min(vals)), "max": float(np.max(vals))}
        compare[pol] = d
    beats = {f"{k}_over_{other}": compare["learned"][k]["min"] > compare[other][k]["max"]
             for other in ("rule", "fixed_heuristic") for k in ("bfs_gteps", "sssp_gteps", "gteps")}
    # other forms of the same queries (one pass each): host-driven level loops,
    # and Bellman-Ford's synchronous rounds (the paper's SSSP)
    forms = {}
    for name, bs, ss in (("host_driven_learned", gi.schedule("learned"), ss_host),
                         ("bellman_ford_graph_driven_learned", None, gi.schedule("learned", persistent=2)),
                         ("bellman_ford_host_driven_learned", None, gi.schedule("learned"))):
        a0, a1 = _events()
        a0.record()
        for s_ in srcs[:16]:
            if bs is not None:
                gi.bfs(g, s_, sched=bs, out=(depth, parent))
            gi.sssp(g, s_, sched=ss, out=dist_)
        a1.record()
        torch.cuda.synchronize()
        forms[name] = {"ms_per_query_pair" if bs is not None else "sssp_ms_per_query": a0.elapsed_time(a1) / 16}
    # exhaustive best direction per level / round: each timed alone from the
    # same state (gi_selector_profile), minima summed
    nx = max(1, min(len(srcs), args.exhaustive_sources))
    ex_ms = {"bfs": 0.0, "sssp": 0.0}
    # the same per-level times summed over the direction each policy picks
    # (its host-driven trace: the levels and rounds do not depend on the
    # directions), so that the policies' direction choices compare without
    # their loop overheads
    replay = {a: {"learned": 0.0, "rule": 0.0, "levels": 0, "unmatched": 0} for a in ("bfs", "sssp")}

    def chosen(algo, t, pol):
        tr = gi.Trace(1 << 14)
        if algo == "bfs":
            gi.bfs(g, s_, want_parent=False, sched=gi.schedule(pol), trace=tr)
        else:
            gi.sssp(g, s_, sched=gi.schedule(pol, delta=delta), trace=tr, out=dist_)
        torch.cuda.synchronize()
        d = tr.as_dict()["direction"]
        k = min(len(t), len(d))
        replay[algo]["unmatched"] += abs(len(t) - len(d))
        return float(sum(t[i, int(d[i])] for i in range(k)))

    for s_ in srcs[:nx]:
        _, t = sel.profile(g, gi.GI_K_BFS, s_)
        ex_ms["bfs"] += float(t.min(axis=1).sum())
        for pol, name in (("learned", "learned"), ("hybrid_pull", "rule")):
            replay["bfs"][name] += chosen("bfs", t, pol)
        replay["bfs"]["levels"] += len(t)
        _, t = sel.profile(g, gi.GI_K_SSSP, s_, sched=gi.schedule("hybrid_pull", delta=delta))
        ex_ms["sssp"] += float(np.where(t > 0, t, np.inf).min(axis=1).sum())
        for pol, name in (("learned", "learned"), ("hybrid_pull", "rule")):
            replay["sssp"][name] += chosen("sssp", t, pol)
        replay["sssp"]["levels"] += len(t)
    for a in replay:
        for k in ("learned", "rule"):
            replay[a][k] /= nx
        replay[a]["best"] = ex_ms[a] / nx
    exhaustive = {"sources": nx, "bfs_ms_per_query": ex_ms["bfs"] / nx, "sssp_ms_per_query": ex_ms["sssp"] / nx,
                  "policies_replayed_ms_per_query": replay,
                  "note": "sum over levels (rounds) of the fastest direction timed alone, without the per-level "
                          "statistics kernel and loop control; BFS without parents.  policies_replayed: the same "
                          "per-level times summed over each policy's own choices"}

    # end to end through the C ABI: CSR + weights from pinned host buffers
    # (gi_load_csr), every query's depth, parent and distance copied back to
    # pinned host memory on a side stream as soon as the query ends
    rp_h = torch.from_numpy(hg.row_ptr).pin_memory()
    col_h = torch.from_numpy(hg.col).pin_memory()
    wt_h = torch.from_numpy(hg.wt).pin_memory()
    slots = 8
    out_h = [[torch.empty(n, dtype=torch.int32).pin_memory() for _ in range(3)] for _ in range(slots)]
    side = torch.cuda.Stream()
    dev_out = [[torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)] for _ in range(slots)]
    slot_free = [None] * slots
    h2d = 4 * (n + 1) + 8 * m
    d2h = len(srcs) * 3 * 4 * n

    bs_l, ss_l = pols["learned"]
    load_stream = torch.cuda.Stream()
    dev = torch.cuda.current_device()

    def load_graph(box):
        # gi_load_csr from the pinned host buffers, then the schedule's per-graph
        # set-up (delta-stepping split, CUDA-graph loops) built ahead of the
        # queries (gi_prepare), on their own stream
        torch.cuda.set_device(dev)
        ge = gi.Graph(rp_h.numpy(), col_h.numpy(), wt_h.numpy(), symmetric=True, stream=load_stream)
        gi.prepare(ge, "bfs", bs_l, stream=load_stream)
        gi.prepare(ge, "sssp", ss_l, stream=load_stream)
        box["g"] = ge

    def queries(ge):
        for i, s_ in enumerate(srcs):
            k = i % slots
            if slot_free[k] is not None:
                slot_free[k].synchronize()  # the host has the slot's previous results
            dd, pp, ds = dev_out[k]
            gi.bfs(ge, s_, sched=bs_l, out=(dd, pp))
            gi.sssp(ge, s_, sched=ss_l, out=ds)
            done = torch.cuda.Event()
            done.record()
            side.wait_event(done)
            with torch.cuda.stream(side):
                for j in range(3):
                    out_h[k][j].copy_(dev_out[k][j], non_blocking=True)
                ev = torch.cuda.Event()
                ev.record()
            slot_free[k] = ev
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.current_stream().synchronize()

    def e2e_run(K):
        # like a data loader: a second host thread loads step k+1's graph (and
        # its set-up) while step k's queries run; the first load, every copy in
        # and every result copy out lie inside the timed region
        box = {}
        load_graph(box)
        for k in range(K):
            ge, box = box["g"], {}
            th = threading.Thread(target=load_graph, args=(box,)) if k + 1 < K else None
            if th:
                th.start()
            queries(ge)
            if th:
                th.join()
            ge.free()

    e2e_run(1)  # warm-up (allocator pool, pinned slabs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(args.e2e_steps)
    e2e_s = time.perf_counter() - t0
    if world > 1:
        from paper_1805_00923_gb300 import replicas
        e2e_s = replicas.max_over_ranks(e2e_s, device="cuda")
    e2e_value = world * args.e2e_steps * arcs_per_step / e2e_s / 1e9

    line = {"metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": l_config(hg, len(srcs), delta),
            "per_algorithm": {"learned": compare["learned"], "rule": compare["rule"],
                              "fixed_heuristic": compare["fixed_heuristic"], "repeats": args.repeats,
                              "learned_beats_beyond_spread": beats, "other_forms": forms,
                              "exhaustive_best_per_level": exhaustive, "gteps_graph500": value / 2,
                              "sssp_autotune": {"schedule": gi.schedule_dict(ss_learned), "tuned_ms": ss_tuned_ms,
                                                "start_ms": ss_start_ms, "source": srcs[0],
                                                "from_library_defaults": tune_defaults}},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_pull_tiled<OpMinInt> (light rounds) / <OpMinIntBounded> (heavy rounds): SSSP "
                                   "delta-stepping DensePull over the row-compacted light / heavy arcs, frontier "
                                   "folded into the gathered start-of-round distances; heavy rounds skip the rows at "
                                   "or below the bucket's end",
                         "bytes_model": "per pull round 4(V+1) + 8m' + 8 m_f + V/4, m' = the arcs the round's pull "
                                        "gathered (library counter: the class's arcs less the long rows its bound "
                                        "filter skipped)",
                         "arcs_gathered": gathered, "arcs_of_the_classes": class_arcs,
                         "timed_in": "the same 64 SSSP queries with the same schedule run host-driven after the "
                                     "timed region, every pull launch bracketed by CUDA events on its stream "
                                     f"({host_ms:.2f} ms per query)",
                         "launches_timed": pull_launches, "pull_rounds_expected": pull_rounds,
                         "avg_launch_ms": pull_ms / max(pull_launches, 1),
                         "peak_kind": f"{peak_kind} hbm_gbs (burst copy)",
                         "traffic_from": PULL_TRAFFIC_NOTE if traffic is not None else None,
                         "gather_ceiling": ceil, "pull_gathers_per_s": pull_rate,
                         "frac_of_gather_ceiling_graph_ids": pull_rate / ceil["graph_ids"]["gathers_per_s"]},
            "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * e2e_s / args.e2e_steps, "steps": args.e2e_steps,
                    "form": "per step gi_load_csr from pinned host CSR + weights and gi_prepare (the schedule's "
                            "per-graph set-up), then the 64 BFS + SSSP queries; each query's depth, parent and "
                            "distance copied to pinned host memory on a side stream (8 result slots reused once the "
                            "host has them); step k+1's load and set-up run in a second host thread on their own "
                            "stream under step k's queries; from the first load on, everything is timed"},
            "gpu_launches": launches, "clocks": clocks}
    if not args.no_extras:
        line["config_m_pr_prd_cc"] = run_rmat22(args, extra=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nq = min(args.cpu_sources, len(srcs))
        qs = [(a_, s_) for s_ in srcs[:nq] for a_ in ("bfs", "sssp")]
        secs, arcs = oracle_queries(hg, qs, len(qs))
        cores, model = host_cpu()
        line["cpu_baseline"] = {"value": arcs / secs / 1e9, "unit": "GTEPS", "cores": len(qs), "kind": "oracle",
                                "sample": f"oracle BFS (depth + parent) and SSSP from {nq} of the {len(srcs)} "
                                          f"sources, each query single-threaded, {len(qs)} queries on {len(qs)} "
                                          f"threads at once ({secs:.1f} s wall)",
                                "host": {"nproc": cores, "model": model,
                                         "used": f"{len(qs)} of {cores} cores"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.free()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def gather_ceiling(col, n, reps=5):
    """Gathers per second of gi_gather_rate (the two memory streams of a pull and
    nothing else) over the graph's own source ids and over uniform random ids
    of the same count, both into an n-float table; best of `reps` launches."""
    import torch
    import paper_1805_00923_gb300 as gi
    idx = torch.from_numpy(col).cuda()
    rnd = torch.randint(0, n, (idx.numel(),), dtype=torch.int32, device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(5))
    table = torch.rand(n, dtype=torch.float32, device="cuda")
    out = {}
    for name, ids in (("graph_ids", idx), ("uniform_random_ids", rnd)):
        best = 1e30
        for _ in range(reps + 1):
            a, b = _events()
            a.record()
            gi.gather_rate(ids, table)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        out[name] = {"gathers_per_s": ids.numel() / (best * 1e-3), "ms": best}
    del idx, rnd, table
    return out


def rmat22_summary(args, hg, g, steps, value, total_ms, per_alg_ms, edges, launches, pr_launches, pr_ms, pr_s,
                   tuned, clocks):
    """The config-M step's numbers, for embedding in the BFS/SSSP line."""
    import paper_1805_00923_gb300 as gi
    m, n = hg.m, hg.n
    peak, peak_kind = measured_hbm()
    avg_ms = pr_ms / max(pr_launches, 1)
    achieved = (8 * m + 12 * n + 4) / (avg_ms * 1e-3) / 1e9
    ceil = gather_ceiling(hg.col, n)
    pull_rate = m / (avg_ms * 1e-3)
    hot = int(pr_s.hot_cache) if pr_s.direction == gi.GI_DIR_DENSE_PULL and pr_s.num_segments == 1 else 0
    kname = {0: "k_pull_tiled_OpPR", 1: "k_pull_hot_OpPR", 2: "k_pull_tiled_hotL1_OpPR"}[hot]
    out = {"workload": workload_config(hg, args.m_scale), "value": value, "unit": "GTEPS", "steps": steps,
           "ms_per_step": total_ms / steps,
           "per_algorithm": {
               "pagerank": {"gteps": edges[0] / (per_alg_ms[0] * 1e-3) / 1e9, "ms": per_alg_ms[0] / steps},
               "pagerank_delta": {"gteps": edges[1] / (per_alg_ms[1] * 1e-3) / 1e9,
                                  "gteps_nominal": PRD_ITERS * m * steps / (per_alg_ms[1] * 1e-3) / 1e9,
                                  "ms": per_alg_ms[1] / steps},
               "cc": {"gteps": edges[2] / (per_alg_ms[2] * 1e-3) / 1e9, "ms": per_alg_ms[2] / steps}},
           "numerators": "PR 20m; PRD m per pull round + m_f per push round; CC m (every vertex reached)",
           "roofline_pr_pull": {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                                "kernel": kname, "traffic": recorded_traffic(kname, f"rmat{args.m_scale}"),
                                "bytes_model": "8m + 12n + 4 per launch", "avg_launch_ms": avg_ms,
                                "launches_timed": pr_launches, "peak_kind": f"{peak_kind} hbm_gbs",
                                "gather_ceiling": ceil, "pull_gathers_per_s": pull_rate,
                                "frac_of_gather_ceiling_graph_ids": pull_rate / ceil["graph_ids"]["gathers_per_s"]},
           "autotuned": tuned, "gpu_launches": launches, "clocks": clocks}
    g.free()
    return out


def _bfs_level_bytes(depth, col, row, row_ptr, deg, levels):
    """Per BFS level d (frontier = depth d): |F|, m_f, |F_next|, n_u and the
    arcs an early-exit pull scans (E_scanned: for each vertex not yet reached,
    its in-arcs up to and including the first one from the frontier, all of
    them if none), from the run's own depths; measurement plumbing in torch."""
    import torch
    m = col.numel()
    local = torch.arange(m, device=col.device, dtype=torch.int32) - row_ptr[row.long()]  # position in the row
    dsrc = depth[col.long()]
    out = []
    for d in range(levels):
        front = depth == d
        unv = (depth > d) | (depth < 0)
        first = deg.clone()
        hit = dsrc == d
        first.scatter_reduce_(0, row[hit].long(), local[hit] + 1, reduce="amin", include_self=True)
        out.append(dict(frontier=int(front.sum()), m_f=int(deg[front].sum()), next=int((depth == d + 1).sum()),
                        n_u=int(unv.sum()), e_scanned=int(first[unv].sum())))
    return out


def run_levels(args):
    """R-MAT scale 24: every BFS level and SSSP round from one source, each of
    SparsePush / DensePush / DensePull timed alone from the same state
    (gi_selector_profile), with the algorithmic bytes of that direction at that
    level and the bandwidth they imply against the measured copy peak."""
    import numpy as np
    import torch
    import graphgen as gg
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import selector as sel
    torch.cuda.set_device(0)
    hg = gg.rmat_graph(24, seed=1, weights=(1, 1000))
    n, m = hg.n, hg.m
    g = gi.Graph.from_host(hg)
    src = int(gg.pick_sources(hg, 1, seed=1)[0])
    peak, peak_kind = measured_hbm()
    deg = torch.from_numpy(np.diff(hg.row_ptr).astype(np.int32)).cuda()
    col = torch.from_numpy(hg.col).cuda()
    row_ptr = torch.from_numpy(hg.row_ptr).cuda()
    row = torch.repeat_interleave(torch.arange(n, device="cuda", dtype=torch.int32), deg.long(), output_size=m)
    names = ("sparse_push", "dense_push", "dense_pull")

    def rows(t, bytes_of):
        res = []
        for i in range(t.shape[0]):
            b = bytes_of(i)
            r = {"level": i}
            r.update(b["sizes"])
            for j, nm in enumerate(names):
                ms = float(t[i, j])
                gbs = b[nm] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
                r[nm] = {"ms": ms, "bytes": b[nm], "gbs": gbs, "frac": gbs / peak}
            res.append(r)
        return res

    depth, _ = gi.bfs(g, src, want_parent=False)
    _, tb = sel.profile(g, gi.GI_K_BFS, src)
    # the same levels with the pull walking every vertex instead of the
    # compacted list of unvisited vertices with in-arcs (gi_schedule.dst_list)
    _, tb0 = sel.profile(g, gi.GI_K_BFS, src, sched=gi.schedule("hybrid_pull", dst_list=0))
    lv = _bfs_level_bytes(depth, col, row, row_ptr, deg, tb.shape[0])
    has_arcs = deg > 0
    for i in range(tb.shape[0]):
        lv[i]["n_u_live"] = int((((depth > i) | (depth < 0)) & has_arcs).sum())

    def bfs_bytes(i):
        x = lv[i]
        push = 12 * x["frontier"] + 8 * x["m_f"] + 8 * x["next"]
        pull = 4 * (x["n_u"] + 1) + 8 * x["e_scanned"] + n // 4 + 8 * x["next"]
        return {"sizes": x, "sparse_push": push, "dense_push": push + n // 8, "dense_pull": pull}

    tr = gi.Trace(1 << 14)
    gi.sssp(g, src, trace=tr)
    d = tr.as_dict()
    _, ts = sel.profile(g, gi.GI_K_SSSP, src)

    def sssp_bytes(i):
        f, mf = int(d["frontier"][i]), int(d["edges"][i])
        nxt = int(d["frontier"][i + 1]) if i + 1 < len(d["frontier"]) else 0
        push = 12 * f + 12 * mf + 8 * nxt
        pull = 4 * (n + 1) + 8 * m + 8 * mf + n // 4 + 4 * nxt
        return {"sizes": {"frontier": f, "m_f": mf, "next": nxt}, "sparse_push": push, "dense_push": push + n // 8,
                "dense_pull": pull}

    bfs_rows = rows(tb, bfs_bytes)
    for r, t0 in zip(bfs_rows, tb0[:, 2]):
        ms = float(t0)
        b = r["dense_pull"]["bytes"]
        gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        r["dense_pull_all_vertices"] = {"ms": ms, "bytes": b, "gbs": gbs, "frac": gbs / peak}
    sssp_rows = rows(ts[:len(d["frontier"])], sssp_bytes)

    def best(rs):
        return max((r[nm]["frac"], r["level"], nm) for r in rs for nm in names)

    print(json.dumps({"metric": METRIC, "workload": "rmat24_levels", "n": n, "m": m, "source": src,
                      "peak_gbs": peak, "peak_kind": peak_kind, "bfs_levels": bfs_rows, "sssp_rounds": sssp_rows,
                      "best_frac": {"bfs": best(bfs_rows), "sssp": best(sssp_rows)},
                      "bytes_model": {
                          "sparse_push": "12|F| + 8 m_f + 8|F_next| (BFS; SSSP adds 4 m_f of weights)",
                          "dense_push": "sparse_push + V/8 (bitmap scan)",
                          "dense_pull_bfs": "4(n_u + 1) + 8 E_scanned + V/4 + 8|F_next|",
                          "dense_pull_sssp": "4(V + 1) + 8m + 8 m_f + V/4 + 4|F_next|"}}))
    return 0


def run_grid4096(args):
    """4096x4096 grid, BFS + SSSP from --sources sources: host-driven drivers vs the batched engine."""
    import numpy as np
    import torch
    import graphgen as gg
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import selector as sel
    torch.cuda.set_device(0)
    sel.install()
    hg = gg.grid_graph(4096, seed=1, weights=(1, 100))
    g = gi.Graph.from_host(hg)
    srcs = gg.pick_sources(hg, args.sources, seed=1)
    out = {}
    for algo in ("bfs", "sssp"):
        t0 = time.perf_counter()
        for s_ in srcs[:2]:
            if algo == "bfs":
                gi.bfs(g, int(s_), want_parent=False, sched=gi.schedule("learned"))
            else:
                gi.sssp(g, int(s_), sched=gi.schedule("learned"))
        torch.cuda.synchronize()
        host_ms = (time.perf_counter() - t0) * 1e3 / 2
        # the same queries as single calls in the whole-GPU persistent mode
        pers = gi.schedule("learned", persistent=1)
        a, b = _events()
        a.record()
        for s_ in srcs[:4]:
            if algo == "bfs":
                gi.bfs(g, int(s_), want_parent=False, sched=pers)
            else:
                gi.sssp(g, int(s_), sched=pers)
        b.record()
        torch.cuda.synchronize()
        pers_ms = a.elapsed_time(b) / 4
        # the level loop as a CUDA graph (BFS; SSSP by delta-stepping at
        # bucket widths of 1x, 2x and 4x the mean weight, and Bellman-Ford)
        graph = {}
        for name, gsc in ((("rule", gi.schedule("hybrid_pull", persistent=2)),
                           ("learned", gi.schedule("learned", persistent=2))) if algo == "bfs" else
                          tuple((f"delta{d}_learned", gi.schedule("learned", persistent=2, delta=d))
                                for d in (50, 100, 200))):
            run = (lambda s_: gi.bfs(g, int(s_), want_parent=False, sched=gsc)) if algo == "bfs" \
                else (lambda s_: gi.sssp(g, int(s_), sched=gsc))
            run(srcs[0])
            a, b = _events()
            a.record()
            for s_ in srcs[:4]:
                run(s_)
            b.record()
            torch.cuda.synchronize()
            graph[name] = a.elapsed_time(b) / 4
        graph_ms = graph
        qs = [(0, int(s_), algo) for s_ in srcs]
        plan = gi.BatchPlan([g], qs, opts=gi.batch_opts(cluster_size=8, selector="learned"))
        plan.launch()
        plan.results()
        a, b = _events()
        a.record()
        plan.launch()
        b.record()
        torch.cuda.synchronize()
        res, ns, lev = plan.results()
        plan.free()
        bms = a.elapsed_time(b)
        out[algo] = {"host_driven_ms_per_query": host_ms, "persistent_ms_per_query": pers_ms,
                     "graph_driven_ms_per_query": graph_ms, "batch_ms_total": bms,
                     "batch_gteps_nominal": len(qs) * hg.m / (bms * 1e-3) / 1e9,
                     "p50_ms": float(np.percentile(ns, 50) / 1e6), "p99_ms": float(np.percentile(ns, 99) / 1e6),
                     "levels_mean": float(lev.mean())}
    val = sum(out[a]["batch_gteps_nominal"] for a in out) / 2
    print(json.dumps({"metric": METRIC, "workload": "grid4096_bfs_sssp", "value": val, "unit": "GTEPS",
                      "n": hg.n, "m": hg.m, "sources": len(srcs), "results": out,
                      "note": "nominal GTEPS = queries * m / time"}))
    return 0


def run_batch512(args):
    """32 graphs (16 R-MAT scale 12-20, ef 8-32; 16 grids 256-2048), 512 BFS/SSSP
    queries in one launch per GPU.  With N ranks the queries are dealt by
    graph size (replicas.shard_balanced) and every rank holds the graphs; the
    time is the slowest rank's, latencies gather on rank 0.  Also the batch
    autotuner's options against the defaults, at identical outputs."""
    import numpy as np
    import torch
    import torch.distributed as dist
    import graphgen as gg
    import paper_1805_00923_gb300 as gi
    from paper_1805_00923_gb300 import replicas
    from paper_1805_00923_gb300 import selector as sel
    world, rank, local = dist_setup()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    sel.install()
    rng = np.random.default_rng(1)
    hgs = [gg.rmat_graph(int(rng.integers(12, 21)), int(rng.choice([8, 16, 32])), seed=100 + i, weights=(1, 1000))
           for i in range(16)]
    hgs += [gg.grid_graph(int(rng.choice([256, 512, 1024, 2048])), seed=200 + i, weights=(1, 1000))
            for i in range(16)]
    gs = [gi.Graph.from_host(h) for h in hgs]
    qs_all = []
    for i in range(512):
        k = int(rng.integers(0, 32))
        qs_all.append((k, int(gg.pick_sources(hgs[k], 1, seed=1000 + i)[0]), "bfs" if i % 2 == 0 else "sssp"))
    mine = replicas.shard_balanced([hgs[q[0]].n for q in qs_all], rank, world) if world > 1 else list(range(512))
    qs = [qs_all[i] for i in mine]
    edges = sum(hgs[q[0]].m for q in qs_all)

    def timed(opts):
        plan = gi.BatchPlan(gs, qs, opts=opts)
        plan.launch()
        plan.results()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = _events()
        a.record()
        plan.launch()
        b.record()
        torch.cuda.synchronize()
        res, ns, lev = plan.results()
        ms = a.elapsed_time(b)
        plan.free()
        ms_all = replicas.max_over_ranks(ms, device="cuda") if world > 1 else ms
        ns_all = np.concatenate(replicas.gather_objects(ns)) if world > 1 else ns
        return ms_all, ns_all

    out = {}
    for cs, order in ((2, 1), (4, 1), (4, 0), (8, 1)):
        ms, ns = timed(gi.batch_opts(cluster_size=cs, selector="learned", order=order))
        out[f"cluster{cs}" + ("" if order == 1 else "_as_given")] = {
            "ms": ms, "gteps_nominal": edges / (ms * 1e-3) / 1e9,
            "p50_ms": float(np.percentile(ns, 50) / 1e6), "p99_ms": float(np.percentile(ns, 99) / 1e6)}
    # the batch autotuner on this rank's queries (untimed search; outputs checked)
    start = gi.batch_opts(cluster_size=4, selector="learned")
    best, best_ms, start_ms = gi.batch_autotune(gs, qs, start=start, budget=args.tune_budget, seed=11)
    ms, ns = timed(best)
    out["autotuned"] = {"ms": ms, "gteps_nominal": edges / (ms * 1e-3) / 1e9,
                        "p50_ms": float(np.percentile(ns, 50) / 1e6), "p99_ms": float(np.percentile(ns, 99) / 1e6),
                        "options": {f: getattr(best, f) for f in ("cluster_size", "t_warp", "t_cta", "sssp_delta",
                                                                  "order")},
                        "search_best_ms": best_ms, "search_start_ms": start_ms}
    best_row = max((v for k, v in out.items()), key=lambda r: r["gteps_nominal"])
    if rank == 0:
        print(json.dumps({"metric": METRIC, "workload": "batch512", "value": best_row["gteps_nominal"],
                          "unit": "GTEPS", "graphs": 32, "queries": 512, "n_gpus": world,
                          "sharding": "queries dealt by graph size over the ranks (each rank holds every graph)"
                          if world > 1 else None, "results": out,
                          "note": "nominal GTEPS = sum over queries of the graph's m / time (slowest rank)"}))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.only:
        return run_only(args)
    if args.impl == "reference":
        return run_reference(args)
    return {"rmat24_bfs_sssp": run_config_l, "rmat22": run_rmat22, "rmat24_levels": run_levels,
            "grid4096": run_grid4096, "batch512": run_batch512, "bc": run_bc}[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
