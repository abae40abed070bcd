"""Replica helpers under torch.distributed with the gloo backend on CPU, world size 2:
sharding covers every query exactly once, the timing reduction takes the
maximum, and each rank's independent results gather back in rank order."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1805_00923_gb300 import replicas
    import graphgen as gg
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_q = 11
        mine = list(replicas.shard(n_q, rank, world))
        # each rank answers its own BFS queries on its own replica of the graph
        hg = gg.rmat_graph(10, seed=3)
        srcs = gg.pick_sources(hg, n_q, seed=5)
        answers = {i: int(oracle.bfs(hg, int(srcs[i]))[0].max()) for i in mine}
        everyone = replicas.gather_objects(answers)
        t = replicas.max_over_ranks(1.5 + rank)
        s = replicas.sum_over_ranks(len(mine))
        q.put((rank, mine, everyone, t, s))
    finally:
        dist.destroy_process_group()


def test_replicas_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, e0, t0, s0), (r1, m1, e1, t1, s1) = out
    assert sorted(m0 + m1) == list(range(11)) and not set(m0) & set(m1)
    assert t0 == t1 == 2.5 and s0 == s1 == 11
    merged = {k: v for d in e0 for k, v in d.items()}
    assert sorted(merged) == list(range(11)) and e0 == e1


def _batch_worker(rank, world, port, q):
    """The sharded batched path of bench.py --workload batch512 with its GPU
    launch replaced by the oracle: queries dealt by cost, each rank answers
    its share and times it, latencies and answers gather on every rank."""
    sys.path.insert(0, ROOT)
    import time
    import numpy as np
    import torch.distributed as dist
    from paper_1805_00923_gb300 import replicas
    import graphgen as gg
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        hgs = [gg.rmat_graph(9, seed=11), gg.rmat_graph(11, seed=12, weights=(1, 1000)), gg.grid_graph(40, seed=13)]
        rng = np.random.default_rng(3)
        qs = [(int(k), int(rng.integers(0, hgs[k].n)), "bfs" if i % 2 == 0 else "sssp")
              for i, k in enumerate(rng.integers(0, 3, 40))]
        qs = [(k, s, "bfs" if hgs[k].wt is None else a) for k, s, a in qs]
        mine = replicas.shard_balanced([hgs[k].m for k, _, _ in qs], rank, world)
        t0 = time.perf_counter()
        res, lat = {}, {}
        for i in mine:
            k, s, a = qs[i]
            t1 = time.perf_counter()
            res[i] = int((oracle.bfs(hgs[k], s)[0] if a == "bfs" else oracle.sssp(hgs[k], s)[0]).sum())
            lat[i] = time.perf_counter() - t1
        total = replicas.max_over_ranks(time.perf_counter() - t0)
        allres = replicas.gather_objects(res)
        q.put((rank, mine, allres, total, [hgs[k].m for k, _, _ in qs]))
    finally:
        dist.destroy_process_group()


def test_sharded_batch_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, m0, a0, t0, costs), (_, m1, a1, t1, _) = out
    assert sorted(m0 + m1) == list(range(40)) and not set(m0) & set(m1)
    assert t0 == t1 > 0
    merged = {k: v for d in a0 for k, v in d.items()}
    assert sorted(merged) == list(range(40)) and a0 == a1
    # dealt longest first: the two loads differ by at most the largest cost
    l0, l1 = sum(costs[i] for i in m0), sum(costs[i] for i in m1)
    assert abs(l0 - l1) <= max(costs)


@pytest.mark.parametrize("n,w", [(0, 3), (5, 8), (17, 4), (100, 7)])
def test_shard_balanced_partition(n, w):
    from paper_1805_00923_gb300 import replicas
    costs = [(7 * i) % 13 + 1 for i in range(n)]
    parts = [replicas.shard_balanced(costs, r, w) for r in range(w)]
    assert sorted(sum(parts, [])) == list(range(n))
    loads = [sum(costs[i] for i in p) for p in parts]
    assert n == 0 or max(loads) - min(loads) <= max(costs)


@pytest.mark.parametrize("n,w", [(0, 3), (5, 8), (17, 4), (100, 7)])
def test_shard_partition(n, w):
    from paper_1805_00923_gb300 import replicas
    parts = [list(replicas.shard(n, r, w)) for r in range(w)]
    assert sum(parts, []) == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
