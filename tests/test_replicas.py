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


@pytest.mark.parametrize("n,w", [(0, 3), (5, 8), (17, 4), (100, 7)])
def test_shard_partition(n, w):
    from paper_1805_00923_gb300 import replicas
    parts = [list(replicas.shard(n, r, w)) for r in range(w)]
    assert sum(parts, []) == list(range(n))
    assert max(map(len, parts)) - min(map(len, parts)) <= 1
