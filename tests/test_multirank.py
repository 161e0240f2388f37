"""Multi-rank host logic on CPU (gloo, world size 2): replicas shard the
problems without overlap or loss, and the job time is the slowest rank's."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1603_03142_gb300 import replicas


def test_shard_partitions_and_balances():
    costs = [replicas.nest_cost(n, L) for n, L in [(128, 1), (1024, 4), (256, 2), (512, 3), (1024, 1), (128, 4)]]
    parts = [replicas.shard_by_cost(costs, r, 3) for r in range(3)]
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(len(costs)))
    loads = [sum(costs[k] for k in p) for p in parts]
    assert max(loads) <= sum(costs) / 3 + max(costs)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.shard_by_cost([5, 1, 3, 2, 4], rank, world)
        t = replicas.max_over_ranks(10.0 * (rank + 1))
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, t, gathered))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, gathered in out:
        assert t == 20.0  # slowest rank
        assert sorted(gathered[0] + gathered[1]) == [0, 1, 2, 3, 4]
        assert not set(gathered[0]) & set(gathered[1])
