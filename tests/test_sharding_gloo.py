"""Multi-rank element assignment, exercised with 2 gloo ranks on the CPU.

Each rank computes its own share of an uneven element list; an all_gather
over gloo checks that the shares are disjoint, cover every element and
balance the estimated cost to within one element's cost.
"""

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1506_08147_gb300 import sharding

DESCS = [dict(n=n, m=m) for n, m in [((24, 24, 24), 24), ((32, 32, 32), 48), ((40, 40, 48), 72),
                                      ((48, 48, 64), 120), ((24, 24, 24), 16), ((48, 64, 40), 48),
                                      ((32, 32, 32), 32), ((40, 40, 48), 96), ((48, 64, 40), 48)]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.my_elements(DESCS, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    if rank == 0:
        out.put(gathered)
    dist.destroy_process_group()


def test_partition_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    shares = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    flat = sorted(i for s in shares for i in s)
    assert flat == list(range(len(DESCS)))
    costs = [sharding.element_cost(d["n"], d["m"]) for d in DESCS]
    loads = [sum(costs[i] for i in s) for s in shares]
    assert max(loads) - min(loads) <= max(costs)


def test_partition_single_rank_and_errors():
    assert sharding.partition([3.0, 1.0, 2.0], 1) == [[0, 1, 2]]
    assert sharding.partition([], 3) == [[], [], []]
    with pytest.raises(ValueError):
        sharding.partition([1.0], 0)


def test_bench_workload_split_two_ranks():
    """bench.py at 2 ranks: two monolayer replicas, each rank a disjoint half
    of their 2 x k elements, replica 0 identical to the 1-rank workload."""
    import bench
    one, _ = bench.workload(2, 0, 1)
    r0, _ = bench.workload(2, 0, 2)
    r1, _ = bench.workload(2, 1, 2)
    keys0 = {e.seed_key for e in r0}
    keys1 = {e.seed_key for e in r1}
    assert not keys0 & keys1
    assert len(keys0) == len(keys1) == 2
    assert {e.seed_key for e in one} <= keys0 | keys1
    assert len(keys0 | keys1) == 4
