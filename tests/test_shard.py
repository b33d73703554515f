"""Batched form over several ranks: LPT partition and the host gather (gloo, CPU)."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2208_01907_gb300.shard import estimated_cost, lpt_partition, run_sharded


def test_lpt_partition_properties():
    costs = [estimated_cost(L) for L in (60000, 2000, 31000, 45000, 5000, 59000, 12000, 2500, 40000)]
    parts = lpt_partition(costs, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))                       # every system exactly once
    loads = [sum(costs[i] for i in p) for p in parts]
    # greedy LPT bound: max load <= 4/3 of the optimum, hence <= 4/3 * (mean + max item)
    assert max(loads) <= (4.0 / 3.0) * max(sum(costs) / 3, max(costs)) + 1e-9
    assert lpt_partition(costs, 3) == parts                       # deterministic
    assert lpt_partition(costs, 1) == [list(range(len(costs)))]
    with pytest.raises(ValueError):
        lpt_partition(costs, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, costs, out_q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a stand-in for the batched GPU calls: each system's "result" names its index and rank
        res = run_sharded(len(costs), costs, lambda idx: {i: (i, rank) for i in idx}, rank, world)
        if rank == 0:
            out_q.put(res)
    finally:
        dist.destroy_process_group()


def test_sharded_gather_world2():
    costs = [estimated_cost(L) for L in (2000, 60000, 30000, 8000, 45000, 15000, 3000)]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, costs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    parts = lpt_partition(costs, 2)
    owner = {i: r for r, p in enumerate(parts) for i in p}
    assert [r[0] for r in res] == list(range(len(costs)))
    assert all(r[1] == owner[r[0]] for r in res)
    assert len(parts[0]) > 0 and len(parts[1]) > 0
