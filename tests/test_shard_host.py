"""Host logic of sharding one batch over replicas (CPU): the split of the
evaluation order into ranges of equal estimated work, and the gather of
per-rank shards to rank 0 over two gloo ranks."""

import os
import socket

import pytest
import torch
import torch.multiprocessing as mp

from paper_2505_08985_gb300 import shard


def _range_work(partials, a, b, block=4096):
    return sum(partials[a // block:(b + block - 1) // block]) if b > a else 0.0


def test_split_balances_work_and_covers_the_order():
    # large footprints first (the sort puts the highest entry levels first)
    partials = [100.0] * 10 + [1.0] * 90
    nq = 100 * 4096 - 17
    for n in (2, 3, 4, 7):
        b = shard.split_by_work(partials, n, nq)
        assert len(b) == n + 1 and b[0] == 0 and b[-1] == nq and all(x <= y for x, y in zip(b, b[1:]))
        assert all(x % 4096 == 0 for x in b[1:-1])  # cuts on block boundaries
        total = sum(partials)
        # each cut is within half a block's work of its target share
        for i in range(1, n):
            cum = sum(partials[:b[i] // 4096])
            assert abs(cum - total * i / n) <= 50.0 + 1e-9


def test_split_edge_cases():
    b = shard.split_by_work([5.0], 3, 10)  # one block: exactly one shard gets it
    assert b[0] == 0 and b[-1] == 10 and sum(1 for i in range(3) if b[i + 1] > b[i]) == 1
    b = shard.split_by_work([0.0, 0.0], 2, 8000)  # no work at all: a valid cover of the order
    assert b[0] == 0 and b[-1] == 8000 and b[1] in (0, 8000)
    assert shard.split_by_work([1.0] * 8, 1, 30000) == [0, 30000]
    assert shard.split_by_work([1.0] * 8, 8, 8 * 4096) == [k * 4096 for k in range(9)]
    with pytest.raises(ValueError):
        shard.split_by_work([1.0], 0, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, nq, bounds, ret):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # a fake evaluation of this rank's range of the evaluation order:
        # position k of the order gets the value 1000 + k
        a, b = bounds[rank], bounds[rank + 1]
        D_local = torch.arange(a, b, dtype=torch.float32) + 1000.0
        out = shard.gather_shards(D_local, bounds, rank, world)
        if rank == 0:
            ret.put(out.tolist())
    finally:
        dist.destroy_process_group()


def test_gather_shards_over_two_gloo_ranks():
    nq = 37
    bounds = [0, 30, 37]  # unequal shards
    ctx = mp.get_context("spawn")
    ret = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, nq, bounds, ret)) for r in range(2)]
    for p in procs:
        p.start()
    out = ret.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out == [1000.0 + k for k in range(nq)]


def test_work_block_adapts_to_the_batch():
    assert shard.work_block(50000, 3) == 260
    assert shard.work_block(1000, 2) == 256
    assert shard.work_block(1 << 22, 8) == 4096
