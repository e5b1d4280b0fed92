"""The N > 1 path of bench.py (replicas: one rank per GPU, slowest rank's time) on CPU with gloo, world size 2."""

import os
import socket

import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(1.0 + rank * 2.5, dist)  # ranks report different times
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1] == 3.5


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(2.0) == 2.0


def _shard_worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1306_4627_gb300 import gen, shard
    pairs = gen.batch_pairs(count=500, seed=77)
    m = [len(x) for x, _ in pairs]
    n = [len(y) for _, y in pairs]
    parts = shard.partition_pairs(m, n, world)
    out[rank] = parts[rank].tolist()  # each rank evaluates the rule itself; nothing is exchanged
    dist.destroy_process_group()


def test_batch_shards_gloo_two_ranks():
    """Two ranks compute their shards independently: together they cover every pair exactly once."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = set(out[0]), set(out[1])
    assert not (a & b) and a | b == set(range(500))


def test_partition_balances_cells():
    import numpy as np
    from paper_1306_4627_gb300 import gen, shard
    pairs = gen.batch_pairs(count=2000, seed=78)
    m = np.array([len(x) for x, _ in pairs])
    n = np.array([len(y) for _, y in pairs])
    for world in (1, 2, 3, 8):
        parts = shard.partition_pairs(m, n, world)
        assert sorted(np.concatenate(parts).tolist()) == list(range(len(pairs)))
        loads = shard.shard_cells(m, n, parts)
        # greedy largest-first: no shard exceeds another by more than the largest pair
        assert max(loads) - min(loads) <= int((m * n).max())
    assert [p.tolist() for p in shard.partition_pairs([3, 1, 2], [1, 1, 1], 2)] == [[0], [1, 2]]


def test_partition_edge_cases():
    from paper_1306_4627_gb300 import shard
    assert [len(p) for p in shard.partition_pairs([], [], 3)] == [0, 0, 0]
    parts = shard.partition_pairs([5], [7], 4)  # more ranks than pairs: one rank works, the others get nothing
    assert [len(p) for p in parts] == [1, 0, 0, 0] and shard.shard_cells([5], [7], parts) == [35, 0, 0, 0]
    parts = shard.partition_pairs([0, 3, 0, 9], [4, 0, 0, 9], 2)  # empty pairs (no cells) are still assigned
    assert sorted(int(k) for p in parts for k in p) == [0, 1, 2, 3]
    import pytest
    with pytest.raises(ValueError):
        shard.partition_pairs([1, 2], [3], 2)
    with pytest.raises(ValueError):
        shard.partition_pairs([1], [1], 0)
