"""Host logic of the multi-GPU bench path on CPU: world-size-2 gloo ranks.
Ranks make disjoint fields (no data exchange) and the timing is the max over
ranks."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = [bench.shard_seed(rank, k) for k in range(8)]
    m = bench.aggregate_max(10.0 * (rank + 1), world)
    q.put((rank, seeds, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_and_max_timing():
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, m0), (r1, s1, m1) = res
    assert m0 == m1 == 20.0
    assert not set(s0) & set(s1)
    assert all(0 <= s < (1 << 24) for s in s0 + s1)


def test_single_rank_identity():
    import bench
    assert bench.aggregate_max(3.5, 1) == 3.5
    assert [bench.shard_seed(0, k) for k in range(5)] == [0, 1, 2, 3, 0]
