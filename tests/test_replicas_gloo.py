"""The multi-GPU path is replicas of independent problems: check the host
logic (sharding, max-over-ranks timing, whole-job throughput) with two
gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2608_17844_b300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        items = list(range(7))
        mine = replicas.shard(items, rank, world)
        elapsed = 1.0 + rank  # rank 1 is the slow one
        tput = replicas.aggregate_throughput(len(mine), elapsed)
        mx = replicas.max_over_ranks(elapsed)
        out.put((rank, mine, tput, mx))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, s0, t0, m0), (r1, s1, t1, m1) = res
    assert s0 == [0, 2, 4, 6] and s1 == [1, 3, 5]
    assert sorted(s0 + s1) == list(range(7))
    assert m0 == m1 == 2.0
    assert t0 == t1 == pytest.approx(7 / 2.0)


def test_single_process_defaults():
    from paper_2608_17844_b300 import replicas
    assert replicas.world() == (1, 0)
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.aggregate_throughput(4, 2.0) == 2.0
    assert replicas.shard([1, 2, 3], 0, 1) == [1, 2, 3]
