"""Host logic of the multi-GPU replica runs, on CPU with gloo (world size 2):
shards are disjoint and complete, the timing reduction is the max over
ranks, and the whole-job rate counts every rank's work."""
import os
import socket

import pytest

from paper_1908_03565_gb300 import replicas


def test_shard_partitions_items():
    for n in (0, 1, 7, 512):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                seen += list(replicas.shard(n, world, r))
            assert seen == list(range(n))
            sizes = [len(replicas.shard(n, world, r)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = 1.5 if rank == 0 else 2.25            # the second replica is slower
        tmax = replicas.max_over_ranks(t, dist)
        dist.barrier()
        rate = replicas.whole_job_rate(16.0, tmax, world)
        q.put((rank, tmax, rate, list(replicas.shard(10, world, rank))))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
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
    assert [r[1] for r in res] == [2.25, 2.25]
    assert res[0][2] == pytest.approx(2 * 16.0 / 2.25)
    assert res[0][3] + res[1][3] == list(range(10))
