"""Multi-process host logic of the replica (weak-scaling) path on CPU with gloo."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1609_01797_gb300.replicas import max_over_ranks, shard_range, sum_over_ranks


def test_shard_range_partitions():
    for n in (0, 1, 7, 65536, 200001):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        step_ms = [3.0, 5.0][rank]
        errors = [11, 31][rank]
        q.put((rank, max_over_ranks(step_ms, world), sum_over_ranks(errors, world), shard_range(10, rank, world)))
    finally:
        dist.destroy_process_group()


def test_reductions_world_size_2():
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
    assert [r[1] for r in res] == [5.0, 5.0]
    assert [r[2] for r in res] == [42, 42]
    assert [r[3] for r in res] == [(0, 5), (5, 10)]
