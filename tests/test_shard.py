"""Frame sharding across ranks and the max-over-ranks timing (CPU, gloo)."""
import os
import socket

import pytest

from paper_1611_05319_gb300.shard import lpt_partition, max_over_ranks


def test_lpt_partition_covers_every_frame_once_and_balances():
    w = [5, 9, 1, 7, 3, 3, 8, 2, 6, 4]
    parts = lpt_partition(w, 3)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(w)))
    loads = [sum(w[i] for i in p) for p in parts]
    assert max(loads) - min(loads) <= max(w)
    assert lpt_partition(w, 1) == [list(range(len(w)))]
    assert lpt_partition([], 2) == [[], []]


def test_lpt_partition_is_deterministic():
    w = [3, 3, 3, 3]
    assert lpt_partition(w, 2) == [[0, 2], [1, 3]]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        weights = [10, 40, 30, 20]
        mine = lpt_partition(weights, world)[rank]
        step_ms = 1.0 + sum(weights[i] for i in mine) / 10.0  # stand-in for a measured step time
        q.put((rank, mine, max_over_ranks(step_ms, dist)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    shards = [r[1] for r in res]
    assert sorted(shards[0] + shards[1]) == [0, 1, 2, 3]
    assert res[0][2] == res[1][2] == max(1.0 + sum([10, 40, 30, 20][i] for i in s) / 10.0 for s in shards)
