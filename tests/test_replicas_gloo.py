"""Host logic of the multi-GPU replica path, on CPU with two gloo ranks."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_1603_09337_gb300 import replicas


def test_shards_partition_the_items():
    for n in (0, 1, 7, 256, 1000):
        for ws in (1, 2, 3, 8):
            got = [list(replicas.shard(n, r, ws)) for r in range(ws)]
            flat = [i for g in got for i in g]
            assert flat == list(range(n))
            assert max(map(len, got)) - min(map(len, got)) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world_size, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world_size), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    ws, r, lr = replicas.world()
    mine = list(replicas.shard(10, r, ws))
    m = replicas.max_over_ranks(1.5 + r)
    dist.barrier()
    q.put((r, mine, m, ws, lr))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_and_reduce():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] + res[1][1] == list(range(10))
    assert all(r[2] == pytest.approx(2.5) for r in res)   # max over ranks
    assert all(r[3] == 2 for r in res)
