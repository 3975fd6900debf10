"""Multi-process host logic on CPU (gloo, world size 2): shards of a grouped
batch cover every image exactly once and balance by blocks, block ranges
tile the whole image, and the timing reduction takes the slowest rank."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import datagen
from paper_1710_07193_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = shard.shard_items(sizes, rank, world)
    b0, b1 = shard.shard_range(262144, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, {"items": mine, "blocks": (b0, b1),
                                      "load": sum(sizes[i] for i in mine)})
    slowest = shard.max_over_ranks(10.0 + rank, dist)
    if rank == 0:
        out.put({"gathered": gathered, "slowest": slowest})
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharding_gloo():
    sizes = [(h // 8) * (w // 8) for h, w in datagen.grouped_sizes()]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = res["gathered"]
    items = sorted(g[0]["items"] + g[1]["items"])
    assert items == list(range(len(sizes)))                  # each image exactly once
    assert not set(g[0]["items"]) & set(g[1]["items"])
    loads = [g[0]["load"], g[1]["load"]]
    assert max(loads) - min(loads) <= max(sizes)              # greedy balance bound
    assert g[0]["blocks"] == (0, 131072) and g[1]["blocks"] == (131072, 262144)
    assert res["slowest"] == 11.0


def test_shard_helpers_single_process():
    assert shard.shard_range(10, 0, 3) == (0, 3)
    assert shard.shard_range(10, 2, 3) == (6, 10)
    assert shard.shard_items([5, 1, 1, 1], 0, 2) == [0]
    assert shard.shard_items([5, 1, 1, 1], 1, 2) == [1, 2, 3]
    assert shard.max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        shard.shard_range(10, 3, 3)
