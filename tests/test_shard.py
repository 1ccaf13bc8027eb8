"""Channel sharding for one process per GPU (host logic; CPU, gloo, world size 2 and 3).

The path shards by 8-channel group with no exchange (Sec. II, Sec. II-C); these tests check the
partition arithmetic and the one collection step, a gather of normalised outputs to rank 0 in
global channel order.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1503_06189_b300 import shard


@pytest.mark.parametrize("n_groups,world", [(128, 1), (128, 2), (128, 3), (16, 8), (3, 8), (0, 2), (129, 4)])
def test_groups_cover_the_band_once_balanced(n_groups, world):
    ranges = [shard.shard_groups(n_groups, world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n_groups
    for (a0, a1), (b0, b1) in zip(ranges, ranges[1:]):
        assert a1 == b0                                   # contiguous, disjoint
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and min(sizes) >= 0


def test_channels_are_whole_groups_and_streams_contiguous():
    assert shard.shard_channels(1024, 16, 3) == (192, 256)   # Pathfinder: 64 channels per server
    for r in range(3):
        f0, f1 = shard.shard_channels(1024, 3, r)
        assert f0 % 8 == 0 and f1 % 8 == 0
    assert shard.streams_of(8, 2, 1) == [4, 5, 6, 7]
    with pytest.raises(ValueError):
        shard.shard_channels(1020, 2, 0)
    with pytest.raises(ValueError):
        shard.shard_groups(8, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gather_worker(rank, world, port, n_chan, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f0, f1 = shard.shard_channels(n_chan, world, rank)
        P = 10
        # each rank's "normalised visibilities" for its channels: a value that names the global
        # channel, the pair and the component, so misplaced rows show up
        f = torch.arange(f0, f1, dtype=torch.float32)[:, None, None]
        p = torch.arange(P, dtype=torch.float32)[None, :, None]
        c = torch.arange(2, dtype=torch.float32)[None, None, :]
        local = 1000.0 * f + 10.0 * p + c
        full = shard.gather_channels(local, f0, n_chan)
        if rank == 0:
            want = (1000.0 * torch.arange(n_chan, dtype=torch.float32)[:, None, None] + 10.0 * p + c)
            q.put(("ok", bool(torch.equal(full, want))))
        else:
            q.put(("ok", full is None))
    except Exception as exc:  # reported to the parent
        q.put(("error", repr(exc)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,n_chan", [(2, 1024), (3, 64)])
def test_gather_orders_shards_by_global_channel(world, n_chan):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gather_worker, args=(r, world, port, n_chan, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for pr in procs:
        pr.join(timeout=60)
    assert all(kind == "ok" and value for kind, value in results), results
    assert all(pr.exitcode == 0 for pr in procs)
