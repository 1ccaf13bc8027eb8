"""Multi-GPU operation by channel sharding (host side).

Channels are independent through the whole hot path: a packet carries one 8-channel group of one
F-engine stream (Sec. II-A.2), each channel's matrix is correlated and normalised on its own (Sec.
II-B, Sec. II-C), and the Pathfinder spreads its band over servers by channel (Sec. II: each
server's GPUs take the channels of their streams). So one process per GPU takes a contiguous range
of whole channel groups, and no data crosses GPUs while frames are assembled, correlated or
normalised. The only exchange is the collection of normalised outputs at the end of an
integration (Sec. II-C: results leave the X-engine for the collection server ordered by stream and
channel), done here as one gather to rank 0 outside the timed hot path.

    g0, g1 = shard_groups(n_groups, world, rank)       # this rank's 8-channel groups [g0, g1)
    f0, f1 = shard_channels(n_chan, world, rank)       # the same as channels [f0, f1)
    full = gather_channels(local_out, f0, n_chan)      # rank 0: [n_chan, ...]; others: None
"""
from __future__ import annotations

CHANNELS_PER_GROUP = 8


def shard_groups(n_groups: int, world: int, rank: int) -> tuple[int, int]:
    """Contiguous, balanced range [g0, g1) of channel groups for `rank` of `world` (sizes differ
    by at most one group; ranks past the last group get an empty range)."""
    if n_groups < 0 or world < 1 or not 0 <= rank < world:
        raise ValueError("need n_groups >= 0, world >= 1 and 0 <= rank < world")
    base, extra = divmod(n_groups, world)
    g0 = rank * base + min(rank, extra)
    return g0, g0 + base + (1 if rank < extra else 0)


def shard_channels(n_chan: int, world: int, rank: int) -> tuple[int, int]:
    """Channel range [f0, f1) of `rank`: whole 8-channel groups (a packet never straddles ranks)."""
    if n_chan % CHANNELS_PER_GROUP:
        raise ValueError("the band must hold whole 8-channel groups")
    g0, g1 = shard_groups(n_chan // CHANNELS_PER_GROUP, world, rank)
    return g0 * CHANNELS_PER_GROUP, g1 * CHANNELS_PER_GROUP


def streams_of(n_streams: int, world: int, rank: int) -> list[int]:
    """F-engine streams (links) whose packets `rank` receives: a contiguous block, so that with
    groups_per_stream groups per stream the rank's channels are contiguous too."""
    s0, s1 = shard_groups(n_streams, world, rank)
    return list(range(s0, s1))


def gather_channels(local, f0: int, n_chan: int, group=None):
    """Collects every rank's channel rows [f0, f0 + len(local)) of a per-channel output (e.g. the
    normalised visibilities [F_local][P][2]) into one [n_chan, ...] tensor on rank 0, in global
    channel order. Returns None on the other ranks. Uses torch.distributed (gloo for host tensors,
    nccl for device tensors); every rank must call it."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    tail = tuple(local.shape[1:])
    meta = torch.tensor([f0, local.shape[0]], dtype=torch.int64, device=local.device)
    metas = [torch.zeros_like(meta) for _ in range(world)]
    dist.all_gather(metas, meta, group=group)
    rows = max(int(m[1]) for m in metas)
    pad = torch.zeros((rows,) + tail, dtype=local.dtype, device=local.device)
    pad[:local.shape[0]] = local
    parts = [torch.empty_like(pad) for _ in range(world)] if rank == 0 else None
    dist.gather(pad, parts, dst=0, group=group)
    if rank != 0:
        return None
    out = torch.empty((n_chan,) + tail, dtype=local.dtype, device=local.device)
    covered = torch.zeros(n_chan, dtype=torch.bool)
    for m, part in zip(metas, parts):
        a, n = int(m[0]), int(m[1])
        if a < 0 or a + n > n_chan or bool(covered[a:a + n].any()):
            raise ValueError("channel shards overlap or fall outside the band")
        out[a:a + n] = part[:n]
        covered[a:a + n] = True
    if not bool(covered.all()):
        raise ValueError("channel shards do not cover the band")
    return out
