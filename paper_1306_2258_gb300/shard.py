"""One molecule's pair work split over ranks, and the sum of the shares.

`set_shard(p, rank, world)` makes a Profile compute shard `rank` of its work list split into
`world` contiguous parts of equal pair work (SAS_OPT_SHARD); its profile is then that shard's
additive share of I(q) (the diagonal and the exact q = 0 pair counts belong to rank 0).  Summing
the shares of all ranks gives the whole profile: `allreduce_shares` does it over a
torch.distributed group in rank order (gather, then a fixed-order sum), so every rank gets the
same bits whatever the backend's reduction tree.
"""
from __future__ import annotations

import torch

from . import _lib


def set_shard(profile, rank: int, world: int):
    if not (1 <= world <= 65535 and 0 <= rank < world):
        raise ValueError("need 1 <= world <= 65535 and 0 <= rank < world")
    profile.set_option(_lib.SAS_OPT_SHARD, world * 65536 + rank)


def sum_shares(shares):
    """Fixed-order sum of share tensors (rank 0 first)."""
    total = shares[0].clone()
    for s in shares[1:]:
        total += s
    return total


def allreduce_shares(share: torch.Tensor, group=None) -> torch.Tensor:
    """The whole profile from every rank's share, identical on all ranks."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(share) for _ in range(world)]
    dist.all_gather(parts, share.contiguous(), group=group)
    return sum_shares(parts)
