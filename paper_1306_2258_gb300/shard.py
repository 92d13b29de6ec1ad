"""One molecule's pair work split over ranks, and the sum of the shares.

`set_shard(p, rank, world)` makes a Profile compute shard `rank` of its work list split into
`world` contiguous parts of equal pair work (SAS_OPT_SHARD); its profile is then that shard's
additive share of I(q) (the diagonal and the exact q = 0 pair counts belong to rank 0).  Summing
the shares of all ranks gives the whole profile: `allreduce_shares` does it over a
torch.distributed group in rank order (gather, then a fixed-order sum), so every rank gets the
same bits whatever the backend's reduction tree.

On a SAS_DETERMINISTIC context the shares can also be put back together bit for bit: every shard's
exact type-pair sums (`Profile.exact_sums`, 128-bit fixed-point integers as int64 (low, high)
pairs) are added exactly (`add_exact` locally, `allreduce_exact` over a group, where integer
addition makes the result independent of the reduction order), and `Profile.assemble_exact`
turns the total into the profile an unsplit call gives.
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


_MASK32 = 0xFFFFFFFF


def _limbs(U: torch.Tensor) -> torch.Tensor:
    """[..., 2] int64 (low, high) of 128-bit two's complement integers -> [..., 4] int64 limbs of
    32 bits, least significant first, the last one signed (sums of up to 2^31 of them are exact)."""
    lo, hi = U[..., 0], U[..., 1]
    return torch.stack([lo & _MASK32, (lo >> 32) & _MASK32, hi & _MASK32, hi >> 32], dim=-1)


def _from_limbs(L: torch.Tensor) -> torch.Tensor:
    """Inverse of _limbs for summed limbs: carries propagated upward, then (low, high)."""
    n0 = L[..., 0] & _MASK32
    c = L[..., 0] >> 32
    t = L[..., 1] + c
    n1 = t & _MASK32
    c = t >> 32
    t = L[..., 2] + c
    n2 = t & _MASK32
    n3 = L[..., 3] + (t >> 32)
    return torch.stack([n0 | (n1 << 32), n2 | (n3 << 32)], dim=-1)


def add_exact(parts) -> torch.Tensor:
    """Exact sum of 128-bit integer arrays [..., 2] int64 (tensors or NumPy arrays)."""
    ts = [torch.as_tensor(p, dtype=torch.int64) for p in parts]
    acc = _limbs(ts[0])
    for t in ts[1:]:
        acc = acc + _limbs(t)
    return _from_limbs(acc)


def allreduce_exact(U: torch.Tensor, group=None) -> torch.Tensor:
    """Exact sum over the group of every rank's 128-bit sums U [..., 2] int64 (the same on all ranks)."""
    import torch.distributed as dist
    L = _limbs(torch.as_tensor(U, dtype=torch.int64)).contiguous()
    dist.all_reduce(L, op=dist.ReduceOp.SUM, group=group)
    return _from_limbs(L)
