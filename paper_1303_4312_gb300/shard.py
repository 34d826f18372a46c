"""Sharding a stable merge across the ranks of a process group.

Algorithm 2 (Section 3) with one processing element per rank: rank g of G
owns the output block [floor(g*(m+n)/G), floor((g+1)*(m+n)/G)), co-ranks both
ends of it (Algorithm 1 / Lemma 1) and merges the input windows those
co-ranks delimit.  Blocks differ in size by at most one element
(Proposition 2) and need no exchange when every rank holds A and B; the
block outputs can be gathered into C when a rank wants the whole result.

The co-rank and local merge steps are parameters: by default they are this
library's CUDA calls on the rank's own GPU (``api.co_rank``, ``api.merge``);
tests pass host implementations to run the plan on CPU ranks.
"""
from __future__ import annotations

from dataclasses import dataclass


@dataclass(frozen=True)
class ShardPlan:
    rank: int
    world: int
    k0: int          # first output rank of this block
    k1: int          # one past the last output rank
    i0: int          # co-rank in A of k0
    i1: int          # co-rank in A of k1
    j0: int          # co-rank in B of k0
    j1: int          # co-rank in B of k1

    @property
    def size(self) -> int:
        return self.k1 - self.k0


def block_bounds(total: int, world: int, rank: int) -> tuple[int, int]:
    """Output block of `rank` (the products are exact integers)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the group")
    return rank * total // world, (rank + 1) * total // world


def plan(m: int, n: int, world: int, rank: int, co_rank) -> ShardPlan:
    """co_rank(k) -> (i, j), i + j == k, for the stable merge of A[m], B[n]."""
    k0, k1 = block_bounds(m + n, world, rank)
    i0, j0 = co_rank(k0)
    i1, j1 = co_rank(k1)
    if i0 + j0 != k0 or i1 + j1 != k1 or not (0 <= i0 <= i1 <= m and 0 <= j0 <= j1 <= n):
        raise RuntimeError("co_rank returned an inconsistent split")
    return ShardPlan(rank, world, k0, k1, i0, i1, j0, j1)


def merge_block(A, B, p: ShardPlan, merge):
    """This rank's block of the output: merge(A[i0:i1], B[j0:j1])."""
    return merge(A[p.i0:p.i1], B[p.j0:p.j1])


def sharded_merge(A, B, group=None, co_rank=None, merge=None, gather: bool = True):
    """Stable merge of A and B (held by every rank) split over the ranks of
    `group` (torch.distributed).  Returns (block, plan) or, with
    gather=True, the whole output assembled on every rank."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if co_rank is None or merge is None:
        from . import api
        co_rank = co_rank or (lambda k: api.co_rank(A, B, k))
        merge = merge or api.merge
    p = plan(A.numel(), B.numel(), world, rank, co_rank)
    block = merge_block(A, B, p, merge)
    if not gather:
        return block, p
    sizes = [block_bounds(A.numel() + B.numel(), world, r) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    padded = torch.zeros(width, dtype=block.dtype, device=block.device)
    padded[: block.numel()] = block
    parts = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(sizes)]), p
