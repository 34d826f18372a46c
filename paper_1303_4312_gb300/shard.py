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


# ---------------------------------------------------------------------------
# Block-distributed inputs: rank r holds only A[a_off[r], a_off[r+1]) and
# B[b_off[r], b_off[r+1]).  The co-ranks of every block boundary are found
# by Algorithm 1 with remote point reads (the library's cr_dist_co_rank_*
# kernels do the arithmetic; this module only runs the collectives), then
# each rank fetches the two windows they delimit from their owners and
# merges them locally.
# ---------------------------------------------------------------------------
def _bits(t):
    """Integer view of a key block (floats travel as their bit patterns)."""
    import torch
    if t.dtype.is_floating_point:
        return t.view(torch.int32 if t.element_size() == 4 else torch.int64)
    return t


def distributed_co_rank(ranks, m, n, A_blk, a_lo, B_blk, b_lo, key_type, group=None,
                        search=None):
    """Algorithm 1 (Section 2) for each output rank in `ranks` -- the same
    list on every rank of the group -- with A and B block-distributed: this
    rank holds A[a_lo, a_lo + len(A_blk)) and B[b_lo, b_lo + len(B_blk)).
    Every rank runs all the searches in lock step; per iteration the
    positions they read are the same everywhere, each rank answers those in
    its own blocks (zero elsewhere) and one all-reduce (sum) delivers every
    key.  After the iteration bound (Proposition 1, corrected: at most
    ceil(log2(min(m, n) + 1)) moves, plus the final check) every search has
    finished.  `search` makes the search object (default: the library's
    kernels, api.DistCoRank).  Returns [(i, j), ...]."""
    import torch
    import torch.distributed as dist
    if search is None:
        from . import api
        search = api.DistCoRank
    s = search(m, n, ranks, key_type, A_blk.device)
    a, b = _bits(A_blk), _bits(B_blk)

    def iterate(times):
        for _ in range(times):
            pa, pb = s.probes()
            ans = torch.cat([s.answer(a, a_lo, pa), s.answer(b, b_lo, pb)])
            dist.all_reduce(ans, group=group)
            s.step(ans[:pa.numel()], ans[pa.numel():])
    iterate(s.iterations())
    res, live = s.result()
    # every rank holds the same state, so all take the same decision here
    extra = 0
    while live and extra < 64:
        iterate(1)
        extra += 1
        res, live = s.result()
    if live:
        raise RuntimeError(f"{live} co-rank searches did not finish")
    return res


def _offsets(local_len, world, group, dev):
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_len], dtype=torch.int64, device=dev)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    off = [0]
    for p in parts:
        off.append(off[-1] + int(p.item()))
    return off


def _fetch_window(blk, off, lo_all, hi_all, rank, world, group):
    """all-to-all: rank g receives the part of [lo_all[g], hi_all[g]) that
    every rank r holds in its block [off[r], off[r+1])."""
    import torch
    import torch.distributed as dist
    send = [max(0, min(hi_all[g], off[rank + 1]) - max(lo_all[g], off[rank]))
            for g in range(world)]
    recv = [max(0, min(hi_all[rank], off[r + 1]) - max(lo_all[rank], off[r]))
            for r in range(world)]
    pieces = []
    for g in range(world):
        if send[g]:
            s0 = max(lo_all[g], off[rank]) - off[rank]
            pieces.append(blk[s0:s0 + send[g]])
    src = torch.cat(pieces) if pieces else blk[:0]
    out = torch.empty(sum(recv), dtype=blk.dtype, device=blk.device)
    dist.all_to_all_single(out, src.contiguous(), recv, send, group=group)
    return out


def distributed_merge(A_blk, B_blk, key_type: str, group=None, Av_blk=None, Bv_blk=None,
                      merge=None, search=None):
    """Stable merge of A and B block-distributed over the ranks of `group`
    (rank r holds the r-th contiguous blocks, any sizes, possibly empty).
    Rank g returns its equal output block C[floor(g(m+n)/G), floor((g+1)(m+n)/G))
    (and its payloads when Av_blk/Bv_blk are given) with its ShardPlan.

    Steps (Section 3's distributed reading of Algorithm 2):
      1. co-rank every block boundary with Algorithm 1 and remote point
         reads (distributed_co_rank; every rank then knows every window);
      2. fetch the windows A[i0, i1) and B[j0, j1) from their owners
         (one all-to-all per array);
      3. merge them locally: `merge(A, B)` or, with payloads,
         `merge(A, Av, B, Bv) -> (C, Cv)`; by default this library's kernels.
    `search` is passed to distributed_co_rank.
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = A_blk.device
    a_off = _offsets(A_blk.numel(), world, group, dev)
    b_off = _offsets(B_blk.numel(), world, group, dev)
    m, n = a_off[-1], b_off[-1]
    # every block boundary, co-ranked by all ranks together
    ks = [block_bounds(m + n, world, g)[0] for g in range(world)] + [m + n]
    cr = distributed_co_rank(ks, m, n, A_blk, a_off[rank], B_blk, b_off[rank], key_type, group,
                             search)
    (i0, j0), (i1, j1) = cr[rank], cr[rank + 1]
    k0, k1 = ks[rank], ks[rank + 1]
    if i0 + j0 != k0 or i1 + j1 != k1 or not (0 <= i0 <= i1 <= m and 0 <= j0 <= j1 <= n):
        raise RuntimeError("co_rank returned an inconsistent split")
    p = ShardPlan(rank, world, k0, k1, i0, i1, j0, j1)
    ia = [c[0] for c in cr[:-1]], [c[0] for c in cr[1:]]
    jb = [c[1] for c in cr[:-1]], [c[1] for c in cr[1:]]
    A = _fetch_window(A_blk, a_off, ia[0], ia[1], rank, world, group)
    B = _fetch_window(B_blk, b_off, jb[0], jb[1], rank, world, group)
    kv = Av_blk is not None
    if kv:
        Av = _fetch_window(Av_blk, a_off, ia[0], ia[1], rank, world, group)
        Bv = _fetch_window(Bv_blk, b_off, jb[0], jb[1], rank, world, group)
    if merge is None:
        from . import api
        if kv:
            return (*api.merge_kv(A, Av, B, Bv, key_type=key_type), p)
        return api.merge(A, B, key_type=key_type), p
    if kv:
        return (*merge(A, Av, B, Bv), p)
    return merge(A, B), p
