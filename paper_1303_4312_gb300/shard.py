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
# B[b_off[r], b_off[r+1]).  The co-ranks of every rank's output block are
# found by Algorithm 1 with remote point reads, then each rank fetches the
# two windows they delimit from their owners and merges them locally.
# ---------------------------------------------------------------------------
_WIDTH = {"i32": 32, "u32": 32, "f32": 32, "i64": 64, "u64": 64, "f64": 64, "pair_u32": 64,
          "pair_i32": 64}


def _as_key(v: int, key_type: str) -> int:
    """A key read back from an int64 carrier (the bits of the stored key,
    sign-extended from its width), as a Python int whose integer order is the
    key type's order: unsigned types are masked to their width; float bits
    (IEEE-754 totalOrder) keep positives and flip the magnitude of negatives;
    ':desc' negates."""
    base, _, mod = key_type.partition(":")
    bits = _WIDTH[base]
    if base.startswith("pair"):
        v &= (1 << 64) - 1
        if base == "pair_i32":
            v ^= (1 << 63) | (1 << 31)      # both halves' sign bits: lexicographic
        return -v if mod == "desc" else v
    if base[0] == "u":
        v &= (1 << bits) - 1
    else:
        v = ((v + (1 << (bits - 1))) & ((1 << bits) - 1)) - (1 << (bits - 1))   # sign-extend
        if base[0] == "f" and v < 0:
            v ^= (1 << (bits - 1)) - 1
    return -v if mod == "desc" else v


def _bits(t):
    """Integer view of a key block (floats travel as their bit patterns)."""
    import torch
    if t.dtype.is_floating_point:
        return t.view(torch.int32 if t.element_size() == 4 else torch.int64)
    return t


class _Prober:
    """Point reads of A and B by global index: every rank all-gathers the
    indices it wants (-1 for none), answers those that fall in its own
    blocks, and an all-reduce (sum) hands each rank its answers (exactly one
    rank owns each index, the others contribute zero)."""

    def __init__(self, A_blk, B_blk, a_off, b_off, rank, world, group):
        import torch
        self.torch = torch
        self.A, self.B = _bits(A_blk), _bits(B_blk)
        self.a0, self.a1 = a_off[rank], a_off[rank + 1]
        self.b0, self.b1 = b_off[rank], b_off[rank + 1]
        self.world, self.group = world, group
        self.dev = A_blk.device

    def read(self, ia, ib):
        import torch.distributed as dist
        torch = self.torch
        ra = len(ia)
        req = torch.tensor(list(ia) + list(ib), dtype=torch.int64, device=self.dev)
        parts = [torch.empty_like(req) for _ in range(self.world)]
        dist.all_gather(parts, req, group=self.group)
        allreq = torch.stack(parts)                       # world x (ra + rb)
        ans = torch.zeros_like(allreq)
        for lo, hi, blk, cols in ((self.a0, self.a1, self.A, slice(0, ra)),
                                  (self.b0, self.b1, self.B, slice(ra, None))):
            idx = allreq[:, cols]
            mine = (idx >= lo) & (idx < hi)
            if bool(mine.any()):
                sub = ans[:, cols]
                sub[mine] = blk[idx[mine] - lo].to(torch.int64)
                ans[:, cols] = sub
        dist.all_reduce(ans, group=self.group)
        mine = ans[dist.get_rank(self.group)].tolist()
        return mine[:ra], mine[ra:]


def distributed_co_rank(ranks, m, n, prober, key_type, group=None):
    """Algorithm 1 (Section 2) for each output rank in `ranks`, run in lock
    step on every rank of the group (each passes the same number of ranks),
    with the keys it compares read remotely: one round of point reads per
    iteration, A[j-1], A[j], B[k-1], B[k] of every unfinished search.
    k_low starts at max(0, i - m) (the printed algorithm leaves it unset and
    argues the first move always sets it).  Returns [(j, k), ...]."""
    import torch
    import torch.distributed as dist
    st = []
    for i in ranks:
        j = min(i, m)
        st.append({"i": i, "j": j, "k": i - j, "jl": max(0, i - n), "kl": max(0, i - m),
                   "done": False})
    while True:
        ia, ib = [], []
        for s in st:
            j, k, live = s["j"], s["k"], not s["done"]
            ia += [j - 1 if live and j > 0 else -1, j if live and j < m else -1]
            ib += [k - 1 if live and k > 0 else -1, k if live and k < n else -1]
        va, vb = prober.read(ia, ib)
        for q, s in enumerate(st):
            if s["done"]:
                continue
            j, k = s["j"], s["k"]
            a_prev, a_cur = _as_key(va[2 * q], key_type), _as_key(va[2 * q + 1], key_type)
            b_prev, b_cur = _as_key(vb[2 * q], key_type), _as_key(vb[2 * q + 1], key_type)
            if j > 0 and k < n and a_prev > b_cur:            # first condition fails
                d = (j - s["jl"] + 1) // 2
                s["kl"] = k
                s["j"], s["k"] = j - d, k + d
            elif k > 0 and j < m and b_prev >= a_cur:         # second condition fails
                d = (k - s["kl"] + 1) // 2
                s["jl"] = j
                s["j"], s["k"] = j + d, k - d
            else:
                s["done"] = True
        live = torch.tensor([sum(not s["done"] for s in st)], dtype=torch.int64,
                            device=prober.dev)
        dist.all_reduce(live, group=group)
        if int(live.item()) == 0:
            return [(s["j"], s["k"]) for s in st]


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
                      merge=None):
    """Stable merge of A and B block-distributed over the ranks of `group`
    (rank r holds the r-th contiguous blocks, any sizes, possibly empty).
    Rank g returns its equal output block C[floor(g(m+n)/G), floor((g+1)(m+n)/G))
    (and its payloads when Av_blk/Bv_blk are given) with its ShardPlan.

    Steps (Section 3's distributed reading of Algorithm 2):
      1. co-rank both block ends with Algorithm 1 and remote point reads;
      2. fetch the windows A[i0, i1) and B[j0, j1) from their owners
         (one all-to-all per array);
      3. merge them locally: `merge(A, B)` or, with payloads,
         `merge(A, Av, B, Bv) -> (C, Cv)`; by default this library's kernels.
    """
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    dev = A_blk.device
    a_off = _offsets(A_blk.numel(), world, group, dev)
    b_off = _offsets(B_blk.numel(), world, group, dev)
    m, n = a_off[-1], b_off[-1]
    k0, k1 = block_bounds(m + n, world, rank)
    prober = _Prober(A_blk, B_blk, a_off, b_off, rank, world, group)
    (i0, j0), (i1, j1) = distributed_co_rank([k0, k1], m, n, prober, key_type, group)
    if i0 + j0 != k0 or i1 + j1 != k1 or not (0 <= i0 <= i1 <= m and 0 <= j0 <= j1 <= n):
        raise RuntimeError("co_rank returned an inconsistent split")
    p = ShardPlan(rank, world, k0, k1, i0, i1, j0, j1)
    import torch
    win = torch.tensor([i0, i1, j0, j1], dtype=torch.int64, device=dev)
    parts = [torch.empty_like(win) for _ in range(world)]
    dist.all_gather(parts, win, group=group)
    w = [t.tolist() for t in parts]
    ia = [x[0] for x in w], [x[1] for x in w]
    jb = [x[2] for x in w], [x[3] for x in w]
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
